"""Planted mistakes in the oracle are caught by its pins.

Each case copies oracle/oracle.c, replaces one expression with a plausible
mistake (a dropped term, a wrong sign, a wrong index, a wrong constant, a
wrong boundary rule, a wrong first-order fallback or refinement rule), compiles the copy
with the oracle's own flags, binds the oracle API to it, and runs the pin
tests of tests/test_oracle_pins.py against it: at least one pin must fail. Mistakes are planted only in a temporary copy
of the oracle, on the CPU.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import build as obuild

from . import test_oracle_pins as pins
from . import test_oracle_amr_pins as amr
from . import test_oracle_rk2_pins as rk2

MUTATIONS = {
    "drop_dp_over_rho": ("((un * dun) + (dp * rc))", "(un * dun)"),
    "drop_rho_du": ("a[d][0] = (un * dW[d][0]) + (Wc[0] * dun);", "a[d][0] = (un * dW[d][0]);"),
    "pressure_predictor_no_gamma": ("double gp = g * Wc[nv - 1];", "double gp = Wc[nv - 1];"),
    "transverse_slope_index": ("(un * dW[d][1 + t])", "(un * dW[d][1 + d])"),
    "predictor_sign": ("Wbar[v] = Wc[v] - s;", "Wbar[v] = Wc[v] + s;"),
    "full_slope_at_faces": ("double hs = 0.5 * dW[d][v];", "double hs = dW[d][v];"),
    "minmod_takes_max": ("if (a > 0.0 && b > 0.0) return (a < b) ? a : b;",
                         "if (a > 0.0 && b > 0.0) return (a > b) ? a : b;"),
    "hll_sign": ("(((SR * FL[v]) - (SL * FR[v]))", "(((SR * FL[v]) + (SL * FR[v]))"),
    "hll_wave_speed": ("double a = WL[1 + d] - cL, b = WR[1 + d] - cR;",
                       "double a = WL[1 + d] - cL, b = WR[1 + d] + cR;"),
    "energy_flux_no_pressure": ("F[nv - 1] = (U[nv - 1] + p) * un;", "F[nv - 1] = U[nv - 1] * un;"),
    "eos_gamma": ("W[nv - 1] = (gamma - 1.0) * (U[nv - 1] - ke);", "W[nv - 1] = gamma * (U[nv - 1] - ke);"),
    "update_sign_y": ("acc[v] = (d == 0) ? t : (acc[v] + t);",
                      "acc[v] = (d == 0) ? t : ((d == 1) ? (acc[v] - t) : (acc[v] + t));"),
    "dt_max_not_sum": ("s = (d == 0) ? sd : (s + sd);", "s = (d == 0) ? sd : ((sd > s) ? sd : s);"),
    "outflow_wraps": ("if (periodic) { gi %= n;", "if (1) { gi %= n;"),
    "outflow_reflects_inner_cell": ("if (gi > n - 1) return n - 1;", "if (gi > n - 1) return n - 2;"),
    "periodic_off_by_one": ("if (periodic) { gi %= n; if (gi < 0) gi += n; return gi; }",
                            "if (periodic) { gi %= n; if (gi < 0) gi += n - 1; return gi; }"),
    # the first-order fallback rule
    "fallback_tests_rho_only": ("if (!(q[0] > 0.0) || !(q[nv - 1] > 0.0)) ok = 0;", "if (!(q[0] > 0.0)) ok = 0;"),
    "fallback_tests_p_only": ("if (!(q[0] > 0.0) || !(q[nv - 1] > 0.0)) ok = 0;", "if (!(q[nv - 1] > 0.0)) ok = 0;"),
    "fallback_reverts_offending_faces_only": (
        """                        if (!(q[0] > 0.0) || !(q[nv - 1] > 0.0)) ok = 0;
                    }
                if (!ok) {""",
        """                        if (!(q[0] > 0.0) || !(q[nv - 1] > 0.0)) {
                            ok = 0;
                            for (int v = 0; v < nv; ++v) ((double*)q)[v] = Wc[v];
                        }
                    }
                if (0) {"""),
    "fallback_to_half_step_state": ("for (int v = 0; v < nv; ++v) fs[(d * 2 + s) * MAXV + v] = Wc[v];",
                                    "for (int v = 0; v < nv; ++v) fs[(d * 2 + s) * MAXV + v] = Wbar[v];"),
    # the two-level AMR step
    "amr_no_flux_correction": ("U0new[oi] = side ? (U0new[oi] + corr) : (U0new[oi] - corr);",
                               "U0new[oi] = U0new[oi] + 0.0 * corr;"),
    "amr_flux_correction_sign": ("U0new[oi] = side ? (U0new[oi] + corr) : (U0new[oi] - corr);",
                                 "U0new[oi] = side ? (U0new[oi] - corr) : (U0new[oi] + corr);"),
    "amr_reflux_far_children": ("int o = ((side ? 0 : 1) << d) | (s1 << a1) | (s2 << a2);",
                                "int o = ((side ? 1 : 0) << d) | (s1 << a1) | (s2 << a2);"),
    "amr_restrict_weight": ("double w = (nd == 3) ? 0.125 : 0.25;", "double w = (nd == 3) ? 0.25 : 0.5;"),
    "amr_octant_order": ("o |= ((f[d] / c->bs[d]) % 2) << d;", "o |= ((f[d] / c->bs[d]) % 2) << (c->ndim - 1 - d);"),
    "amr_fine_cell_width": ("for (int d = 0; d < c->ndim; ++d) f.nb[d] = 2 * c->nb[d];",
                            "for (int d = 0; d < c->ndim; ++d) f.nb[d] = c->nb[d];"),
    # the Heun RK2 integrator
    "rk2_forward_euler_twice": ("Unew[o] = Ubase ? (0.5 * (Ubase[o] + us)) : us;", "Unew[o] = us;"),
    "rk2_stage_weights": ("(0.5 * (Ubase[o] + us))", "((0.25 * Ubase[o]) + (0.75 * us))"),
    "rk2_boundary_flux_weight": ("bflux[v] = 0.5 * (b1[v] + b2[v]);", "bflux[v] = b1[v] + b2[v];"),
    "rk2_stages_use_half_step": ("return sweep(m, U, Ubase, 0, dt, Unew, bflux);",
                                 "return sweep(m, U, Ubase, 1, dt, Unew, bflux);"),
    "rk2_second_stage_from_old_state": ("long f2 = (f1 < 0) ? -1 : ora_stage(m, Us, U, dt, Unew, b2);",
                                        "long f2 = (f1 < 0) ? -1 : ora_stage(m, U, Us, dt, Unew, b2);"),
}

# cheapest first; a mutation is caught as soon as one of them fails
PIN_TESTS = [
    ("minmod", lambda o: pins.test_minmod_brute_force(o)),
    ("hll_identical", lambda o: pins.test_hll_identical_states_is_physical_flux(o)),
    ("hll_subsonic", lambda o: pins.test_hll_subsonic_against_hand_values(o)),
    ("fallback_hand_p", lambda o: pins.test_first_order_fallback_hand_case(o, "p")),
    ("fallback_hand_rho", lambda o: pins.test_first_order_fallback_hand_case(o, "rho")),
    ("dt_closed_form", lambda o: pins.test_dt_closed_form(o)),
    ("sod_exact", lambda o: pins.test_sod_2d_matches_exact_solution_and_rows_are_identical(o)),
    ("free_stream", lambda o: pins.test_free_stream_is_preserved_bitwise(o, 3, (0, 0, 0))),
    ("conservation_periodic", lambda o: pins.test_conservation_periodic(o, 1)),
    ("conservation_bflux", lambda o: pins.test_conservation_with_boundary_fluxes(o, "sod")),
    ("mirror_x", lambda o: pins.test_mirror_symmetry_bitwise(o, 0)),
    ("permute_xy", lambda o: pins.test_axis_permutation_symmetry(o, 0, 1)),
    ("outflow_at_rest", lambda o: pins.test_outflow_boundary_flux_is_physical_flux_at_rest(o)),
    ("sod_outflow", lambda o: pins.test_sod_outflow_after_shock_exits(o)),
    ("homologous_2d", lambda o: pins.test_homologous_expansion_matches_exact_density(o, 2)),
    ("order_acoustic_x", lambda o: pins.test_second_order_on_smooth_acoustic_wave(o, (1, 0))),
    ("order_acoustic_diag", lambda o: pins.test_second_order_on_smooth_acoustic_wave(o, (1, 1))),
    ("order_advection", lambda o: pins.test_second_order_on_advected_density_wave(o)),
    ("rk2_free_stream", lambda o: rk2.test_rk2_free_stream_is_preserved_bitwise(o, 3, (1, 1, 1))),
    ("rk2_conservation_bflux", lambda o: rk2.test_rk2_conservation_with_boundary_fluxes(o, "sod")),
    ("rk2_sod_exact", lambda o: rk2.test_rk2_sod_matches_exact_solution_and_rows_are_identical(o)),
    ("rk2_order_advection", lambda o: rk2.test_rk2_second_order_on_advected_density_wave(o)),
    ("rk2_order_acoustic", lambda o: rk2.test_rk2_second_order_on_smooth_acoustic_wave(o)),
    ("amr_free_stream", lambda o: amr.test_free_stream_is_preserved_across_levels(o, 3)),
    ("amr_all_refined", lambda o: amr.test_everything_refined_is_the_uniform_fine_step(o, 3)),
    ("amr_conservation", lambda o: amr.test_leaf_totals_are_conserved_on_a_periodic_box(o, 3)),
    ("amr_conservation_2d", lambda o: amr.test_leaf_totals_are_conserved_on_a_periodic_box(o, 2)),
]


def _build_variant(tmp_path, name, old, new):
    src = open(obuild.SRC).read()
    assert src.count(old) == 1, f"mutation {name}: pattern must occur exactly once"
    path = os.path.join(tmp_path, f"oracle_{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp_path, f"liboracle_{name}.so")
    subprocess.run(["gcc", *obuild.CFLAGS, path, "-o", so, "-lm"], check=True)
    return so


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    variant = oracle.Variant(_build_variant(str(tmp_path), name, old, new))
    variant.set_threads(min(8, os.cpu_count() or 1))
    for pin, fn in PIN_TESTS:
        try:
            with np.errstate(all="ignore"):
                fn(variant)
        except (AssertionError, FloatingPointError, ValueError):
            print(f"{name}: caught by {pin}")
            return                                  # caught
    pytest.fail(f"no pin caught mutation {name}")
