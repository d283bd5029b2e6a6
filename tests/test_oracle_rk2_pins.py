"""Pins of the oracle's second integrator, Heun's two-stage Runge-Kutta
method with the plain MUSCL operator (the paper's Spark solver is explicit
finite volume with 2nd-order Runge-Kutta, section "Experiments"), against
things fixed outside it: exact solutions, conservation, symmetry, free
stream and second-order convergence. No GPU is used here."""
import math

import numpy as np
import pytest

from paper_2507_09337_b300 import workloads as wl

from .test_oracle_pins import omesh


def run_to_rk2(oracle_mod, spec, U0, tend):
    """Drive the RK2 oracle to time tend (last step shortened to land on it)."""
    m = omesh(oracle_mod, spec)
    U, t = U0.copy(), 0.0
    while t < tend:
        dt = min(oracle_mod.dt(m, U), tend - t)
        U, _, _ = oracle_mod.step_rk2(m, U, dt)
        t += dt
    return U


@pytest.mark.parametrize("ndim,periodic", [(2, (0, 0, 0)), (3, (1, 1, 1))])
def test_rk2_free_stream_is_preserved_bitwise(oracle_mod, ndim, periodic):
    rng = np.random.default_rng(17)
    if ndim == 2:
        spec = wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(8, 8, 1), periodic=periodic)
    else:
        spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8), periodic=periodic)
    U0 = wl.uniform_state(spec, rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
    U, _, _ = oracle_mod.run(omesh(oracle_mod, spec), U0, 4, rk2=True)
    assert np.array_equal(U, U0)


def test_rk2_sod_matches_exact_solution_and_rows_are_identical(oracle_mod):
    from oracle import exact_riemann
    spec = wl.sod_spec(64, 8)
    U, dts, _ = oracle_mod.run(omesh(oracle_mod, spec), wl.sod_state(spec), 20, rk2=True)
    G = wl.from_blocks(spec, U)[:, 0]
    for v in range(4):
        assert all(np.array_equal(G[v, 0], G[v, j]) for j in range(64))
    assert np.all(G[2] == 0.0)
    t = float(dts.sum())
    x = (np.arange(64) + 0.5) / 64
    ex = exact_riemann.sample((x - 0.5) / t, (1, 0, 1), (0.125, 0, 0.1))
    assert np.mean(np.abs(G[0, 0] - ex[0])) < 0.015
    assert np.mean(np.abs(G[1, 0] / G[0, 0] - ex[1])) < 0.04


def test_rk2_sod_converges_to_exact_solution(oracle_mod):
    from oracle import exact_riemann
    errs = []
    for N in (64, 128, 256):
        spec = wl.sod_spec(N, 8, ny_cells=8)
        U = run_to_rk2(oracle_mod, spec, wl.sod_state(spec), 0.2)
        x = (np.arange(N) + 0.5) / N
        ex = exact_riemann.sample((x - 0.5) / 0.2, (1, 0, 1), (0.125, 0, 0.1))
        errs.append(np.mean(np.abs(wl.from_blocks(spec, U)[0, 0, 0] - ex[0])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[0] < 0.015 and np.all(orders > 0.7), (errs, orders)


@pytest.mark.parametrize("seed", [1, 2])
def test_rk2_conservation_periodic(oracle_mod, seed):
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8), periodic=(1, 1, 1))
    U0 = wl.random_blocky_state(spec, seed) if seed == 1 else wl.random_smooth_state(spec, seed)
    U, _, bf = oracle_mod.run(omesh(oracle_mod, spec), U0, 5, rk2=True)
    assert np.all(bf == 0.0)
    s0, s1 = U0.sum(axis=(0, 2, 3, 4)), U.sum(axis=(0, 2, 3, 4))
    scale = np.abs(U0).sum(axis=(0, 2, 3, 4))
    scale[1:4] = np.maximum(scale[1:4], U0[:, 0].sum())
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale


@pytest.mark.parametrize("case", ["sod", "blocky3d"])
def test_rk2_conservation_with_boundary_fluxes(oracle_mod, case):
    """sum U_new = sum U - (B1 + B2)/2: the boundary fluxes of the two stages,
    weighted as the stages are."""
    if case == "sod":
        spec = wl.sod_spec(64, 8, ny_cells=16)
        U0 = wl.sod_state(spec, split=0.3)
        n = 40
    else:
        spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8))
        U0 = wl.random_blocky_state(spec, 5)
        n = 5
    U, _, bf = oracle_mod.run(omesh(oracle_mod, spec), U0, n, rk2=True)
    s0, s1 = U0.sum(axis=(0, 2, 3, 4)), U.sum(axis=(0, 2, 3, 4))
    scale = np.abs(U0).sum(axis=(0, 2, 3, 4)) + np.abs(bf)
    scale[1:spec.nvar - 1] = np.maximum(scale[1:spec.nvar - 1], U0[:, 0].sum())
    assert np.any(np.abs(bf) > 1e-6 * scale)
    assert np.all(np.abs(s1 - (s0 - bf)) <= 1e-13 * scale)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_rk2_mirror_symmetry_bitwise(oracle_mod, axis):
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8))
    U0 = wl.random_blocky_state(spec, 11)
    m = omesh(oracle_mod, spec)
    Ua, _, _ = oracle_mod.run(m, U0, 3, rk2=True)
    Ub, _, _ = oracle_mod.run(m, wl.mirror(spec, U0, axis), 3, rk2=True)
    assert np.array_equal(wl.mirror(spec, Ua, axis), Ub)


def test_rk2_results_do_not_depend_on_block_size(oracle_mod):
    """Each stage refreshes guards from its own state: 8^3 blocks, 16^3 blocks
    and one 32 x 16 x 16 block give bitwise the same result."""
    specs = [wl.MeshSpec(ndim=3, nb=(4, 2, 2), bs=(8, 8, 8)),
             wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(16, 16, 16)),
             wl.MeshSpec(ndim=3, nb=(1, 1, 1), bs=(32, 16, 16))]
    Ug0 = wl.from_blocks(specs[0], wl.random_blocky_state(specs[0], 3))
    outs = []
    for s in specs:
        U, _, _ = oracle_mod.run(omesh(oracle_mod, s), wl.to_blocks(s, Ug0), 3, rk2=True)
        outs.append(wl.from_blocks(s, U))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_rk2_second_order_on_advected_density_wave(oracle_mod):
    """Exact solution rho(x - u t). Both stages are needed: a forward-Euler
    step (or two) is first order in time at a fixed CFL number."""
    errs = []
    for N in (32, 64, 128):
        spec = wl.MeshSpec(ndim=2, nb=(N // 8, 1, 1), bs=(8, 8, 1), periodic=(1, 1, 0))
        U = run_to_rk2(oracle_mod, spec, wl.advected_wave_state(spec), 0.25)
        ex = wl.advected_wave_state(spec, t=0.25)
        errs.append(np.abs(U[:, 0] - ex[:, 0]).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.7), (errs, orders)


def test_rk2_second_order_on_smooth_acoustic_wave(oracle_mod):
    """A diagonal sound wave at CFL 0.4: the summed-direction CFL limit of the
    forward-Euler MUSCL stage that Heun's method is strong-stability
    preserving for is 1/2 (at 0.8 the diagonal wave's order drops to ~1.2 on
    the coarse grids)."""
    from .test_oracle_pins import _acoustic, _coarsen2
    sols = []
    for N in (32, 64, 128):
        spec = wl.MeshSpec(ndim=2, nb=(N // 8, N // 8, 1), bs=(8, 8, 1), periodic=(1, 1, 0), cfl=0.4)
        U = run_to_rk2(oracle_mod, spec, _acoustic(spec, (1, 1)), 0.25)
        sols.append(wl.from_blocks(spec, U)[:, 0])
    e1 = np.abs(_coarsen2(sols[1]) - sols[0]).mean()
    e2 = np.abs(_coarsen2(sols[2]) - sols[1]).mean()
    assert math.log2(e1 / e2) > 1.6, (e1, e2)


def test_rk2_and_hancock_agree_on_a_smooth_wave(oracle_mod):
    """Two second-order schemes for the same equations: on a smooth wave their
    difference is far below either one's distance from the initial state."""
    spec = wl.MeshSpec(ndim=2, nb=(16, 1, 1), bs=(8, 8, 1), periodic=(1, 1, 0))
    U0 = wl.advected_wave_state(spec)
    m = omesh(oracle_mod, spec)
    A = run_to_rk2(oracle_mod, spec, U0, 0.1)
    B, t, n = U0.copy(), 0.0, 0
    while t < 0.1:
        dt = min(oracle_mod.dt(m, B), 0.1 - t)
        B, _, _ = oracle_mod.step(m, B, dt)
        t += dt
    assert np.abs(A - B).max() < 0.05 * np.abs(A - U0).max()
