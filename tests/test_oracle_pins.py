"""Pins of the CPU oracle against things fixed outside it: published values,
exact solutions, closed forms, conservation, symmetry and convergence.

Each test names the part of the scheme a plausible mistake would break.
No GPU is used here.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2507_09337_b300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    vals = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def omesh(oracle_mod, spec):
    return oracle_mod.Mesh(**spec.oracle_kwargs())


def run_to(oracle_mod, spec, U0, tend):
    """Drive the oracle to time tend (last step shortened to land on tend)."""
    m = omesh(oracle_mod, spec)
    U, t, n = U0.copy(), 0.0, 0
    while t < tend:
        dt = min(oracle_mod.dt(m, U), tend - t)
        U, _, _ = oracle_mod.step(m, U, dt)
        t += dt
        n += 1
    return U, n


# ------------------------------------------------------------------ exact solutions

def test_exact_riemann_matches_published_sod_star_state():
    from oracle import exact_riemann
    g = golden("sod_star_state.txt")
    ps, us = exact_riemann.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert ps == pytest.approx(g["p_star"], abs=1e-5)
    assert us == pytest.approx(g["u_star"], abs=1e-5)
    # densities either side of the contact
    w = exact_riemann.sample([us - 1e-6, us + 1e-6], (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert w[0, 0] == pytest.approx(g["rho_star_left"], abs=1e-5)
    assert w[0, 1] == pytest.approx(g["rho_star_right"], abs=1e-5)


def test_exact_riemann_integral_conservation():
    """On [-L, L], int U(x, t) dx = int U(x, 0) dx + t (F(U_L) - F(U_R)) while the
    waves stay inside: checks the sampled fan, shock and contact states."""
    from oracle import exact_riemann
    g = 1.4
    for left, right in [((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
                        ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),
                        ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01)),
                        ((5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.095))]:
        t, L, n = 0.01, 1.0, 400001
        x = np.linspace(-L, L, n)
        W = exact_riemann.sample(x / t, left, right, g)
        U = np.array([W[0], W[0] * W[1], W[2] / (g - 1) + 0.5 * W[0] * W[1] ** 2])

        def cons(w):
            r, u, p = w
            return np.array([r, r * u, p / (g - 1) + 0.5 * r * u * u])

        def flux(w):
            r, u, p = w
            E = p / (g - 1) + 0.5 * r * u * u
            return np.array([r * u, r * u * u + p, u * (E + p)])

        lhs = np.trapezoid(U, x, axis=1)
        rhs = L * (cons(left) + cons(right)) + t * (flux(left) - flux(right))
        np.testing.assert_allclose(lhs, rhs, rtol=2e-4, atol=2e-4 * np.abs(rhs).max())


def test_sedov_xi0_matches_published_constants():
    from oracle import sedov
    gold = golden("sedov_xi0.txt")
    assert sedov.xi0(1.4) == pytest.approx(gold["xi0_gamma_1.4"], abs=1.5e-3)
    assert sedov.xi0(5.0 / 3.0) == pytest.approx(gold["xi0_gamma_5/3"], abs=1e-3)


# ------------------------------------------------------------------ point functions

def test_minmod_brute_force(oracle_mod):
    cases = [((1.0, 2.0), 1.0), ((2.0, 1.0), 1.0), ((-1.0, -2.0), -1.0), ((-2.0, -1.0), -1.0),
             ((1.0, -1.0), 0.0), ((-1.0, 1.0), 0.0), ((0.0, 1.0), 0.0), ((1.0, 0.0), 0.0),
             ((-0.0, -1.0), 0.0), ((3.0, 3.0), 3.0), ((1e-300, 1e300), 1e-300)]
    for (a, b), want in cases:
        assert oracle_mod.minmod(a, b) == want


def _phys_flux_x(g, rho, u, v, p):
    E = p / (g - 1) + 0.5 * rho * (u * u + v * v)
    return np.array([rho * u, rho * u * u + p, rho * u * v, u * (E + p)])


def test_hll_identical_states_is_physical_flux(oracle_mod):
    # rho=1, u=2, v=0.5, p=1: E = 1/0.4 + 0.5*(4.25) = 4.625
    F = oracle_mod.hll(2, 0, 1.4, [1.0, 2.0, 0.5, 1.0], [1.0, 2.0, 0.5, 1.0])
    np.testing.assert_allclose(F, [2.0, 5.0, 1.0, 11.25], rtol=1e-15)
    # the same state seen along y: the roles of u and v swap
    F = oracle_mod.hll(2, 1, 1.4, [1.0, 0.5, 2.0, 1.0], [1.0, 0.5, 2.0, 1.0])
    np.testing.assert_allclose(F, [2.0, 1.0, 5.0, 11.25], rtol=1e-15)


def test_hll_supersonic_upwinding(oracle_mod):
    g = 1.4
    WL, WR = [1.0, 5.0, 0.0, 1.0], [0.5, 4.0, 0.3, 0.8]      # both faster than sound, rightward
    assert np.array_equal(oracle_mod.hll(2, 0, g, WL, WR), _phys_flux_x(g, *WL))
    WL, WR = [1.0, -5.0, 0.0, 1.0], [0.5, -4.0, 0.3, 0.8]    # leftward: right state upwind
    assert np.array_equal(oracle_mod.hll(2, 0, g, WL, WR), _phys_flux_x(g, *WR))


def test_hll_symmetric_collision_has_zero_mass_flux(oracle_mod):
    F = oracle_mod.hll(3, 2, 1.4, [1.3, 0.1, 0.2, 0.7, 2.0], [1.3, 0.1, 0.2, -0.7, 2.0])
    assert F[0] == 0.0 and F[4] == 0.0
    assert F[3] > 2.0           # pressure plus the ram pressure term


def test_hll_subsonic_against_hand_values(oracle_mod):
    """HLL between (1, 0, 0, 1) and (0.125, 0, 0, 0.1): the initial Sod face."""
    g = 1.4
    cL, cR = math.sqrt(1.4), math.sqrt(1.4 * 0.1 / 0.125)
    assert cL > cR                      # so S_L = -c_L and S_R = +c_L
    SL, SR = -cL, cL
    UL = np.array([1.0, 0.0, 0.0, 2.5])
    UR = np.array([0.125, 0.0, 0.0, 0.25])
    FL = np.array([0.0, 1.0, 0.0, 0.0])
    FR = np.array([0.0, 0.1, 0.0, 0.0])
    want = (SR * FL - SL * FR + SL * SR * (UR - UL)) / (SR - SL)
    got = oracle_mod.hll(2, 0, g, [1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1])
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-16)


def test_dt_closed_form(oracle_mod):
    """rho = 1, p = 1/gamma gives c = 1; with u = (1, 0, 0) the summed signal
    speed is (2 + 1 + 1) N in 3D and (2 + 1) N in 2D."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8))
    U = wl.uniform_state(spec, 1.0, (1.0, 0.0, 0.0), 1.0 / 1.4)
    assert oracle_mod.dt(omesh(oracle_mod, spec), U) == pytest.approx(0.8 / (4 * 16), rel=1e-15)
    spec = wl.MeshSpec(ndim=2, nb=(4, 2, 1), bs=(8, 8, 1))
    U = wl.uniform_state(spec, 1.0, (0.0, -1.0), 1.0 / 1.4)
    assert oracle_mod.dt(omesh(oracle_mod, spec), U) == pytest.approx(0.8 / (32 + 2 * 16), rel=1e-15)


def test_sedov_deposit_count_brute_force():
    """Cells whose centres lie within 3.5 cells of a cell vertex: count odd
    integer triples (half-cell units) with a^2 + b^2 + c^2 <= 49."""
    n = sum(1 for a, b, c in itertools.product(range(-7, 8, 2), repeat=3) if a * a + b * b + c * c <= 49)
    assert n == 160
    for N, b in ((32, 8), (128, 16)):
        assert int(wl.sedov_deposit_mask(wl.sedov_spec(N, b)).sum()) == n


# ------------------------------------------------------------------ Sod shock tube

def test_sod_2d_matches_exact_solution_and_rows_are_identical(oracle_mod):
    """The 64 x 64 Sod tube, 20 steps: every row is bitwise identical (no
    transverse flux is created) and the density profile is within the L1
    bound of the exact solution."""
    from oracle import exact_riemann
    spec = wl.sod_spec(64, 8)
    U, dts, _ = oracle_mod.run(omesh(oracle_mod, spec), wl.sod_state(spec), 20)
    G = wl.from_blocks(spec, U)[:, 0]
    for v in range(4):
        assert all(np.array_equal(G[v, 0], G[v, j]) for j in range(64))
    assert np.all(G[2] == 0.0)                          # no y-momentum appears
    t = float(dts.sum())
    x = (np.arange(64) + 0.5) / 64
    ex = exact_riemann.sample((x - 0.5) / t, (1, 0, 1), (0.125, 0, 0.1))
    assert np.mean(np.abs(G[0, 0] - ex[0])) < 0.012
    u = G[1, 0] / G[0, 0]
    assert np.mean(np.abs(u - ex[1])) < 0.03


def test_sod_converges_to_exact_solution(oracle_mod):
    from oracle import exact_riemann
    errs = []
    for N in (64, 128, 256):
        spec = wl.sod_spec(N, 8, ny_cells=8)
        U, _ = run_to(oracle_mod, spec, wl.sod_state(spec), 0.2)
        x = (np.arange(N) + 0.5) / N
        ex = exact_riemann.sample((x - 0.5) / 0.2, (1, 0, 1), (0.125, 0, 0.1))
        errs.append(np.mean(np.abs(wl.from_blocks(spec, U)[0, 0, 0] - ex[0])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[0] < 0.012
    assert np.all(orders > 0.7), (errs, orders)


def test_y_extent_does_not_change_rows(oracle_mod):
    """1D reduction: a 64 x 8 tube gives bitwise the rows of the 64 x 64 one."""
    a = wl.sod_spec(64, 8)
    b = wl.sod_spec(64, 8, ny_cells=8)
    Ua, _, _ = oracle_mod.run(omesh(oracle_mod, a), wl.sod_state(a), 12)
    Ub, _, _ = oracle_mod.run(omesh(oracle_mod, b), wl.sod_state(b), 12)
    Ga, Gb = wl.from_blocks(a, Ua)[:, 0], wl.from_blocks(b, Ub)[:, 0]
    assert np.array_equal(Ga[:, :8], Gb)


def test_sod_outflow_after_shock_exits(oracle_mod):
    """Outflow faces transmit waves: after the shock has left the right end
    (t = 0.35), the profile stays within the L1 bound of the exact solution."""
    from oracle import exact_riemann
    spec = wl.sod_spec(64, 8, ny_cells=8)
    U, _ = run_to(oracle_mod, spec, wl.sod_state(spec), 0.35)
    x = (np.arange(64) + 0.5) / 64
    ex = exact_riemann.sample((x - 0.5) / 0.35, (1, 0, 1), (0.125, 0, 0.1))
    G = wl.from_blocks(spec, U)[:, 0, 0]
    assert np.abs(G[0] - ex[0]).mean() < 0.012
    assert np.abs(G[1] / G[0] - ex[1]).mean() < 0.012


def test_outflow_boundary_flux_is_physical_flux_at_rest(oracle_mod):
    """Zero-gradient outflow, gas at rest, varying only along x: the boundary
    cell's slope and the guard's slope vanish, so each boundary face carries
    the boundary cell's own physical flux: no mass or energy, momentum = p."""
    rng = np.random.default_rng(3)
    spec = wl.sod_spec(32, 8, ny_cells=8)
    rho = np.repeat(rng.uniform(0.5, 2.0, 32)[None, :], 8, axis=0)
    p = np.repeat(rng.uniform(0.5, 2.0, 32)[None, :], 8, axis=0)
    U0 = wl.to_blocks(spec, wl.cons_from_prim_global(spec, rho, [0 * rho, 0 * rho], p)[:, None])
    m = omesh(oracle_mod, spec)
    dt = oracle_mod.dt(m, U0)
    _, bf, _ = oracle_mod.step(m, U0, dt)
    cd = dt * 32
    assert bf[0] == 0.0 and bf[3] == 0.0
    assert bf[1] == pytest.approx(cd * 8 * (p[0, -1] - p[0, 0]), rel=1e-13)
    assert abs(bf[2]) <= 1e-13 * cd * p.sum()


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("ndim,periodic", [(2, (0, 0, 0)), (3, (0, 0, 0)), (3, (1, 1, 1))])
def test_free_stream_is_preserved_bitwise(oracle_mod, ndim, periodic):
    rng = np.random.default_rng(7)
    if ndim == 2:
        spec = wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(8, 8, 1), periodic=periodic)
    else:
        spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8), periodic=periodic)
    U0 = wl.uniform_state(spec, rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
    U, _, _ = oracle_mod.run(omesh(oracle_mod, spec), U0, 5)
    assert np.array_equal(U, U0)


def test_results_do_not_depend_on_block_size(oracle_mod):
    """Guards of interior block faces are exact copies, so 8^3 blocks, 16^3
    blocks and a single 32 x 16 x 16 block give bitwise the same result."""
    specs = [wl.MeshSpec(ndim=3, nb=(4, 2, 2), bs=(8, 8, 8)),
             wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(16, 16, 16)),
             wl.MeshSpec(ndim=3, nb=(1, 1, 1), bs=(32, 16, 16))]
    base = specs[0]
    Ug0 = wl.from_blocks(base, wl.random_blocky_state(base, 3))
    outs = []
    for s in specs:
        U, _, _ = oracle_mod.run(omesh(oracle_mod, s), wl.to_blocks(s, Ug0), 3)
        outs.append(wl.from_blocks(s, U))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def _rule12_scale(G0):
    """Per-variable scale of the parity rule: |value| for rho and E; the largest
    |momentum| of the field for the momenta."""
    nv = G0.shape[0]
    scale = np.abs(G0).copy()
    for v in range(1, nv - 1):
        scale[v] = np.maximum(scale[v], np.abs(G0[1:nv - 1]).max())
    return scale


@pytest.mark.parametrize("seed", [1, 2])
def test_conservation_periodic(oracle_mod, seed):
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8), periodic=(1, 1, 1))
    U0 = wl.random_blocky_state(spec, seed) if seed == 1 else wl.random_smooth_state(spec, seed)
    U, _, bf = oracle_mod.run(omesh(oracle_mod, spec), U0, 6)
    assert np.all(bf == 0.0)
    s0, s1 = U0.sum(axis=(0, 2, 3, 4)), U.sum(axis=(0, 2, 3, 4))
    scale = np.abs(U0).sum(axis=(0, 2, 3, 4))
    scale[1:4] = np.maximum(scale[1:4], U0[:, 0].sum())       # momenta: sum rho * O(1) speed
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale


@pytest.mark.parametrize("case", ["sod", "blocky3d"])
def test_conservation_with_boundary_fluxes(oracle_mod, case):
    if case == "sod":
        spec = wl.sod_spec(64, 8, ny_cells=16)
        U0 = wl.sod_state(spec, split=0.3)          # waves reach the outflow faces
        n = 40
    else:
        spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8))
        U0 = wl.random_blocky_state(spec, 5)
        n = 6
    U, _, bf = oracle_mod.run(omesh(oracle_mod, spec), U0, n)
    s0, s1 = U0.sum(axis=(0, 2, 3, 4)), U.sum(axis=(0, 2, 3, 4))
    scale = np.abs(U0).sum(axis=(0, 2, 3, 4)) + np.abs(bf)
    scale[1:spec.nvar - 1] = np.maximum(scale[1:spec.nvar - 1], U0[:, 0].sum())
    assert np.any(np.abs(bf) > 1e-6 * scale)              # the boundary flux is not trivial
    assert np.all(np.abs(s1 - (s0 - bf)) <= 1e-13 * scale)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry_bitwise(oracle_mod, axis):
    """run(mirror(U)) == mirror(run(U)) bitwise, on random jumps in every direction."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8))
    U0 = wl.random_blocky_state(spec, 11)
    m = omesh(oracle_mod, spec)
    Ua, _, _ = oracle_mod.run(m, U0, 4)
    Ub, _, _ = oracle_mod.run(m, wl.mirror(spec, U0, axis), 4)
    assert np.array_equal(wl.mirror(spec, Ua, axis), Ub)


def test_sedov_is_mirror_symmetric_bitwise(oracle_mod):
    spec = wl.sedov_spec(32, 8)
    U, _, _ = oracle_mod.run(omesh(oracle_mod, spec), wl.sedov_state(spec), 8)
    for axis in range(3):
        assert np.array_equal(wl.mirror(spec, U, axis), U)


@pytest.mark.parametrize("a,b", [(0, 1), (1, 2), (0, 2)])
def test_axis_permutation_symmetry(oracle_mod, a, b):
    """Exchanging two axes commutes with the scheme up to the order of the
    x, y, z sums (rule: |diff| <= 1e-13 of the per-variable scale)."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8))
    U0 = wl.random_blocky_state(spec, 13)
    m = omesh(oracle_mod, spec)
    Ua, _, _ = oracle_mod.run(m, U0, 4)
    Ub, _, _ = oracle_mod.run(m, wl.swap_axes(spec, U0, a, b), 4)
    Ga = wl.from_blocks(spec, wl.swap_axes(spec, Ua, a, b))
    Gb = wl.from_blocks(spec, Ub)
    scale = _rule12_scale(Ga)
    assert np.all(np.abs(Ga - Gb) <= 1e-13 * scale)


def test_sedov_blast_radius(oracle_mod):
    """64^3 Sedov (E = 1 within 3.5 cells of the centre, rho0 = 1, p0 = 1e-5)
    run to the time at which the similarity radius is 0.3: the peak of the
    shell-averaged density lies within 1.5 cells of it; total energy and mass
    are unchanged (the shock has not reached the boundary)."""
    from oracle import sedov
    spec = wl.sedov_spec(64, 16)
    U0 = wl.sedov_state(spec)
    tend = (0.3 / sedov.xi0(1.4)) ** 2.5
    U, n = run_to(oracle_mod, spec, U0, tend)
    G = wl.from_blocks(spec, U)
    x, y, z = spec.centers()
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2).ravel()
    dx = 1.0 / 64
    shell = np.floor(r / dx).astype(int)
    rho = G[0].ravel()
    prof = np.bincount(shell, weights=rho) / np.maximum(np.bincount(shell), 1)
    r_peak = (np.argmax(prof) + 0.5) * dx
    assert abs(r_peak - sedov.shock_radius(tend)) <= 1.5 * dx
    G0 = wl.from_blocks(spec, U0)
    for v in (0, 4):
        assert abs(G[v].sum() - G0[v].sum()) <= 1e-13 * G0[v].sum()


# ------------------------------------------------------------------ order of accuracy

def _acoustic(spec, k, eps=1e-2):
    x, y, _ = spec.centers()
    k = np.asarray(k, float)
    s = np.sin(2 * np.pi * (k[0] * x + k[1] * y))[0]
    kn = k / np.linalg.norm(k)
    vel = [eps * s * kn[d] for d in range(2)]
    U = wl.cons_from_prim_global(spec, 1 + eps * s, vel, 1 / 1.4 + eps * s)
    return wl.to_blocks(spec, U[:, None])


def _coarsen2(G):
    nv, ny, nx = G.shape
    return G.reshape(nv, ny // 2, 2, nx // 2, 2).mean(axis=(2, 4))


@pytest.mark.parametrize("k", [(1, 0), (1, 1)])
def test_second_order_on_smooth_acoustic_wave(oracle_mod, k):
    """Self-convergence of a small-amplitude sound wave (density, velocity and
    pressure all vary, along x and along the diagonal): the L1 order over
    N = 32, 64, 128 is well above 1 (every predictor term matters)."""
    sols = []
    for N in (32, 64, 128):
        spec = wl.MeshSpec(ndim=2, nb=(N // 8, N // 8, 1), bs=(8, 8, 1), periodic=(1, 1, 0))
        U, _ = run_to(oracle_mod, spec, _acoustic(spec, k), 0.25)
        sols.append(wl.from_blocks(spec, U)[:, 0])
    e1 = np.abs(_coarsen2(sols[1]) - sols[0]).mean()
    e2 = np.abs(_coarsen2(sols[2]) - sols[1]).mean()
    assert math.log2(e1 / e2) > 1.6, (e1, e2)


@pytest.mark.parametrize("ndim", [2, 3])
def test_homologous_expansion_matches_exact_density(oracle_mod, ndim):
    """u = a (x - x0) (along x in 2D, radially in 3D) with uniform rho and p is
    an exact solution with rho(t) = rho0 / (1 + a t)^ndim_expanding, uniform in
    space; the density predictor's rho du term is the only one that acts. In the
    region the outflow boundaries have not yet reached, the density error is
    small and falls at second order."""
    a, tend = 2.0, 0.05
    errs = []
    for N in ((64, 128) if ndim == 2 else (32, 64)):
        if ndim == 2:
            spec = wl.MeshSpec(ndim=2, nb=(N // 8, 1, 1), bs=(8, 8, 1), hi=(1, 8 / N, 1))
        else:
            spec = wl.MeshSpec(ndim=3, nb=(N // 8,) * 3, bs=(8,) * 3)
        x, y, z = spec.centers()
        if ndim == 2:
            x = x[0]
            vel = [a * (x - 0.5), 0 * x]
            rho = np.ones_like(x)
            U0 = wl.to_blocks(spec, wl.cons_from_prim_global(spec, rho, vel, np.ones_like(x))[:, None])
            k = 1
        else:
            vel = [a * (x - 0.5), a * (y - 0.5), a * (z - 0.5)]
            U0 = wl.to_blocks(spec, wl.cons_from_prim_global(spec, np.ones_like(x), vel, np.ones_like(x)))
            k = 3
        U, _ = run_to(oracle_mod, spec, U0, tend)
        G = wl.from_blocks(spec, U)[0]
        reach = (1.2 + a * 0.5) * tend + 4.0 / N
        c = (np.arange(N) + 0.5) / N
        inner = np.abs(c - 0.5) < 0.5 - reach
        sub = G[0][:, inner] if ndim == 2 else G[np.ix_(inner, inner, inner)]
        errs.append(np.abs(sub - 1.0 / (1.0 + a * tend) ** k).max())
    assert errs[0] < (5e-6 if ndim == 2 else 2e-5) and math.log2(errs[0] / errs[1]) > 1.8, errs


def test_second_order_on_advected_density_wave(oracle_mod):
    """Exact solution rho(x - u t): L1 order > 1.8 over N = 32, 64, 128."""
    errs = []
    for N in (32, 64, 128):
        spec = wl.MeshSpec(ndim=2, nb=(N // 8, 1, 1), bs=(8, 8, 1), periodic=(1, 1, 0))
        U, _ = run_to(oracle_mod, spec, wl.advected_wave_state(spec), 0.25)
        ex = wl.advected_wave_state(spec, t=0.25)
        errs.append(np.abs(U[:, 0] - ex[:, 0]).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), orders


def test_first_order_fallback_is_conservative_and_symmetric(oracle_mod):
    """Random jumps smeared by two steps, then one step at 40x the CFL time
    step: the Hancock predictor drives many face states negative and those
    cells fall back to first order. The fallback path must keep exact
    conservation (periodic box) and bitwise mirror symmetry."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8), periodic=(1, 1, 1))
    m = omesh(oracle_mod, spec)
    U0, _, _ = oracle_mod.run(m, wl.random_blocky_state(spec, 21), 2)
    dt = 40.0 * oracle_mod.dt(m, U0)
    U, bf, nfirst = oracle_mod.step(m, U0, dt)
    assert nfirst > 50
    s0, s1 = U0.sum(axis=(0, 2, 3, 4)), U.sum(axis=(0, 2, 3, 4))
    scale = np.abs(U0).sum(axis=(0, 2, 3, 4))
    scale[1:4] = np.maximum(scale[1:4], U0[:, 0].sum())
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale)
    for axis in range(3):
        Um, _, nfm = oracle_mod.step(m, wl.mirror(spec, U0, axis), dt)
        assert nfm == nfirst
        assert np.array_equal(wl.mirror(spec, U, axis), Um)


def test_serving_sphere_count_matches_full_mask():
    """The windowed deposit count of the serving recipes equals the count of
    the full-mesh mask (the initial states use it for the energy per cell)."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        req = wl.serving_request(rng, max_blocks=12, sizes=(8,))
        if req["kind"] != 1:
            continue
        assert wl.sphere_count(req["spec"], req["region"]) == int(
            wl.region_mask(req["spec"], 1, req["region"]).sum())


# ------------------------------------------------------------------ first-order fallback, by hand

def _euler_x_flux(gamma, rho, u, p):
    """Physical x flux (rho u, rho u^2 + p, 0, (E + p) u) of a 2D state moving
    along x (textbook Euler flux; v = 0)."""
    E = p / (gamma - 1.0) + 0.5 * rho * u * u
    return np.stack([rho * u, rho * u * u + p, np.zeros_like(rho), (E + p) * u])


@pytest.mark.parametrize("var", ["p", "rho"])
def test_first_order_fallback_hand_case(oracle_mod, var):
    """Fallback rule (a cell with any face state of rho <= 0 or p <= 0 takes
    W for ALL its face states), checked against a closed form.

    Uniform supersonic flow u = 10 along x, a linear ramp delta (i + 1) in
    pressure (or density) and the other variable 1, uniform in y. At half
    Courant number K = (dt/2)(u/dx) = 4.25 the Hancock state of ramp cell i
    has p_bar = delta (i + 1 - K) and low/high x face states
    delta (i + 1 - K -+ 1/2): cells 1, 2, 3 have a non-positive face, cell 3
    only on its low x and y faces; cell 0 has zero slope (outflow clamp).
    With S_L > 0 on every face, HLL is the left state's physical flux, so
    cells 0..3 update exactly as first-order upwind:
        U_i+ = U_i - (dt/dx) (F(W_i) - F(W_{i-1})),   U_0+ = U_0,
    and exactly 3 cells per row fall back. Testing only one of rho / p, or
    reverting only the offending faces, or reverting to the half-step state,
    breaks this."""
    spec = wl.MeshSpec(ndim=2, nb=(2, 1, 1), bs=(16, 8, 1), periodic=(0, 1, 0))
    delta, u, K = 0.1, 10.0, 4.25
    U0 = wl.ramp_state(spec, var, delta, u)
    dx = spec.dx(0)
    dt = 2.0 * K * dx / u
    U, _, nfirst = oracle_mod.step(omesh(oracle_mod, spec), U0, dt)
    G0, G = wl.from_blocks(spec, U0), wl.from_blocks(spec, U)
    assert np.all(np.isfinite(G))
    assert nfirst == 3 * spec.ncells[1]
    # rows stay identical and v stays exactly 0
    assert np.array_equal(G, np.broadcast_to(G[:, :, :1, :], G.shape)) and np.all(G[2] == 0.0)
    i = np.arange(4)
    ramp = delta * (i + 1.0)
    rho, p = (np.ones(4), ramp) if var == "p" else (ramp, np.ones(4))
    F = _euler_x_flux(spec.gamma, rho, np.full(4, u), p)
    c = dt / dx
    want = G0[:, 0, 0, :4].copy()
    want[:, 1:] -= c * (F[:, 1:] - F[:, :-1])
    got = G[:, 0, 0, :4]
    scale = np.abs(G0[:, 0, 0, :4]) + c * np.abs(F) + 1e-300
    assert np.all(np.abs(got - want) <= 1e-13 * scale.max(axis=1, keepdims=True)), (got, want)
    assert np.array_equal(got[:, 0], G0[:, 0, 0, 0])


def test_plain_muscl_stage_never_falls_back(oracle_mod):
    """Without the half step, minmod face states W -+ dW/2 lie between the
    cell's value and a neighbour's, so they stay positive and the Runge-Kutta
    stages never take the fallback, even at 40x the CFL time step (the
    MUSCL-Hancock step does, on the same input)."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8), periodic=(1, 1, 1))
    m = omesh(oracle_mod, spec)
    U0, _, _ = oracle_mod.run(m, wl.random_blocky_state(spec, 21), 2)
    dt = 40.0 * oracle_mod.dt(m, U0)
    _, _, nf_stage = oracle_mod.stage(m, U0, dt)
    _, _, nf_step = oracle_mod.step(m, U0, dt)
    assert nf_stage == 0 and nf_step > 50
