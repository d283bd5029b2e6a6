"""Pins of the oracle's two-level AMR step (block refinement with flux
correction at coarse-fine faces; oracle.c, "two-level AMR") against things
fixed outside it: the uniform-mesh step it must reduce to when nothing or
everything is refined, exact preservation of a free stream across levels,
exact conservation of sum U dV over the leaf cells (the point of the flux
correction), mirror symmetry, and the exact Sod solution across a
refinement boundary. No GPU is used here."""
import numpy as np
import pytest

from paper_2507_09337_b300 import workloads as wl

from .test_oracle_pins import omesh


def _fine_state(spec, make, *a):
    fs = wl.fine_spec(spec)
    return make(fs, *a)


def leaf_totals(spec, refined, U0, U1):
    """sum over leaf cells of U dV, per variable."""
    dv = np.prod([spec.dx(d) for d in range(spec.ndim)])
    leaf = np.ones(spec.nblocks, dtype=bool)
    leaf[np.asarray(refined, dtype=int)] = False
    t0 = U0[leaf].sum(axis=(0, 2, 3, 4)) * dv
    t1 = U1.sum(axis=(0, 2, 3, 4)) * dv / (1 << spec.ndim)
    return t0 + t1


@pytest.mark.parametrize("ndim", [2, 3])
def test_no_refinement_is_the_uniform_step(oracle_mod, ndim):
    spec = (wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8), periodic=(1, 0, 1)) if ndim == 3
            else wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(8, 8, 1), periodic=(0, 1, 0)))
    U0 = wl.random_blocky_state(spec, 3)
    m = omesh(oracle_mod, spec)
    dt = oracle_mod.dt(m, U0)
    U, _, _ = oracle_mod.step(m, U0, dt)
    A0, A1, _ = oracle_mod.amr_step(m, [], U0, np.zeros((0,) + U0.shape[1:]), dt)
    assert np.array_equal(A0, U) and A1.shape[0] == 0
    assert oracle_mod.amr_dt(m, [], U0, np.zeros((0,) + U0.shape[1:])) == dt


@pytest.mark.parametrize("ndim", [2, 3])
def test_everything_refined_is_the_uniform_fine_step(oracle_mod, ndim):
    """With every coarse block refined the fine level is a whole uniform mesh
    of half the cell width: its step (guards, cell widths, octant order) is
    the uniform step on that mesh, bit for bit, and the parents are its
    restriction."""
    spec = (wl.MeshSpec(ndim=3, nb=(2, 1, 2), bs=(8, 8, 8), periodic=(1, 1, 0)) if ndim == 3
            else wl.MeshSpec(ndim=2, nb=(2, 3, 1), bs=(8, 8, 1), periodic=(0, 1, 0)))
    fs = wl.fine_spec(spec)
    Uf = wl.random_blocky_state(fs, 7)
    refined = np.arange(spec.nblocks, dtype=np.int32)
    U0, U1 = wl.amr_split(spec, refined, Uf)
    mf = omesh(oracle_mod, fs)
    m = omesh(oracle_mod, spec)
    dt = oracle_mod.dt(mf, Uf)
    assert oracle_mod.amr_dt(m, refined, U0, U1) == dt
    Ff, _, _ = oracle_mod.step(mf, Uf, dt)
    A0, A1, _ = oracle_mod.amr_step(m, refined, U0, U1, dt)
    _, B1 = wl.amr_split(spec, refined, Ff)
    assert np.array_equal(A1, B1)
    C0, _ = wl.amr_split(spec, refined, Ff)
    scale = np.abs(C0).max(axis=(0, 2, 3, 4))[None, :, None, None, None]
    assert np.all(np.abs(A0 - C0) <= 1e-14 * scale)


@pytest.mark.parametrize("ndim", [2, 3])
def test_free_stream_is_preserved_across_levels(oracle_mod, ndim):
    rng = np.random.default_rng(11)
    spec = (wl.MeshSpec(ndim=3, nb=(3, 3, 3), bs=(8, 8, 8), periodic=(0, 1, 1)) if ndim == 3
            else wl.MeshSpec(ndim=2, nb=(4, 3, 1), bs=(8, 8, 1), periodic=(1, 0, 0)))
    fs = wl.fine_spec(spec)
    Uf = wl.uniform_state(fs, rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
    refined = wl.refined_blocks(spec, "sphere", 0.3)
    assert 0 < len(refined) < spec.nblocks
    U0, U1 = wl.amr_split(spec, refined, Uf)
    m = omesh(oracle_mod, spec)
    A0, A1, _ = oracle_mod.amr_run(m, refined, U0, U1, 3)
    assert np.array_equal(A0, U0) and np.array_equal(A1, U1)


@pytest.mark.parametrize("ndim", [2, 3])
def test_leaf_totals_are_conserved_on_a_periodic_box(oracle_mod, ndim):
    """The flux correction makes each coarse-fine face carry one flux (the
    fine fluxes' average), so sum U dV over the leaves is conserved to
    rounding on a periodic box."""
    spec = (wl.MeshSpec(ndim=3, nb=(3, 3, 3), bs=(8, 8, 8), periodic=(1, 1, 1)) if ndim == 3
            else wl.MeshSpec(ndim=2, nb=(4, 4, 1), bs=(8, 8, 1), periodic=(1, 1, 0)))
    Uf = _fine_state(spec, wl.random_blocky_state, 5)
    refined = wl.refined_blocks(spec, "sphere", 0.3)
    U0, U1 = wl.amr_split(spec, refined, Uf)
    m = omesh(oracle_mod, spec)
    t0 = leaf_totals(spec, refined, U0, U1)
    A0, A1, _ = oracle_mod.amr_run(m, refined, U0, U1, 4)
    t1 = leaf_totals(spec, refined, A0, A1)
    scale = leaf_totals(spec, refined, np.abs(U0), np.abs(U1))
    scale[1:-1] = np.maximum(scale[1:-1], scale[0])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def test_mirror_symmetry(oracle_mod):
    """A refinement pattern and state mirrored in x give the mirrored result
    (to rounding: the flux correction sums the fine fluxes in index order)."""
    spec = wl.MeshSpec(ndim=3, nb=(4, 2, 2), bs=(8, 8, 8), periodic=(0, 1, 0))
    fs = wl.fine_spec(spec)
    Uf = wl.random_blocky_state(fs, 9)
    refined = wl.refined_blocks(spec, "sphere", 0.4)
    U0, U1 = wl.amr_split(spec, refined, Uf)
    V0, V1 = wl.amr_split(spec, refined, wl.mirror(fs, Uf, 0))
    m = omesh(oracle_mod, spec)
    A0, A1, _ = oracle_mod.amr_run(m, refined, U0, U1, 3)
    B0, B1, _ = oracle_mod.amr_run(m, refined, V0, V1, 3)
    scale = np.abs(A0).max(axis=(0, 2, 3, 4))[None, :, None, None, None]
    assert np.all(np.abs(wl.mirror(spec, A0, 0) - B0) <= 1e-13 * scale)


def test_sod_across_a_refinement_boundary(oracle_mod):
    """2D Sod with the right half of the tube refined: every row stays the
    same bit for bit, and the density profile (fine level injected to the
    fine grid) is within the first-order bound of the exact solution."""
    from oracle import exact_riemann
    spec = wl.sod_spec(64, 8, ny_cells=16)
    fs = wl.fine_spec(spec)
    refined = wl.refined_blocks(spec, "half")
    U0, U1 = wl.amr_split(spec, refined, wl.sod_state(fs))
    m = omesh(oracle_mod, spec)
    t, n = 0.0, 0
    while t < 0.15:
        dt = min(oracle_mod.amr_dt(m, refined, U0, U1), 0.15 - t)
        U0, U1, _ = oracle_mod.amr_step(m, refined, U0, U1, dt)
        t += dt
        n += 1
    G0 = wl.from_blocks(spec, U0)[0, 0]
    assert np.all(G0 == G0[:1])
    rho = np.repeat(G0[0], 2)                      # coarse cells onto the fine grid
    B1 = np.zeros((fs.nblocks,) + U1.shape[1:])
    nch = 4
    for r, b in enumerate(refined):
        bc = (b % spec.nb[0], b // spec.nb[0])
        for o in range(nch):
            B1[(2 * bc[0] + (o & 1)) + fs.nb[0] * (2 * bc[1] + (o >> 1))] = U1[r * nch + o]
    Gf = wl.from_blocks(fs, B1)[0, 0]
    assert np.all(Gf == Gf[:1])
    xf = (np.arange(128) + 0.5) / 128
    right = xf > 0.5
    rho[right] = Gf[0][right]
    ex = exact_riemann.sample((xf - 0.5) / t, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))[0]
    l1 = np.abs(rho - ex).mean()
    print(f"AMR Sod t = {t:.3f} ({n} steps): L1(rho) vs exact {l1:.4f}")
    assert l1 < 0.02
