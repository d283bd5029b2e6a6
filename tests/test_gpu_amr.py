"""The two-level AMR step on the GPU (orcha_amr_*) against the oracle's
two-level step: both levels' states (leaves and parents) and the dt sequence
under the parity rule, free stream bitwise, leaf totals conserved on a
periodic box. The exact-FP64 library reproduces the oracle bit for bit
(tests/test_gpu_exact_build.py)."""
import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import rule12_error
from .test_oracle_amr_pins import leaf_totals

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def gpu_amr_run(spec, refined, U0, U1, nsteps):
    """nsteps GPU steps, one call each; returns (U0, U1, dts)."""
    a = B.AmrMesh(spec, refined)
    try:
        a.load(U0, U1)
        dts = []
        for n in range(nsteps):
            a.advance(1, init_dt=(n == 0))
            dts.append(None)
        err = a.poll()
        G0, G1 = a.store()
        return G0, G1, err
    finally:
        a.close()


def gpu_amr_dts(spec, refined, U0, U1, nsteps):
    a = B.AmrMesh(spec, refined)
    try:
        a.load(U0, U1)
        a.advance(0, init_dt=True)
        dts = [a.dt_value()]
        for _ in range(nsteps):
            a.advance(1, init_dt=False)
            dts.append(a.dt_value())
        return np.array(dts)
    finally:
        a.close()


def _case(ndim, bs, periodic, seed, frac=0.35):
    if ndim == 3:
        spec = wl.MeshSpec(ndim=3, nb=(3, 3, 3), bs=(bs, bs, bs), periodic=periodic)
    else:
        spec = wl.MeshSpec(ndim=2, nb=(4, 3, 1), bs=(bs, bs, 1), periodic=periodic[:2] + (0,))
    fs = wl.fine_spec(spec)
    refined = wl.refined_blocks(spec, "sphere", frac)
    U0, U1 = wl.amr_split(spec, refined, wl.random_blocky_state(fs, seed))
    return spec, refined, U0, U1


@pytest.mark.parametrize("ndim,bs,periodic", [(3, 8, (0, 0, 0)), (3, 8, (1, 1, 1)), (3, 16, (1, 0, 1)),
                                              (2, 16, (0, 1, 0)), (2, 8, (1, 1, 0))])
def test_amr_steps_match_the_oracle(oracle_mod, ndim, bs, periodic):
    spec, refined, U0, U1 = _case(ndim, bs, periodic, 13)
    assert 0 < len(refined) < spec.nblocks
    m = oracle_mod.Mesh(**spec.oracle_kwargs())
    O0, O1, odts = oracle_mod.amr_run(m, refined, U0, U1, 4)
    G0, G1, err = gpu_amr_run(spec, refined, U0, U1, 4)
    assert err == 0
    e0, e1 = rule12_error(G0, O0, spec.nvar), rule12_error(G1, O1, spec.nvar)
    print(f"AMR {ndim}D bs {bs} periodic {periodic}: {len(refined)} refined, rule-12 error coarse {e0:.3e} "
          f"fine {e1:.3e}, bitwise {np.mean(G0 == O0):.4f} / {np.mean(G1 == O1):.4f}")
    assert e0 <= TOL and e1 <= TOL
    gdts = gpu_amr_dts(spec, refined, U0, U1, 3)
    np.testing.assert_allclose(gdts[:4], odts[:4], rtol=TOL, atol=0)


def test_amr_free_stream_is_kept_bitwise():
    rng = np.random.default_rng(2)
    spec = wl.MeshSpec(ndim=3, nb=(3, 3, 3), bs=(8, 8, 8), periodic=(0, 1, 1))
    fs = wl.fine_spec(spec)
    refined = wl.refined_blocks(spec, "sphere", 0.3)
    U0, U1 = wl.amr_split(spec, refined,
                          wl.uniform_state(fs, rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2)))
    G0, G1, err = gpu_amr_run(spec, refined, U0, U1, 3)
    assert err == 0 and np.array_equal(G0, U0) and np.array_equal(G1, U1)


def test_amr_leaf_totals_conserved_periodic():
    spec, refined, U0, U1 = _case(3, 8, (1, 1, 1), 21)
    G0, G1, err = gpu_amr_run(spec, refined, U0, U1, 6)
    assert err == 0
    t0, t1 = leaf_totals(spec, refined, U0, U1), leaf_totals(spec, refined, G0, G1)
    scale = leaf_totals(spec, refined, np.abs(U0), np.abs(U1))
    scale[1:-1] = np.maximum(scale[1:-1], scale[0])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)


def test_amr_validation():
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(8, 8, 8))
    with pytest.raises(B.OrchaError) as ei:
        B.AmrMesh(spec, [0, 0])
    assert ei.value.status == B.ORCHA_ERR_INVALID
    with pytest.raises(B.OrchaError):
        B.AmrMesh(spec, [8])
