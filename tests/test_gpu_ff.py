"""The FF task: primitives, reconstruction, predictor and HLL fluxes in
double-word arithmetic (pairs of FP32 numbers, ~48 bits), FP64 update, guard
fill and dt. It is held to the FP64 path's parity rule: per cell and
variable |gpu - oracle| <= 1e-12 * max(|oracle|, s_v) against the FP64
oracle; the tests print the observed difference."""
import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import gpu_batch_steps, gpu_steps, oracle_steps, rule12_error

pytestmark = pytest.mark.gpu
TOL = 1e-12
FF = B.ORCHA_TASK_HYDRO_FF
U2 = 2.0 ** -48      # u^2, u = 2^-24 the binary32 unit roundoff


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def test_dword_building_blocks_error_bounds():
    """Largest errors of the double-word operations on 2^26 operand pairs,
    in units of u^2, against bounds from their error analysis: the split
    (2^-49 relative = u^2 / 2); the sum, relative to |x| + |y|: u^2 from
    adding the low parts, 2 u^2 from adding that to the high parts' rounding
    error, 2 u^2 from Fast2Sum when cancellation leaves |w| > |sh|, plus the
    FP64 reference's own 2^-53; the product 7 u^2
    (the dropped lo*lo term u^2, two roundings of the cross terms 3 u^2, the
    final sum 3 u^2); reciprocal, rsqrt and sound speed a few u^2 (roundings
    of the Newton correction, whose size is about u)."""
    e = B.orcha_selftest_dword(1 << 26, seed=99)
    names = ["split", "sum", "product", "reciprocal", "rsqrt", "sound speed"]
    print("double-word max errors in u^2:", {n: round(v / U2, 3) for n, v in zip(names, e)})
    bounds = [0.5, 5.1, 7.0, 8.0, 10.0, 20.0]
    for n, v, b in zip(names, e, bounds):
        assert np.isfinite(v) and v <= b * U2, (n, v / U2)


def test_sod_2d_64x64_20_steps(oracle_mod):
    spec = wl.sod_spec(64, 8)
    U0 = wl.sod_state(spec)
    G, gdts, err = gpu_steps(spec, U0, 20, task=FF, record_dt=True)
    O, odts = oracle_steps(oracle_mod, spec, U0, 20)
    assert err == 0
    e = rule12_error(G, O, spec.nvar)
    print(f"FF sod64 20 steps: rule-12 error {e:.3e}, dt max rel {np.max(np.abs(gdts - odts) / odts):.3e}")
    np.testing.assert_allclose(gdts, odts, rtol=TOL, atol=0)
    assert e <= TOL


def test_sedov_128_packets_of_64_10_steps(oracle_mod):
    spec, packets = wl.sedov128_packets(64)
    U0 = wl.sedov_state(spec)
    G, gdts, err = gpu_steps(spec, U0, 10, task=FF, packets=packets, record_dt=True)
    O, odts = oracle_steps(oracle_mod, spec, U0, 10)
    assert err == 0
    e = rule12_error(G, O, spec.nvar)
    print(f"FF sedov128 10 steps: rule-12 error {e:.3e}")
    np.testing.assert_allclose(gdts, odts, rtol=TOL, atol=0)
    assert e <= TOL


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 0, 1)])
def test_random_jumps_every_tile_shape(oracle_mod, periodic):
    """Random jumps (limiter and upwind branches; the first-order fallback is
    driven in tests/test_gpu_fallback.py); every tile variant gives the same
    bits."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=periodic)
    U0 = wl.random_blocky_state(spec, 17)
    O, _ = oracle_steps(oracle_mod, spec, U0, 4)
    outs = []
    for tile in [(8, 8), (16, 8), (16, 16)]:
        G, _, err = gpu_steps(spec, U0, 4, task=FF, tile=tile)
        assert err == 0
        e = rule12_error(G, O, spec.nvar)
        print(f"FF tile {tile}: rule-12 error {e:.3e}")
        assert e <= TOL
        outs.append(G)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_2d_and_block_sizes(oracle_mod):
    for spec in [wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(32, 16, 1), periodic=(1, 0, 0)),
                 wl.MeshSpec(ndim=3, nb=(3, 2, 2), bs=(8, 8, 8)),
                 wl.MeshSpec(ndim=3, nb=(1, 2, 3), bs=(32, 16, 8))]:
        U0 = wl.random_blocky_state(spec, 9)
        G, _, err = gpu_steps(spec, U0, 5, task=FF)
        O, _ = oracle_steps(oracle_mod, spec, U0, 5)
        assert err == 0
        e = rule12_error(G, O, spec.nvar)
        print(f"FF {spec.ndim}D bs={spec.bs}: rule-12 error {e:.3e}")
        assert e <= TOL


def test_batch_path_matches_packet_path_and_conserves():
    """Persistent batch launches give the packet path's bits; on a periodic
    Sedov mass and energy totals are conserved to 1e-13 after 20 steps."""
    spec = wl.sedov_spec(64, 16, periodic=True)
    U0 = wl.sedov_state(spec)
    A, _, err = gpu_steps(spec, U0, 20, task=FF)
    (G,), errs = gpu_batch_steps([(spec, U0, None)], 20, task=FF, use_graph=True)
    assert err == 0 and errs == [0]
    assert np.array_equal(A, G)
    for v in (0, 4):
        s0, s1 = U0[:, v].sum(), G[:, v].sum()
        assert abs(s1 - s0) <= 1e-13 * abs(s0)


def test_sedov128_100_steps_error_reported(oracle_mod):
    """The precision workload run with the FF task: 100 steps of the 128^3
    Sedov, still within the FP64 parity rule."""
    spec, packets = wl.sedov128_packets(64)
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, packets)], 100, task=FF)
    O, _ = oracle_steps(oracle_mod, spec, U0, 100)
    assert errs == [0]
    e = rule12_error(G, O, spec.nvar)
    l1 = float(np.abs(G[:, 0] - O[:, 0]).mean() / np.abs(O[:, 0]).mean())
    print(f"FF sedov128 100 steps: rule-12 error {e:.3e}, relative L1(rho) {l1:.3e}")
    assert e <= TOL
