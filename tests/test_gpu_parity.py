"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 path: per cell and variable |gpu - oracle| <= 1e-12 * max(|oracle|, s_v)
(s_v = the field's largest |momentum| for momentum components). The default
build fuses multiply-adds (a few ulp per step from the unfused definition; the
tests print the observed difference); a build with ORCHA_FP64_CONTRACT=0
evaluates the oracle's expression trees unfused and matches it bit for bit.
"""
import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import gpu_steps, oracle_steps, rule12_error

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()
    yield


def test_sod_2d_64x64_20_steps(oracle_mod):
    """2D Sod, 64 x 64 cells as 8 x 8 blocks of 8 x 8, one packet of 64 blocks,
    20 steps: states and the dt sequence."""
    spec = wl.sod_spec(64, 8)
    U0 = wl.sod_state(spec)
    G, gdts, err = gpu_steps(spec, U0, 20, record_dt=True)
    O, odts = oracle_steps(oracle_mod, spec, U0, 20)
    assert err == 0
    np.testing.assert_allclose(gdts, odts, rtol=TOL, atol=0)
    e = rule12_error(G, O, spec.nvar)
    print(f"sod64 rule-12 error {e:.3e}, bitwise-equal {np.mean(G == O):.6f}")
    assert e <= TOL


def test_sedov_128_packets_of_64_10_steps(oracle_mod):
    """3D Sedov, 128^3 cells as 512 blocks of 16^3, packets of 64 blocks, 10
    steps, every cell."""
    spec, packets = wl.sedov128_packets(64)
    U0 = wl.sedov_state(spec)
    G, gdts, err = gpu_steps(spec, U0, 10, packets=packets, record_dt=True)
    O, odts = oracle_steps(oracle_mod, spec, U0, 10)
    assert err == 0
    np.testing.assert_allclose(gdts, odts, rtol=TOL, atol=0)
    e = rule12_error(G, O, spec.nvar)
    print(f"sedov128 rule-12 error {e:.3e}, bitwise-equal {np.mean(G == O):.6f}")
    assert e <= TOL


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1), (1, 0, 1)])
def test_random_jumps_every_tile_shape(oracle_mod, periodic):
    """Random jumps in every direction (limiter and upwind branches; at the CFL
    time step no cell takes the first-order fallback, which
    tests/test_gpu_fallback.py drives), two blocks of 16^3 per axis; every
    tile variant gives the same bits."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=periodic)
    U0 = wl.random_blocky_state(spec, 17)
    O, _ = oracle_steps(oracle_mod, spec, U0, 4)
    outs = []
    for tile in [(8, 8), (16, 8), (16, 16)]:
        G, _, err = gpu_steps(spec, U0, 4, tile=tile)
        assert err == 0
        e = rule12_error(G, O, spec.nvar)
        print(f"tile {tile} rule-12 error {e:.3e}")
        assert e <= TOL
        outs.append(G)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("bs,nb", [((8, 8, 8), (3, 2, 2)), ((32, 32, 32), (2, 1, 1)), ((32, 16, 8), (1, 2, 3))])
def test_block_shapes(oracle_mod, bs, nb):
    """Block sizes 8, 16, 32 (also mixed per axis) and non-cubic block grids."""
    spec = wl.MeshSpec(ndim=3, nb=nb, bs=bs)
    Ug = wl.from_blocks(wl.MeshSpec(ndim=3, nb=nb, bs=bs), wl.random_smooth_state(spec, 5, amp=0.6))
    U0 = wl.to_blocks(spec, Ug)
    G, _, err = gpu_steps(spec, U0, 3)
    O, _ = oracle_steps(oracle_mod, spec, U0, 3)
    assert err == 0
    assert rule12_error(G, O, spec.nvar) <= TOL


def test_2d_blocks_and_tiles(oracle_mod):
    spec = wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(32, 16, 1), periodic=(1, 0, 0))
    U0 = wl.random_blocky_state(spec, 9)
    O, _ = oracle_steps(oracle_mod, spec, U0, 6)
    for tile in [(8, 8), (16, 8), (16, 16)]:
        G, _, err = gpu_steps(spec, U0, 6, tile=tile)
        assert err == 0 and rule12_error(G, O, spec.nvar) <= TOL


def test_uneven_shuffled_packets_match_one_packet():
    """A ragged partition of the blocks into packets, in shuffled order, gives
    the bits of a single packet."""
    spec = wl.MeshSpec(ndim=3, nb=(4, 3, 2), bs=(8, 8, 8))
    U0 = wl.random_blocky_state(spec, 23)
    rng = np.random.default_rng(4)
    ids = rng.permutation(spec.nblocks).astype(np.int32)
    cuts = np.sort(rng.choice(np.arange(1, spec.nblocks), size=5, replace=False))
    packets = np.split(ids, cuts)
    A, _, _ = gpu_steps(spec, U0, 5, packets=packets)
    Bv, _, _ = gpu_steps(spec, U0, 5)
    assert np.array_equal(A, Bv)


def test_single_block_meshes(oracle_mod):
    for spec in [wl.MeshSpec(ndim=3, nb=(1, 1, 1), bs=(16, 16, 16)),
                 wl.MeshSpec(ndim=3, nb=(1, 1, 1), bs=(8, 8, 8), periodic=(1, 1, 1)),
                 wl.MeshSpec(ndim=2, nb=(1, 1, 1), bs=(8, 8, 1))]:
        U0 = wl.random_blocky_state(spec, 31)
        G, _, err = gpu_steps(spec, U0, 3)
        O, _ = oracle_steps(oracle_mod, spec, U0, 3)
        assert err == 0 and rule12_error(G, O, spec.nvar) <= TOL


def test_graph_replay_matches_eager():
    spec, packets = wl.sedov128_packets(64)
    spec = wl.sedov_spec(64, 16)
    packets = [np.arange(0, 30, dtype=np.int32), np.arange(30, 64, dtype=np.int32)]
    U0 = wl.sedov_state(spec)
    A, _, _ = gpu_steps(spec, U0, 6, packets=packets)
    G, _, _ = gpu_steps(spec, U0, 6, packets=packets, use_graph=True)
    assert np.array_equal(A, G)


def test_f32flux_error_and_conservation(oracle_mod):
    """FP32 reconstruction/flux with FP64 update on a 64^3 periodic Sedov: the
    L1 density error against the FP64 oracle is reported; mass and energy
    totals are conserved to 1e-13 (promoted face fluxes telescope)."""
    spec = wl.sedov_spec(64, 16, periodic=True)
    U0 = wl.sedov_state(spec)
    G, _, err = gpu_steps(spec, U0, 20, task=B.ORCHA_TASK_HYDRO_F32FLUX)
    O, _ = oracle_steps(oracle_mod, spec, U0, 20)
    assert err == 0
    l1 = float(np.abs(G[:, 0] - O[:, 0]).mean())
    print(f"f32flux 64^3 Sedov, 20 steps: L1(rho) vs FP64 oracle = {l1:.3e}")
    assert np.isfinite(l1) and l1 < 1e-4
    for v in (0, 4):
        s0, s1 = U0[:, v].sum(), G[:, v].sum()
        assert abs(s1 - s0) <= 1e-13 * abs(s0)


def test_nonphysical_input_is_reported():
    spec = wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(8, 8, 8))
    U0 = wl.uniform_state(spec, 1.0, (0.0, 0.0, 0.0), 1.0)
    U0[1, 4, 3, 3, 3] = -1.0          # negative total energy -> p < 0
    mesh = B.Mesh(spec)
    try:
        mesh.load(U0)
        mesh.run(B.ORCHA_TASK_SIGNAL_SPEED)
        with pytest.raises(B.OrchaError) as ei:
            mesh.poll()
        assert ei.value.status == B.ORCHA_ERR_NONFINITE
        assert mesh.poll() == 0          # the word was cleared
    finally:
        mesh.close()


def test_packet_validation():
    spec = wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(8, 8, 8))
    mesh = B.Mesh(spec)
    try:
        for bad in ([], [0, 2], [1, 1], [-1]):
            with pytest.raises(B.OrchaError) as ei:
                B.orcha_packet_create(mesh.handle, np.array(bad, dtype=np.int32))
            assert ei.value.status == B.ORCHA_ERR_INVALID
        with pytest.raises(B.OrchaError):
            mesh.set_tile(16, 16)        # does not divide 8^3 blocks
        with pytest.raises(B.OrchaError):
            B.orcha_mesh_advance(mesh.handle, mesh.packets[:0], B.ORCHA_TASK_HYDRO_FP64, 1, True, False)
    finally:
        mesh.close()


def test_integer_pipe_conversions_match_hardware():
    """Every binary32 pattern (FP32 -> FP64) and 2^32 pseudo-random binary64
    patterns, half of them steered to the binary32 range edges (FP64 -> FP32,
    round to nearest even)."""
    assert B.orcha_selftest_conversions(0, 1 << 32, seed=12345) == 0


@pytest.mark.parametrize("task", [B.ORCHA_TASK_HYDRO_F32FLUX, B.ORCHA_TASK_HYDRO_F32FLUX_FFSUM])
def test_c4_f32flux_100_steps_error_against_fp64_oracle(oracle_mod, task):
    """The precision workload: 128^3 Sedov, FP32 reconstruction/flux, 100
    steps, in the configured arithmetic (face fluxes promoted to FP64 before
    the difference, FP64 update and signal speed) and in the shortcut (float-
    float flux sums, FP32 signal speed). Reports L1(rho) against the FP64
    oracle; totals of mass and energy are conserved to 1e-13 (the blast stays
    inside)."""
    spec, packets = wl.sedov128_packets(64)
    U0 = wl.sedov_state(spec)
    G, _, err = gpu_steps(spec, U0, 100, task=task, packets=packets)
    O, _ = oracle_steps(oracle_mod, spec, U0, 100)
    assert err == 0
    l1 = float(np.abs(G[:, 0] - O[:, 0]).mean())
    l1_rel = l1 / float(np.abs(O[:, 0]).mean())
    name = "f32flux" if task == B.ORCHA_TASK_HYDRO_F32FLUX else "f32flux_ffsum"
    print(f"C4 {name} 128^3 Sedov, 100 steps: L1(rho) = {l1:.3e} (relative {l1_rel:.3e}), "
          f"max |drho| = {np.abs(G[:, 0] - O[:, 0]).max():.3e}")
    assert l1_rel < 1e-5
    for v in (0, 4):
        s0, s1 = U0[:, v].sum(), G[:, v].sum()
        assert abs(s1 - s0) <= 1e-13 * abs(s0)


def test_integer_pipe_fp64_arithmetic_matches_hardware():
    """The integer-pipe binary64 add/sub/mul give the hardware's bits on 2^31
    pseudo-random operand pairs (carries, ties, cancellation, zeros), and the
    FP64 task's integer sign tests, wave-speed order, minmod and halving
    agree with FP64 comparisons and 0.5 * x on the same pairs; the FP32
    tasks' median-of-three minmod gives the bits of its sign-test definition
    on binary32 pairs cut from them (zeros of both signs, ties)."""
    assert B.orcha_selftest_fp64_emulation(1 << 31, seed=2024) == 0


@pytest.mark.parametrize("task", [B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_F32FLUX, B.ORCHA_TASK_HYDRO_FF,
                                  B.ORCHA_TASK_HYDRO_RK2, B.ORCHA_TASK_HYDRO_F32FLUX_FFSUM])
@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1)])
def test_free_stream_is_preserved_bitwise(task, periodic):
    """A uniform state with an arbitrary velocity is the degenerate case of the
    scheme: every slope is zero and both faces of a cell carry the same flux,
    so every variant keeps it bit for bit, through the packet path and the
    persistent path."""
    rng = np.random.default_rng(3)
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=periodic)
    U0 = wl.uniform_state(spec, rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
    G, _, err = gpu_steps(spec, U0, 4, task=task)
    assert err == 0 and np.array_equal(G, U0)
    from .gpu_helpers import gpu_batch_steps
    (H,), errs = gpu_batch_steps([(spec, U0, None)], 4, task=task)
    assert errs == [0] and np.array_equal(H, U0)


def test_nonphysical_state_is_reported_by_the_batch_path():
    spec = wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(16, 16, 16))
    U0 = wl.uniform_state(spec, 1.0, (0.0, 0.0, 0.0), 1.0)
    U0[1, 4, 3, 3, 3] = -1.0          # negative total energy -> p < 0
    from .gpu_helpers import gpu_batch_steps
    with pytest.raises(B.OrchaError) as ei:
        gpu_batch_steps([(spec, U0, None)], 1)
    assert ei.value.status == B.ORCHA_ERR_NONFINITE
