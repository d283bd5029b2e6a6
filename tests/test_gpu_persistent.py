"""The persistent multi-packet path (orcha_batch_*): one launch per time step
drains a work queue of (mesh, block, tile) items, gathers halos directly and
forms each mesh's dt on the device. It must give bitwise the packet path's
result (and so the oracle's)."""
import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import gpu_batch_steps, gpu_steps, oracle_steps, rule12_error

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def test_sedov128_batch_matches_packet_path_and_oracle(oracle_mod):
    spec, packets = wl.sedov128_packets(64)
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, packets)], 10)
    A, _, _ = gpu_steps(spec, U0, 10, packets=packets)
    assert errs == [0]
    assert np.array_equal(G, A)
    O, _ = oracle_steps(oracle_mod, spec, U0, 10)
    assert rule12_error(G, O, spec.nvar) <= TOL


@pytest.mark.parametrize("task", [B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_FF])
def test_sedov256_uneven_packets_two_steps(oracle_mod, task):
    """256^3 cells as 4096 blocks of 16^3, packet sizes seed-uniform in
    [1, 256]: every cell after two steps (graph-captured), in FP64 and in the
    double-word arithmetic, both held to the FP64 rule."""
    spec, packets = wl.sedov256_uneven_packets(0)
    assert min(len(p) for p in packets) >= 1 and sum(len(p) for p in packets) == 4096
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, packets)], 2, task=task, use_graph=True)
    assert errs == [0]
    O, _ = oracle_steps(oracle_mod, spec, U0, 2)
    e = rule12_error(G, O, spec.nvar)
    print(f"sedov256 uneven packets, 2 steps, task {task}: rule-12 error {e:.3e}")
    assert e <= TOL


def test_sedov256_f32flux_error_and_conservation(oracle_mod):
    """The same 256^3 mesh in the configured FP32-flux arithmetic: L1(rho)
    against the FP64 oracle after two steps, stated; mass and energy totals
    conserved to 1e-13 (the blast stays inside)."""
    spec, packets = wl.sedov256_uneven_packets(0)
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, packets)], 2, task=B.ORCHA_TASK_HYDRO_F32FLUX, use_graph=True)
    assert errs == [0]
    O, _ = oracle_steps(oracle_mod, spec, U0, 2)
    l1 = float(np.abs(G[:, 0] - O[:, 0]).mean()) / float(np.abs(O[:, 0]).mean())
    print(f"sedov256 FP32 flux, 2 steps: relative L1(rho) {l1:.3e}")
    assert l1 < 1e-6
    for v in (0, 4):
        assert abs(G[:, v].sum() - U0[:, v].sum()) <= 1e-13 * abs(U0[:, v].sum())


@pytest.mark.parametrize("tile", [(8, 8), (16, 8), (16, 16)])
def test_batch_tiles_and_graph_replay(tile):
    spec = wl.MeshSpec(ndim=3, nb=(2, 3, 2), bs=(16, 16, 16), periodic=(1, 0, 0))
    U0 = wl.random_blocky_state(spec, 41)
    ref, _, _ = gpu_steps(spec, U0, 6)
    (G,), _ = gpu_batch_steps([(spec, U0, None)], 6, tile=tile)
    assert np.array_equal(G, ref)
    # the same 6 steps as 3 + 3 replays of one captured 3-step graph
    (H,), _ = gpu_batch_steps([(spec, U0, None)], 3, tile=tile, use_graph=True, repeat=2)
    assert np.array_equal(H, ref)


@pytest.mark.parametrize("task", [B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_RK2, B.ORCHA_TASK_HYDRO_FF])
def test_multi_mesh_batch_mixed_block_sizes(task):
    """Meshes with 8^3, 16^3 and 32^3 blocks (different dt each) in one batch of
    8x8 tiles: each result equals the mesh advanced alone (for RK2 each mesh's
    two stages share the launches, and dt stays per mesh)."""
    probs = [
        (wl.MeshSpec(ndim=3, nb=(3, 2, 2), bs=(8, 8, 8)), 51),
        (wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(16, 16, 16), periodic=(1, 1, 1)), 52),
        (wl.MeshSpec(ndim=3, nb=(1, 1, 2), bs=(32, 32, 32)), 53),
    ]
    problems = []
    alone = []
    for spec, seed in probs:
        U0 = wl.random_blocky_state(spec, seed)
        rng = np.random.default_rng(seed)
        ids = rng.permutation(spec.nblocks).astype(np.int32)
        pk = np.array_split(ids, 2) if spec.nblocks > 1 else [ids]
        problems.append((spec, U0, pk))
        alone.append(gpu_steps(spec, U0, 4, task=task)[0])
    outs, errs = gpu_batch_steps(problems, 4, tile=(8, 8), task=task)
    assert errs == [0, 0, 0]
    for G, A in zip(outs, alone):
        assert np.array_equal(G, A)


def test_2d_batch(oracle_mod):
    spec = wl.sod_spec(64, 8)
    U0 = wl.sod_state(spec)
    (G,), _ = gpu_batch_steps([(spec, U0, [np.arange(0, 40, dtype=np.int32), np.arange(40, 64, dtype=np.int32)])], 20)
    O, _ = oracle_steps(oracle_mod, spec, U0, 20)
    assert rule12_error(G, O, spec.nvar) <= TOL


@pytest.mark.parametrize("task", [B.ORCHA_TASK_HYDRO_F32FLUX, B.ORCHA_TASK_HYDRO_F32FLUX_FFSUM])
def test_batch_f32flux_matches_packet_path(task):
    spec = wl.sedov_spec(64, 16)
    U0 = wl.sedov_state(spec)
    (G,), _ = gpu_batch_steps([(spec, U0, None)], 5, task=task)
    A, _, _ = gpu_steps(spec, U0, 5, task=task)
    assert np.array_equal(G, A)


def test_batch_validation():
    spec = wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(8, 8, 8))
    m = B.Mesh(spec, packets=[np.array([0], dtype=np.int32)])       # covers 1 of 2 blocks
    try:
        with pytest.raises(B.OrchaError) as ei:
            B.orcha_batch_create(m.packets)
        assert ei.value.status == B.ORCHA_ERR_INVALID
    finally:
        m.close()
    m = B.Mesh(spec)
    try:
        with pytest.raises(B.OrchaError):
            B.orcha_batch_create(m.packets, 16, 16)                    # tile larger than the blocks
    finally:
        m.close()


@pytest.mark.parametrize("tile", [(16, 16), (16, 8)])
def test_tail_wave_split_into_z_slabs_keeps_the_bits(tile):
    """512 blocks of 16^3 leave a partial last wave of resident CTAs, whose
    items the batch splits into z slabs (two, or three for the FF variant with
    16x8 tiles on a B300): the result is bitwise the packet path's (every face
    flux is the same expression whichever item computes it), in every
    arithmetic variant."""
    spec, packets = wl.sedov128_packets(64)
    U0 = wl.random_blocky_state(spec, 71)
    for task in (B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_F32FLUX, B.ORCHA_TASK_HYDRO_FF,
                 B.ORCHA_TASK_HYDRO_F32FLUX_FFSUM):
        A, _, _ = gpu_steps(spec, U0, 3, packets=packets, task=task)
        (G,), errs = gpu_batch_steps([(spec, U0, packets)], 3, tile=tile, task=task)
        assert errs == [0]
        assert np.array_equal(G, A), task
