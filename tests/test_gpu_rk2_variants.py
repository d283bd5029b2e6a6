"""Heun two-stage Runge-Kutta steps with the plain MUSCL operator evaluated in
double-word arithmetic (RK2_FF, held to the FP64 parity rule against the RK2
oracle: per cell and variable |gpu - oracle| <= 1e-12 * max(|oracle|, s_v))
and in FP32 (RK2_F32FLUX: its L1 density error against the FP64 RK2 oracle
is reported; totals are conserved to 1e-13). In both, the packet stages, the
packet path's whole steps, the persistent batch and every tile shape give the
same bits."""
import dataclasses

import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import gpu_batch_steps, gpu_steps, oracle_steps, rule12_error

pytestmark = pytest.mark.gpu
TOL = 1e-12
RK2_FF = B.ORCHA_TASK_HYDRO_RK2_FF
RK2_F32 = B.ORCHA_TASK_HYDRO_RK2_F32FLUX
STAGES = {RK2_FF: (B.ORCHA_TASK_RK2_FF_STAGE1, B.ORCHA_TASK_RK2_FF_STAGE2),
          RK2_F32: (B.ORCHA_TASK_RK2_F32FLUX_STAGE1, B.ORCHA_TASK_RK2_F32FLUX_STAGE2)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def _stage_by_stage(spec, U0, nsteps, task):
    """FF steps written out with the packet-level stage tasks; returns (U, dts)."""
    s1, s2 = STAGES[task]
    mesh = B.Mesh(spec)
    try:
        mesh.load(U0)
        mesh.run(B.ORCHA_TASK_SIGNAL_SPEED)
        B.orcha_dt_reduce(mesh.handle)
        dts = []
        for _ in range(nsteps):
            dts.append(mesh.dt_value())
            mesh.run(B.ORCHA_TASK_GUARD_FILL)
            mesh.run(s1)
            B.orcha_mesh_swap(mesh.handle)
            mesh.run(B.ORCHA_TASK_GUARD_FILL)
            mesh.run(s2)
            B.orcha_dt_reduce(mesh.handle)
            B.orcha_mesh_swap(mesh.handle)
        assert mesh.poll() == 0
        return mesh.store(), np.array(dts)
    finally:
        mesh.close()


def test_ff_sod_2d_64x64_20_steps(oracle_mod):
    spec = wl.sod_spec(64, 8)
    U0 = wl.sod_state(spec)
    G, gdts = _stage_by_stage(spec, U0, 20, RK2_FF)
    O, odts = oracle_steps(oracle_mod, spec, U0, 20, rk2=True)
    e = rule12_error(G, O, spec.nvar)
    print(f"RK2 FF sod64 20 steps: rule-12 error {e:.3e}")
    np.testing.assert_allclose(gdts, odts, rtol=TOL, atol=0)
    assert e <= TOL
    A, _, err = gpu_steps(spec, U0, 20, task=RK2_FF)
    assert err == 0 and np.array_equal(A, G)


def test_ff_sedov_128_packets_of_64_10_steps(oracle_mod):
    spec, packets = wl.sedov128_packets(64)
    spec = dataclasses.replace(spec, cfl=0.4)
    U0 = wl.sedov_state(spec)
    A, _, err = gpu_steps(spec, U0, 10, task=RK2_FF, packets=packets)
    (G,), errs = gpu_batch_steps([(spec, U0, packets)], 10, task=RK2_FF, use_graph=True)
    O, _ = oracle_steps(oracle_mod, spec, U0, 10, rk2=True)
    assert err == 0 and errs == [0]
    assert np.array_equal(A, G)
    e = rule12_error(G, O, spec.nvar)
    print(f"RK2 FF sedov128 10 steps: rule-12 error {e:.3e}")
    assert e <= TOL


@pytest.mark.parametrize("task", [RK2_FF, RK2_F32])
def test_random_jumps_every_tile_shape(oracle_mod, task):
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=(1, 0, 1), cfl=0.4)
    U0 = wl.random_blocky_state(spec, 17)
    O, _ = oracle_steps(oracle_mod, spec, U0, 4, rk2=True)
    outs = []
    for tile in [(8, 8), (16, 8), (16, 16)]:
        G, _, err = gpu_steps(spec, U0, 4, task=task, tile=tile)
        assert err == 0
        e = rule12_error(G, O, spec.nvar)
        print(f"RK2 task {task} tile {tile}: rule-12 error {e:.3e}")
        if task == RK2_FF:
            assert e <= TOL
        else:
            assert np.all(np.isfinite(G)) and e < 1e-3
        outs.append(G)
        (H,), _ = gpu_batch_steps([(spec, U0, None)], 4, task=task, tile=tile)
        assert np.array_equal(H, G)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("task", [RK2_FF, RK2_F32])
def test_2d_blocks_and_graph_replay(oracle_mod, task):
    spec = wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(32, 16, 1), periodic=(1, 0, 0), cfl=0.4)
    U0 = wl.random_blocky_state(spec, 9)
    O, _ = oracle_steps(oracle_mod, spec, U0, 6, rk2=True)
    G, _, err = gpu_steps(spec, U0, 6, task=task, use_graph=True)
    e = rule12_error(G, O, spec.nvar)
    assert err == 0 and (e <= TOL if task == RK2_FF else e < 1e-3)
    (H,), _ = gpu_batch_steps([(spec, U0, None)], 3, task=task, use_graph=True, repeat=2)
    assert np.array_equal(H, G)


def test_f32_sedov_100_steps_error_and_conservation(oracle_mod):
    """The FP32-flux Heun step on the 128^3 Sedov set-up: relative L1 density
    error against the FP64 RK2 oracle after 100 steps (a stated number), and
    mass and energy totals conserved to 1e-13 (the blast stays inside)."""
    spec, packets = wl.sedov128_packets(64)
    spec = dataclasses.replace(spec, cfl=0.4)
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, packets)], 100, task=RK2_F32)
    assert errs == [0]
    O, _ = oracle_steps(oracle_mod, spec, U0, 100, rk2=True)
    l1 = np.abs(G[:, 0] - O[:, 0]).sum() / np.abs(O[:, 0]).sum()
    print(f"RK2 F32 sedov128 100 steps: relative L1(rho) {l1:.3e}, "
          f"largest |drho| {np.abs(G[:, 0] - O[:, 0]).max():.3e}")
    assert np.isfinite(l1) and l1 < 1e-5
    for v in (0, 4):
        s0, s1 = U0[:, v].sum(), G[:, v].sum()
        assert abs(s1 - s0) <= 1e-13 * abs(s0)


@pytest.mark.parametrize("task", [RK2_FF, RK2_F32])
def test_free_stream_is_preserved_bitwise(task):
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=(1, 1, 1), cfl=0.4)
    U0 = wl.uniform_state(spec, 1.3, (0.4, -0.25, 0.15), 0.9)
    (G,), errs = gpu_batch_steps([(spec, U0, None)], 3, task=task)
    assert errs == [0] and np.array_equal(G, U0)
