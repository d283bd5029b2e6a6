"""Heun two-stage Runge-Kutta steps on the GPU (FP64, plain MUSCL operator)
against the RK2 oracle, under the FP64 parity rule: per cell and variable
|gpu - oracle| <= 1e-12 * max(|oracle|, s_v). Packet path (guard fill per
stage), persistent batch path (halo gather per stage) and the packet-level
stage tasks all give the same bits."""
import dataclasses

import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import gpu_batch_steps, gpu_steps, oracle_steps, rule12_error

pytestmark = pytest.mark.gpu
TOL = 1e-12
RK2 = B.ORCHA_TASK_HYDRO_RK2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def _stage_by_stage(spec, U0, nsteps, packets=None):
    """Steps written out with the packet-level tasks; returns (U, dts)."""
    mesh = B.Mesh(spec, packets=packets)
    try:
        mesh.load(U0)
        mesh.run(B.ORCHA_TASK_SIGNAL_SPEED)
        B.orcha_dt_reduce(mesh.handle)
        dts = []
        for _ in range(nsteps):
            dts.append(mesh.dt_value())
            mesh.run(B.ORCHA_TASK_GUARD_FILL)
            mesh.run(B.ORCHA_TASK_RK2_STAGE1)
            B.orcha_mesh_swap(mesh.handle)
            mesh.run(B.ORCHA_TASK_GUARD_FILL)
            mesh.run(B.ORCHA_TASK_RK2_STAGE2)
            B.orcha_dt_reduce(mesh.handle)
            B.orcha_mesh_swap(mesh.handle)
        assert mesh.poll() == 0
        return mesh.store(), np.array(dts)
    finally:
        mesh.close()


def test_sod_2d_64x64_20_steps(oracle_mod):
    spec = wl.sod_spec(64, 8)
    U0 = wl.sod_state(spec)
    G, gdts = _stage_by_stage(spec, U0, 20)
    O, odts = oracle_steps(oracle_mod, spec, U0, 20, rk2=True)
    e = rule12_error(G, O, spec.nvar)
    print(f"RK2 sod64 20 steps: rule-12 error {e:.3e}")
    np.testing.assert_allclose(gdts, odts, rtol=TOL, atol=0)
    assert e <= TOL
    A, _, err = gpu_steps(spec, U0, 20, task=RK2)           # mesh_advance drives the same stages
    assert err == 0 and np.array_equal(A, G)


def test_sedov_128_packets_of_64_10_steps(oracle_mod):
    spec, packets = wl.sedov128_packets(64)
    spec = dataclasses.replace(spec, cfl=0.4)
    U0 = wl.sedov_state(spec)
    A, _, err = gpu_steps(spec, U0, 10, task=RK2, packets=packets)
    (G,), errs = gpu_batch_steps([(spec, U0, packets)], 10, task=RK2, use_graph=True)
    O, _ = oracle_steps(oracle_mod, spec, U0, 10, rk2=True)
    assert err == 0 and errs == [0]
    assert np.array_equal(A, G)
    e = rule12_error(G, O, spec.nvar)
    print(f"RK2 sedov128 10 steps: rule-12 error {e:.3e}")
    assert e <= TOL


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 0, 1)])
def test_random_jumps_every_tile_shape(oracle_mod, periodic):
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=periodic, cfl=0.4)
    U0 = wl.random_blocky_state(spec, 17)
    O, _ = oracle_steps(oracle_mod, spec, U0, 4, rk2=True)
    outs = []
    for tile in [(8, 8), (16, 8), (16, 16)]:
        G, _, err = gpu_steps(spec, U0, 4, task=RK2, tile=tile)
        assert err == 0
        e = rule12_error(G, O, spec.nvar)
        print(f"RK2 tile {tile}: rule-12 error {e:.3e}")
        assert e <= TOL
        outs.append(G)
        (H,), _ = gpu_batch_steps([(spec, U0, None)], 4, task=RK2, tile=tile)
        assert np.array_equal(H, G)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_2d_blocks_and_graph_replay(oracle_mod):
    spec = wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(32, 16, 1), periodic=(1, 0, 0), cfl=0.4)
    U0 = wl.random_blocky_state(spec, 9)
    O, _ = oracle_steps(oracle_mod, spec, U0, 6, rk2=True)
    G, _, err = gpu_steps(spec, U0, 6, task=RK2, use_graph=True)
    assert err == 0 and rule12_error(G, O, spec.nvar) <= TOL
    (H,), _ = gpu_batch_steps([(spec, U0, None)], 3, task=RK2, use_graph=True, repeat=2)
    assert np.array_equal(H, G)


def test_conservation_periodic():
    spec = wl.sedov_spec(64, 16, periodic=True)
    spec = dataclasses.replace(spec, cfl=0.4)
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, None)], 20, task=RK2)
    assert errs == [0]
    for v in (0, 4):
        s0, s1 = U0[:, v].sum(), G[:, v].sum()
        assert abs(s1 - s0) <= 1e-13 * abs(s0)
