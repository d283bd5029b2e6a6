"""Two operator applications per launch (the fused batch tasks) against the
one-step launches and the oracle.

TB2 (temporal blocking): two MUSCL-Hancock steps per launch with the dt of
the pair's first state. Each pass of the fused launch is the one-step
sweep's code, so a TB2 launch gives the bits of two single-step launches
with the same dt; FP64 is held to the parity rule against two oracle steps
with that dt. RK2_FUSED: both Heun stages per launch; the bits of the
two-launch Heun step, and the parity rule against the RK2 oracle. The
exact-FP64 library reproduces the oracle bit for bit (test_gpu_exact_build).
"""
import dataclasses

import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import gpu_batch_fixed_dt, gpu_batch_steps, gpu_one_step, rule12_error

pytestmark = pytest.mark.gpu
TOL = 1e-12
TILES = [(8, 8), (16, 8), (16, 16)]
TB2 = {B.ORCHA_TASK_HYDRO_TB2: B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_F32FLUX_TB2: B.ORCHA_TASK_HYDRO_F32FLUX}
FUSED_RK = {B.ORCHA_TASK_HYDRO_RK2_FUSED: B.ORCHA_TASK_HYDRO_RK2,
            B.ORCHA_TASK_HYDRO_RK2_F32FLUX_FUSED: B.ORCHA_TASK_HYDRO_RK2_F32FLUX}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def _case(periodic, ndim=3, seed=17):
    if ndim == 3:
        spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=periodic)
    else:
        spec = wl.MeshSpec(ndim=2, nb=(3, 2, 1), bs=(16, 16, 1), periodic=periodic)
    return spec, wl.random_blocky_state(spec, seed)


@pytest.mark.parametrize("task", list(TB2))
@pytest.mark.parametrize("periodic,ndim", [((0, 0, 0), 3), ((1, 1, 1), 3), ((1, 0, 1), 3), ((0, 1, 0), 2)])
def test_tb2_launch_is_two_single_steps(oracle_mod, task, periodic, ndim):
    spec, U0 = _case(periodic, ndim)
    m = oracle_mod.Mesh(**spec.oracle_kwargs())
    dt = oracle_mod.dt(m, U0)
    O1, _, _ = oracle_mod.step(m, U0, dt)
    O2, _, _ = oracle_mod.step(m, O1, dt)
    one = B.ORCHA_TASK_HYDRO_FP64 if task == B.ORCHA_TASK_HYDRO_TB2 else B.ORCHA_TASK_HYDRO_F32FLUX
    for tile in TILES:
        S1 = gpu_one_step(spec, U0, dt, one, tile, "batch")
        S2 = gpu_one_step(spec, S1, dt, one, tile, "batch")
        G, err, _ = gpu_batch_fixed_dt(spec, U0, dt, task, tile, 2)
        assert err == 0
        assert np.array_equal(G, S2), tile
        if task == B.ORCHA_TASK_HYDRO_TB2:
            e = rule12_error(G, O2, spec.nvar)
            print(f"TB2 {periodic} {ndim}D tile {tile}: rule-12 error {e:.3e} (bitwise two single steps)")
            assert e <= TOL
        else:
            l1 = float(np.abs(G[:, 0] - O2[:, 0]).sum() / np.abs(O2[:, 0]).sum())
            print(f"TB2 FP32 flux {periodic} {ndim}D tile {tile}: relative L1(rho) {l1:.3e}")
            assert l1 < 1e-5


def test_tb2_sedov_pairs_against_the_oracle_with_the_same_dts(oracle_mod):
    """Sedov 64^3, 10 steps as 5 launches: each pair takes the dt of its first
    state; the oracle is driven with the same dt rule."""
    spec = wl.sedov_spec(64, 16)
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, None)], 10, task=B.ORCHA_TASK_HYDRO_TB2, tile=(16, 8))
    assert errs == [0]
    m = oracle_mod.Mesh(**spec.oracle_kwargs())
    U = U0
    for _ in range(5):
        dt = oracle_mod.dt(m, U)
        U, _, _ = oracle_mod.step(m, U, dt)
        U, _, _ = oracle_mod.step(m, U, dt)
    e = rule12_error(G, U, spec.nvar)
    print(f"TB2 sedov64 10 steps: rule-12 error {e:.3e}")
    assert e <= TOL
    for v in (0, 4):
        assert abs(G[:, v].sum() - U0[:, v].sum()) <= 1e-13 * abs(U0[:, v].sum())


@pytest.mark.parametrize("task", list(FUSED_RK))
@pytest.mark.parametrize("periodic,ndim", [((0, 0, 0), 3), ((1, 1, 1), 3), ((0, 1, 0), 2)])
def test_fused_heun_is_the_two_launch_step(oracle_mod, task, periodic, ndim):
    spec, U0 = _case(periodic, ndim, seed=23)
    spec = dataclasses.replace(spec, cfl=0.4)
    m = oracle_mod.Mesh(**spec.oracle_kwargs())
    dt = oracle_mod.dt(m, U0)
    O, _, _ = oracle_mod.step_rk2(m, U0, dt)
    for tile in TILES:
        A, _, _ = gpu_batch_fixed_dt(spec, U0, dt, FUSED_RK[task], tile, 1)
        G, err, _ = gpu_batch_fixed_dt(spec, U0, dt, task, tile, 1)
        assert err == 0
        assert np.array_equal(G, A), tile
        if task == B.ORCHA_TASK_HYDRO_RK2_FUSED:
            e = rule12_error(G, O, spec.nvar)
            print(f"fused Heun {periodic} {ndim}D tile {tile}: rule-12 error {e:.3e}")
            assert e <= TOL


def test_fused_heun_sedov_steps_match_the_rk2_oracle(oracle_mod):
    spec = dataclasses.replace(wl.sedov_spec(64, 16), cfl=0.4)
    U0 = wl.sedov_state(spec)
    (G,), errs = gpu_batch_steps([(spec, U0, None)], 6, task=B.ORCHA_TASK_HYDRO_RK2_FUSED, tile=(16, 8))
    (A,), _ = gpu_batch_steps([(spec, U0, None)], 6, task=B.ORCHA_TASK_HYDRO_RK2, tile=(16, 8))
    assert errs == [0] and np.array_equal(G, A)
    O, _, _ = oracle_mod.run(oracle_mod.Mesh(**spec.oracle_kwargs()), U0, 6, rk2=True)
    e = rule12_error(G, O, spec.nvar)
    print(f"fused Heun sedov64 6 steps: rule-12 error {e:.3e}")
    assert e <= TOL


def test_free_stream_and_graph_replay():
    rng = np.random.default_rng(5)
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=(1, 0, 1))
    U0 = wl.uniform_state(spec, rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
    for task in list(TB2) + list(FUSED_RK):
        (G,), errs = gpu_batch_steps([(spec, U0, None)], 4, task=task, use_graph=True, repeat=2)
        assert errs == [0] and np.array_equal(G, U0), task


def test_second_step_beyond_the_stability_limit_is_reported():
    """A pair whose shared dt is 1.3 / s(U0): the intermediate state's speed
    is about the initial one, so dt s(U1) > 1 and the launch flags it."""
    spec, U0 = _case((1, 1, 1))
    import oracle
    s0 = oracle.max_signal_speed(oracle.Mesh(**spec.oracle_kwargs()), U0)
    _, err, _ = gpu_batch_fixed_dt(spec, U0, 1.3 / s0, B.ORCHA_TASK_HYDRO_TB2, (16, 8), 2)
    assert err & B.ORCHA_DEVERR_CFL
    _, err, _ = gpu_batch_fixed_dt(spec, U0, 0.5 / s0, B.ORCHA_TASK_HYDRO_TB2, (16, 8), 2)
    assert err == 0


def test_fused_task_validation():
    spec, U0 = _case((0, 0, 0))
    mesh = B.Mesh(spec)
    try:
        batch = B.orcha_batch_create(mesh.packets, 16, 8)
        try:
            with pytest.raises(B.OrchaError) as ei:
                B.orcha_batch_advance(batch, B.ORCHA_TASK_HYDRO_TB2, 3, True, False)
            assert ei.value.status == B.ORCHA_ERR_INVALID
        finally:
            B.orcha_batch_destroy(batch)
        with pytest.raises(B.OrchaError) as ei:
            mesh.advance(2, B.ORCHA_TASK_HYDRO_TB2)
        assert ei.value.status == B.ORCHA_ERR_UNSUPPORTED
    finally:
        mesh.close()
