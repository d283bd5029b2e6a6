"""The signal-speed filter of the persistent one-step tasks: a cell's FP64
signal speed is evaluated only when its FP32 upper bound reaches a quarter of
the previous step's largest speed, and the step's reducer re-evaluates in FP64
whenever a skipped bound could exceed the maximum. dt = CFL / max_cells
sum_d (|u_d| + c) / dx_d must keep the bits of the unfiltered evaluation (the
packet path, which evaluates every cell), whatever the threshold."""
import dataclasses

import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import _poll

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def _packet_steps(spec, U0, task, nsteps, dt0=None):
    """nsteps through the packet path (every cell's speed in FP64): returns
    (state, dt after each step, device error word). dt0: start from this dt
    instead of the CFL dt of U0."""
    mesh = B.Mesh(spec)
    try:
        mesh.load(U0)
        dts = []
        if dt0 is None:
            mesh.advance(0, task, init_dt=True)
            dts.append(mesh.dt_value())       # the first dt: every cell's speed in FP64
        else:
            mesh.dt.fill_(dt0)
        for _ in range(nsteps):
            mesh.advance(1, task, init_dt=False)
            dts.append(mesh.dt_value())
        return mesh.store(), np.array(dts), _poll(mesh)
    finally:
        mesh.close()


def _batch_steps(spec, U0, task, nsteps, dt0=None, use_graph=False):
    """The same through one persistent launch per step (the filtered path)."""
    import torch
    mesh = B.Mesh(spec)
    batch = None
    try:
        mesh.load(U0)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        batch = B.orcha_batch_create(mesh.packets, 0, 0)
        dts = []
        if dt0 is None:
            B.orcha_batch_advance(batch, task, 0, True, False, s)
            s.synchronize()
            dts.append(mesh.dt_value())       # the first dt: filtered for the FP64 rule
        else:
            mesh.dt.fill_(dt0)
            s.wait_stream(torch.cuda.current_stream())
        for _ in range(nsteps):
            B.orcha_batch_advance(batch, task, 1, False, use_graph, s)
            s.synchronize()
            dts.append(mesh.dt_value())
        return mesh.store(), np.array(dts), _poll(mesh, s)
    finally:
        if batch:
            B.orcha_batch_destroy(batch)
        mesh.close()


def test_bound_is_an_upper_bound():
    """2^24 random states, heavy cancellation included: the FP32 bound never
    lies below the FP64 speed (and the lower bound that the filtered first
    time step pairs with it never above it), never applies to a state the FP64 path finds
    non-physical, and applies to about half of them (the rest lie outside
    its range or cancel to below 2^-40 E). Where the pressure is a
    near-cancellation the bound is loose (its FP32 interval for p is
    ~2^-22 (E + ke) wide), by a few parts per thousand at most."""
    n = 1 << 24
    bad, applied, nonphys, ratio = B.orcha_selftest_speed_bound(n, seed=7)
    print(f"speed bound: applied to {applied} of {n} states, largest bound/speed {ratio:.9f}")
    assert bad == 0
    assert nonphys == 0
    assert applied > n // 3
    assert 1.0 <= ratio < 1.01


TASKS = [B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_F32FLUX, B.ORCHA_TASK_HYDRO_FF, B.ORCHA_TASK_HYDRO_RK2]


@pytest.mark.parametrize("task", TASKS)
def test_sedov_dt_sequence_and_state_bitwise(task):
    """Sedov 64^3 (blocks of 16^3): nearly every cell lies far below the
    blast's speed and is skipped; dt after every step and the final state
    equal the unfiltered packet path bit for bit."""
    spec = wl.MeshSpec(ndim=3, nb=(4, 4, 4), bs=(16, 16, 16))
    U0 = wl.sedov_state(spec)
    if task == B.ORCHA_TASK_HYDRO_RK2:
        spec = dataclasses.replace(spec, cfl=0.4)
    A, da, ea = _packet_steps(spec, U0, task, 8)
    G, dg, eg = _batch_steps(spec, U0, task, 8)
    assert ea == 0 and eg == 0
    assert np.array_equal(da, dg), (da, dg)
    assert np.array_equal(A, G)


@pytest.mark.parametrize("task", TASKS)
def test_random_state_bitwise(task):
    """Random jumps (speeds of every size in every block), graph-captured."""
    spec = wl.MeshSpec(ndim=3, nb=(3, 2, 2), bs=(16, 16, 16), periodic=(1, 0, 1),
                       cfl=0.4 if task == B.ORCHA_TASK_HYDRO_RK2 else wl.CFL)
    U0 = wl.random_blocky_state(spec, 23)
    A, da, _ = _packet_steps(spec, U0, task, 4)
    G, dg, _ = _batch_steps(spec, U0, task, 4, use_graph=True)
    assert np.array_equal(da, dg)
    assert np.array_equal(A, G)


@pytest.mark.parametrize("state", ["sedov", "random"])
def test_threshold_above_every_cell_falls_back(state):
    """A caller-written dt of 1e-12 puts the threshold (CFL / (4 dt)) above
    every cell's bound, so the step skips every FP64 speed; the reducer must
    find a skipped bound above the (empty) maximum and evaluate the blocks in
    FP64. Without that the step would end with no maximum (BAD_DT)."""
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16))
    U0 = wl.sedov_state(spec) if state == "sedov" else wl.random_blocky_state(spec, 9)
    A, da, ea = _packet_steps(spec, U0, B.ORCHA_TASK_HYDRO_FP64, 1, dt0=1e-12)
    G, dg, eg = _batch_steps(spec, U0, B.ORCHA_TASK_HYDRO_FP64, 1, dt0=1e-12)
    assert ea == 0 and eg == 0
    assert np.array_equal(da, dg)
    assert np.array_equal(A, G)


@pytest.mark.parametrize("task", [B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_FF])
def test_first_dt_mixed_bounds_bitwise(task):
    """The filtered first time step on a state whose cells take every branch:
    fast cells whose pressure is below 2^-40 of their energy (no FP32 bounds:
    evaluated in FP64 by the first pass), a two-state jump whose faster half
    ties at the maximum (every cell of it evaluated), and a slow background
    (skipped). The first dt and two steps equal the unfiltered packet path
    bit for bit; with the fast cells (first dt only: their near-vacuum jet is
    not meant to be stepped) the largest speed lies among the cells without
    bounds, without them among the tied ones."""
    spec = wl.MeshSpec(ndim=3, nb=(3, 2, 2), bs=(8, 8, 8))
    for fast in (True, False):
        U0 = wl.uniform_state(spec, 1.0, (0.0, 0.0, 0.0), 1.0)
        U0[:6, 4] = 10.0 / 0.4                       # blocks 0..5: p = 10, the faster half
        if fast:
            rho, u, p = 1.0, 30.0, 1.0e-12           # p / E ~ 2e-15: no FP32 bounds
            U0[7, :, 2:4, 3, 5] = 0.0
            U0[7, 0, 2:4, 3, 5] = rho
            U0[7, 2, 2:4, 3, 5] = rho * u
            U0[7, 4, 2:4, 3, 5] = p / 0.4 + 0.5 * rho * u * u
        n = 0 if fast else 2
        A, da, ea = _packet_steps(spec, U0, task, n)
        G, dg, eg = _batch_steps(spec, U0, task, n)
        assert len(da) == n + 1
        assert ea == 0 and eg == 0
        assert np.array_equal(da, dg), (fast, da, dg)
        assert np.array_equal(A, G)


def test_2d_sod_bitwise():
    """2D (the sweep's single-plane form): Sod, whose two states' speeds are
    within a factor 1.2, so every cell is evaluated; still bitwise."""
    spec = wl.sod_spec(64, 8)
    U0 = wl.sod_state(spec)
    A, da, _ = _packet_steps(spec, U0, B.ORCHA_TASK_HYDRO_FP64, 6)
    G, dg, _ = _batch_steps(spec, U0, B.ORCHA_TASK_HYDRO_FP64, 6)
    assert np.array_equal(da, dg)
    assert np.array_equal(A, G)
