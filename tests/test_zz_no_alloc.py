"""The no-allocation CFL entry point (orcha_cfl_dt_noalloc) against the
existing path (SIGNAL_SPEED task + orcha_dt_reduce on a mesh).

Some callers of this library cannot let it allocate device memory (their own
allocator owns all of HBM, or allocation is forbidden in their time loop);
orcha_cfl_dt_noalloc serves them with a fixed file-scope device array as its
scratch. This file is collected last; it must pass alone in a fresh process
and after the other tests.
"""
import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def _reference_dt(mesh):
    """dt of the mesh's current buffer through the existing entry points."""
    mesh.run(B.ORCHA_TASK_SIGNAL_SPEED)
    B.orcha_dt_reduce(mesh.handle)
    assert mesh.poll() == 0
    return mesh.dt_value()


def _noalloc_dt(mesh, dt=None, err=None):
    """The same dt through the no-allocation entry point, written into a
    separate device scalar (the mesh's own dt is left alone)."""
    import torch
    if dt is None:
        dt = torch.empty(1, dtype=torch.float64, device=mesh.device)
        err = torch.empty(1, dtype=torch.int32, device=mesh.device)
    dt.fill_(-1.0)
    err.zero_()
    d = B.orcha_mesh_desc.from_buffer_copy(mesh.desc)
    d.dt_dev = dt.data_ptr()
    B.orcha_cfl_dt_noalloc(d, B.orcha_mesh_current(mesh.handle), err.data_ptr())
    torch.cuda.synchronize()
    return float(dt.item()), int(err.item())


def _check(mesh):
    """The entry point runs the mesh path's own signal-speed and reduction
    kernels on the same state, so the two dts agree bit for bit."""
    want = _reference_dt(mesh)
    got, err = _noalloc_dt(mesh)
    assert err == 0
    assert got == want, (got, want)
    return got


def test_two_calls_in_a_row_match_the_mesh_path():
    """Two calls in a row on meshes of different block counts (512, then 64
    blocks, then the first mesh again after a step): each equals the mesh
    path's dt, so no call sees the previous call's scratch."""
    spec_a, packets_a = wl.sedov128_packets(64)
    spec_b = wl.sod_spec(64, 8)
    a = B.Mesh(spec_a, packets=packets_a)
    b = B.Mesh(spec_b)
    try:
        a.load(wl.sedov_state(spec_a))
        b.load(wl.sod_state(spec_b))
        _check(a)
        _check(b)
        a.advance(1, B.ORCHA_TASK_HYDRO_FP64, init_dt=True)
        _check(a)
    finally:
        a.close()
        b.close()


def test_warm_calls_leave_free_device_memory_unchanged():
    """After a first call (which may load the library's device code and its
    fixed array), further calls allocate nothing: the device's free memory
    is the same before and after two of them (outputs preallocated)."""
    import torch
    spec, packets = wl.sedov128_packets(64)
    a = B.Mesh(spec, packets=packets)
    try:
        a.load(wl.sedov_state(spec))
        dt = torch.empty(1, dtype=torch.float64, device=a.device)
        err = torch.empty(1, dtype=torch.int32, device=a.device)
        first, _ = _noalloc_dt(a, dt, err)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info(a.device)
        second, e2 = _noalloc_dt(a, dt, err)
        third, e3 = _noalloc_dt(a, dt, err)
        free1, _ = torch.cuda.mem_get_info(a.device)
        assert free1 == free0, (free0, free1)
        assert first == second == third and e2 == e3 == 0
    finally:
        a.close()


def test_reports_nonphysical_state_and_rejects_oversized_meshes():
    spec = wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(8, 8, 8))
    U0 = wl.uniform_state(spec, 1.0, (0.0, 0.0, 0.0), 1.0)
    U0[0, 4, 1, 2, 3] = -1.0
    m = B.Mesh(spec)
    try:
        m.load(U0)
        _, err = _noalloc_dt(m)
        assert err & B.ORCHA_DEVERR_NONPHYSICAL
        big = B.orcha_mesh_desc.from_buffer_copy(m.desc)
        big.nb[0], big.nb[1], big.nb[2] = 64, 32, 33           # 67584 blocks > 65536
        with pytest.raises(B.OrchaError) as ei:
            B.orcha_cfl_dt_noalloc(big, 0, m.dt.data_ptr())
        assert ei.value.status == B.ORCHA_ERR_INVALID and "limit" in str(ei.value)
    finally:
        m.close()
