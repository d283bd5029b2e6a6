"""Thin ctypes binding of liborcha.so (include/orcha.h), same names.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. PyTorch provides device memory (the two state buffers and dt) and
streams. If the library is missing the import of :func:`lib` raises; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
# ORCHA_LIBRARY_VARIANT=exact loads liborcha_exact.so, the build in which every
# FP64 operation is one unfused round-to-nearest operation
LIB_PATH = os.path.join(HERE, {"": "liborcha.so", "default": "liborcha.so",
                               "exact": "liborcha_exact.so"}[os.environ.get("ORCHA_LIBRARY_VARIANT", "")])

ORCHA_OK = 0
ORCHA_ERR_INVALID = -1
ORCHA_ERR_OOM = -2
ORCHA_ERR_CUDA = -3
ORCHA_ERR_TIMEOUT = -4
ORCHA_ERR_NONFINITE = -5
ORCHA_ERR_UNSUPPORTED = -6

ORCHA_DEVERR_NONPHYSICAL = 1
ORCHA_DEVERR_BAD_DT = 2
ORCHA_DEVERR_CFL = 8

ORCHA_TASK_GUARD_FILL = 0
ORCHA_TASK_HYDRO_FP64 = 1
ORCHA_TASK_HYDRO_F32FLUX = 2
ORCHA_TASK_SIGNAL_SPEED = 3
ORCHA_TASK_HYDRO_FF = 4
ORCHA_TASK_RK2_STAGE1 = 5
ORCHA_TASK_RK2_STAGE2 = 6
ORCHA_TASK_HYDRO_RK2 = 7
ORCHA_TASK_RK2_F32FLUX_STAGE1 = 8
ORCHA_TASK_RK2_F32FLUX_STAGE2 = 9
ORCHA_TASK_HYDRO_RK2_F32FLUX = 10
ORCHA_TASK_RK2_FF_STAGE1 = 11
ORCHA_TASK_RK2_FF_STAGE2 = 12
ORCHA_TASK_HYDRO_RK2_FF = 13
ORCHA_TASK_HYDRO_F32FLUX_FFSUM = 14
ORCHA_TASK_HYDRO_TB2 = 15
ORCHA_TASK_HYDRO_F32FLUX_TB2 = 16
ORCHA_TASK_HYDRO_RK2_FUSED = 17
ORCHA_TASK_HYDRO_RK2_F32FLUX_FUSED = 18

ORCHA_INIT_FROM_HOST = 0
ORCHA_INIT_SPHERE = 1
ORCHA_INIT_HALF_SPACE = 2

TASKS = {"fp64": ORCHA_TASK_HYDRO_FP64, "f32flux": ORCHA_TASK_HYDRO_F32FLUX, "ff": ORCHA_TASK_HYDRO_FF,
         "f32flux_ffsum": ORCHA_TASK_HYDRO_F32FLUX_FFSUM,
         "tb2": ORCHA_TASK_HYDRO_TB2, "tb2_f32": ORCHA_TASK_HYDRO_F32FLUX_TB2,
         "rk2_fused": ORCHA_TASK_HYDRO_RK2_FUSED, "rk2_fused_f32": ORCHA_TASK_HYDRO_RK2_F32FLUX_FUSED,
         "rk2": ORCHA_TASK_HYDRO_RK2, "rk2_f32": ORCHA_TASK_HYDRO_RK2_F32FLUX, "rk2_ff": ORCHA_TASK_HYDRO_RK2_FF}


class OrchaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"orcha status {status}: {msg}")
        self.status = status


class orcha_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("nb", ctypes.c_int32 * 3),
        ("bs", ctypes.c_int32 * 3),
        ("periodic", ctypes.c_int32 * 3),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("state_dev", ctypes.c_void_p * 2),
        ("dt_dev", ctypes.c_void_p),
    ]


class orcha_request_desc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32), ("nb", ctypes.c_int32 * 3), ("bs", ctypes.c_int32 * 3),
        ("periodic", ctypes.c_int32 * 3), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("nsteps", ctypes.c_int32),
        ("task", ctypes.c_int32), ("init_kind", ctypes.c_int32), ("region", ctypes.c_int32 * 4),
        ("u_in", ctypes.c_double * 5), ("u_out", ctypes.c_double * 5),
        ("init_host", ctypes.c_void_p), ("out_host", ctypes.c_void_p),
    ]


class orcha_request_stats(ctypes.Structure):
    _fields_ = [
        ("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double), ("t_ready_us", ctypes.c_double),
        ("t_done_us", ctypes.c_double), ("zone_updates", ctypes.c_int64), ("totals", ctypes.c_double * 5),
        ("dt_next", ctypes.c_double), ("device_error", ctypes.c_int32), ("status", ctypes.c_int32),
    ]


class orcha_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("steps_launched", ctypes.c_int64),
        ("zone_updates", ctypes.c_int64), ("now_us", ctypes.c_double), ("pool_bytes", ctypes.c_size_t),
        ("pool_peak_bytes", ctypes.c_size_t),
    ]


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_st = ctypes.c_int32

# name -> (restype, argtypes), in the order of include/orcha.h
SIGNATURES = {
    "orcha_state_elems": (ctypes.c_size_t, [ctypes.POINTER(orcha_mesh_desc)]),
    "orcha_mesh_create": (_st, [ctypes.POINTER(orcha_mesh_desc), ctypes.POINTER(_vp)]),
    "orcha_mesh_destroy": (_st, [_vp]),
    "orcha_mesh_current": (_i32, [_vp]),
    "orcha_mesh_swap": (_st, [_vp]),
    "orcha_mesh_set_tile": (_st, [_vp, _i32, _i32]),
    "orcha_mesh_get_tile": (_st, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "orcha_mesh_load": (_st, [_vp, _vp, _i32, _vp]),
    "orcha_mesh_store": (_st, [_vp, _vp, _i32, _vp]),
    "orcha_mesh_init_region": (_st, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), _vp]),
    "orcha_packet_create": (_st, [_vp, ctypes.POINTER(_i32), _i32, ctypes.POINTER(_vp)]),
    "orcha_packet_destroy": (_st, [_vp]),
    "orcha_packet_run": (_st, [_vp, ctypes.c_int, _vp]),
    "orcha_packet_unpack": (_st, [_vp, _vp, _i32, _vp]),
    "orcha_packet_pack": (_st, [_vp, _vp, _i32, _vp]),
    "orcha_dt_reduce": (_st, [_vp, _vp]),
    "orcha_mesh_advance": (_st, [_vp, ctypes.POINTER(_vp), _i32, ctypes.c_int, _i32, _i32, _i32, _vp]),
    "orcha_batch_create": (_st, [ctypes.POINTER(_vp), _i32, _i32, _i32, ctypes.POINTER(_vp)]),
    "orcha_batch_destroy": (_st, [_vp]),
    "orcha_batch_advance": (_st, [_vp, ctypes.c_int, _i32, _i32, _i32, _vp]),
    "orcha_server_create": (_st, [ctypes.c_size_t, _i32, ctypes.POINTER(_vp)]),
    "orcha_server_destroy": (_st, [_vp]),
    "orcha_server_submit": (_st, [_vp, ctypes.POINTER(orcha_request_desc), ctypes.POINTER(ctypes.c_int64)]),
    "orcha_server_wait": (_st, [_vp, ctypes.c_int64, _i32, ctypes.POINTER(orcha_request_stats)]),
    "orcha_server_get_stats": (_st, [_vp, ctypes.POINTER(orcha_server_stats)]),
    "orcha_autotune": (_st, [_i32, ctypes.POINTER(_i32), ctypes.c_int, _i32, ctypes.c_char_p, ctypes.POINTER(_i32),
                             ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)]),
    "orcha_cfl_dt_noalloc": (_st, [ctypes.POINTER(orcha_mesh_desc), _i32, _vp, _vp]),
    "orcha_mesh_poll": (_st, [_vp, _vp, ctypes.POINTER(_i32)]),
    "orcha_selftest_conversions": (_st, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "orcha_selftest_fp64_emulation": (_st, [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "orcha_selftest_dword": (_st, [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "orcha_selftest_speed_bound": (_st, [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_double)]),
    "orcha_measure_fp64_rate": (_st, [_i32, ctypes.POINTER(ctypes.c_double)]),
    "orcha_amr_fine_elems": (ctypes.c_size_t, [ctypes.POINTER(orcha_mesh_desc), _i32]),
    "orcha_amr_create": (_st, [ctypes.POINTER(orcha_mesh_desc), ctypes.POINTER(_i32), _i32, _vp, _vp,
                               ctypes.POINTER(_vp)]),
    "orcha_amr_destroy": (_st, [_vp]),
    "orcha_amr_load": (_st, [_vp, _vp, _vp, _i32, _vp]),
    "orcha_amr_store": (_st, [_vp, _vp, _vp, _i32, _vp]),
    "orcha_amr_advance": (_st, [_vp, _i32, _i32, _vp]),
    "orcha_amr_poll": (_st, [_vp, _vp, ctypes.POINTER(_i32)]),
    "orcha_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load liborcha.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2507_09337_b300.build`"
                              + (" --exact" if LIB_PATH.endswith("_exact.so") else ""))
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != ORCHA_OK:
        raise OrchaError(status, lib().orcha_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------- same-name wrappers

def orcha_state_elems(desc: orcha_mesh_desc) -> int:
    return int(lib().orcha_state_elems(ctypes.byref(desc)))


def orcha_mesh_create(desc: orcha_mesh_desc) -> int:
    h = _vp()
    _check(lib().orcha_mesh_create(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def orcha_mesh_destroy(mesh: int) -> None:
    _check(lib().orcha_mesh_destroy(mesh))


def orcha_mesh_current(mesh: int) -> int:
    return int(lib().orcha_mesh_current(mesh))


def orcha_mesh_swap(mesh: int) -> None:
    _check(lib().orcha_mesh_swap(mesh))


def orcha_mesh_set_tile(mesh: int, tx: int, ty: int) -> None:
    _check(lib().orcha_mesh_set_tile(mesh, tx, ty))


def orcha_mesh_get_tile(mesh: int) -> tuple:
    tx, ty = _i32(), _i32()
    _check(lib().orcha_mesh_get_tile(mesh, ctypes.byref(tx), ctypes.byref(ty)))
    return tx.value, ty.value


def orcha_mesh_load(mesh: int, interior_ptr: int, host_ptr: bool, stream=None) -> None:
    _check(lib().orcha_mesh_load(mesh, interior_ptr, int(bool(host_ptr)), _stream_ptr(stream)))


def orcha_mesh_store(mesh: int, interior_ptr: int, host_ptr: bool, stream=None) -> None:
    _check(lib().orcha_mesh_store(mesh, interior_ptr, int(bool(host_ptr)), _stream_ptr(stream)))


def orcha_mesh_init_region(mesh: int, kind: int, region, u_in, u_out, stream=None) -> None:
    r = (_i32 * 4)(*[int(x) for x in region])
    a = (ctypes.c_double * 5)(*[float(x) for x in u_in])
    b = (ctypes.c_double * 5)(*[float(x) for x in u_out])
    _check(lib().orcha_mesh_init_region(mesh, int(kind), r, a, b, _stream_ptr(stream)))


def orcha_packet_create(mesh: int, block_ids) -> int:
    ids = np.ascontiguousarray(block_ids, dtype=np.int32)
    h = _vp()
    _check(lib().orcha_packet_create(mesh, ids.ctypes.data_as(ctypes.POINTER(_i32)), int(ids.size),
                                     ctypes.byref(h)))
    return h.value


def orcha_packet_destroy(packet: int) -> None:
    _check(lib().orcha_packet_destroy(packet))


def orcha_packet_run(packet: int, task: int, stream=None) -> None:
    _check(lib().orcha_packet_run(packet, int(task), _stream_ptr(stream)))


def orcha_packet_unpack(packet: int, dst_ptr: int | None, dst_is_host: bool, stream=None) -> None:
    _check(lib().orcha_packet_unpack(packet, dst_ptr, int(bool(dst_is_host)), _stream_ptr(stream)))


def orcha_packet_pack(packet: int, src_ptr: int, src_is_host: bool, stream=None) -> None:
    _check(lib().orcha_packet_pack(packet, src_ptr, int(bool(src_is_host)), _stream_ptr(stream)))


def orcha_dt_reduce(mesh: int, stream=None) -> None:
    _check(lib().orcha_dt_reduce(mesh, _stream_ptr(stream)))


def orcha_mesh_advance(mesh: int, packets, task: int, nsteps: int, init_dt: bool, use_graph: bool,
                       stream=None) -> None:
    arr = (_vp * len(packets))(*packets)
    _check(lib().orcha_mesh_advance(mesh, arr, len(packets), int(task), int(nsteps), int(bool(init_dt)),
                                    int(bool(use_graph)), _stream_ptr(stream)))


def orcha_batch_create(packets, tx: int = 0, ty: int = 0) -> int:
    arr = (_vp * len(packets))(*packets)
    h = _vp()
    _check(lib().orcha_batch_create(arr, len(packets), tx, ty, ctypes.byref(h)))
    return h.value


def orcha_batch_destroy(batch: int) -> None:
    _check(lib().orcha_batch_destroy(batch))


def orcha_batch_advance(batch: int, task: int, nsteps: int, init_dt: bool, use_graph: bool, stream=None) -> None:
    _check(lib().orcha_batch_advance(batch, int(task), int(nsteps), int(bool(init_dt)), int(bool(use_graph)),
                                     _stream_ptr(stream)))


def orcha_server_create(hbm_budget_bytes: int, max_active: int = 1024) -> int:
    h = _vp()
    _check(lib().orcha_server_create(int(hbm_budget_bytes), int(max_active), ctypes.byref(h)))
    return h.value


def orcha_server_destroy(server: int) -> None:
    _check(lib().orcha_server_destroy(server))


def orcha_server_submit(server: int, req: orcha_request_desc) -> int:
    t = ctypes.c_int64()
    _check(lib().orcha_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def orcha_server_wait(server: int, ticket: int, timeout_ms: int = -1) -> orcha_request_stats:
    st = orcha_request_stats()
    _check(lib().orcha_server_wait(server, int(ticket), int(timeout_ms), ctypes.byref(st)))
    return st


def orcha_server_get_stats(server: int) -> orcha_server_stats:
    st = orcha_server_stats()
    _check(lib().orcha_server_get_stats(server, ctypes.byref(st)))
    return st


DEFAULT_TUNE_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "orcha_b300", "tiles.json")


def orcha_autotune(ndim: int, bs, task: int, nblocks: int = 296, cache_path: str | None = DEFAULT_TUNE_CACHE):
    """Fastest (tx, ty, ms_per_step) tile for this block geometry and task."""
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    b = (_i32 * 3)(*[int(x) for x in bs])
    tx, ty, ms = _i32(), _i32(), ctypes.c_double()
    _check(lib().orcha_autotune(int(ndim), b, int(task), int(nblocks),
                                cache_path.encode() if cache_path else None,
                                ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(ms)))
    return tx.value, ty.value, ms.value


def orcha_cfl_dt_noalloc(desc: orcha_mesh_desc, current: int, err_dev_ptr: int, stream=None) -> None:
    """dt of desc.state_dev[current] into desc.dt_dev with no device allocation
    (see include/orcha.h)."""
    _check(lib().orcha_cfl_dt_noalloc(ctypes.byref(desc), int(current), err_dev_ptr, _stream_ptr(stream)))


def orcha_mesh_poll(mesh: int, stream=None) -> int:
    """Wait for the stream and return the device error word (raises if set)."""
    err = _i32()
    _check(lib().orcha_mesh_poll(mesh, _stream_ptr(stream), ctypes.byref(err)))
    return err.value


def orcha_selftest_conversions(first_pattern: int, count: int, seed: int = 1) -> int:
    bad = ctypes.c_uint64()
    _check(lib().orcha_selftest_conversions(int(first_pattern), int(count), int(seed), ctypes.byref(bad)))
    return bad.value


def orcha_selftest_fp64_emulation(count: int, seed: int = 1) -> int:
    bad = ctypes.c_uint64()
    _check(lib().orcha_selftest_fp64_emulation(int(count), int(seed), ctypes.byref(bad)))
    return bad.value


def orcha_selftest_dword(count: int, seed: int = 1) -> list:
    err = (ctypes.c_double * 6)()
    _check(lib().orcha_selftest_dword(int(count), int(seed), err))
    return list(err)


def orcha_selftest_speed_bound(count: int, seed: int = 1) -> tuple:
    """(states where the bound lies below the FP64 speed, states where it
    applied, states where it applied to a non-physical state, largest
    bound / speed ratio)."""
    counts = (ctypes.c_uint64 * 3)()
    ratio = ctypes.c_double()
    _check(lib().orcha_selftest_speed_bound(int(count), int(seed), counts, ctypes.byref(ratio)))
    return counts[0], counts[1], counts[2], ratio.value


def orcha_measure_fp64_rate(op: int = 0) -> float:
    """FP64 pipe throughput of the current device in lane operations/s
    (op 0 FMA, 1 add, 2 multiply)."""
    r = ctypes.c_double()
    _check(lib().orcha_measure_fp64_rate(int(op), ctypes.byref(r)))
    return r.value


def orcha_amr_fine_elems(desc: orcha_mesh_desc, nref: int) -> int:
    return int(lib().orcha_amr_fine_elems(ctypes.byref(desc), int(nref)))


def orcha_amr_create(desc: orcha_mesh_desc, refined, fine0_ptr: int, fine1_ptr: int) -> int:
    ids = np.ascontiguousarray(refined, dtype=np.int32)
    h = _vp()
    _check(lib().orcha_amr_create(ctypes.byref(desc), ids.ctypes.data_as(ctypes.POINTER(_i32)), len(ids),
                                  fine0_ptr, fine1_ptr, ctypes.byref(h)))
    return h.value


def orcha_amr_destroy(amr: int) -> None:
    _check(lib().orcha_amr_destroy(amr))


def orcha_amr_load(amr: int, coarse_ptr: int, fine_ptr: int | None, host_ptr: bool, stream=None) -> None:
    _check(lib().orcha_amr_load(amr, coarse_ptr, fine_ptr, int(bool(host_ptr)), _stream_ptr(stream)))


def orcha_amr_store(amr: int, coarse_ptr: int, fine_ptr: int | None, host_ptr: bool, stream=None) -> None:
    _check(lib().orcha_amr_store(amr, coarse_ptr, fine_ptr, int(bool(host_ptr)), _stream_ptr(stream)))


def orcha_amr_advance(amr: int, nsteps: int, init_dt: bool, stream=None) -> None:
    _check(lib().orcha_amr_advance(amr, int(nsteps), int(bool(init_dt)), _stream_ptr(stream)))


def orcha_amr_poll(amr: int, stream=None) -> int:
    err = _i32()
    _check(lib().orcha_amr_poll(amr, _stream_ptr(stream), ctypes.byref(err)))
    return err.value


def orcha_last_error() -> str:
    return lib().orcha_last_error().decode()


# ---------------------------------------------------------------- torch-owned mesh

class Mesh:
    """A mesh whose two state buffers and dt are torch tensors on one CUDA
    device; wraps the handle and its packets."""

    def __init__(self, spec: wl.MeshSpec, device: str = "cuda:0", packets=None):
        import torch
        self.spec = spec
        self.device = torch.device(device)
        d = orcha_mesh_desc()
        d.ndim = spec.ndim
        for a in range(3):
            d.nb[a] = spec.nb[a]
            d.bs[a] = spec.bs[a]
            d.periodic[a] = spec.periodic[a]
            d.lo[a] = spec.lo[a]
            d.hi[a] = spec.hi[a]
        d.gamma = spec.gamma
        d.cfl = spec.cfl
        n = orcha_state_elems(d)
        if n == 0:
            raise OrchaError(ORCHA_ERR_INVALID, "invalid mesh geometry")
        with torch.cuda.device(self.device):
            self.state = [torch.zeros(n, dtype=torch.float64, device=self.device) for _ in range(2)]
            self.dt = torch.zeros(1, dtype=torch.float64, device=self.device)
            d.state_dev[0] = self.state[0].data_ptr()
            d.state_dev[1] = self.state[1].data_ptr()
            d.dt_dev = self.dt.data_ptr()
            self.desc = d
            self.handle = orcha_mesh_create(d)
        self.packets = []
        if packets is None:
            packets = [np.arange(spec.nblocks, dtype=np.int32)]
        for ids in packets:
            self.packets.append(orcha_packet_create(self.handle, ids))

    def close(self):
        if getattr(self, "handle", None):
            for p in self.packets:
                orcha_packet_destroy(p)
            self.packets = []
            orcha_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, U, stream=None):
        """Copy an interior block array (numpy host array or CUDA tensor) in."""
        import torch
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64)
            assert U.shape == self.spec.block_shape()
            self._host_keep = torch.from_numpy(U).pin_memory()
            orcha_mesh_load(self.handle, self._host_keep.data_ptr(), True, stream)
        else:
            assert U.is_cuda and U.dtype == torch.float64 and U.is_contiguous()
            orcha_mesh_load(self.handle, U.data_ptr(), False, stream)

    def store(self, out=None, stream=None):
        """Copy the current interiors out; returns a numpy array (host) or fills
        `out` (a CUDA tensor of the block shape)."""
        import torch
        if out is not None:
            orcha_mesh_store(self.handle, out.data_ptr(), False, stream)
            return out
        host = torch.empty(self.spec.block_shape(), dtype=torch.float64).pin_memory()
        orcha_mesh_store(self.handle, host.data_ptr(), True, stream)
        torch.cuda.current_stream(self.device).synchronize() if stream is None else stream.synchronize()
        return host.numpy().copy()

    def run(self, task, stream=None):
        for p in self.packets:
            orcha_packet_run(p, task, stream)

    def advance(self, nsteps: int, task=ORCHA_TASK_HYDRO_FP64, init_dt: bool = True, use_graph: bool = False,
                stream=None):
        orcha_mesh_advance(self.handle, self.packets, task, nsteps, init_dt, use_graph, stream)

    def poll(self, stream=None) -> int:
        return orcha_mesh_poll(self.handle, stream)

    def set_tile(self, tx: int, ty: int):
        orcha_mesh_set_tile(self.handle, tx, ty)

    def dt_value(self) -> float:
        return float(self.dt.item())


class AmrMesh:
    """A two-level mesh (orcha_amr_*) whose coarse and fine state buffers and
    dt are torch tensors on one CUDA device."""

    def __init__(self, spec: wl.MeshSpec, refined, device: str = "cuda:0"):
        import torch
        self.spec = spec
        self.refined = np.ascontiguousarray(refined, dtype=np.int32)
        self.coarse = Mesh(spec, device=device)
        self.device = self.coarse.device
        n1 = orcha_amr_fine_elems(self.coarse.desc, len(self.refined))
        with torch.cuda.device(self.device):
            self.fine = [torch.zeros(max(n1, 2), dtype=torch.float64, device=self.device) for _ in range(2)]
        # the AMR object makes its own coarse-level mesh over the same buffers
        self.handle = orcha_amr_create(self.coarse.desc, self.refined, self.fine[0].data_ptr(),
                                       self.fine[1].data_ptr())

    @property
    def nfine(self) -> int:
        return len(self.refined) << self.spec.ndim

    def close(self):
        if getattr(self, "handle", None):
            orcha_amr_destroy(self.handle)
            self.handle = None
        if getattr(self, "coarse", None) is not None:
            self.coarse.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, U0: np.ndarray, U1: np.ndarray):
        import torch
        a = torch.from_numpy(np.ascontiguousarray(U0, dtype=np.float64)).pin_memory()
        b = torch.from_numpy(np.ascontiguousarray(U1, dtype=np.float64)).pin_memory()
        orcha_amr_load(self.handle, a.data_ptr(), b.data_ptr() if self.nfine else None, True)

    def store(self):
        import torch
        a = torch.empty(self.spec.block_shape(), dtype=torch.float64).pin_memory()
        b = torch.empty((self.nfine,) + self.spec.block_shape()[1:], dtype=torch.float64).pin_memory()
        orcha_amr_store(self.handle, a.data_ptr(), b.data_ptr() if self.nfine else None, True)
        return a.numpy().copy(), b.numpy().copy()

    def advance(self, nsteps: int, init_dt: bool = True, stream=None):
        orcha_amr_advance(self.handle, nsteps, init_dt, stream)

    def poll(self, stream=None) -> int:
        return orcha_amr_poll(self.handle, stream)

    def dt_value(self) -> float:
        return float(self.coarse.dt.item())
