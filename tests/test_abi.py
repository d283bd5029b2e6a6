"""The C-ABI library loads and exports every function include/orcha.h declares;
host-side argument checks. No GPU needed (no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import build as pkgbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*ORCHA_API\s+[^(;]*?\b(orcha_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    pkgbuild.build()
    return B.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_the_header():
    assert sorted(B.SIGNATURES) == declared_functions()


def test_only_the_abi_is_exported(L):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert {s for s in syms if s.startswith("orcha_")} == set(declared_functions())


def test_exact_build_exports_the_same_abi():
    """The exact-FP64 library variant (every FP64 operation unfused) is the
    same C ABI."""
    import subprocess
    path = pkgbuild.build(variant="exact")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert {s for s in syms if s.startswith("orcha_")} == set(declared_functions())


def _desc(**kw):
    d = B.orcha_mesh_desc()
    d.ndim = kw.get("ndim", 3)
    nb, bs = kw.get("nb", (2, 2, 2)), kw.get("bs", (16, 16, 16))
    for a in range(3):
        d.nb[a], d.bs[a] = nb[a], bs[a]
        d.lo[a], d.hi[a] = 0.0, 1.0
    d.gamma, d.cfl = kw.get("gamma", 1.4), 0.8
    return d


def test_state_elems_counts_padded_cells(L):
    assert B.orcha_state_elems(_desc()) == 8 * 5 * 20 ** 3
    assert B.orcha_state_elems(_desc(ndim=2, nb=(8, 8, 1), bs=(8, 8, 1))) == 64 * 4 * 12 * 12
    assert B.orcha_state_elems(_desc(ndim=4)) == 0


@pytest.mark.parametrize("kw,msg", [
    (dict(ndim=4), "ndim"),
    (dict(bs=(12, 16, 16)), "bs[0]"),
    # the kernels split a block's cell index by masks and shifts: only 8, 16 or 32
    (dict(bs=(16, 24, 16)), "bs[1]"),
    (dict(bs=(16, 16, 64)), "bs[2]"),
    (dict(bs=(4, 16, 16)), "bs[0]"),
    (dict(ndim=2, nb=(2, 2, 2), bs=(8, 8, 1)), "2D"),
    (dict(gamma=1.0), "gamma"),
])
def test_mesh_create_rejects_bad_geometry(L, kw, msg):
    d = _desc(**kw)
    d.state_dev[0], d.state_dev[1], d.dt_dev = 256, 512, 1024      # never dereferenced: rejected first
    h = ctypes.c_void_p()
    st = L.orcha_mesh_create(ctypes.byref(d), ctypes.byref(h))
    assert st == B.ORCHA_ERR_INVALID and h.value is None
    assert msg in B.orcha_last_error()


def test_mesh_create_rejects_missing_buffers(L):
    d = _desc()
    h = ctypes.c_void_p()
    assert L.orcha_mesh_create(ctypes.byref(d), ctypes.byref(h)) == B.ORCHA_ERR_INVALID
    d.state_dev[0], d.state_dev[1], d.dt_dev = 256, 256, 1024
    assert L.orcha_mesh_create(ctypes.byref(d), ctypes.byref(h)) == B.ORCHA_ERR_INVALID
    d.state_dev[0], d.state_dev[1], d.dt_dev = 256, 516, 1024
    assert L.orcha_mesh_create(ctypes.byref(d), ctypes.byref(h)) == B.ORCHA_ERR_INVALID
    assert "aligned" in B.orcha_last_error()
    d.state_dev[0], d.state_dev[1], d.dt_dev = 256, 520, 1024       # 8-byte but not 16-byte aligned
    assert L.orcha_mesh_create(ctypes.byref(d), ctypes.byref(h)) == B.ORCHA_ERR_INVALID
    assert "16-byte" in B.orcha_last_error()


def test_null_handles_are_rejected(L):
    assert L.orcha_packet_run(None, 0, None) == B.ORCHA_ERR_INVALID
    assert L.orcha_dt_reduce(None, None) == B.ORCHA_ERR_INVALID
    assert L.orcha_mesh_destroy(None) == B.ORCHA_OK
    assert L.orcha_mesh_current(None) == -1
