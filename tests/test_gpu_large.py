"""A mesh past 2^31 state elements: 65,536 blocks of 16^3 (512 x 512 x 1024
cells, 268 M zones; 21 GB per padded state buffer), where global offsets no
longer fit in 32 bits. The initial states are built on the device (a host
copy would need 10.7 GB); the checks are properties that hold at any size:
a free stream stays bitwise, the persistent batch path gives the packet
path's bits, and a periodic mesh conserves its totals."""
import math

import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

pytestmark = pytest.mark.gpu
NB = (32, 32, 64)
BS = (16, 16, 16)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def _spec():
    return wl.MeshSpec(ndim=3, nb=NB, bs=BS, periodic=(1, 1, 1))


def _smooth_state(spec):
    """Periodic smooth state, cell centres from block and cell indices:
    rho = 1 + 0.2 sin(2 pi x) sin(2 pi y), velocities of 0.1 - 0.3 varying
    along the other axes, p = 1 + 0.1 cos(2 pi (x + z))."""
    import torch
    dev = torch.device("cuda")
    nbx, nby, nbz = spec.nb
    bs = spec.bs
    b = torch.arange(spec.nblocks, device=dev, dtype=torch.int64)

    def coord(bidx, a, shape):
        i = torch.arange(bs[a], device=dev, dtype=torch.float64)
        return ((bidx.to(torch.float64)[:, None] * bs[a] + i[None, :] + 0.5) / (spec.nb[a] * bs[a])).reshape(shape)

    x = coord(b % nbx, 0, (-1, 1, 1, bs[0]))
    y = coord((b // nbx) % nby, 1, (-1, 1, bs[1], 1))
    z = coord(b // (nbx * nby), 2, (-1, bs[2], 1, 1))
    tp = 2.0 * math.pi
    rho = 1.0 + 0.2 * torch.sin(tp * x) * torch.sin(tp * y)
    u = 0.3 * torch.sin(tp * y) + 0.0 * z
    v = 0.2 * torch.cos(tp * z) + 0.0 * x
    w = 0.1 * torch.sin(tp * x) + 0.0 * y
    p = 1.0 + 0.1 * torch.cos(tp * (x + z))
    U = torch.empty(spec.block_shape(), dtype=torch.float64, device=dev)
    U[:, 0] = rho
    U[:, 1] = rho * u
    U[:, 2] = rho * v
    U[:, 3] = rho * w
    U[:, 4] = p / (spec.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return U


def _run(spec, U0, path):
    """One FP64 step through the persistent batch or the packet path; returns
    the new interiors (device) and frees the mesh."""
    import torch
    ids = torch.arange(spec.nblocks, dtype=torch.int32).numpy()
    mesh = B.Mesh(spec, packets=[ids[k:k + 4096] for k in range(0, spec.nblocks, 4096)])
    try:
        mesh.load(U0)
        if path == "batch":
            batch = B.orcha_batch_create(mesh.packets)
            try:
                B.orcha_batch_advance(batch, B.ORCHA_TASK_HYDRO_FP64, 1, True, False)
            finally:
                B.orcha_batch_destroy(batch)
        else:
            mesh.advance(1, B.ORCHA_TASK_HYDRO_FP64)
        assert mesh.poll() == 0
        out = torch.empty_like(U0)
        mesh.store(out)
        torch.cuda.synchronize()
        return out
    finally:
        mesh.close()
        del mesh
        torch.cuda.empty_cache()


def test_state_is_past_32_bit_offsets():
    d = B.orcha_mesh_desc()
    d.ndim = 3
    for a in range(3):
        d.nb[a], d.bs[a], d.periodic[a], d.hi[a] = NB[a], BS[a], 1, 1.0
    d.gamma, d.cfl = 1.4, 0.8
    assert B.orcha_state_elems(d) > 2 ** 31


def test_free_stream_stays_bitwise():
    import torch
    spec = _spec()
    U0 = torch.empty(spec.block_shape(), dtype=torch.float64, device="cuda")
    rho, vel, p = 1.3, (0.4, -0.25, 0.15), 0.9
    U0[:, 0] = rho
    for k in range(3):
        U0[:, 1 + k] = rho * vel[k]
    U0[:, 4] = p / (spec.gamma - 1.0) + 0.5 * rho * sum(c * c for c in vel)
    out = _run(spec, U0, "batch")
    assert torch.equal(out, U0)


def test_batch_equals_packet_path_and_conserves():
    import torch
    spec = _spec()
    U0 = _smooth_state(spec)
    A = _run(spec, U0, "batch")
    G = _run(spec, U0, "packets")
    assert torch.equal(A, G)
    s0 = U0.sum(dim=(0, 2, 3, 4))
    s1 = A.sum(dim=(0, 2, 3, 4))
    scale = U0.abs().sum(dim=(0, 2, 3, 4))
    scale[1:4] = torch.maximum(scale[1:4], U0[:, 0].sum())
    assert bool(torch.all((s1 - s0).abs() <= 1e-13 * scale)), ((s1 - s0) / scale).tolist()
    assert not torch.equal(A, U0)


def test_one_packet_of_65536_blocks():
    """A packet of more blocks than one launch has grid rows (65,535): the
    packet path fills its guards over several launches and matches the
    persistent batch bit for bit (8^3 blocks, 64 x 32 x 32 of them)."""
    import torch
    spec = wl.MeshSpec(ndim=3, nb=(64, 32, 32), bs=(8, 8, 8), periodic=(1, 1, 1))
    U0 = _smooth_state(spec)
    outs = []
    for path in ("batch", "packets"):
        mesh = B.Mesh(spec)                  # one packet of every block
        try:
            assert len(mesh.packets) == 1 and spec.nblocks == 65536
            mesh.load(U0)
            if path == "batch":
                batch = B.orcha_batch_create(mesh.packets)
                try:
                    B.orcha_batch_advance(batch, B.ORCHA_TASK_HYDRO_FP64, 2, True, False)
                finally:
                    B.orcha_batch_destroy(batch)
            else:
                mesh.advance(2, B.ORCHA_TASK_HYDRO_FP64)
            assert mesh.poll() == 0
            out = torch.empty_like(U0)
            mesh.store(out)
            torch.cuda.synchronize()
            outs.append(out)
        finally:
            mesh.close()
    assert torch.equal(outs[0], outs[1]) and not torch.equal(outs[0], U0)
