"""Packing and unpacking one data packet (orcha_packet_pack / _unpack): the
interiors of the packet's blocks in packet order, to and from host or device
memory, equal the corresponding blocks of the whole-mesh copy; the other
blocks are untouched; unpacking to NULL is a no-op (state stays resident)."""
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


def _ragged_packets(n, seed):
    rng = np.random.default_rng(seed)
    ids = rng.permutation(n).astype(np.int32)
    cuts = np.sort(rng.choice(np.arange(1, n), size=3, replace=False))
    return np.split(ids, cuts)


@pytest.mark.parametrize("ndim,nb,bs", [(3, (3, 2, 2), (8, 8, 8)), (2, (4, 3, 1), (16, 8, 1))])
def test_unpack_equals_the_packet_blocks_after_steps(ndim, nb, bs):
    import torch
    spec = wl.MeshSpec(ndim=ndim, nb=nb, bs=bs)
    U0 = wl.random_blocky_state(spec, 5)
    packets = _ragged_packets(spec.nblocks, 8)
    mesh = B.Mesh(spec, packets=packets)
    st = torch.cuda.current_stream()
    try:
        mesh.load(U0)
        mesh.advance(2, B.ORCHA_TASK_HYDRO_FP64, init_dt=True)
        full = mesh.store()
        for h, ids in zip(mesh.packets, packets):
            shape = (len(ids),) + spec.block_shape()[1:]
            host = torch.empty(shape, dtype=torch.float64).pin_memory()
            dev = torch.empty(shape, dtype=torch.float64, device="cuda")
            B.orcha_packet_unpack(h, host.data_ptr(), True, st)
            B.orcha_packet_unpack(h, dev.data_ptr(), False, st)
            B.orcha_packet_unpack(h, None, True, st)           # resident: nothing to move
            st.synchronize()
            assert np.array_equal(host.numpy(), full[ids])
            assert np.array_equal(dev.cpu().numpy(), full[ids])
    finally:
        mesh.close()


def test_pack_writes_only_the_packet_blocks():
    import torch
    spec = wl.MeshSpec(ndim=3, nb=(3, 2, 2), bs=(8, 8, 8))
    U0 = wl.random_blocky_state(spec, 6)
    packets = _ragged_packets(spec.nblocks, 9)
    mesh = B.Mesh(spec, packets=packets)
    st = torch.cuda.current_stream()
    try:
        mesh.load(U0)
        ids = packets[1]
        new = np.ascontiguousarray(1.5 * U0[ids])
        host = torch.from_numpy(new).pin_memory()
        B.orcha_packet_pack(mesh.packets[1], host.data_ptr(), True, st)
        got = mesh.store()
        want = U0.copy()
        want[ids] = new
        assert np.array_equal(got, want)
        dev = torch.from_numpy(np.ascontiguousarray(U0[packets[2]])).cuda()
        B.orcha_packet_pack(mesh.packets[2], dev.data_ptr(), False, st)
        B.orcha_packet_pack(mesh.packets[1], torch.from_numpy(np.ascontiguousarray(U0[ids])).cuda().data_ptr(),
                            False, st)
        assert np.array_equal(mesh.store(), U0)
        with pytest.raises(B.OrchaError):
            B.orcha_packet_pack(mesh.packets[0], None, True, st)
    finally:
        mesh.close()
