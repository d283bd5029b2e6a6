"""Continuous-batching server (orcha_server_*): each request's result is the
same alone and in the mix (bitwise), the device recipes give the numpy initial
states, admission waits for memory under a tight budget, and a served request
matches the oracle and the plain packet path."""
import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import serve
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import oracle_steps, rule12_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


def _requests(n, seed, max_blocks=8, sizes=(8, 16), nsteps=3):
    rng = np.random.default_rng(seed)
    return [wl.serving_request(rng, max_blocks=max_blocks, sizes=sizes, nsteps=nsteps) for _ in range(n)]


def _host_buffers(req):
    import torch
    spec = req["spec"]
    U0 = wl.region_state(spec, req["kind"], req["region"], req["u_in"], req["u_out"])
    init = torch.from_numpy(U0).pin_memory()
    out = torch.empty(spec.block_shape(), dtype=torch.float64).pin_memory()
    return U0, init, out


def _serve(reqs, task=B.ORCHA_TASK_HYDRO_FP64, budget=8 << 30, together=True, from_host=True):
    """Run requests through one server; returns (outputs, stats)."""
    srv = serve.Server(budget)
    keep, outs, stats = [], [], []
    try:
        descs = []
        for r in reqs:
            if from_host:
                U0, init, out = _host_buffers(r)
                keep.append((init, out))
                descs.append(serve.request_desc(r, task, init.data_ptr(), out.data_ptr()))
                outs.append(out)
            else:
                import torch
                out = torch.empty(r["spec"].block_shape(), dtype=torch.float64).pin_memory()
                keep.append(out)
                descs.append(serve.request_desc(r, task, None, out.data_ptr()))
                outs.append(out)
        if together:
            tickets = [srv.submit(d) for d in descs]
            stats = [srv.wait(t) for t in tickets]
        else:
            stats = [srv.wait(srv.submit(d)) for d in descs]
        peak = srv.stats().pool_peak_bytes
    finally:
        srv.close()
    return [o.numpy().copy() for o in outs], stats, peak


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _requests(8, 3)
    alone = [_serve([r])[0][0] for r in reqs]
    mixed, stats, _ = _serve(reqs)
    for a, m, s in zip(alone, mixed, stats):
        assert s.status == 0 and s.device_error == 0
        assert np.array_equal(a, m)


def test_mixed_precision_and_block_sizes_in_flight_together():
    """FP64, FP32-flux (configured and shortcut) and FF requests of block
    sizes 8, 16 and 32 in flight together: each result equals the same
    request served alone."""
    reqs = _requests(12, 5, sizes=(8, 16, 32), max_blocks=4, nsteps=2)
    tasks = ([B.ORCHA_TASK_HYDRO_FP64] * 3 + [B.ORCHA_TASK_HYDRO_F32FLUX] * 3 + [B.ORCHA_TASK_HYDRO_FF] * 3
             + [B.ORCHA_TASK_HYDRO_F32FLUX_FFSUM] * 3)
    alone = [_serve([r], task=t)[0][0] for r, t in zip(reqs, tasks)]
    srv = serve.Server(8 << 30)
    try:
        keep, tickets = [], []
        for r, task in zip(reqs, tasks):
            U0, init, out = _host_buffers(r)
            keep.append((init, out))
            tickets.append(srv.submit(serve.request_desc(r, task, init.data_ptr(), out.data_ptr())))
        for t in tickets:
            assert srv.wait(t).status == 0
    finally:
        srv.close()
    for (init, out), a in zip(keep, alone):
        assert np.array_equal(out.numpy(), a)


def test_device_recipe_equals_host_initial_state():
    reqs = _requests(4, 7)
    host, _, _ = _serve(reqs, from_host=True)
    recipe, stats, _ = _serve(reqs, from_host=False)
    for h, r, s in zip(host, recipe, stats):
        assert np.array_equal(h, r)
        nv = 5
        tot = r.sum(axis=(0, 2, 3, 4))
        np.testing.assert_allclose(s.totals[:nv], tot, rtol=1e-12, atol=1e-12 * np.abs(tot).max())


def test_admission_waits_for_memory_under_a_tight_budget():
    reqs = _requests(6, 11, max_blocks=8, sizes=(16,))
    need = max(2 * r["spec"].nblocks * 5 * 20 ** 3 * 8 for r in reqs)
    budget = int(2.2 * need) + (1 << 20)
    alone = [_serve([r])[0][0] for r in reqs]
    mixed, stats, peak = _serve(reqs, budget=budget)
    assert peak <= budget
    assert all(s.t_admit_us >= 0 for s in stats)
    for a, m in zip(alone, mixed):
        assert np.array_equal(a, m)


def test_served_request_matches_oracle_and_packet_path(oracle_mod):
    req = _requests(1, 13, max_blocks=6, sizes=(8,), nsteps=4)[0]
    spec = req["spec"]
    U0 = wl.region_state(spec, req["kind"], req["region"], req["u_in"], req["u_out"])
    (G,), (s,), _ = _serve([req])
    O, dts = oracle_steps(oracle_mod, spec, U0, 4)
    assert rule12_error(G, O, spec.nvar) <= 1e-12
    m = oracle_mod.Mesh(**spec.oracle_kwargs())
    assert s.dt_next == pytest.approx(oracle_mod.dt(m, O), rel=1e-12)
    from .gpu_helpers import gpu_steps
    P, _, _ = gpu_steps(spec, U0, 4)
    assert np.array_equal(G, P)


@pytest.mark.parametrize("task", [B.ORCHA_TASK_HYDRO_FP64, B.ORCHA_TASK_HYDRO_FF])
def test_non_cubic_blocks_join_a_fitting_tile(oracle_mod, task):
    """The server runs FP64 and FF requests whose blocks are 16 or more cells
    across on 16x16 tiles; blocks 8 cells across y (16 x 8 x 16, 32 x 8 x 8)
    join the 16x8 launch instead. Served together with a cubic request, each
    result is within the FP64 parity rule of the oracle."""
    reqs = []
    for nb, bs in [((2, 3, 1), (16, 8, 16)), ((1, 2, 2), (32, 8, 8)), ((2, 1, 1), (16, 16, 16))]:
        ncell = [nb[d] * bs[d] for d in range(3)]
        L = max(ncell)
        spec = wl.MeshSpec(ndim=3, nb=nb, bs=bs, hi=tuple(c / L for c in ncell))
        g = spec.gamma
        reqs.append(dict(spec=spec, kind=2, region=(0, ncell[0] // 2, 0, 0), u_in=tuple(wl._cons(g, 1.0, 1.0, 3)),
                         u_out=tuple(wl._cons(g, 0.125, 0.1, 3)), nsteps=3))
    outs, stats, _ = _serve(reqs, task=task)
    for r, G, st in zip(reqs, outs, stats):
        assert st.status == 0
        spec = r["spec"]
        U0 = wl.region_state(spec, 2, r["region"], r["u_in"], r["u_out"])
        O, _ = oracle_steps(oracle_mod, spec, U0, 3)
        e = rule12_error(G, O, spec.nvar)
        print(f"served {spec.bs} task {task}: rule-12 error {e:.3e}")
        assert e <= 1e-12


def test_submit_validation_and_timeout():
    import torch
    srv = serve.Server(64 << 20)
    try:
        big = wl.serving_request(np.random.default_rng(1), max_blocks=1, sizes=(32,))
        big["spec"] = wl.MeshSpec(ndim=3, nb=(4, 4, 4), bs=(32, 32, 32))
        with pytest.raises(B.OrchaError) as ei:
            srv.submit(serve.request_desc(big, B.ORCHA_TASK_HYDRO_FP64))
        assert ei.value.status == B.ORCHA_ERR_OOM
        bad = dict(big, nsteps=0)
        bad["spec"] = wl.MeshSpec(ndim=3, nb=(1, 1, 1), bs=(8, 8, 8))
        with pytest.raises(B.OrchaError) as ei:
            srv.submit(serve.request_desc(bad, B.ORCHA_TASK_HYDRO_FP64))
        assert ei.value.status == B.ORCHA_ERR_INVALID
        slow = dict(bad, nsteps=400)
        slow["spec"] = wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(32, 32, 32))
        t = srv.submit(serve.request_desc(slow, B.ORCHA_TASK_HYDRO_FP64))
        with pytest.raises(B.OrchaError) as ei:
            srv.wait(t, 0)
        assert ei.value.status == B.ORCHA_ERR_TIMEOUT
        st = srv.wait(t)                       # the ticket survives the timeout
        assert st.zone_updates == 2 * 32 ** 3 * 400
    finally:
        srv.close()


def test_nonphysical_request_reports_device_error():
    import torch
    spec = wl.MeshSpec(ndim=3, nb=(2, 1, 1), bs=(8, 8, 8))
    U0 = wl.uniform_state(spec, 1.0, (0.0, 0.0, 0.0), 1.0)
    U0[0, 4, 2, 2, 2] = -1.0
    init = torch.from_numpy(U0).pin_memory()
    out = torch.empty_like(init).pin_memory()
    req = dict(spec=spec, kind=0, region=(0, 0, 0, 0), u_in=(0,) * 5, u_out=(0,) * 5, nsteps=1)
    srv = serve.Server(64 << 20)
    try:
        t = srv.submit(serve.request_desc(req, B.ORCHA_TASK_HYDRO_FP64, init.data_ptr(), out.data_ptr()))
        with pytest.raises(B.OrchaError) as ei:
            srv.wait(t)
        assert ei.value.status == B.ORCHA_ERR_NONFINITE
        # the server keeps serving after a failed request
        good = _requests(1, 17)[0]
        t2 = srv.submit(serve.request_desc(good, B.ORCHA_TASK_HYDRO_FP64))
        assert srv.wait(t2).status == 0
    finally:
        srv.close()


def test_2d_requests_in_flight_with_3d_ones(oracle_mod):
    """2D requests (their own launch groups) served together with 3D ones:
    each 2D result matches the oracle and the packet path, and the 3D results
    equal those served alone."""
    from .gpu_helpers import gpu_steps
    g = 1.4
    reqs2d = []
    for nb, bs, axis in [((4, 2, 1), (16, 16, 1), 0), ((3, 5, 1), (8, 8, 1), 1)]:
        spec = wl.MeshSpec(ndim=2, nb=nb, bs=bs, hi=(1.0, nb[1] * bs[1] / (nb[0] * bs[0]), 1.0))
        n_ax = nb[axis] * bs[axis]
        u_in = tuple(wl._cons(g, 1.0, 1.0, 2))         # (rho, m_x, m_y, E), padded to five
        u_out = tuple(wl._cons(g, 0.125, 0.1, 2))
        reqs2d.append(dict(spec=spec, kind=B.ORCHA_INIT_HALF_SPACE, region=(axis, n_ax // 2, 0, 0),
                           u_in=u_in, u_out=u_out, nsteps=3))
    reqs3d = _requests(3, 21, max_blocks=6, sizes=(8, 16), nsteps=3)
    alone3d = [_serve([r])[0][0] for r in reqs3d]
    mixed, stats, _ = _serve(reqs2d + reqs3d)
    assert all(s.status == 0 for s in stats)
    for r, G in zip(reqs2d, mixed[:2]):
        spec = r["spec"]
        U0 = wl.region_state(spec, r["kind"], r["region"], r["u_in"], r["u_out"])
        O, _ = oracle_steps(oracle_mod, spec, U0, 3)
        assert rule12_error(G, O, spec.nvar) <= 1e-12
        P, _, _ = gpu_steps(spec, U0, 3)
        assert np.array_equal(G, P)
    for A, M in zip(alone3d, mixed[2:]):
        assert np.array_equal(A, M)
