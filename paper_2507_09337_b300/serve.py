"""Serving driver: Poisson-arriving requests through the continuous-batching
server (orcha_server_*) or through plain per-request packet launches.

    python -m paper_2507_09337_b300.serve [--rates 1000,2000,...] [--requests N]
           [--task f32flux|f32flux_ffsum|fp64|ff] [--budget-gb 64] [--max-blocks 512] [--out FILE]

Each request is an independent 3D problem (K ~ U[1, max_blocks] blocks of
8^3, 16^3 or 32^3 cells, Sedov-like or Sod-like two-region initial state
written on the device, `nsteps` steps). For each arrival rate the requests
are submitted at their arrival times; latency = completion - submission (the
server clock), throughput = zone updates of all requests / (last completion
- first submission). The baseline runs the same requests one at a time
through the packet path (mesh + one packet per request, per-step guard-fill,
hydro and dt launches) and is timed the same way.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as B
from . import workloads as wl


def request_desc(req: dict, task: int, init_host=None, out_host=None) -> B.orcha_request_desc:
    spec = req["spec"]
    d = B.orcha_request_desc()
    d.ndim = spec.ndim
    for a in range(3):
        d.nb[a], d.bs[a], d.periodic[a] = spec.nb[a], spec.bs[a], spec.periodic[a]
        d.lo[a], d.hi[a] = spec.lo[a], spec.hi[a]
    d.gamma, d.cfl = spec.gamma, spec.cfl
    d.nsteps = req["nsteps"]
    d.task = task
    if init_host is not None:
        d.init_kind = B.ORCHA_INIT_FROM_HOST
        d.init_host = init_host
    else:
        d.init_kind = req["kind"]
        for i in range(4):
            d.region[i] = req["region"][i]
        for v in range(5):
            d.u_in[v], d.u_out[v] = req["u_in"][v], req["u_out"][v]
    d.out_host = out_host
    return d


class Server:
    """Owner of an orcha_server handle."""

    def __init__(self, budget_bytes: int, max_active: int = 1024):
        self.h = B.orcha_server_create(budget_bytes, max_active)

    def submit(self, desc) -> int:
        return B.orcha_server_submit(self.h, desc)

    def wait(self, ticket: int, timeout_ms: int = -1):
        return B.orcha_server_wait(self.h, ticket, timeout_ms)

    def stats(self):
        return B.orcha_server_get_stats(self.h)

    def close(self):
        if self.h:
            B.orcha_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _pct(a, q):
    return float(np.percentile(np.asarray(a), q)) if len(a) else None


def run_server(stream, task: int, budget_bytes: int, warm: int = 8) -> dict:
    """Submit the stream at its arrival times; return latency/throughput stats."""
    srv = Server(budget_bytes)
    try:
        # warm-up: a few requests before the clock starts (first-launch costs)
        for _, req in stream[:warm]:
            srv.wait(srv.submit(request_desc(req, task)))
        tickets = []
        t0 = time.perf_counter()
        for t_arr, req in stream:
            while time.perf_counter() - t0 < t_arr:
                pass
            tickets.append(srv.submit(request_desc(req, task)))
        stats = [srv.wait(t) for t in tickets]
        s = srv.stats()
    finally:
        srv.close()
    lat_ms = [(x.t_done_us - x.t_submit_us) * 1e-3 for x in stats]
    span_s = (max(x.t_done_us for x in stats) - min(x.t_submit_us for x in stats)) * 1e-6
    zu = sum(x.zone_updates for x in stats)
    return {"mode": "server", "requests": len(stats), "p50_ms": _pct(lat_ms, 50), "p99_ms": _pct(lat_ms, 99),
            "mean_ms": float(np.mean(lat_ms)), "zone_updates_per_s": zu / span_s, "span_s": span_s,
            "zone_updates": zu, "pool_peak_gb": s.pool_peak_bytes / 1e9,
            "wait_p50_ms": _pct([(x.t_ready_us - x.t_submit_us) * 1e-3 for x in stats], 50),
            "totals": [list(x.totals) for x in stats]}


def run_plain(stream, task: int, warm: int = 8) -> dict:
    """The same requests one at a time through plain per-packet launches."""
    import torch
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()

    def one(req):
        spec = req["spec"]
        mesh = B.Mesh(spec, device="cuda")
        try:
            B.orcha_mesh_init_region(mesh.handle, req["kind"], req["region"], req["u_in"], req["u_out"], st)
            mesh.advance(req["nsteps"], task, init_dt=True, use_graph=False, stream=st)
            st.synchronize()
        finally:
            mesh.close()
        return spec.zones * req["nsteps"]

    for _, req in stream[:warm]:
        one(req)
    lat_ms, zu = [], 0
    t0 = time.perf_counter()
    for t_arr, req in stream:
        while time.perf_counter() - t0 < t_arr:
            pass
        zu += one(req)
        lat_ms.append((time.perf_counter() - t0 - t_arr) * 1e3)
    span_s = time.perf_counter() - t0 - stream[0][0]
    return {"mode": "plain", "requests": len(stream), "p50_ms": _pct(lat_ms, 50), "p99_ms": _pct(lat_ms, 99),
            "mean_ms": float(np.mean(lat_ms)), "zone_updates_per_s": zu / span_s, "span_s": span_s,
            "zone_updates": zu}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="1000,2000,5000,10000,20000,50000")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--task", choices=["f32flux", "f32flux_ffsum", "fp64", "ff"], default="f32flux")
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--max-blocks", type=int, default=512)
    ap.add_argument("--nsteps", type=int, default=1)
    ap.add_argument("--plain", action="store_true", help="also run the plain per-request baseline")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from . import build
    build.build()
    task = B.TASKS[args.task]
    out = open(args.out, "w") if args.out else None

    def emit(res):
        line = json.dumps(res)
        print(line, flush=True)
        if out:
            out.write(line + "\n")
            out.flush()

    base = wl.serving_stream(args.requests, 1.0, max_blocks=args.max_blocks, nsteps=args.nsteps)
    try:
        for rate in [float(r) for r in args.rates.split(",")]:
            stream = [(t / rate, req) for t, req in base]
            res = run_server(stream, task, int(args.budget_gb * 1e9))
            res.pop("totals")
            res.update(rate_per_s=rate, task=args.task, budget_gb=args.budget_gb, max_blocks=args.max_blocks)
            emit(res)
            if args.plain:
                p = run_plain(stream, task)
                p.update(rate_per_s=rate, task=args.task, max_blocks=args.max_blocks)
                emit(p)
    finally:
        if out:
            out.close()


if __name__ == "__main__":
    main()
