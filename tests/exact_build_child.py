"""Child process of tests/test_gpu_exact_build.py: runs the parity cases with
the exact-FP64 library (ORCHA_LIBRARY_VARIANT=exact, set by the parent) and
prints one JSON line per case comparing it with the oracle bit for bit."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2507_09337_b300 import binding as B  # noqa: E402
from paper_2507_09337_b300 import workloads as wl  # noqa: E402
from tests.gpu_helpers import gpu_batch_fixed_dt, gpu_batch_steps, gpu_one_step, gpu_steps, oracle_steps  # noqa: E402


def main():
    assert B.LIB_PATH.endswith("liborcha_exact.so"), B.LIB_PATH
    spec2 = wl.sod_spec(64, 8)
    sedov, packets = wl.sedov128_packets(64)
    jumps = wl.MeshSpec(ndim=3, nb=(2, 2, 2), bs=(16, 16, 16), periodic=(1, 0, 1))
    cases = [("sod64", spec2, wl.sod_state(spec2), None, 20, False, [(8, 8)]),
             ("sedov128", sedov, wl.sedov_state(sedov), packets, 10, False, [(16, 16)]),
             ("jumps", jumps, wl.random_blocky_state(jumps, 17), None, 4, False, [(8, 8), (16, 8), (16, 16)]),
             ("sod64_rk2", spec2, wl.sod_state(spec2), None, 20, True, [(8, 8)])]
    for name, spec, U0, pk, n, rk2, tiles in cases:
        O, odts = oracle_steps(oracle, spec, U0, n, rk2=rk2)
        task = B.ORCHA_TASK_HYDRO_RK2 if rk2 else B.ORCHA_TASK_HYDRO_FP64
        res = {"case": name, "steps": n}
        if not rk2:
            G, gdts, err = gpu_steps(spec, U0, n, task=task, packets=pk, record_dt=True)
            res["packet_path_bitwise"] = bool(np.array_equal(G, O)) and err == 0
            res["dt_bitwise"] = bool(np.array_equal(gdts, odts))
        for tile in tiles:
            (H,), errs = gpu_batch_steps([(spec, U0, pk)], n, task=task, tile=tile)
            res[f"batch_{tile[0]}x{tile[1]}_bitwise"] = bool(np.array_equal(H, O)) and errs == [0]
            res[f"batch_{tile[0]}x{tile[1]}_max_abs_diff"] = float(np.abs(H - O).max())
        print(json.dumps(res), flush=True)
    # the first-order fallback: one step at 40x the CFL time step of smeared
    # random jumps, and the ramp hand case
    oracle.set_threads(8)
    m = oracle.Mesh(**jumps.oracle_kwargs())
    U1, _, _ = oracle.run(m, wl.random_blocky_state(jumps, 21), 2)
    dt = 40.0 * oracle.dt(m, U1)
    ramp = wl.MeshSpec(ndim=2, nb=(2, 1, 1), bs=(16, 16, 1), periodic=(0, 1, 0))
    cases = [("fallback40", jumps, U1, dt)]
    for var in ("p", "rho"):
        cases.append((f"fallback_ramp_{var}", ramp, wl.ramp_state(ramp, var, 0.1, 10.0), 0.85 * ramp.dx(0)))
    for name, spec, U0, step_dt in cases:
        O, _, nfirst = oracle.step(oracle.Mesh(**spec.oracle_kwargs()), U0, step_dt)
        res = {"case": name, "nfirst": nfirst}
        for tile in [(8, 8), (16, 8), (16, 16)]:
            for path in ("packet", "batch"):
                G = gpu_one_step(spec, U0, step_dt, B.ORCHA_TASK_HYDRO_FP64, tile, path)
                res[f"{path}_{tile[0]}x{tile[1]}_bitwise"] = bool(np.array_equal(G, O))
        print(json.dumps(res), flush=True)
    # two operator applications per launch: two Hancock steps at one dt, and
    # a whole Heun step
    import dataclasses
    U2 = wl.random_blocky_state(jumps, 17)
    m = oracle.Mesh(**jumps.oracle_kwargs())
    dt = oracle.dt(m, U2)
    O1, _, _ = oracle.step(m, U2, dt)
    O2, _, _ = oracle.step(m, O1, dt)
    rk = dataclasses.replace(jumps, cfl=0.4)
    mr = oracle.Mesh(**rk.oracle_kwargs())
    dtr = oracle.dt(mr, U2)
    OR, _, _ = oracle.step_rk2(mr, U2, dtr)
    res_tb = {"case": "tb2"}
    res_rk = {"case": "rk2_fused"}
    for tile in [(8, 8), (16, 8), (16, 16)]:
        G, err, _ = gpu_batch_fixed_dt(jumps, U2, dt, B.ORCHA_TASK_HYDRO_TB2, tile, 2)
        res_tb[f"batch_{tile[0]}x{tile[1]}_bitwise"] = bool(np.array_equal(G, O2)) and err == 0
        G, err, _ = gpu_batch_fixed_dt(rk, U2, dtr, B.ORCHA_TASK_HYDRO_RK2_FUSED, tile, 1)
        res_rk[f"batch_{tile[0]}x{tile[1]}_bitwise"] = bool(np.array_equal(G, OR)) and err == 0
    print(json.dumps(res_tb), flush=True)
    print(json.dumps(res_rk), flush=True)
    # the two-level AMR step
    amr = wl.MeshSpec(ndim=3, nb=(3, 3, 3), bs=(8, 8, 8), periodic=(1, 0, 1))
    refined = wl.refined_blocks(amr, "sphere", 0.35)
    A0, A1 = wl.amr_split(amr, refined, wl.random_blocky_state(wl.fine_spec(amr), 13))
    O0, O1, _ = oracle.amr_run(oracle.Mesh(**amr.oracle_kwargs()), refined, A0, A1, 4)
    a = B.AmrMesh(amr, refined)
    try:
        a.load(A0, A1)
        a.advance(4, init_dt=True)
        err = a.poll()
        G0, G1 = a.store()
    finally:
        a.close()
    print(json.dumps({"case": "amr", "coarse_bitwise": bool(np.array_equal(G0, O0)) and err == 0,
                      "fine_bitwise": bool(np.array_equal(G1, O1))}), flush=True)


if __name__ == "__main__":
    main()
