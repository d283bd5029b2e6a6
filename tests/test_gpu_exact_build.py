"""The exact-FP64 build (ORCHA_FP64_CONTRACT=0: every FP64 operation one
unfused round-to-nearest operation, evaluated in the order of the scheme's
definition) reproduces the oracle bit for bit: 2D Sod (20 steps, the dt
sequence too), 3D Sedov 128^3 in packets of 64 (10 steps), random jumps with
every tile shape (4 steps), through the packet path and the persistent batch,
Heun RK2 steps on 2D Sod, and one step with many first-order fallback cells
(smeared random jumps at 40x the CFL time step; the ramp hand cases), and the
fused launches (two Hancock steps at one dt; a whole Heun step), and four
two-level AMR steps. The library variant is loaded in a child
process (a process holds one liborcha)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def results():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build(variant="exact")
    env = dict(os.environ, ORCHA_LIBRARY_VARIANT="exact")
    r = subprocess.run([sys.executable, os.path.join(HERE, "exact_build_child.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    out = {}
    for line in r.stdout.splitlines():
        if line.startswith("{"):
            d = json.loads(line)
            out[d["case"]] = d
    print(json.dumps(out, indent=1))
    return out


@pytest.mark.parametrize("case", ["sod64", "sedov128", "jumps", "sod64_rk2", "fallback40", "fallback_ramp_p",
                                  "fallback_ramp_rho", "tb2", "rk2_fused", "amr"])
def test_exact_build_is_bitwise_the_oracle(results, case):
    d = results[case]
    flags = {k: v for k, v in d.items() if k.endswith("_bitwise")}
    assert flags and all(flags.values()), d
