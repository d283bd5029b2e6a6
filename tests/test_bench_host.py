"""Host-side pieces of bench.py that run without a GPU: the full-size parity
measure (rule 12 of the parity tests) and the CPU baseline leg, whose final
state the parity block compares the GPU tasks against."""
import numpy as np

import bench
import oracle
from paper_2507_09337_b300 import workloads as wl


def test_parity_error_is_rule_12():
    rng = np.random.default_rng(5)
    O = rng.uniform(0.5, 2.0, size=(3, 5, 4, 4, 4))
    O[:, 1:4] -= 1.25                     # momenta of both signs
    assert bench.parity_error(O.copy(), O, 5) == 0.0
    G = O.copy()
    G[1, 0, 2, 2, 2] *= 1.0 + 3e-13       # density: relative to the cell's own value
    assert np.isclose(bench.parity_error(G, O, 5), 3e-13, rtol=1e-3)
    O2 = O.copy()
    O2[0, 2, 0, 0, 0] = 0.0               # a momentum that vanishes: scaled by the largest |momentum|
    G = O2.copy()
    G[0, 2, 0, 0, 0] = 1e-12
    mom = np.abs(O2[:, 1:4]).max()
    assert np.isclose(bench.parity_error(G, O2, 5), 1e-12 / mom, rtol=1e-12)


def test_cpu_baseline_returns_the_oracle_state_it_reached():
    spec = wl.MeshSpec(ndim=3, nb=(2, 2, 1), bs=(8, 8, 8))
    U0 = wl.sedov_state(spec)
    rate, cores, n, el, U = bench.oracle_rate(spec, U0, 0.0)
    assert n == 1 and rate > 0 and cores >= 1
    m = oracle.Mesh(**spec.oracle_kwargs())
    W, _, _ = oracle.step(m, U0.copy(), oracle.dt(m, U0))
    assert np.array_equal(U, W)
