"""Tile autotuner: returns a built variant that divides the block, caches it
per (GPU, geometry, task), and the tuned tile gives the default's bits."""
import json
import os

import numpy as np
import pytest

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl

from .gpu_helpers import gpu_batch_steps

pytestmark = pytest.mark.gpu

BUILT = {(16, 16), (16, 8), (8, 8)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09337_b300 import build
    build.build()


@pytest.mark.parametrize("ndim,bs,task", [(3, (16, 16, 16), B.ORCHA_TASK_HYDRO_FP64),
                                          (3, (8, 8, 8), B.ORCHA_TASK_HYDRO_F32FLUX),
                                          (3, (16, 16, 16), B.ORCHA_TASK_HYDRO_F32FLUX_FFSUM),
                                          (2, (32, 16, 1), B.ORCHA_TASK_HYDRO_FP64),
                                          (3, (16, 16, 16), B.ORCHA_TASK_HYDRO_FF),
                                          (3, (16, 16, 16), B.ORCHA_TASK_HYDRO_RK2)])
def test_autotune_picks_a_valid_tile_and_caches_it(tmp_path, ndim, bs, task):
    cache = str(tmp_path / "tiles.json")
    tx, ty, ms = B.orcha_autotune(ndim, bs, task, nblocks=64, cache_path=cache)
    assert (tx, ty) in BUILT and bs[0] % tx == 0 and bs[1] % ty == 0 and ms > 0
    entries = json.load(open(cache))
    assert len(entries) == 1 and list(entries.values())[0][:2] == [tx, ty]
    assert B.orcha_autotune(ndim, bs, task, nblocks=64, cache_path=cache)[:2] == (tx, ty)   # cache hit


def test_tuned_tile_gives_the_same_bits():
    spec = wl.MeshSpec(ndim=3, nb=(3, 2, 2), bs=(16, 16, 16))
    U0 = wl.random_blocky_state(spec, 61)
    tx, ty, _ = B.orcha_autotune(3, spec.bs, B.ORCHA_TASK_HYDRO_FP64, nblocks=64, cache_path=None)
    (A,), _ = gpu_batch_steps([(spec, U0, None)], 3, tile=(tx, ty))
    (D,), _ = gpu_batch_steps([(spec, U0, None)], 3)
    assert np.array_equal(A, D)
