"""The persistent kernel's column work list (csrc/worklist.h), on the CPU:
every plane of every block column tile is queued exactly once, no piece is
shorter than two planes, pieces are queued longest first, and every cut
inside a column lies on a rounded multiple of W / G (W planes in all, G
resident CTAs)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_09337_b300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("worklist") / "worklist_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr",
                        "-gencode", "arch=compute_103a,code=sm_103a",
                        f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                        os.path.join(ROOT, "tests", "worklist_check.cu"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def run(exe, G, meshes):
    args = [str(G)] + [str(v) for m in meshes for v in m]
    out = subprocess.run([exe] + args, capture_output=True, text=True, check=True).stdout
    return [tuple(int(v) for v in line.split()) for line in out.splitlines()]


CASES = {
    # 128^3 Sedov: 512 blocks of 16^3, one 16x16 tile per block plane, 148 CTAs
    "sedov128_16x16": (148, [(0, 8, 8, 8, 16, 16, 16, 1)]),
    # the same with 16x8 tiles (two per plane) and three CTAs per SM
    "sedov128_16x8": (444, [(0, 8, 8, 8, 16, 16, 16, 2)]),
    # two meshes of different block sizes in one launch
    "two_meshes": (296, [(0, 4, 4, 4, 16, 16, 16, 1), (1, 3, 2, 5, 8, 8, 8, 1)]),
    # more CTAs than planes per column would give
    "many_ctas": (1000, [(0, 2, 2, 2, 8, 8, 8, 1)]),
    # one resident CTA: every column whole
    "one_cta": (1, [(0, 3, 3, 3, 16, 16, 16, 4)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_column_items(harness, name):
    G, meshes = CASES[name]
    items = run(harness, G, meshes)
    cols = {}
    W = 0
    for slot, nbx, nby, nbz, bsx, bsy, bsz, ntile in meshes:
        depth = nbz * bsz
        for blk in range(nbx * nby):
            for t in range(ntile):
                cols[(slot, blk, t)] = depth
                W += depth
    # coverage: each column's pieces tile [0, depth) exactly once
    pieces = {}
    for slot, blk, tile, z0, z1 in items:
        assert (slot, blk, tile) in cols
        assert 0 <= z0 < z1 <= cols[(slot, blk, tile)]
        pieces.setdefault((slot, blk, tile), []).append((z0, z1))
    assert set(pieces) == set(cols)
    for key, ps in pieces.items():
        ps.sort()
        assert ps[0][0] == 0 and ps[-1][1] == cols[key]
        assert all(a[1] == b[0] for a, b in zip(ps, ps[1:]))
        assert all(z1 - z0 >= 2 for z0, z1 in ps)
    # queue order: longest first
    lengths = [z1 - z0 for *_, z0, z1 in items]
    assert lengths == sorted(lengths, reverse=True)
    # cuts inside a column sit on rounded multiples of W / G of the plane stream
    seg = W / G
    base = 0
    order = []
    for slot, nbx, nby, nbz, bsx, bsy, bsz, ntile in meshes:
        for by in range(nby):
            for bx in range(nbx):
                for t in range(ntile):
                    order.append((slot, bx + nbx * by, t))
    for key in order:
        for z0, _ in pieces[key][1:]:
            pos = base + z0
            k = round(pos / seg)
            assert any(abs(round(kk * seg) - pos) == 0 for kk in (k - 1, k, k + 1)), (key, z0)
        base += cols[key]
    if G == 1:
        assert len(items) == len(cols)
    else:
        # about one segment per CTA: no more pieces than columns plus cuts
        assert len(items) <= len(cols) + G
