"""The committed ncu summaries under profiles/ against the kernel sources:
bench.py reports a kernel's DRAM traffic from them only while the code they
were captured on is unchanged, so a summary whose hash is stale would leave
the bench line's roofline.traffic empty."""
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# summary -> kernel variants bench.py may time on that workload
CAPTURED = {
    "persistent_kernel_fp64_sedov128.md": ["persistent_kernel<3,16,16,rd>"],
    "persistent_kernel_fp64_sedov256.md": ["persistent_kernel<3,16,16,rd>"],
    "persistent_kernel_f32flux_sedov128.md": ["persistent_kernel<3,16,8,float>",
                                              "persistent_kernel<3,16,8,float,false,true>"],
    "persistent_kernel_ff_sedov128.md": ["persistent_kernel<3,16,16,dw>"],
    "persistent_kernel_rk2_sedov128.md": ["persistent_kernel<3,16,16,rd,true>"],
    "fused_kernel_sedov128.md": ["fused_kernel<3,16,16,rd,false>", "fused_kernel<3,16,16,float,false>",
                                 "fused_kernel<3,16,16,rd,true>"],
}


def _summary_hash(md):
    """The summary's recorded hash and the extra sources it covers."""
    sha, extra = None, ()
    for line in open(os.path.join(ROOT, "profiles", md)):
        if line.strip().startswith("kernel_source_sha256:"):
            sha = line.split(":", 1)[1].strip()
        elif line.strip().startswith("kernel_sources:"):
            extra = tuple(t.strip() for t in line.split(":", 1)[1].split(",") if t.strip())
    return sha, extra


@pytest.mark.parametrize("md", sorted(CAPTURED))
def test_summary_traffic_only_while_current(md):
    """A summary captured on the current kernel code gives each kernel it
    lists a positive traffic; a summary from older code gives none (the
    bench line then carries traffic null instead of a stale number)."""
    sha, extra = _summary_hash(md)
    current = sha == bench.kernel_source_hash(extra)
    for kernel in CAPTURED[md]:
        t = bench.profiled_traffic(md, kernel)
        assert (t is not None and t > 0) if current else t is None, (md, kernel, current)
    assert bench.profiled_traffic(md, "persistent_kernel<3,8,8,rd>") is None


def test_persistent_summaries_do_not_cover_amr_or_fused_sources():
    """An edit to the AMR or fused sources leaves the persistent kernel's
    captures current: their hash covers only the headers it is built from."""
    sha, extra = _summary_hash("persistent_kernel_fp64_sedov256.md")
    assert extra == ()
    assert "amr.cu" not in bench.KERNEL_SOURCES and "fused.cuh" not in bench.KERNEL_SOURCES
    assert _summary_hash("fused_kernel_sedov128.md")[1] == ("fused.cuh",)
    assert _summary_hash("amr_step_sedov128.md")[1] == ("amr.cu",)


def test_stale_hash_gives_no_traffic(tmp_path, monkeypatch):
    text = open(os.path.join(ROOT, "profiles", "persistent_kernel_fp64_sedov128.md")).read()
    current = bench.kernel_source_hash()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "x.md").write_text(text.replace(current, "0" * 64))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda extra=(): current)
    assert bench.profiled_traffic("x.md", "persistent_kernel<3,16,16,rd>") is None
