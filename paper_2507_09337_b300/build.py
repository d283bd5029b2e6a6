"""Build the C-ABI library liborcha.so (CUDA for sm_103a) in the package directory.

    python -m paper_2507_09337_b300.build [--force] [--verbose] [--exact]

The library is compiled with nvcc directly (no JIT cache): each .cu source
to an object in parallel, then one link, so the built file sits in-tree next
to this script. --exact builds liborcha_exact.so instead:
the same sources with ORCHA_FP64_CONTRACT=0, where every FP64 operation is
one unfused round-to-nearest operation (loaded by the binding when
ORCHA_LIBRARY_VARIANT=exact).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liborcha.so")
# library variant -> (file, extra nvcc flags)
VARIANTS = {"default": ("liborcha.so", []),
            "exact": ("liborcha_exact.so", ["-DORCHA_FP64_CONTRACT=0"])}
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
           "--expt-relaxed-constexpr", "-shared", "-cudart", "shared"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(INCLUDE, "orcha.h"), __file__]


def lib_path(variant: str = "default") -> str:
    return os.path.join(HERE, VARIANTS[variant][0])


def up_to_date(variant: str = "default") -> bool:
    lib = lib_path(variant)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, variant: str = "default") -> str:
    """Compile every .cu source to an object (in parallel, in a temporary
    folder) and link them into the library."""
    import tempfile
    from concurrent.futures import ThreadPoolExecutor
    lib = lib_path(variant)
    if not force and up_to_date(variant):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    flags = [*ARCH, *[f for f in NVFLAGS if f not in ("-shared",)], *VARIANTS[variant][1], f"-I{INCLUDE}"]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    with tempfile.TemporaryDirectory(prefix="orcha_build_") as tmp:
        def compile_one(src):
            obj = os.path.join(tmp, os.path.basename(src) + ".o")
            r = subprocess.run([nvcc, *flags, "-c", src, "-o", obj], capture_output=True, text=True)
            return src, obj, r
        with ThreadPoolExecutor(max_workers=max(1, min(len(sources()), os.cpu_count() or 1))) as ex:
            results = list(ex.map(compile_one, sources()))
        for src, _, r in results:
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n" + r.stdout + r.stderr)
            if verbose:
                sys.stderr.write(r.stdout + r.stderr)
        r = subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "shared", *[o for _, o, _ in results],
                            "-o", lib + ".tmp"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                variant="exact" if "--exact" in sys.argv else "default"))
