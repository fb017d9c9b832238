"""Build the in-tree shared library ``libdsm.so`` (sm_103a) from ``csrc/``.

    python -m paper_2308_10896_b300.build        # or build() from Python

Every translation unit is compiled with nvcc for ``sm_103a`` only and linked
into one shared library next to this file; the Python binding loads it from
there.  Objects go to ``_build/`` (not committed).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libdsm.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
          "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _sources(src_dir=CSRC):
    return sorted(glob.glob(os.path.join(src_dir, "*.cu")) + glob.glob(os.path.join(src_dir, "*.cpp")))


def _stale(src_dir=CSRC, out=OUT) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = _sources(src_dir) + glob.glob(os.path.join(src_dir, "*.h")) + glob.glob(os.path.join(src_dir, "*.cuh")) \
        + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list | None = None, src_dir: str = CSRC,
          out: str = OUT) -> str:
    """Compile src_dir/*.cu, *.cpp into the shared library `out` (skipped when up to date)."""
    OUTP = out
    if not force and not _stale(src_dir, OUTP):
        return OUTP
    objdir = BUILD if src_dir == CSRC else os.path.join(os.path.dirname(OUTP), "_build")
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    extra = list(extra or [])
    inc = ["-I", os.path.join(ROOT, "include"), "-I", src_dir]

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        flags = [f for f in COMMON if f not in ("-I", CSRC, os.path.join(ROOT, "include"))] + inc
        cmd = [nvcc, *ARCH, *flags, *extra, "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, *flags, "-x", "c++", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, _sources(src_dir)))
    tmp = OUTP + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUTP)
    return OUTP


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
