"""Build the engine's shared library in-tree: ``_build/libmcmie.so``.

One nvcc invocation, sm_103a only, IEEE-strict device arithmetic (no
fast-math, no implicit multiply-add contraction: only the fmaf calls the
source writes are fused).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "_build", "libmcmie.so")
# the same engine with every table, pixel, bin and voxel index checked at run
# time (MC_CHECKED: an out-of-range index sets MC_EFLAG_BOUNDS and is clamped);
# for tests, built only on request
LIB_CHECKED = os.path.join(HERE, "_build", "libmcmie_checked.so")
# the same engine with CUDA's accurate logf / expf / exp2f / sincosf and
# correctly rounded division and square root in place of the hardware
# approximations (MC_STRICT), for trace comparisons at the tightest tolerance;
# built only on request, loaded instead of the normal one when MC_STRICT=1
LIB_STRICT = os.path.join(HERE, "_build", "libmcmie_strict.so")
SOURCES = ["walk.cu", "api.cu", "mie_table.cpp", "noalloc.cu", "metrics.cu", "grid.cu", "phase_weights.cu"]
HEADERS = ["engine.h", "table_format.h"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true",
              "-prec-sqrt=true", "-ftz=false", "-Xcompiler", "-fPIC,-O2", "-shared",
              "--threads", "4"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


PEAKS_LIB = os.path.join(HERE, "_build", "libmcpeaks.so")


def _compile(lib, sources, deps, force, verbose, extra):
    if not force and not _stale(lib, deps):
        return None
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc()] + NVCC_FLAGS + list(extra) + ["-I", os.path.join(ROOT, "include"),
                                                 "-o", tmp] + [os.path.join(CSRC, s) for s in sources]
    if verbose:
        print(" ".join(cmd))
    return subprocess.Popen(cmd), tmp, lib


def build_checked(force=False, verbose=False):
    """Compile the checked engine (-DMC_CHECKED) if missing or stale; return
    its path. Loaded instead of the normal one when MC_CHECKED=1."""
    me = os.path.abspath(__file__)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [
        os.path.join(ROOT, "include", "mcmie.h"), me]
    job = _compile(LIB_CHECKED, SOURCES, deps, force, verbose, ["-DMC_CHECKED"])
    if job is not None:
        proc, tmp, lib = job
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, "nvcc")
        os.replace(tmp, lib)
    return LIB_CHECKED


def build_strict(force=False, verbose=False):
    """Compile the IEEE-strict engine (-DMC_STRICT) if missing or stale;
    return its path. Loaded instead of the normal one when MC_STRICT=1."""
    me = os.path.abspath(__file__)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [
        os.path.join(ROOT, "include", "mcmie.h"), me]
    job = _compile(LIB_STRICT, SOURCES, deps, force, verbose, ["-DMC_STRICT"])
    if job is not None:
        proc, tmp, lib = job
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, "nvcc")
        os.replace(tmp, lib)
    return LIB_STRICT


def build(force=False, verbose=False, extra=()):
    """Compile the engine (and the issue-rate microbenchmarks) if missing or
    older than their sources; return the engine library's path."""
    me = os.path.abspath(__file__)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [
        os.path.join(ROOT, "include", "mcmie.h"), me]
    jobs = [_compile(LIB, SOURCES, deps, force, verbose, extra),
            _compile(PEAKS_LIB, ["peaks.cu"], [os.path.join(CSRC, "peaks.cu"),
                                               os.path.join(ROOT, "include", "mcpeaks.h"), me],
                     force, verbose, extra)]
    for job in jobs:
        if job is None:
            continue
        proc, tmp, lib = job
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, "nvcc")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
