"""Build libdg_gb300.so for sm_103a (in-tree, one nvcc job per translation unit).

Each polynomial degree lives in its own translation unit (csrc/op_n<N>.cu)
so the units compile in parallel; the host geometry and the C ABI are two
more units.  The result is ``paper_2606_18927_gb300/_build/libdg_gb300.so``.

The bounds-checking variant (``variant="debug"``) compiles the same sources
with DG_DEBUG_BOUNDS: every index the kernels gather through the mesh tables
is checked against its range, and one that is out of range sets a device flag
(reported as DG_ERR_DEVICE_BOUNDS by dg_check_status) and is replaced by 0
instead of being used.  It is ``_build/debug/libdg_gb300_debug.so``, loaded
by the binding when DG_LIBRARY_VARIANT=debug.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdg_gb300.so")
VARIANTS = {"release": (OUT, LIB, []),
            "debug": (os.path.join(OUT, "debug"), os.path.join(OUT, "debug", "libdg_gb300_debug.so"),
                      ["-DDG_DEBUG_BOUNDS"])}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _sources() + _headers())


def _compile(src, extra, out):
    obj = os.path.join(out, os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj


def build(force=False, jobs=None, extra=(), variant="release"):
    """Compile the library (or its bounds-checking variant) if it is missing
    or older than its sources."""
    out, lib, flags = VARIANTS[variant]
    os.makedirs(out, exist_ok=True)
    if not force and not _stale(lib):
        return lib
    srcs = _sources()
    jobs = jobs or min(len(srcs), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags + list(extra), out), srcs))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


def build_all(force=False):
    """Both variants, compiled side by side."""
    with cf.ThreadPoolExecutor(2) as ex:
        libs = list(ex.map(lambda v: build(force=force, jobs=max(1, (os.cpu_count() or 2) // 2), variant=v),
                           ("release", "debug")))
    return libs


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv))
