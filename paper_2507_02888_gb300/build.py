"""Build libewald_gb300.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel into ``_build/`` and linked into
``paper_2507_02888_gb300/libewald_gb300.so``.  The debug variant
(``-DEWALD_DEBUG``: every kernel checks its ring, queue, list and particle
indices and reports a miss through the status word) goes to ``_build_debug/``
and ``libewald_gb300_debug.so``.  Usage: ``python -m
paper_2507_02888_gb300.build [--force] [--debug | --all]``.
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libewald_gb300.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libewald_gb300_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
VARIANTS = {"release": (BUILD, LIB, []), "debug": (BUILD_DEBUG, LIB_DEBUG, ["-DEWALD_DEBUG"])}


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build_variants(variants=("release",), force=False, verbose=False):
    """Compile every CUDA/C++ source once per variant, all translation units
    in one thread pool; link each variant's library; return their paths."""
    todo = [v for v in variants if force or not up_to_date(VARIANTS[v][1])]
    if not todo:
        return [VARIANTS[v][1] for v in variants]
    nvcc = _nvcc()

    def compile_one(job):
        v, src = job
        bdir, _, extra = VARIANTS[v]
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s (%s):\n%s%s" % (src, v, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    for v in todo:
        os.makedirs(VARIANTS[v][0], exist_ok=True)
    jobs = [(v, src) for v in todo for src in sources()]
    # the longest translation units first: they set the wall time
    jobs.sort(key=lambda j: -os.path.getsize(j[1]))
    with ThreadPoolExecutor(max_workers=max(1, min(32, os.cpu_count() or 1))) as ex:
        objs = dict(zip(jobs, ex.map(compile_one, jobs)))
    for v in todo:
        lib = VARIANTS[v][1]
        tmp = lib + ".%d.tmp" % os.getpid()
        r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + [objs[(v, s)] for s in sources()],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed (%s):\n%s%s" % (v, r.stdout, r.stderr))
        os.replace(tmp, lib)
    return [VARIANTS[v][1] for v in variants]


def build(force=False, verbose=False):
    """Compile the release library; return the .so path."""
    return build_variants(("release",), force, verbose)[0]


def build_debug(force=False, verbose=False):
    """Compile the debug library (-DEWALD_DEBUG); return the .so path."""
    return build_variants(("debug",), force, verbose)[0]


def build_all(force=False, verbose=False):
    """Compile both libraries in one pool; return their paths."""
    return build_variants(("release", "debug"), force, verbose)


if __name__ == "__main__":
    v = ("release", "debug") if "--all" in sys.argv else ("debug",) if "--debug" in sys.argv else ("release",)
    print(build_variants(v, force="--force" in sys.argv, verbose="-v" in sys.argv))
