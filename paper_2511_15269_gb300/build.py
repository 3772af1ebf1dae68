"""Builds the CUDA library libfmm_gb300.so in-tree for sm_103a.

Each translation unit in csrc/ is compiled by nvcc in parallel, then linked
into a shared library next to this file.  Rebuilds only when a source or the
public header is newer than the library.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfmm_gb300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2", "-I", os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
            [GEN, os.path.join(ROOT, "include", "fmm.h")])


def _compile(src, verbose):
    obj = os.path.join(OBJ, os.path.basename(src) + ".o")
    cmd = [NVCC] + ARCH + FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-8000:]))
    return obj, r.stderr


GEN = os.path.join(CSRC, "gen_tables.py")
GEN_OUT = os.path.join(CSRC, "tables_gen.h")


def _generate():
    if not os.path.exists(GEN_OUT) or os.path.getmtime(GEN_OUT) < os.path.getmtime(GEN):
        subprocess.run([sys.executable, GEN, GEN_OUT], check=True)


def build(force=False, verbose=False, jobs=None):
    """Compile every CUDA source for sm_103a and link libfmm_gb300.so."""
    _generate()
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in _deps())
        if os.path.getmtime(LIB) >= newest:
            return LIB
    os.makedirs(OBJ, exist_ok=True)
    srcs = _sources()
    # compile the heaviest translation units first
    srcs.sort(key=lambda p: -os.path.getsize(p) - (10**7 if "eval_f" in p else 0))
    logs = {}
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        futs = {ex.submit(_compile, s, verbose): s for s in srcs}
        objs = []
        for f in cf.as_completed(futs):
            obj, log = f.result()
            objs.append(obj)
            logs[futs[f]] = log
    tmp = LIB + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + sorted(objs)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
    os.replace(tmp, LIB)
    if verbose:
        for s, log in logs.items():
            sys.stderr.write("== %s\n%s\n" % (os.path.basename(s), log))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
