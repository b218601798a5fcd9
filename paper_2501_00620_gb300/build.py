"""Build the CUDA library (liblbm.so) in-tree for sm_103a with nvcc.

Each .cu translation unit compiles in parallel into _build/, then links into
paper_2501_00620_gb300/liblbm.so.  No cmake, one -gencode.
"""
import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build liblbm.so")
    return p


# Translation units that take longest to compile start first.
_HEAVY = ("gen3", "fast3", "fast2", "serve", "noalloc", "d2")


def _sources():
    def rank(p):
        b = os.path.basename(p)
        return next((k for k, h in enumerate(_HEAVY) if h in b), len(_HEAVY)), b
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")), key=rank)


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stamp(extra=""):
    h = hashlib.sha256()
    for f in _sources() + _headers() + [os.path.abspath(__file__)]:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode() + extra.encode())
    return h.hexdigest()


def _headers_digest():
    h = hashlib.sha256()
    for f in _headers():
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _compile(src, verbose, headers_digest):
    """Compile one translation unit unless its object was built from the same
    source, headers and flags (a stamp beside the object)."""
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    h = hashlib.sha256()
    with open(src, "rb") as fh:
        h.update(fh.read())
    h.update((headers_digest + " ".join(ARCH + NVCC_FLAGS) + str(verbose)).encode())
    stamp = obj + ".stamp"
    if not verbose and os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == h.hexdigest():
        return obj, ""
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    with open(stamp, "w") as fh:
        fh.write(h.hexdigest())
    return obj, r.stderr


def build(force=False, verbose=False, jobs=None):
    """Compile every translation unit and link liblbm.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp_file = os.path.join(BUILD, "liblbm.stamp")
    stamp = _stamp()
    if (not force and os.path.exists(LIB) and os.path.exists(stamp_file)
            and open(stamp_file).read() == stamp):
        return LIB
    srcs = _sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    logs = {}
    hd = _headers_digest()
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = {ex.submit(_compile, s, verbose, hd): s for s in srcs}
        objs = []
        for fu in cf.as_completed(futs):
            obj, log = fu.result()
            objs.append(obj)
            logs[futs[fu]] = log
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *sorted(objs), "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    if verbose:
        for s, log in sorted(logs.items()):
            sys.stderr.write("== %s\n%s" % (os.path.basename(s), log))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
