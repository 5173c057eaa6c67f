"""Build libhelr.so (the CUDA library behind include/he_lr.h) in-tree for sm_103a.

Each translation unit compiles in parallel with nvcc; the objects link into one
shared library with the CUDA runtime linked statically.  Usage:
    python -m paper_2406_13221_gb300.build [--force]
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhelr.so")
UNITS = ["ntt.cu", "ks.cu", "ks_tensor.cu", "ops.cu", "encode.cu", "eval.cu", "helr_ctx.cu", "helr_lr.cu", "noalloc.cu",
         "autotune.cu", "boot.cu"]
HEADERS = ["helr_internal.cuh", "ntt_core.cuh", os.path.join("..", "..", "include", "he_lr.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-Xptxas", "-O3"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=()):
    os.makedirs(OUT, exist_ok=True)
    nv = nvcc()
    hdrs = [os.path.join(SRC, h) for h in HEADERS]
    jobs = []
    for u in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(OUT, u.replace(".cu", ".o"))
        if force or _stale(obj, [src] + hdrs):
            jobs.append(([nv] + ARCH + FLAGS + list(extra) + ["-c", src, "-o", obj], u))
    def run(job):
        cmd, u = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (u, r.stdout, r.stderr))
        return r.stderr if verbose else ""
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for msg in ex.map(run, jobs):
                if msg:
                    sys.stderr.write(msg)
    objs = [os.path.join(OUT, u.replace(".cu", ".o")) for u in UNITS]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [nv] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
