"""Build libifilt.so in-tree for sm_103a (GB300) with nvcc.

    python -m paper_2404_07398_gb300.build          # or __graft_entry__.build()

Every translation unit is compiled in parallel into _build/, then linked into
paper_2404_07398_gb300/libifilt.so (static CUDA runtime, no torch dependency).
IFILT_NVCC_FLAGS adds nvcc flags (e.g. -DIFILT_MG_MINB_XFER=3 to change a kernel's
resident-block target); objects are not rebuilt when only these flags change, so
build with force=True (or remove _build/) after changing them.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libifilt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(ptxas_verbose=False):
    # host code without contracted multiply-adds: the same host results on x86 and Arm, and the
    # same bits as the device kernels that restate host arithmetic with IEEE operations
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3,-ffp-contract=off",
                "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", SRC]
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f + os.environ.get("IFILT_NVCC_FLAGS", "").split()


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cu", ".cpp")))


def _newer(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, ptxas_verbose=False, force=False):
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "ifilt.h"))
    jobs = []
    objs = []
    for s in sources():
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        if force or _newer(o, [s] + headers):
            lang = ["-x", "cu"] if s.endswith(".cu") else ["-x", "c++"]
            jobs.append([cc] + _flags(ptxas_verbose) + lang + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    failed = []
    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0 or ptxas_verbose:
                sys.stderr.write(" ".join(cmd[-3:]) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    if force or jobs or _newer(LIB, objs):
        tmp = LIB + ".tmp"
        cmd = [cc] + ARCH + ["-shared", "-cudart", "static", "-Xcompiler", "-fPIC", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv, force="--force" in sys.argv)
    print(LIB)
