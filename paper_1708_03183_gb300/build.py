"""Build libslt.so in-tree with nvcc for sm_103a (GB300).

    python paper_1708_03183_gb300/build.py [-v] [-f]

Each translation unit is compiled in parallel, then linked into
paper_1708_03183_gb300/_build/libslt.so.  Rebuilds only when a source or header is newer.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libslt.so")
SOURCES = ["api.cpp", "refelem.cpp", "tune.cpp", "sort.cu", "inspect.cu", "exec.cu", "exec_batched.cu",
           "adjoint.cu", "noalloc.cu", "peak.cu", "contract.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "slt.h"))
    return files


def build(verbose=False, force=False):
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in _inputs())):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    # build-time generator: nonzero pattern of the reference differentiation matrices
    gen = os.path.join(OUT, "refgen")
    r = subprocess.run([nvcc, "-x", "c++", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        os.path.join(CSRC, "refgen.cpp"), os.path.join(CSRC, "refelem.cpp"), "-o", gen],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("refgen build failed:\n%s%s" % (r.stdout, r.stderr))
    r = subprocess.run([gen], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("refgen failed:\n%s" % r.stderr)
    with open(os.path.join(OUT, "refmask.h"), "w") as f:
        f.write(r.stdout)
    common = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
              "-I", CSRC, "-I", OUT] + ARCH

    def compile_one(src):
        obj = os.path.join(OUT, src + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + common
        if src.endswith(".cu"):
            # device code of a translation unit compiled by parallel jobs (the executor's many
            # template instances dominate the build)
            cmd += ["--split-compile=0"] + (["-Xptxas", "-v"] if verbose else [])
        else:
            cmd += ["-x", "c++"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
