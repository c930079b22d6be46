"""Build the CUDA library libsipg.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into ``paper_2405_18982_gb300/_lib/libsipg.so``.  No cmake, no torch
extension machinery: the library exposes a plain C ABI (include/sipg.h) and
the Python side loads it with ctypes.
"""
import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
# objects per host architecture: a tree copied between an x86 and an Arm
# machine never reuses the other's objects
BUILD_DIR = os.path.join(PKG, "_build", platform.machine())
LIB = os.path.join(OUT_DIR, "libsipg.so")
STAMP = os.path.join(OUT_DIR, "libsipg.machine")
# the colour-pass instantiation units are the slowest: they go first
SOURCES = (sorted(f for f in os.listdir(CSRC) if f.startswith("smooth_i_") and f.endswith(".cu")) +
           ["smooth_tc3.cu", "smooth_batch2.cu", "apply.cu", "setup.cu", "transfer.cu", "smoother.cu", "smooth_full.cu", "api.cu",
            "krylov.cu", "noalloc.cu"])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if os.path.exists(cand):
        return cand
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found (set CUDA_HOME)")
    return found


def cuda_lib_dir():
    home = os.path.dirname(os.path.dirname(nvcc_path()))
    for sub in ("lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"),
                os.path.join("targets", "x86_64-linux", "lib")):
        d = os.path.join(home, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(home, "lib64")


def _headers_mtime():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs += [os.path.join(ROOT, "include", "sipg.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(h) for h in hdrs)


def _compile(src, verbose, force):
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
    if (not verbose and not force and os.path.exists(obj) and
            os.path.getmtime(obj) >= max(os.path.getmtime(os.path.join(CSRC, src)), _headers_mtime())):
        return obj, ""  # object newer than its source and every header
    cmd = [nvcc_path(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17",
           "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-diag-suppress", "177",
           "-I", os.path.join(ROOT, "include")] + ARCH
    if verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr[-6000:]}")
    return obj, res.stderr


def up_to_date():
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return False
    with open(STAMP) as fh:
        if fh.read().strip() != platform.machine():
            return False
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "sipg.h"),
                                                                   os.path.abspath(__file__)]
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force=False, verbose=False, jobs=None):
    """Compile and link libsipg.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, force), SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    libdir = cuda_lib_dir()
    tmp = LIB + ".tmp"
    cmd = [nvcc_path(), "-shared", "-o", tmp] + objs + ARCH + [
        "-cudart", "shared", "-L", libdir, "-Xlinker", "-rpath=" + libdir]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(platform.machine() + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
