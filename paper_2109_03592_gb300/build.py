"""Build libsem.so in-tree: every .cu for sm_103a with nvcc, every .cpp with
g++, compiled in parallel and linked (static cudart) into
paper_2109_03592_gb300/libsem.so."""

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsem.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsem.so")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers_digest():
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".h", ".cuh")):
            h.update(open(os.path.join(CSRC, f), "rb").read())
    h.update(open(os.path.join(HERE, "..", "include", "sem.h"), "rb").read())
    return h.hexdigest()


def _compile(src, cuda, hdr):
    path = os.path.join(CSRC, src)
    # objects are cached by source, headers and host machine (x86_64 vs aarch64)
    digest = hashlib.sha256(open(path, "rb").read() + hdr.encode() + platform.machine().encode()).hexdigest()[:16]
    obj = os.path.join(BUILD, f"{src}.{digest}.o")
    if os.path.exists(obj):
        return obj
    if src.endswith(".cu"):
        cmd = [os.path.join(cuda, "bin", "nvcc"), ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-O3", "-c", path, "-o", obj + ".tmp"]
    else:
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-I" + os.path.join(cuda, "include"), "-c", path, "-o",
               obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose=False):
    cuda = _cuda_home()
    os.makedirs(BUILD, exist_ok=True)
    hdr = _headers_digest()
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, cuda, hdr), srcs))
    tmp = LIB + ".tmp"
    cmd = [os.path.join(cuda, "bin", "nvcc"), ARCH, "-shared", "-o", tmp] + objs + [
        "-cudart", "static", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    keep = {os.path.basename(o) for o in objs}
    for f in os.listdir(BUILD):
        if f.endswith(".o") and f not in keep:
            os.remove(os.path.join(BUILD, f))
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
