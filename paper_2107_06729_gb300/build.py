"""Builds libmmx.so in-tree for sm_103a (nvcc + g++, no cmake).

The three translation units compile in parallel; the result is
paper_2107_06729_gb300/libmmx.so (git-ignored)."""
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmmx.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kernels.cu", "stage_f32.cu", "stage_f64.cu", "fft_fused_f32.cu", "fft_fused_f64.cu", "fft_split.cu", "fft_pipe.cu",
           "mmx_api.cu", "static_demag.cu", "rnet.cu", "tensor_host.cpp"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "mmx.h"))
    return files


STAMP = os.path.join(OUT, "machine.txt")


def _stale():
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    if open(STAMP).read().strip() != platform.machine():
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps() + [__file__])


def _compile(src):
    s = os.path.join(CSRC, src)
    o = os.path.join(OUT, src + ".o")
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xptxas", "-v" if os.environ.get("MMX_PTXAS_V") else "-O3", "-c", s, "-o", o]
    else:
        cmd = ["g++", "-O2", "-std=gnu++17", "-fPIC", "-pthread", "-c", s, "-o", o]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return o, r.stderr


def build(force=False, verbose=False):
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), max(2, os.cpu_count() or 2))) as ex:
        results = list(ex.map(_compile, SOURCES))
    if verbose:
        for _, err in results:
            if err:
                print(err)
    objs = [o for o, _ in results]
    libs = ["-lpthread"]
    if platform.machine() in ("x86_64", "AMD64"):
        libs.append("-lquadmath")
    tmp = LIB + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, *libs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(platform.machine())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
