"""In-tree build of libm2m.so for sm_103a with nvcc (no cmake, one TU).

Flags: -fmad=false so that every expression that decides a bin or cell, or
feeds one, rounds exactly as written (the kernels spell out fmaf/fma where
contraction is wanted); IEEE division and square root (the nvcc defaults)
for the same reason.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRCS = [os.path.join(HERE, "csrc", f)
        for f in ("m2m_api.cu", "m2m_pass_f32.cu", "m2m_pass_f32x.cu", "m2m_pass_f32b.cu", "m2m_pass_f64.cu",
                  "m2m_static.cu", "m2m_steps_f32.cu")]
HDRS = [os.path.join(HERE, "csrc", f)
        for f in ("m2m_device.cuh", "m2m_kernels.cuh", "m2m_analysis.cuh", "m2m_steps.cuh")] + [
    os.path.join(ROOT, "include", "m2m.h")]
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libm2m.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libm2m.so")


def flags(verbose=False):
    f = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
         "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in SRCS + HDRS + [__file__])


def build(force=False, verbose=False):
    """Compile libm2m.so in place (skipped when newer than its sources)."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objs, procs = [], []
    for src in SRCS:           # one translation unit per precision, in parallel
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc()] + flags(verbose) + ["-c", "-o", obj, src],
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    failed = False
    for pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            sys.stderr.write(out)
        failed |= pr.returncode != 0
    if failed:
        raise RuntimeError("nvcc failed building libm2m.so")
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc(), ARCH, "--shared", "-o", tmp] + objs + ["-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking libm2m.so")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
