"""In-tree build of the CUDA library libvlb.so (sm_103a only)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libvlb.so")
SOURCES = ["lb_api.cu", "lb_fused.cu", "lb_strip.cu", "lb_sweep.cu", "lb_nodes.cu", "lb_lut.cu", "lb_diffuse.cu",
           "lb_batch.cu", "lb_unet.cu", "lb_learned.cu", "lb_ckpt.cu", "lb3d.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no automatic contraction of a product and a sum into one FMA.  The one-cell
# kernels fuse exactly where the source calls fmaf, so the same device code rounds identically
# in every kernel it is inlined into (single-lattice and batched launches agree bitwise).
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         "--expt-relaxed-constexpr", "-fmad=false"]
# Sources with no bitwise counterpart in another kernel: the compiler may contract products and
# sums into FMAs there (the three-dimensional step is checked against the oracle to a tolerance).
FMA_SOURCES = ("lb3d.cu",)


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvlb.so")


def _deps():
    headers = sorted(f for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    return [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, f) for f in headers] + [
        os.path.join(ROOT, "include", "lb.h"), os.path.join(ROOT, "include", "lb3d.h"),
        os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libvlb.so next to this file."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        flags = [("-fmad=true" if f == "-fmad=false" and src in FMA_SOURCES else f) for f in FLAGS]
        cmd = [cc, *ARCH, *flags, "-I", os.path.join(ROOT, "include"), "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for obj, log in results:
            print(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
