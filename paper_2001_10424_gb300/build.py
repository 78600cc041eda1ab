"""Build the sm_103a shared library ``libgkb.so`` in-tree with nvcc.

The translation units are compiled in parallel (one nvcc process each) and
linked into ``paper_2001_10424_gb300/libgkb.so`` with the CUDA runtime linked
statically, so loading the library needs nothing beyond the CUDA driver.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgkb.so")

# (source, defines): the stencil / smoother instantiations are split by
# GKB_PART into units that compile in parallel
SOURCES = ([("kernels_f64.cu", ["-DGKB_PART=%d" % k]) for k in range(1, 8)]
           + [("kernels_f32.cu", ["-DGKB_PART=%d" % k]) for k in range(1, 8)]
           + [(f, []) for f in ("solver.cu", "api.cu", "noalloc.cu", "unet.cu", "fgmres.cu", "lockstep.cu", "tail.cu")])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgkb.so")


def _stamp(paths):
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False):
    """Compile every .cu under csrc/ for sm_103a and link libgkb.so."""
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "gkb.h"))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _stamp(deps):
        return LIB
    nvcc = nvcc_path()
    inc = ["-I", os.path.join(os.path.dirname(HERE), "include")]

    def compile_one(unit):
        src, defs = unit
        tag = "".join(d.split("=")[-1] for d in defs)
        obj = os.path.join(BUILD, src.replace(".cu", (("_p" + tag) if tag else "") + ".o"))
        cmd = [nvcc] + ARCH + FLAGS + defs + inc + ["-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr))
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        return obj

    workers = max(1, min(len(SOURCES), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
