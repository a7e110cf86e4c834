"""Builds libsg.so (the C-ABI library) in-tree for sm_103a.

Every translation unit is compiled in parallel with nvcc, then linked into
paper_2605_21046_gb300/libsg.so.  Objects go to paper_2605_21046_gb300/_build/.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["sg_setup.cpp", "sg_apply.cu", "sg_apply_f64.cu", "sg_apply_dw.cu", "sg_apply_f32.cu", "sg_mg.cu", "sg_vanka_factor.cu", "sg_vanka_tc.cu",
           "sg_krylov.cu", "sg_noalloc.cu", "sg_manufactured.cu", "sg_mc.cu", "sg_mc_apply.cu", "sg_adjoint.cu", "sg_api.cu",
           "sg_debug.cu"]
# the build with device bounds checks (-DSG_DEBUG_BOUNDS): libsg_debug.so
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libsg_debug.so")


def _nvcc():
    cand = [shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _compile(src, verbose, debug_bounds=False):
    out = os.path.join(BUILD_DEBUG if debug_bounds else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", *ARCH,
           "-I", os.path.join(PKG, "..", "include"), "-c", os.path.join(CSRC, src), "-o", out]
    if debug_bounds:
        cmd[1:1] = ["-DSG_DEBUG_BOUNDS=1"]
    if src.endswith(".cu"):
        cmd[1:1] = ["-Xptxas", "-v"] if verbose else []
    if src in ("sg_mg.cu", "sg_vanka_factor.cu", "sg_vanka_tc.cu", "sg_manufactured.cu", "sg_mc.cu"):
        cmd[1:1] = ["-Xcompiler", "-fopenmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return out, r.stderr


def build(verbose=False, force=False, debug_bounds=False):
    """Compile and link libsg.so (or, with debug_bounds, libsg_debug.so: every
    unit compiled with -DSG_DEBUG_BOUNDS); returns its path."""
    lib = LIB_DEBUG if debug_bounds else LIB
    os.makedirs(BUILD_DEBUG if debug_bounds else BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(PKG, "..", "include", "sg.h"))
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) > max(os.path.getmtime(f) for f in srcs + hdrs)):
        return lib
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, debug_bounds), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    tmp = lib + ".tmp"
    cmd = [_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
