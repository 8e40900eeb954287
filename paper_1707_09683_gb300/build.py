"""Build libmpf.so (the CUDA scan library) in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled by nvcc in parallel (the
scan-kernel instantiations, ``mpf_inst.cu``, once per lane-group size and
once more for the tensor-memory variants) and
the objects are linked into ``paper_1707_09683_gb300/libmpf.so``.  Objects are
rebuilt only when a source or header is newer.  No CMake, no torch
extension machinery: plain nvcc, one ``-gencode``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmpf.so")
# Debug build: the same sources with the kernels' index checks
# (-DMPF_DEBUG_CHECKS): a failed check sets the context's status word and
# skips the access; mpf_sync then returns MPF_EDEVICE.
OBJ_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libmpf_debug.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _cuda_lib_dir() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        p = os.path.join(home, d)
        if os.path.isdir(p):
            return p
    return os.path.join(home, "lib64")


def _newest_header() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    hs.append(os.path.join(ROOT, "include", "mpf.h"))
    return max(os.path.getmtime(h) for h in hs if os.path.exists(h))


# The scan-kernel instantiations: one source compiled once per lane-group size.
INST_SRC = "mpf_inst.cu"
INST_LANES = (1, 2, 4, 8, 16, 32)
QP_LANES = (1, 2, 4, 8, 16)   # packed tensor-memory variants: 32 / lanes queries per warp


def _units():
    """(source, object name, extra defines) of every translation unit."""
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.basename(src)
        if base == INST_SRC:
            units += [(src, f"mpf_inst_lg{lg}.o", [f"-DMPF_LG={lg}"]) for lg in INST_LANES]
            units.append((src, "mpf_inst_lg32_tm.o", ["-DMPF_LG=32", "-DMPF_TM=1"]))
            units += [(src, f"mpf_inst_qp{lg}_tm.o", [f"-DMPF_LG={lg}", "-DMPF_QP=1"]) for lg in QP_LANES]
        else:
            units.append((src, base.replace(".cu", ".o"), []))
    # The largest units first, so the parallel build ends sooner.
    units.sort(key=lambda u: (os.path.basename(u[0]) != INST_SRC, u[1]))
    return units


def _compile(unit, hdr_time: float, verbose: bool, debug: bool = False) -> str:
    src, obj_name, defines = unit
    obj = os.path.join(OBJ_DEBUG if debug else OBJ, obj_name)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time):
        return obj
    cmd = [_nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O2", *defines, "-I", os.path.join(ROOT, "include"), "-c", src,
           "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    if debug:
        cmd.insert(1, "-DMPF_DEBUG_CHECKS")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        print(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None, debug: bool = False) -> str:
    """Compile and link libmpf.so (libmpf_debug.so with debug=True); returns
    its path."""
    obj_dir, lib = (OBJ_DEBUG, LIB_DEBUG) if debug else (OBJ, LIB)
    os.makedirs(obj_dir, exist_ok=True)
    units = _units()
    hdr = _newest_header()
    jobs = jobs or min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda u: _compile(u, hdr, verbose, debug), units))
    # Objects of translation units that no longer exist must not be linked.
    stale = set(glob.glob(os.path.join(obj_dir, "*.o"))) - set(objs)
    for o in stale:
        os.remove(o)
    newest = max(os.path.getmtime(o) for o in objs)
    if os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    libdir = _cuda_lib_dir()
    cmd = [_nvcc(), ARCH, "-shared", "-cudart", "shared", "-o", lib + ".tmp", *objs,
           "-Xlinker", f"-rpath,{libdir}", "-L", libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(lib + ".tmp", lib)
    return lib


UBENCH_SRC = os.path.join(HERE, "ubench", "mpf_ubench.cu")
UBENCH_LIB = os.path.join(HERE, "libmpf_ubench.so")


def build_ubench() -> str:
    """Compile the roofline microbenchmarks (ubench/mpf_ubench.cu) into
    libmpf_ubench.so, apart from the scan library; returns its path."""
    if os.path.exists(UBENCH_LIB) and os.path.getmtime(UBENCH_LIB) >= os.path.getmtime(UBENCH_SRC):
        return UBENCH_LIB
    libdir = _cuda_lib_dir()
    cmd = [_nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-cudart", "shared", "-o", UBENCH_LIB + ".tmp", UBENCH_SRC,
           "-Xlinker", f"-rpath,{libdir}", "-L", libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {UBENCH_SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(UBENCH_LIB + ".tmp", UBENCH_LIB)
    return UBENCH_LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
