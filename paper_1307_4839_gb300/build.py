"""Build libswof.so in-tree with nvcc for sm_103a.

Each .cu file under csrc/ is compiled separately (in parallel); the FP64
units get -fmad=false so no multiply-add is contracted, and the same FP64
sources are compiled once more with contraction (swof_fp64c*.cu).  The result lands in
paper_1307_4839_gb300/_build/libswof.so (git-ignored).  build(debug=True)
builds the index-checking variant (-DSWOF_BOUNDS_CHECK=1) into
_build/debug/libswof_debug.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libswof.so")
BUILD_DEBUG = os.path.join(BUILD, "debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libswof_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
          "--expt-relaxed-constexpr"]
PER_FILE = {
    "swof_fp64.cu": ["-fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    "swof_fp32.cu": [],
    "swof_fp64_reg.cu": ["-fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    # the same two units with a*b+c contracted into FMAs (swof_set_fp64_contraction)
    "swof_fp64c.cu": ["-fmad=true", "-prec-div=true", "-prec-sqrt=true"],
    "swof_fp64c_reg.cu": ["-fmad=true", "-prec-div=true", "-prec-sqrt=true"],
    # the ensemble kernel reads, within one launch, data other CTAs wrote:
    # global loads bypass the (non-coherent) L1
    "swof_ens_fp64.cu": ["-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-Xptxas", "-dlcm=cg"],
    "swof_ens_fp32.cu": ["-Xptxas", "-dlcm=cg"],
}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libswof")


def sources() -> list[str]:
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


# units that include another .cu file
INCLUDES = {"swof_fp64c.cu": "swof_fp64.cu", "swof_fp64c_reg.cu": "swof_fp64_reg.cu"}


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    inc = INCLUDES.get(os.path.basename(src))
    deps = [src] + ([os.path.join(CSRC, inc)] if inc else []) + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "swof.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, debug: bool = False) -> str:
    out_dir = BUILD_DEBUG if debug else BUILD
    lib = LIB_DEBUG if debug else LIB
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for f in sources():
        src = os.path.join(CSRC, f)
        obj = os.path.join(out_dir, f.replace(".cu", ".o"))
        if force or _stale(obj, src):
            cmd = [nvcc, *ARCH, *COMMON, *PER_FILE.get(f, []), *(["-DSWOF_BOUNDS_CHECK=1"] if debug else []),
                   "-c", src, "-o", obj]
            if ptxas_v:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((f, cmd))
    objs = [os.path.join(out_dir, f.replace(".cu", ".o")) for f in sources()]

    def run(job):
        name, cmd = job
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_v:
            sys.stdout.write(r.stdout + r.stderr)
        return name

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if jobs or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv, debug="--debug" in sys.argv))
