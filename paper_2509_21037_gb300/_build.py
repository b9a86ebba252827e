"""In-tree build of the native libraries (sm_103a CUDA + host C++).

Produces, next to this file in ``_lib/``:
  libsc.so        -- the Schur-complement C ABI (include/sc.h), CUDA kernels
  libsc_dense.so  -- dense cuBLAS TRSM+SYRK comparator (include/sc_dense.h)
  libscfactor.so  -- host sparse Cholesky input producer (include/sc_factor.h)
  libscpipe.so    -- CPU/GPU pipeline of the numeric stage (include/sc_pipeline.h),
                     linked against the two above
Translation units compile in parallel; one -gencode (sm_103a) only.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from typing import List

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_lib")
OBJ = os.path.join(OUT, "obj")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _nvcc_obj(src: str, obj: str, extra: List[str]) -> List[str]:
    cuda = _cuda_home()
    return [os.path.join(cuda, "bin", "nvcc"), *ARCH, "-O3", "-lineinfo", "-std=c++17",
            "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC, "--expt-relaxed-constexpr",
            *extra, "-c", src, "-o", obj]


def _run_parallel(cmds: List[List[str]]) -> None:
    procs = [(c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for c in cmds]
    failed = []
    for c, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((c, out.decode(errors="replace")))
    if failed:
        msg = "\n\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("native build failed:\n" + msg)


def build(verbose: bool = False, extra_nvcc: List[str] = ()) -> str:
    os.makedirs(OBJ, exist_ok=True)
    cuda = _cuda_home()
    cu_main = ["sc_plan.cpp", "sc_api.cu", "sc_kernels.cu", "sc_static.cu", "sc_split.cu", "sc_mlp.cu",
               "sc_implicit.cu", "sc_apply_fixed.cu", "sc_probe.cu", "sc_syrk_tc.cu", "sc_select.cu",
               "sc_apply_digits.cu"]
    objs_main = []
    cmds = []
    for s in cu_main:
        o = os.path.join(OBJ, s + ".o")
        objs_main.append(o)
        cmds.append(_nvcc_obj(os.path.join(CSRC, s), o, list(extra_nvcc)))
    o_pipe = os.path.join(OBJ, "sc_pipeline.cpp.o")
    cmds.append(_nvcc_obj(os.path.join(CSRC, "sc_pipeline.cpp"), o_pipe, list(extra_nvcc)))
    o_dense = os.path.join(OBJ, "sc_dense.cu.o")
    cmds.append(_nvcc_obj(os.path.join(CSRC, "sc_dense.cu"), o_dense, list(extra_nvcc)))
    cmds.append(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-I", INC,
                 os.path.join(CSRC, "host_factor.cpp"), os.path.join(CSRC, "host_apply.cpp"), "-pthread",
                 "-o", os.path.join(OUT, "libscfactor.so")])
    if verbose:
        for c in cmds:
            print(" ".join(c), file=sys.stderr)
    _run_parallel(cmds)
    nvcc = os.path.join(cuda, "bin", "nvcc")
    links = [
        [nvcc, *ARCH, "-shared", *objs_main, "-o", os.path.join(OUT, "libsc.so"), "-lcudart", "-lpthread"],
        [nvcc, *ARCH, "-shared", o_dense, "-o", os.path.join(OUT, "libsc_dense.so"),
         "-lcudart", "-lcublas"],
    ]
    _run_parallel(links)
    _run_parallel([[nvcc, *ARCH, "-shared", o_pipe, "-o", os.path.join(OUT, "libscpipe.so"), "-L", OUT, "-lsc",
                    "-lscfactor", "-lcudart", "-Xlinker", "-rpath,$ORIGIN"]])
    return OUT


if __name__ == "__main__":
    print(build(verbose=True))
