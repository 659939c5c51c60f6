"""Build libnpweno.so (the CUDA library behind include/npweno.h) in-tree for sm_103a.

Seven translation units are compiled in parallel with nvcc and linked into one shared
object next to this file:
  npw_fp64.cu  -- double-precision kernels, --fmad=false (each operation rounded as written)
  npw_fp32.cu  -- mixed-precision kernels, also --fmad=false: every fused multiply-add is an
                  explicit fmaf, so the per-stage and the resident kernels (and any batch mix)
                  produce the same bits from the same data
  npw_queue_fp64.cu, npw_queue_fp32.cu -- the work-queue kernels of each precision, one per
                  instance shape (also --fmad=false)
  npw_api.cu   -- host runtime and the C ABI
  npw_noalloc.cu -- npweno_rk3_step_noalloc and its fixed device scratch array
  npw_format.cu  -- npw_format_check, the self-check of the integer float<->double format changes
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libnpweno.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}",
          "--expt-relaxed-constexpr", "-diag-suppress", "128"]
UNITS = {
    "npw_fp64.cu": ["--fmad=false"],
    "npw_fp32.cu": ["--fmad=false"],
    "npw_queue_fp64.cu": ["--fmad=false"],
    "npw_queue_fp32.cu": ["--fmad=false"],
    "npw_api.cu": [],
    "npw_noalloc.cu": [],
    "npw_format.cu": ["--fmad=false"],
}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    out = [os.path.join(INCLUDE, "npweno.h")]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(item):
        src, extra = item
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS.items()))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
