"""Builds liblagflux.so in-tree with nvcc for sm_103a (GB300).

Each .cu file is compiled to an object in parallel, then linked into a shared
library next to this file.  `-Xptxas -v` register and spill reports go to
_build/ptxas.log.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "liblagflux.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                 "-Xptxas", "-v"]


# Per-file extra flags: the FP32 kernels flush denormals (FP32 values below
# 1e-38 play no role in the scheme, and it keeps the special-function paths short).
# Both kernel units pin their rounding (-fmad=false; fused multiply-adds are
# written out where wanted), so results do not depend on how an expression
# was inlined.
EXTRA = {"lf_kernels_f32.cu": ["-ftz=true", "-fmad=false"], "lf_kernels_f64.cu": ["-fmad=false"],
         "lf_species_f32.cu": ["-ftz=true", "-fmad=false"], "lf_species_f64.cu": ["-fmad=false"],
         "lf_kernels3d_f32.cu": ["-ftz=true", "-fmad=false"], "lf_kernels3d_f64.cu": ["-fmad=false"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"),
                 shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set CUDA_HOME or NVCC)")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps() -> list[str]:
    inc = os.path.join(os.path.dirname(HERE), "include")
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(inc, f) for f in os.listdir(inc)]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, defines: dict | None = None, out: str | None = None) -> str:
    """Compiles and links the library.  `defines` (-D NAME=VALUE) and `out`
    (another library path, objects in a separate build folder) serve tuning
    sweeps of the launch shape; the default build uses neither."""
    lib = out or LIB
    if not force and not defines and out is None and up_to_date():
        return LIB
    bdir = BUILD if out is None else os.path.join(BUILD, os.path.basename(out) + ".d")
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    dflags = [f"-D{k}={v}" for k, v in (defines or {}).items()]

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *CFLAGS, *dflags, *EXTRA.get(os.path.basename(src), []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, sources()))
    with open(os.path.join(bdir, "ptxas.log"), "w") as f:
        for obj, log in results:
            f.write(f"== {os.path.basename(obj)}\n{log}\n")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
