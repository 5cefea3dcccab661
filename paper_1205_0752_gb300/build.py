"""Builds libgfc.so in-tree with nvcc for sm_103a (one -gencode, translation
units compiled in parallel). Run ``python -m paper_1205_0752_gb300.build``."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgfc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["gfc_kernels.cu", "gfc_capi.cpp", "gfc_server.cpp", "gfc_router.cpp", "gfc_noalloc.cu",
           "gfc_diag.cu", "gfc_probe.cu"]
# gfc_eval_inst.cu is compiled once per (arithmetic, unrolled angular pair
# count) so that the kernel instantiations build in parallel; double-float
# has the generic loop only
INSTANCES = [(t, n) for t in ("double", "float") for n in (32, 64, 128, 0)] + [("df", 0)]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "gfc.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.isfile(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    # no FMA contraction in host code: the grid checks must round like the
    # kernels' explicitly rounded grid arithmetic on every host architecture
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
                     "-I", INCLUDE, "-I", CSRC]
    units = [(s, []) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    units += [("gfc_eval_inst.cu", [f"-DGFC_INST_T={t}", f"-DGFC_INST_NP={n}"]) for t, n in INSTANCES]

    def compile_one(unit):
        src, defs = unit
        tag = "".join(d.split("=")[1] for d in defs)
        obj = os.path.join(BUILD, src + tag + f".{os.getpid()}.o")
        cmd = [nvcc] + common + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    # largest units first, so the longest compiles start at once
    units.sort(key=lambda u: (not u[1], u[0] != "gfc_kernels.cu"))
    workers = max(1, min(len(units), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
