"""Build the CUDA library liblbm.so in-tree (paper_1510_08886_gb300/_build).

nvcc for sm_103a only, one object per translation unit compiled in
parallel, then one shared-library link.  ``python -m
paper_1510_08886_gb300.build [-v]`` rebuilds; ``-v`` adds ``-Xptxas -v``
(registers, spills, shared memory per kernel).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "liblbm.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["k_fp64.cu", "k_cluster.cu", "k_fp32.cu", "k_fp16.cu", "k_bf16.cu", "engine_fp32.cu", "engine_fp16.cu",
           "engine_fp64.cu", "engine_res_fp64.cu",
           "engine_bf16.cu", "engine_res_fp32.cu", "engine_res_half.cu", "engine_res_bf16.cu",
           "lbm_engine.cu", "lbm_api.cu", "lbm_noalloc.cu", "peak_probe.cu", "dvm.cpp", "dvm_gen.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "lbm.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False):
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              "-I", CSRC] + ARCH
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-c",
                   os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ([nvcc, "-shared", "-cudart", "static"] + ARCH + ["-o", tmp]
           + [o for o, _ in results])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
