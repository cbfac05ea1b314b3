"""Build libshacsim.so in-tree with nvcc for sm_103a (GB300).

Four translation units compiled in parallel, one -gencode, no cmake.  A fifth,
generated here, embeds the batched kernels' device sources for the library's
run-time compiler (model-specialised builds, shac_batch_specialize).
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
LIB = os.path.join(HERE, "libshacsim.so")
SOURCES = ["shac_api.cu", "shac_kernels.cu", "shac_learner.cu", "shac_jit.cu"]
HEADERS = ["shac_device.cuh", "shac_kernels.cuh", "shac_batched.cuh", "shac_jit.h"]
# device sources compiled again at run time, embedded as string constants
EMBEDDED = [("shac_jit_src_device", "shac_device.cuh"), ("shac_jit_src_kernels", "shac_kernels.cuh"),
            ("shac_jit_src_batched", "shac_batched.cuh")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def cuda_lib_dir() -> str:
    """lib64 of the CUDA toolkit whose nvcc builds the library (NVRTC lives there)."""
    path = shutil.which(nvcc()) or nvcc()
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(path))), "lib64")


def write_embedded_sources(path: str) -> None:
    """A C++ file defining each embedded device source as a string constant."""
    parts = ["// Generated by build.py: device sources compiled again at run time.\n"]
    for sym, name in EMBEDDED:
        text = open(os.path.join(CSRC, name)).read()
        assert ")SHACSRC\"" not in text
        parts.append(f'extern const char* const {sym};\nconst char* const {sym} = R"SHACSRC({text})SHACSRC";\n')
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write("".join(parts))
    os.replace(tmp, path)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "shacsim.h")]
    objs = []
    jobs = []
    emb = os.path.join(BUILD, "shac_jit_sources.cpp")
    if force or _stale(emb, [os.path.join(CSRC, n) for _, n in EMBEDDED] + [os.path.abspath(__file__)]):
        write_embedded_sources(emb)
    for src in SOURCES + [emb]:
        s = src if os.path.isabs(src) else os.path.join(CSRC, src)
        o = os.path.join(BUILD, os.path.basename(src).rsplit(".", 1)[0] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc(), *ARCH, *FLAGS, "-c", s, "-o", o]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for r in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs):
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
                if verbose:
                    sys.stderr.write(r.stderr)
    if force or jobs or _stale(LIB, objs):
        lib = cuda_lib_dir()
        cmd = [nvcc(), *ARCH, "-shared", "--cudart", "static", *objs, "-o", LIB + ".tmp", "-L" + lib, "-lnvrtc",
               "-Xlinker", "-rpath", "-Xlinker", lib]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
