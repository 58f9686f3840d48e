"""Build liblope.so in-tree for sm_103a (GB300).

Each CUDA translation unit under csrc/ is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a), then linked into one shared library
with the CUDA runtime linked statically, so the library loads on hosts without
a GPU driver (the driver is reached through cudaGetDriverEntryPointByVersion at
run time).  Usage: python -m paper_1502_03504_gb300.build [--force] [-v]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblope.so")
SOURCES = ["k_tma.cu", "k_tma_stage.cu", "k_generic.cu", "k_generic_rk.cu", "k_batch.cu",
           "k_reduce.cu", "jit.cu", "api.cu"]
# Device headers embedded in the library for run-time compiled local functions
# (jit.cu hands them to NVRTC); they compile under nvcc and NVRTC alike.
JIT_HEADERS = ["lope_internal.h", "device_common.cuh", "tma_device.cuh", "trap.cuh",
               "generic_device.cuh"]
JIT_GEN = "jit_headers.cpp"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the LOPe CUDA library cannot be built")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "lope.h"))
    return files


def _write_jit_headers() -> str:
    """Generate the C++ file holding the device headers as string constants."""
    delim = "LOPE_EMBED"
    out = ["// Generated by build.py: device headers for run-time compilation.",
           "namespace lope {", f"extern const int kJitHeaderCount = {len(JIT_HEADERS)};",
           "extern const char* const kJitHeaderNames[] = {"]
    out += [f'    "{h}",' for h in JIT_HEADERS]
    out += ["};", "extern const char* const kJitHeaderTexts[] = {"]
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h)) as fh:
            text = fh.read()
        if f"){delim}" in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        out.append(f'    R"{delim}({text}){delim}",')
    out += ["};", "}  // namespace lope", ""]
    path = os.path.join(BUILD, JIT_GEN)
    with open(path, "w") as fh:
        fh.write("\n".join(out))
    return path


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
    path = src if os.path.isabs(src) else os.path.join(CSRC, src)
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, "-c", path, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link liblope.so next to this file; returns its path."""
    newest = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    sources = SOURCES + [_write_jit_headers()]
    with cf.ThreadPoolExecutor(max_workers=len(sources)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), sources))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
