"""Builds liblqcd.so in-tree with nvcc for sm_103a (GB300).

Each csrc/*.cu is compiled to an object in parallel, then linked into
paper_1105_2279_gb300/liblqcd.so with the CUDA runtime linked statically
(the library shares the device's primary context with PyTorch).

    python -m paper_1105_2279_gb300.build          # or build_library()
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblqcd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def nvcc_path():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (set NVCC or put CUDA on PATH)")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(nvcc, src, verbose_ptxas=False):
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale(objs_srcs, lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(PKG), "include", "lqcd.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


JIT_PRELUDE_PARTS = ("geom.cuh", "su3.cuh", "expr_ops.cuh", "reduce.cuh")
JIT_PRELUDE = os.path.join(CSRC, "jit_prelude.inc")


def write_jit_prelude():
    """Embeds the NVRTC-compatible device headers as one raw string literal for
    the JIT (csrc/jit.cu); rewritten only when its content changes."""
    parts = []
    for name in JIT_PRELUDE_PARTS:
        with open(os.path.join(CSRC, name)) as f:
            lines = [ln for ln in f.read().splitlines()
                     if not ln.startswith('#include "') and ln.strip() != "#pragma once"]
        parts.append("\n".join(lines))
    text = 'R"LQJIT(\n' + "\n".join(parts) + '\n)LQJIT"\n'
    old = None
    if os.path.exists(JIT_PRELUDE):
        with open(JIT_PRELUDE) as f:
            old = f.read()
    if old != text:
        with open(JIT_PRELUDE, "w") as f:
            f.write(text)


def build_library(force=False, verbose_ptxas=False, jobs=None):
    """Compiles and links liblqcd.so if any source is newer; returns its path."""
    write_jit_prelude()
    if not force and not verbose_ptxas and not _stale(None, LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()
    srcs = sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, nvcc, s, verbose_ptxas) for s in srcs]
        objs = []
        for f in futs:
            o, log = f.result()
            objs.append(o)
            logs.append(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose_ptxas:
        sys.stderr.write("".join(logs))
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
