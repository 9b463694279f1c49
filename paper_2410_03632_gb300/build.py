"""Build the in-tree CUDA library ``_lib/libblast.so`` for sm_103a with nvcc.

Each ``csrc/*.cu`` is compiled to an object in parallel, then linked into one
shared library against the shared CUDA runtime.  Rebuilds only when a source
or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_lib")
SO = os.path.join(OUT_DIR, "libblast.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
# Host code (the plan's quadrature nodes) is compiled without fused multiply-add
# contraction, so every node is the plain IEEE evaluation of its formula on any
# host: the basis integrand oscillates as j_l(k chi) with k chi up to ~1e5, so a
# node one ulp off shifts its phase by ~1e-11.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-I", INC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INC, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(SO):
        return False
    t = os.path.getmtime(SO)
    return all(os.path.getmtime(f) <= t for f in _deps())


PROBE_SRC = os.path.join(HERE, "probe", "peaks.cu")
PROBE_SO = os.path.join(OUT_DIR, "libpeaks.so")


def build_probe(force: bool = False) -> str:
    """The CUDA-core FMA peak microbenchmark (a separate library the benchmark
    loads to state ALU roofline denominators)."""
    if not force and os.path.exists(PROBE_SO) and os.path.getmtime(PROBE_SO) >= os.path.getmtime(PROBE_SRC):
        return PROBE_SO
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = PROBE_SO + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", PROBE_SRC, "-o", tmp,
                           "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {PROBE_SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_SO)
    return PROBE_SO


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    build_probe(force)
    if not force and up_to_date():
        return SO
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC] + ARCH + FLAGS + (extra or []) + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + [
        "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose=True))
