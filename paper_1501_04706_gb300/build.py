"""Build libqh.so (the C-ABI hull library) in-tree for sm_103a with nvcc.

The translation units compile in parallel; the shared library links the CUDA
runtime statically.  The result goes to ``paper_1501_04706_gb300/_build/``.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libqh.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["qh_rounds.cu", "qh_finish.cu", "qh_api.cu", "qh_noalloc.cu", "qh_sorted.cu"]
# Translation units: (source, object name, flags).  The grid-wide kernel is compiled once per variant
# (threads per CTA, points per thread, CTAs per SM it is built for), each in its own namespace; the plan
# picks one at run time.
UNITS = [("qh_rounds.cu", "qh_rounds_v256", ["-DQH_NT=256", "-DQH_IPT=16", "-DQH_MINB=2", "-DQH_VARIANT_NS=v256"]),
         ("qh_rounds.cu", "qh_rounds_v256i8", ["-DQH_NT=256", "-DQH_IPT=8", "-DQH_MINB=3", "-DQH_VARIANT_NS=v256i8"]),
         ("qh_rounds.cu", "qh_rounds_v128", ["-DQH_NT=128", "-DQH_IPT=16", "-DQH_MINB=4", "-DQH_VARIANT_NS=v128"]),
         ("qh_rounds.cu", "qh_rounds_v128i8", ["-DQH_NT=128", "-DQH_IPT=8", "-DQH_MINB=6", "-DQH_VARIANT_NS=v128i8"]),
         ("qh_finish.cu", "qh_finish", []),
         ("qh_api.cu", "qh_api", []),
         ("qh_noalloc.cu", "qh_noalloc", []),
         ("qh_sorted.cu", "qh_sorted", [])]
HEADERS = ["qh_internal.cuh", "qh_predicates.cuh", "qh_sorted.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
              "-Xptxas", "-warn-spills", "-I", INCLUDE]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "qh.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          out_path: str | None = None) -> str:
    """Compile (if sources changed) and return the path of libqh.so.

    ``extra`` adds nvcc flags; with ``out_path`` the library (and its objects)
    go to another file, e.g. for an experiment build with extra defines.
    """
    lib_path = out_path or LIB_PATH
    if out_path is None and not force and not _stale():
        return LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = "" if out_path is None else "_" + os.path.splitext(os.path.basename(out_path))[0]
    nvcc = _nvcc()
    extra = list(extra or [])

    def compile_one(unit) -> str:
        src, name, flags = unit
        obj = os.path.join(OUT_DIR, name + tag + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *flags, *extra]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=OUT_DIR)
    os.close(fd)
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
