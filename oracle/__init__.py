"""CPU oracle for the 2D convex hull -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (``paper_1501_04706_gb300``) never
imports, links or runs it, and the two share no code.

The C source ``qh_oracle.c`` holds the arithmetic; this module compiles it with
gcc into ``oracle/_build`` on first use and wraps it with ctypes.

Functions (all inputs are float32 point arrays of shape [n, 2]):

``hull2d(points)``            monotone chain with exact predicates; returns the
                              CCW hull vertex indices starting at the
                              lexicographically smallest point (problem
                              statement, Sec. 1).
``quickhull(points, mode)``   generation-synchronous QuickHull (Sec. 3-4.4);
                              returns (indices, live counts per generation).
``hull2d_batched(points, offsets)``  per-set monotone chain over a CSR batch.
``orient_sign`` / ``dist_cmp``  the exact predicates themselves, for pinning.

Parity status: pinned.  The tests check every function against brute force on
small inputs (exact rational arithmetic), closed forms, invariants that hold at
any size and metamorphic relations; see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

STATUS = {0: "ok", 1: "invalid argument", 2: "non-finite input", 4: "out of memory",
          7: "internal inconsistency"}
NONFINITE = 2

_libs: dict[int, ctypes.CDLL] = {}


def build(mutation: int = 0, force: bool = False) -> str:
    """Compile the oracle (optionally with a planted mistake); return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    name = "liboracle.so" if mutation == 0 else f"liboracle_m{mutation}.so"
    out = os.path.join(_BUILD, name)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
        os.close(fd)
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               f"-DQHO_MUTATION={mutation}", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _lib(mutation: int = 0) -> ctypes.CDLL:
    if mutation not in _libs:
        lib = ctypes.CDLL(build(mutation))
        f32, i32, i64 = ctypes.c_float, ctypes.c_int32, ctypes.c_int64
        vp = ctypes.c_void_p
        lib.qho_orient_sign.argtypes = [f32] * 6 + [ctypes.c_int]
        lib.qho_orient_sign.restype = ctypes.c_int
        lib.qho_dist_cmp.argtypes = [f32] * 8 + [ctypes.c_int]
        lib.qho_dist_cmp.restype = ctypes.c_int
        lib.qho_hull2d.argtypes = [vp, i64, vp, vp, ctypes.c_int]
        lib.qho_hull2d.restype = ctypes.c_int
        lib.qho_hull2d_batched.argtypes = [vp, vp, i32, vp, vp, ctypes.c_int]
        lib.qho_hull2d_batched.restype = ctypes.c_int
        lib.qho_quickhull.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp, ctypes.c_int, vp]
        lib.qho_quickhull.restype = ctypes.c_int
        _libs[mutation] = lib
    return _libs[mutation]


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle rejected the input: {STATUS.get(status, status)}")
        self.status = status


def _points(points) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(points, dtype=np.float32))
    if p.ndim != 2 or p.shape[1] != 2:
        raise ValueError("points must have shape [n, 2]")
    return p


def orient_sign(a, b, c, always_exact: bool = False, mutation: int = 0) -> int:
    return _lib(mutation).qho_orient_sign(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                          float(c[0]), float(c[1]), int(always_exact))


def dist_cmp(u, v, p, q, always_exact: bool = False, mutation: int = 0) -> int:
    """sign(dist(p) - dist(q)) where dist(x) = -orient(u, v, x) (distance right of u->v)."""
    return _lib(mutation).qho_dist_cmp(float(u[0]), float(u[1]), float(v[0]), float(v[1]),
                                       float(p[0]), float(p[1]), float(q[0]), float(q[1]),
                                       int(always_exact))


def hull2d(points, always_exact: bool = False, mutation: int = 0) -> np.ndarray:
    p = _points(points)
    n = p.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    cnt = ctypes.c_int64(0)
    st = _lib(mutation).qho_hull2d(p.ctypes.data, n, out.ctypes.data, ctypes.byref(cnt),
                                   int(always_exact))
    if st != 0:
        raise OracleError(st)
    return out[: cnt.value].copy()


def hull2d_batched(points, offsets, always_exact: bool = False):
    """Returns (out int32[N], counts int32[num_sets]); set s's hull is out[offsets[s]:][:counts[s]]."""
    p = _points(points)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    num_sets = off.shape[0] - 1
    out = np.zeros(max(p.shape[0], 1), dtype=np.int32)
    counts = np.zeros(max(num_sets, 1), dtype=np.int32)
    _lib().qho_hull2d_batched(p.ctypes.data, off.ctypes.data, num_sets, out.ctypes.data,
                              counts.ctypes.data, int(always_exact))
    return out[: p.shape[0]], counts[:num_sets]


def quickhull(points, mode: str = "quad", max_gen: int = 4096, mutation: int = 0):
    """Returns (hull indices, live point count after each generation)."""
    p = _points(points)
    n = p.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    live = np.zeros(max_gen, dtype=np.int64)
    cnt = ctypes.c_int64(0)
    ngen = ctypes.c_int(0)
    m = {"chord": 0, "quad": 1}[mode]
    st = _lib(mutation).qho_quickhull(p.ctypes.data, n, m, out.ctypes.data, ctypes.byref(cnt),
                                      live.ctypes.data, max_gen, ctypes.byref(ngen))
    if st != 0:
        raise OracleError(st)
    g = min(ngen.value, max_gen)
    return out[: cnt.value].copy(), live[:g].copy()


# ---------------------------------------------------------------------------
# All-core timing build (the CPU baseline of bench.py): the same source plus a
# driver that hulls contiguous chunks in threads and then the union of the
# chunk hulls; its output is hull2d's output.
# ---------------------------------------------------------------------------
_SRC_PAR = os.path.join(_HERE, "qh_oracle_parallel.c")
_par_lib: list = []


def build_parallel(force: bool = False) -> str:
    """Compile the all-core driver (includes qh_oracle.c unchanged); return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liboracle_par.so")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PAR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
        os.close(fd)
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-pthread",
               "-DQHO_MUTATION=0", "-o", tmp, _SRC_PAR, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def host_threads() -> int:
    """Threads the all-core driver uses: the cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def hull2d_parallel(points, threads: int | None = None) -> np.ndarray:
    """hull2d's result, computed on `threads` host threads (default: all cores)."""
    if not _par_lib:
        lib = ctypes.CDLL(build_parallel())
        lib.qho_hull2d_parallel.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int]
        lib.qho_hull2d_parallel.restype = ctypes.c_int
        _par_lib.append(lib)
    p = _points(points)
    n = p.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    cnt = ctypes.c_int64(0)
    st = _par_lib[0].qho_hull2d_parallel(p.ctypes.data, n, out.ctypes.data, ctypes.byref(cnt),
                                         int(threads or host_threads()))
    if st != 0:
        raise OracleError(st)
    return out[: cnt.value].copy()
