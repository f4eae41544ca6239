"""Python binding of libqh.so, the GB300 segmented-QuickHull library.

Argument marshalling only: every step of the hull runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  The library must have
been built (``__graft_entry__.build()`` or ``python -m paper_1501_04706_gb300.build``);
loading fails loudly otherwise -- there is no CPU fallback.

Method: Zhang, Mei, Xu, Zhao, "A Novel Implementation of QuickHull Algorithm on
the GPU" (segmented QuickHull, Sec. 3-4).  Output: CCW hull vertex indices from
the lexicographically smallest point, collinear boundary points excluded,
duplicates represented by their lowest index.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

__all__ = [
    "QhError", "Plan", "load", "hull2d", "hull2d_batched", "hull2d_host", "check_orient_host",
    "check_orient_device", "check_dist_host", "check_dist_device", "MODE_QUAD", "MODE_CHORD",
    "PREC_F32", "PREC_F64", "STATUS",
]

MODE_QUAD, MODE_CHORD = 0x0, 0x1
PREC_F32, PREC_F64 = 0x0, 0x2
MAX_GEN = 512

STATUS = {0: "ok", 1: "invalid argument", 2: "non-finite input coordinate", 3: "CUDA runtime error",
          4: "out of device memory", 5: "capacity exceeded", 6: "device-side wait timed out",
          7: "internal error", 8: "unsupported in this context"}


class QhError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class _Stats(ctypes.Structure):
    _fields_ = [("device_status", ctypes.c_int32), ("global_rounds", ctypes.c_int32),
                ("generations", ctypes.c_int32), ("small_problems", ctypes.c_int32),
                ("nodes", ctypes.c_int32), ("big_sets", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("pad0", ctypes.c_int32), ("live", ctypes.c_int64 * MAX_GEN), ("exact_orient", ctypes.c_int64),
                ("exact_compare", ctypes.c_int64), ("phase_ms", ctypes.c_float * 5),
                ("grid_phase_us", ctypes.c_float * 16), ("grid_points", ctypes.c_int64), ("grid_read", ctypes.c_int64), ("grid_written", ctypes.c_int64),
                ("small_points", ctypes.c_int64)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libqh.so (built in-tree); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libqh.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    lib.qh_plan_create.argtypes = [i64, i32, u32, ctypes.POINTER(vp)]
    lib.qh_plan_destroy.argtypes = [vp]
    lib.qh_plan_set_flags.argtypes = [vp, u32]
    lib.qh_plan_set_tuning.argtypes = [vp, i32, i32, i32]
    lib.qh_plan_set_block.argtypes = [vp, i32]
    lib.qh_plan_set_debug.argtypes = [vp, u32, i32]
    lib.qh_plan_set_items_per_thread.argtypes = [vp, i32]
    lib.qh_hull2d_noalloc.argtypes = [vp, i64, vp, vp, vp]
    lib.qh_plan_get_tuning.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                       ctypes.POINTER(i32)]
    lib.qh_plan_autotune.argtypes = [vp, vp, vp, i32, i64, vp, vp, i32, vp]
    lib.qh_hull2d_p.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.qh_hull2d.argtypes = [vp, i64, vp, vp, vp]
    lib.qh_hull2d_batched.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    lib.qh_hull2d_host.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.qh_hull2d_sorted.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.qh_plan_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    lib.qh_status_string.argtypes = [ctypes.c_int]
    lib.qh_status_string.restype = ctypes.c_char_p
    lib.qh_version.restype = i32
    lib.qh_check_orient_host.argtypes = [vp, i64, i32, vp, vp]
    lib.qh_check_orient_device.argtypes = [vp, i64, i32, vp, vp, vp]
    lib.qh_check_dist_host.argtypes = [vp, i64, vp]
    lib.qh_check_dist_device.argtypes = [vp, i64, vp, vp]
    for f in ("qh_plan_create", "qh_plan_destroy", "qh_plan_set_flags", "qh_plan_set_tuning", "qh_plan_set_block",
              "qh_plan_set_debug", "qh_hull2d_noalloc", "qh_plan_set_items_per_thread",
              "qh_plan_get_tuning", "qh_plan_autotune", "qh_hull2d_p",
              "qh_hull2d", "qh_hull2d_batched", "qh_hull2d_host", "qh_hull2d_sorted", "qh_plan_get_stats",
              "qh_check_orient_host",
              "qh_check_orient_device", "qh_check_dist_host", "qh_check_dist_device"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st: int, where: str) -> None:
    if st != 0:
        raise QhError(st, where)


def _stream(device=None) -> int:
    import torch

    return torch.cuda.current_stream(device).cuda_stream


TUNE_CACHE_ENV = "QH_TUNE_CACHE"
_build_id: list = []


def library_build_id() -> str:
    """Content hash of the library's sources: a tuning stored by another build is not reused."""
    if not _build_id:
        import hashlib

        h = hashlib.sha256()
        here = os.path.dirname(os.path.abspath(__file__))
        csrc = os.path.join(here, "csrc")
        for f in sorted(os.listdir(csrc)) + [os.path.join("..", "..", "include", "qh.h")]:
            path = os.path.join(csrc, f)
            if os.path.isfile(path):
                with open(path, "rb") as fh:
                    h.update(fh.read())
        _build_id.append(h.hexdigest()[:12])
    return _build_id[0]


def tune_cache_key(device_name: str, capability, flags: int, num_sets: int, n: int) -> str:
    """Key of a stored tuning: GPU, library build and the call's configuration."""
    return (f"{device_name}|sm{int(capability[0])}{int(capability[1])}|build={library_build_id()}"
            f"|flags={int(flags)}|sets={int(num_sets)}|n={int(n)}")


def tune_cache_load(path: str) -> dict:
    """The stored tunings (empty when the file is missing or unreadable)."""
    import json

    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get("entries", {})
        return e if isinstance(e, dict) else {}
    except (OSError, ValueError):
        return {}


def tune_cache_store(path: str, key: str, tuning: dict) -> None:
    """Add one tuning to the file (written to a temporary file, then renamed into place)."""
    import json
    import tempfile

    entries = tune_cache_load(path)
    entries[key] = {k: int(tuning[k]) for k in ("threads_per_block", "items_per_thread", "cutover",
                                                  "grid_ctas_per_sm")}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".json", dir=d)
    with os.fdopen(fd, "w") as f:
        json.dump({"version": 1, "entries": entries}, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Plan:
    """Device scratch for hulls of up to ``max_points`` points in up to ``max_sets`` sets."""

    def __init__(self, max_points: int, max_sets: int = 1, mode: int = MODE_QUAD, prec: int = PREC_F32):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.qh_plan_create(int(max_points), int(max_sets), mode | prec, ctypes.byref(h)), "qh_plan_create")
        self.handle = h
        self.max_points = int(max_points)
        self.max_sets = int(max_sets)
        self.flags = mode | prec

    def close(self) -> None:
        if self.handle:
            load().qh_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_flags(self, mode: int = MODE_QUAD, prec: int = PREC_F32) -> None:
        _check(load().qh_plan_set_flags(self.handle, mode | prec), "qh_plan_set_flags")
        self.flags = mode | prec

    def set_tuning(self, cutover: int = 4096, timing: bool = False, ctas_per_sm: int = 0) -> None:
        _check(load().qh_plan_set_tuning(self.handle, int(cutover), int(bool(timing)), int(ctas_per_sm)),
               "qh_plan_set_tuning")

    def set_block(self, threads: int) -> None:
        """Block size of the grid-wide kernel: 256 or 128 threads."""
        _check(load().qh_plan_set_block(self.handle, int(threads)), "qh_plan_set_block")

    def set_items_per_thread(self, ipt: int) -> None:
        """Points per thread per tile of the grid-wide kernel: 16 or 8 (a tile is threads x ipt points)."""
        _check(load().qh_plan_set_items_per_thread(self.handle, int(ipt)), "qh_plan_set_items_per_thread")

    def set_debug(self, spin_limit: int = 0, max_tree_nodes: int = 0) -> None:
        """Debug limits for the device-side error paths (0 = default): grid-barrier polls before a
        wait gives up (QH_ERR_TIMEOUT) and the segment-tree capacity (QH_ERR_CAPACITY)."""
        _check(load().qh_plan_set_debug(self.handle, int(spin_limit), int(max_tree_nodes)), "qh_plan_set_debug")

    def tuning(self) -> dict:
        v = [ctypes.c_int32() for _ in range(4)]
        _check(load().qh_plan_get_tuning(self.handle, *[ctypes.byref(x) for x in v]), "qh_plan_get_tuning")
        return {"threads_per_block": v[0].value, "items_per_thread": v[1].value, "cutover": v[2].value,
                "grid_ctas_per_sm": v[3].value}

    def apply_tuning(self, t: dict) -> None:
        """Set block size, points per thread, cutover and grid CTAs per SM from a tuning dict."""
        self.set_block(int(t["threads_per_block"]))
        self.set_items_per_thread(int(t["items_per_thread"]))
        self.set_tuning(int(t["cutover"]), False, int(t["grid_ctas_per_sm"]))

    def autotune(self, points, offsets=None, out=None, counts=None, reps: int = 3, cache: str | None = None) -> dict:
        """Time every candidate setting on this input (each one's output checked against the plan's current
        setting on the device), keep the fastest; returns the chosen tuning with ``cached``.

        With a cache file (``cache``, else the ``QH_TUNE_CACHE`` environment variable) the result is stored
        under a key of GPU name, compute capability, library build, flags, set count and point count, and a
        later call with the same key applies the stored tuning without timing anything."""
        import torch

        pts = _points_tensor(points)
        dev = pts.device
        if offsets is None:
            num_sets, off_ptr = 1, None
        else:
            off = offsets.to(device=dev, dtype=torch.int64).contiguous()
            num_sets, off_ptr = off.shape[0] - 1, off.data_ptr()
        path = cache if cache is not None else os.environ.get(TUNE_CACHE_ENV)
        key = None
        if path:
            key = tune_cache_key(torch.cuda.get_device_name(dev), torch.cuda.get_device_capability(dev),
                                 self.flags, num_sets, pts.shape[0])
            hit = tune_cache_load(path).get(key)
            if hit is not None:
                self.apply_tuning(hit)
                return dict(self.tuning(), cached=True)
        if out is None:
            out = torch.empty(max(pts.shape[0], 1), dtype=torch.int32, device=dev)
        if counts is None:
            counts = torch.empty(max(num_sets, 1), dtype=torch.int32, device=dev)
        _check(load().qh_plan_autotune(self.handle, pts.data_ptr(), off_ptr, num_sets, pts.shape[0], out.data_ptr(),
                                       counts.data_ptr(), int(reps), _stream(dev)), "qh_plan_autotune")
        t = self.tuning()
        if path:
            tune_cache_store(path, key, t)
        return dict(t, cached=False)

    def stats(self) -> dict:
        s = _Stats()
        _check(load().qh_plan_get_stats(self.handle, ctypes.byref(s)), "qh_plan_get_stats")
        g = s.generations
        return {"device_status": s.device_status, "global_rounds": s.global_rounds, "generations": g,
                "small_problems": s.small_problems, "nodes": s.nodes, "big_sets": s.big_sets, "levels": s.levels,
                "live": [int(v) for v in s.live[: min(g, MAX_GEN)]], "exact_orient": int(s.exact_orient),
                "exact_compare": int(s.exact_compare), "phase_ms": [float(v) for v in s.phase_ms],
                "grid_phase_us": [float(v) for v in s.grid_phase_us if v > 0], "grid_points": int(s.grid_points),
                "grid_read": int(s.grid_read), "grid_written": int(s.grid_written),
                "small_points": int(s.small_points)}


def _points_tensor(points):
    import torch

    if not isinstance(points, torch.Tensor) or not points.is_cuda:
        raise ValueError("points must be a CUDA tensor")
    if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 2:
        raise ValueError("points must be float32 of shape [n, 2]")
    return points.contiguous()


def hull2d(points, plan: Plan | None = None, out=None, count=None, sync: bool = True):
    """Hull of one point set (CUDA float32 tensor [n, 2]).

    Returns the int32 index tensor (synchronizes to read the count) or, with
    ``sync=False``, the (out, count) device tensors without synchronizing.
    """
    import torch

    lib = load()
    pts = _points_tensor(points)
    n = pts.shape[0]
    dev = pts.device
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if count is None:
        count = torch.empty(1, dtype=torch.int32, device=dev)
    s = _stream(dev)
    if plan is None:
        st = lib.qh_hull2d(pts.data_ptr(), n, out.data_ptr(), count.data_ptr(), s)
    else:
        st = lib.qh_hull2d_p(plan.handle, pts.data_ptr(), n, out.data_ptr(), count.data_ptr(), s)
    _check(st, "qh_hull2d")
    if not sync:
        return out, count
    c = int(count.item())
    if c < 0:
        raise QhError(-c, "qh_hull2d (device)")
    return out[:c]


def hull2d_batched(points, offsets, plan: Plan, out=None, counts=None):
    """Hulls of a CSR batch; returns (out int32[N], counts int32[num_sets]) without synchronizing.

    Set s's hull (indices local to the set) is out[offsets[s] : offsets[s] + counts[s]].
    """
    import torch

    lib = load()
    pts = _points_tensor(points)
    off = offsets.to(device=pts.device, dtype=torch.int64).contiguous()
    num_sets = off.shape[0] - 1
    if out is None:
        out = torch.empty(max(pts.shape[0], 1), dtype=torch.int32, device=pts.device)
    if counts is None:
        counts = torch.empty(max(num_sets, 1), dtype=torch.int32, device=pts.device)
    _check(lib.qh_hull2d_batched(plan.handle, pts.data_ptr(), off.data_ptr(), num_sets, out.data_ptr(),
                                 counts.data_ptr(), _stream(pts.device)), "qh_hull2d_batched")
    return out, counts[:num_sets]


def hull2d_sorted(points, plan: Plan, out=None, count=None):
    """Hull of one point set by the x-sorted form of the rounds (qh_hull2d_sorted).

    Same result as ``hull2d`` for the plan's flags; the call synchronizes the stream.
    Returns the int32 index tensor.
    """
    import torch

    lib = load()
    pts = _points_tensor(points)
    n = pts.shape[0]
    dev = pts.device
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if count is None:
        count = torch.empty(1, dtype=torch.int32, device=dev)
    _check(lib.qh_hull2d_sorted(plan.handle, pts.data_ptr(), n, out.data_ptr(), count.data_ptr(), _stream(dev)),
           "qh_hull2d_sorted")
    c = int(count.item())
    if c < 0:
        raise QhError(-c, "qh_hull2d_sorted (device)")
    return out[:c]


def hull2d_host(points: np.ndarray, plan: Plan, out: np.ndarray | None = None) -> np.ndarray:
    """End-to-end form with host buffers (copies inside the call); synchronizes."""
    lib = load()
    p = np.ascontiguousarray(points, dtype=np.float32)
    n = p.shape[0]
    if out is None:
        out = np.empty(max(n, 1), dtype=np.int32)
    cnt = ctypes.c_int32(0)
    _check(lib.qh_hull2d_host(plan.handle, p.ctypes.data, n, out.ctypes.data, ctypes.byref(cnt), _stream()),
           "qh_hull2d_host")
    return out[: cnt.value]


def check_orient_host(tri: np.ndarray, prec: int = 0):
    """Filtered orientation of triples (float32 [n, 6]) on the CPU: (sign, certified)."""
    lib = load()
    t = np.ascontiguousarray(tri, dtype=np.float32).reshape(-1, 6)
    n = t.shape[0]
    sign = np.zeros(n, dtype=np.int32)
    cert = np.zeros(n, dtype=np.int32)
    _check(lib.qh_check_orient_host(t.ctypes.data, n, int(prec), sign.ctypes.data, cert.ctypes.data),
           "qh_check_orient_host")
    return sign, cert


def check_orient_device(tri, prec: int = 0):
    import torch

    lib = load()
    t = tri.contiguous()
    n = t.shape[0]
    sign = torch.zeros(n, dtype=torch.int32, device=t.device)
    cert = torch.zeros(n, dtype=torch.int32, device=t.device)
    _check(lib.qh_check_orient_device(t.data_ptr(), n, int(prec), sign.data_ptr(), cert.data_ptr(),
                                      _stream(t.device)), "qh_check_orient_device")
    return sign, cert


def check_dist_host(quads: np.ndarray):
    lib = load()
    q = np.ascontiguousarray(quads, dtype=np.float32).reshape(-1, 8)
    sign = np.zeros(q.shape[0], dtype=np.int32)
    _check(lib.qh_check_dist_host(q.ctypes.data, q.shape[0], sign.ctypes.data), "qh_check_dist_host")
    return sign


def check_dist_device(quads):
    import torch

    lib = load()
    q = quads.contiguous()
    sign = torch.zeros(q.shape[0], dtype=torch.int32, device=q.device)
    _check(lib.qh_check_dist_device(q.data_ptr(), q.shape[0], sign.data_ptr(), _stream(q.device)),
           "qh_check_dist_device")
    return sign
