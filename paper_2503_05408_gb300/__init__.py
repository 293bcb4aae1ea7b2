"""Thin Python binding of ``libsptrsv.so`` (the C ABI declared in include/sptrsv.h).

Argument marshalling only: every step of the solve runs in the library's own
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback - if the in-tree library has not been built the import of this
module succeeds but every call raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsptrsv.so")

# ---------------------------------------------------------------- constants
OK = 0
ERR_ARG, ERR_NOT_LOWER, ERR_UNSORTED_OR_DUP, ERR_ZERO_DIAG = -1, -2, -3, -4
ERR_OOM, ERR_BUDGET, ERR_CUDA, ERR_LAUNCH, ERR_TIMEOUT = -5, -6, -7, -8, -9
ERR_NOT_CONVERGED, ERR_PENDING, ERR_NO_DEVICE, ERR_IO = -10, -11, -12, -13

SCHED_LEVELS, SCHED_GROWLOCAL = 0, 1
TRI_LOWER, TRI_UPPER, TRI_LOWER_TRANSPOSED = 0, 1, 2
_TRI = {"lower": TRI_LOWER, "upper": TRI_UPPER, "lower_transposed": TRI_LOWER_TRANSPOSED}
COARSEN_NONE, COARSEN_FUNNEL = 0, 1
_COARSEN = {"none": COARSEN_NONE, "funnel": COARSEN_FUNNEL}
VALUES_F64, VALUES_F32 = 1, 2
F64, F32 = 0, 1
SYNC_AUTO, SYNC_GRID, SYNC_FLAGS, SYNC_CTA, SYNC_CTA_REGS, SYNC_LOCAL, SYNC_CHUNKS, SYNC_RESIDENT = range(8)
PART_AUTO, PART_PARENTS, PART_RANGES, PART_GRID = 0, 1, 2, 3
PREC_F64, PREC_F32_REFINE = 0, 1

SYNC_NAMES = {SYNC_AUTO: "auto", SYNC_GRID: "grid", SYNC_FLAGS: "flags", SYNC_CTA: "cta",
              SYNC_CTA_REGS: "cta_regs", SYNC_LOCAL: "local", SYNC_CHUNKS: "chunks",
              SYNC_RESIDENT: "resident"}
_SYNC = {v: k for k, v in SYNC_NAMES.items()}
_MODE = {"levels": SCHED_LEVELS, "growlocal": SCHED_GROWLOCAL}
_PREC = {"f64": PREC_F64, "f32_refine": PREC_F32_REFINE}
_PART = {"auto": PART_AUTO, "parents": PART_PARENTS, "ranges": PART_RANGES, "grid": PART_GRID}


class SptrsvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


# ---------------------------------------------------------------- structs
class CSRStruct(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class AnalyzeOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("k", ctypes.c_int32), ("alpha0", ctypes.c_double),
                ("growth", ctypes.c_double), ("L", ctypes.c_double), ("accept", ctypes.c_double),
                ("values", ctypes.c_int32), ("device", ctypes.c_int32), ("triangle", ctypes.c_int32),
                ("sched_blocks", ctypes.c_int32), ("sched_threads", ctypes.c_int32),
                ("coarsen", ctypes.c_int32), ("coarsen_max_weight", ctypes.c_double),
                ("analyze_on_device", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("supersteps", ctypes.c_int32), ("k", ctypes.c_int32), ("max_level_rows", ctypes.c_int32),
                ("avg_wavefront", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("analyze_ms", ctypes.c_double), ("phases", ctypes.c_int32), ("ring_rows", ctypes.c_int32),
                ("schedule_ms", ctypes.c_double), ("sched_blocks", ctypes.c_int32),
                ("coarse_vertices", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("sync", ctypes.c_int32), ("lanes", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("refine_tol", ctypes.c_double),
                ("blocks_per_sm", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("timeout_s", ctypes.c_double), ("rhs_tile", ctypes.c_int32),
                ("eager_sum", ctypes.c_int32), ("partition", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("barriers", ctypes.c_int64),
                ("flag_waits", ctypes.c_int64), ("dnorm", ctypes.c_double), ("sync", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("grid", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("berr", ctypes.c_double), ("cross_edges", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("latency_s", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["sync_name"] = SYNC_NAMES.get(self.sync, str(self.sync))
        return d


class ServeOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("refine_tol", ctypes.c_double),
                ("threads", ctypes.c_int32), ("device", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("peak_workspace_bytes", ctypes.c_int64),
                ("arena_bytes", ctypes.c_int64), ("factor_bytes", ctypes.c_int64)]


SERVE_CONTINUOUS, SERVE_SERIAL_F64 = 0, 1

_lib = None


def lib():
    """Load the in-tree library; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "sptrsv_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "sptrsv_last_error": (ctypes.c_char_p, []),
            "sptrsv_version": (ctypes.c_int, []),
            "sptrsv_analyze_opts_default": (None, [ctypes.POINTER(AnalyzeOpts)]),
            "sptrsv_analyze": (ctypes.c_int, [ctypes.POINTER(CSRStruct), ctypes.POINTER(AnalyzeOpts),
                                              ctypes.POINTER(vp)]),
            "sptrsv_plan_stats": (ctypes.c_int, [vp, ctypes.POINTER(Stats)]),
            "sptrsv_plan_export": (ctypes.c_int, [vp, vp, vp, vp, vp]),
            "sptrsv_local_partition": (ctypes.c_int, [ctypes.POINTER(CSRStruct), i32, i32, vp, vp]),
            "sptrsv_block_partition": (ctypes.c_int, [ctypes.POINTER(CSRStruct), i32, i32, i32, vp, vp]),
            "sptrsv_plan_export_parts": (ctypes.c_int, [vp, vp]),
            "sptrsv_plan_save": (ctypes.c_int, [vp, ctypes.POINTER(CSRStruct), ctypes.c_char_p]),
            "sptrsv_plan_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(AnalyzeOpts),
                                                ctypes.POINTER(vp)]),
            "sptrsv_destroy": (None, [vp]),
            "sptrsv_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
            "sptrsv_solve_host": (ctypes.c_int, [vp, vp, vp, i32, i64, i32, ctypes.POINTER(SolveOpts), vp,
                                                 ctypes.POINTER(Report)]),
            "sptrsv_solve": (ctypes.c_int, [vp, vp, vp, i32, i64, i32, ctypes.POINTER(SolveOpts), vp,
                                            ctypes.POINTER(Report)]),
            "sptrsv_autotune": (ctypes.c_int, [vp, vp, vp, i32, i64, i32, ctypes.POINTER(SolveOpts), vp,
                                               ctypes.POINTER(SolveOpts), ctypes.POINTER(dbl)]),
        }
        pp = ctypes.POINTER(vp)
        sig.update({
            "sptrsv_batch_create": (ctypes.c_int, [pp, i32, ctypes.POINTER(i32), i32, ctypes.POINTER(SolveOpts),
                                                   pp]),
            "sptrsv_batch_run": (ctypes.c_int, [vp, pp, pp, ctypes.POINTER(i64), vp, ctypes.POINTER(Report)]),
            "sptrsv_batch_destroy": (None, [vp]),
            "sptrsv_batch_solve": (ctypes.c_int, [pp, i32, pp, pp, ctypes.POINTER(i32), ctypes.POINTER(i64), i32,
                                                  ctypes.POINTER(SolveOpts), vp, ctypes.POINTER(Report)]),
        })
        sig.update({
            "sptrsv_serve_opts_default": (None, [ctypes.POINTER(ServeOpts)]),
            "sptrsv_serve_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(ServeOpts), pp]),
            "sptrsv_serve_register": (ctypes.c_int, [vp, vp, ctypes.POINTER(i32)]),
            "sptrsv_serve_submit": (ctypes.c_int, [vp, i32, vp, vp, i32, i64, ctypes.POINTER(ctypes.c_uint64)]),
            "sptrsv_serve_submit_host": (ctypes.c_int, [vp, i32, vp, i64, vp, i64, i32,
                                                        ctypes.POINTER(ctypes.c_uint64)]),
            "sptrsv_serve_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(Report)]),
            "sptrsv_serve_wait": (ctypes.c_int, [vp, ctypes.c_uint64, dbl, ctypes.POINTER(Report)]),
            "sptrsv_serve_drain": (ctypes.c_int, [vp, dbl]),
            "sptrsv_serve_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServeStats)]),
            "sptrsv_serve_destroy": (None, [vp]),
        })
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        L = lib()
        raise SptrsvError(status, f"{L.sptrsv_status_string(status).decode()}: "
                                  f"{L.sptrsv_last_error().decode()}")


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().sptrsv_solve_opts_default(ctypes.byref(o))
    for key, v in kw.items():
        if v is None:
            continue
        if key == "sync" and isinstance(v, str):
            v = _SYNC[v]
        if key == "precision" and isinstance(v, str):
            v = _PREC[v]
        if key == "partition" and isinstance(v, str):
            v = _PART[v]
        setattr(o, key, v)
    return o


@dataclass
class ScheduleExport:
    level: np.ndarray
    sigma: np.ndarray
    pi: np.ndarray
    perm: np.ndarray


def block_partition(A, blocks, kind="parents", row_cap=0):
    """Host-only: (block of each row, position in its block's list) of the partition of
    kind ``parents``, ``ranges`` or ``grid`` for ``blocks`` thread blocks
    (``sptrsv_block_partition``)."""
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    csr = CSRStruct(int(A.n), int(col.size), _ptr(rowptr), _ptr(col), _ptr(val))
    blk = np.zeros(int(A.n), dtype=np.int32)
    pos = np.zeros(int(A.n), dtype=np.int32)
    k = _PART[kind] if isinstance(kind, str) else int(kind)
    _check(lib().sptrsv_block_partition(ctypes.byref(csr), k, int(blocks), int(row_cap), _ptr(blk), _ptr(pos)))
    return blk, pos


def local_partition(A, blocks, row_cap=0):
    """Host-only: (block of each row, position in its block's list) of the block-local
    executor's partition for ``blocks`` thread blocks (``sptrsv_local_partition``)."""
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    csr = CSRStruct(int(A.n), int(col.size), _ptr(rowptr), _ptr(col), _ptr(val))
    blk = np.zeros(int(A.n), dtype=np.int32)
    pos = np.zeros(int(A.n), dtype=np.int32)
    _check(lib().sptrsv_local_partition(ctypes.byref(csr), int(blocks), int(row_cap), _ptr(blk), _ptr(pos)))
    return blk, pos


class Plan:
    """An analysed factor: ``Plan(A)`` with ``A`` having ``n, rowptr, col, val`` (numpy).
    ``triangle``: "lower" (L x = b), "upper" (U x = b, diagonal first in each row) or
    "lower_transposed" (L^T x = b from L's rows).
    ``sched_blocks`` > 1 (GrowLocal only): block-parallel scheduling (Sec. 3.1) on
    ``sched_threads`` host threads (0: one per hardware thread).
    ``coarsen="funnel"`` (GrowLocal only): schedule the Funnel-coarsened DAG (Sec. 4),
    parts of weight <= ``coarsen_max_weight`` (0: 500).
    ``analyze_on_device=True`` (LEVELS): wavefronts, order and layout computed by kernels
    on ``device``."""

    def __init__(self, A, mode="levels", k=0, alpha0=20.0, growth=1.5, L=500.0, accept=0.97,
                 values=VALUES_F64 | VALUES_F32, device=0, triangle="lower", sched_blocks=0,
                 sched_threads=0, coarsen="none", coarsen_max_weight=0.0, analyze_on_device=False):
        lb = lib()
        self._rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
        self._col = np.ascontiguousarray(A.col, dtype=np.int32)
        self._val = np.ascontiguousarray(A.val, dtype=np.float64)
        if self._rowptr.size != int(A.n) + 1 or self._val.size != self._col.size:
            raise ValueError("rowptr must have n + 1 entries and val as many as col")
        csr = CSRStruct(int(A.n), int(self._col.size), _ptr(self._rowptr),
                        _ptr(self._col), _ptr(self._val))
        o = AnalyzeOpts()
        lb.sptrsv_analyze_opts_default(ctypes.byref(o))
        o.mode = _MODE[mode] if isinstance(mode, str) else int(mode)
        o.k, o.alpha0, o.growth, o.L, o.accept = int(k), alpha0, growth, L, accept
        o.values, o.device = int(values), int(device)
        o.triangle = _TRI[triangle] if isinstance(triangle, str) else int(triangle)
        o.sched_blocks, o.sched_threads = int(sched_blocks), int(sched_threads)
        o.coarsen = _COARSEN[coarsen] if isinstance(coarsen, str) else int(coarsen)
        o.coarsen_max_weight = float(coarsen_max_weight)
        o.analyze_on_device = int(bool(analyze_on_device))
        h = ctypes.c_void_p()
        self.handle = None
        _check(lb.sptrsv_analyze(ctypes.byref(csr), ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value
        self.n = int(A.n)
        self.device = int(device)
        del self._rowptr, self._col, self._val       # analyze copied what it needs

    def funnel_parts(self) -> np.ndarray:
        """The Funnel part of every row (``sptrsv_plan_export_parts``)."""
        part = np.empty(self.n, dtype=np.int32)
        _check(lib().sptrsv_plan_export_parts(self.handle, _ptr(part)))
        return part

    def save(self, A, path):
        """Write this plan and the factor ``A`` (the one it was analysed from, in the
        plan's triangle format) to ``path`` (``sptrsv_plan_save``)."""
        rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
        col = np.ascontiguousarray(A.col, dtype=np.int32)
        val = np.ascontiguousarray(A.val, dtype=np.float64)
        csr = CSRStruct(int(A.n), int(col.size), _ptr(rowptr), _ptr(col), _ptr(val))
        _check(lib().sptrsv_plan_save(self.handle, ctypes.byref(csr), os.fsencode(path)))

    @classmethod
    def load(cls, path, values=VALUES_F64 | VALUES_F32, device=0):
        """Rebuild a saved plan on ``device`` without scheduling again (``sptrsv_plan_load``)."""
        lb = lib()
        o = AnalyzeOpts()
        lb.sptrsv_analyze_opts_default(ctypes.byref(o))
        o.values, o.device = int(values), int(device)
        h = ctypes.c_void_p()
        _check(lb.sptrsv_plan_load(os.fsencode(path), ctypes.byref(o), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.handle = h.value
        self.device = int(device)
        self.n = self.stats()["n"]
        return self

    def close(self):
        if self.handle:
            lib().sptrsv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = Stats()
        _check(lib().sptrsv_plan_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def export(self) -> ScheduleExport:
        arrs = [np.empty(self.n, dtype=np.int32) for _ in range(4)]
        _check(lib().sptrsv_plan_export(self.handle, *[_ptr(a) for a in arrs]))
        return ScheduleExport(*arrs)

    def autotune(self, b, x, *, stream=None, **base):
        """Time the candidate launch shapes on (b, x) and remember the fastest in the plan;
        returns the winning options as a dict (usable as ``solve(**opts)``)."""
        nrhs, ld, dtype = self._shape(b, x)
        best = SolveOpts()
        ms = ctypes.c_double()
        _check(lib().sptrsv_autotune(self.handle, _ptr(b), _ptr(x), nrhs, ld, dtype,
                                     ctypes.byref(solve_opts(**base)), _stream_handle(stream),
                                     ctypes.byref(best), ctypes.byref(ms)))
        out = {"sync": best.sync, "lanes": best.lanes, "threads": best.threads,
               "blocks_per_sm": best.blocks_per_sm, "rhs_tile": best.rhs_tile, "eager_sum": best.eager_sum,
               "partition": best.partition}
        self.tuned_ms = ms.value
        return out

    def _shape(self, b, x):
        import torch
        if not (isinstance(b, torch.Tensor) and b.is_cuda):
            raise TypeError("b must be a CUDA tensor")
        if b.dtype == torch.float64:
            dtype = F64
        elif b.dtype == torch.float32:
            dtype = F32
        else:
            raise TypeError("b must be float64 or float32")
        if b.dim() == 1:
            nrhs, ld = 1, max(self.n, 1)
            if b.stride(0) != 1:
                raise ValueError("b must be contiguous")
        elif b.dim() == 2:
            nrhs = b.shape[1]
            if b.stride(0) != 1:
                raise ValueError("b must be column-major: stride (1, ld)")
            ld = b.stride(1) if nrhs > 1 else max(self.n, 1)
        else:
            raise ValueError("b must be 1-D or 2-D")
        if b.shape[0] != self.n:
            raise ValueError("b has the wrong number of rows")
        if x is not None and (x.dtype != b.dtype or x.shape != b.shape or x.stride() != b.stride()):
            raise ValueError("x must match b in dtype, shape and strides")
        return nrhs, ld, dtype

    def solve_host(self, b, x=None, *, stream=None, report=True, **opts):
        """Solve with ``b`` and ``x`` in host memory (CPU tensors, float64 or float32, (n,) or
        (n, nrhs) column-major; pinned memory keeps the copies asynchronous): the library
        copies b in, solves and copies x out on the stream (``sptrsv_solve_host``)."""
        import torch
        if b.is_cuda or (x is not None and x.is_cuda):
            raise TypeError("solve_host takes CPU tensors")
        dtype = F64 if b.dtype == torch.float64 else F32 if b.dtype == torch.float32 else None
        if dtype is None:
            raise TypeError("b must be float64 or float32")
        nrhs, ld = _colmajor_info(b, self.n)
        if x is None:
            x = torch.empty_strided(b.shape, b.stride(), dtype=b.dtype).pin_memory()
        if x.dtype != b.dtype or _colmajor_info(x, self.n) != (nrhs, ld):
            raise ValueError("x must match b in dtype, shape and leading dimension")
        rep = Report()
        o = solve_opts(**opts)
        st = lib().sptrsv_solve_host(self.handle, _ptr(b), _ptr(x), int(nrhs), int(ld), dtype,
                                     ctypes.byref(o), _stream_handle(stream),
                                     ctypes.byref(rep) if report else None)
        _check(st)
        return x, (rep.as_dict() if report else None)

    def solve(self, b, x=None, *, stream=None, report=True, **opts):
        """Solve L x = b for a CUDA tensor ``b`` of shape (n,) or (n, nrhs) column-major
        (stride (1, ld)); ``x`` is allocated like ``b`` if not given.  Returns (x, report)."""
        import torch
        nrhs, ld, dtype = self._shape(b, x)
        if x is None:
            x = torch.empty_strided(b.shape, b.stride(), dtype=b.dtype, device=b.device)
        rep = Report()
        o = solve_opts(**opts)
        st = lib().sptrsv_solve(self.handle, _ptr(b), _ptr(x), int(nrhs), int(ld), dtype,
                                ctypes.byref(o), _stream_handle(stream),
                                ctypes.byref(rep) if report else None)
        _check(st)
        return x, (rep.as_dict() if report else None)


def _colmajor_info(t, n):
    if t.dim() == 1:
        return 1, max(n, 1)
    if t.stride(0) != 1:
        raise ValueError("right-hand sides must be column-major: stride (1, ld)")
    return t.shape[1], (t.stride(1) if t.shape[1] > 1 else max(n, 1))


class Batch:
    """Many factors solved by one persistent launch replayed from a CUDA graph.

    ``Batch(plans, nrhs, precision="f64"|"f32_refine", **opts)``; ``run(bs, xs)`` with
    lists of CUDA float64 tensors shaped (n_f,) or (n_f, nrhs_f) column-major."""

    def __init__(self, plans, nrhs, precision="f64", **opts):
        self.plans = list(plans)
        self.nrhs = [int(r) for r in nrhs]
        cnt = len(self.plans)
        arr = (ctypes.c_void_p * cnt)(*[p.handle for p in self.plans])
        nr = (ctypes.c_int32 * cnt)(*self.nrhs)
        o = solve_opts(precision=precision, **opts)
        h = ctypes.c_void_p()
        self.handle = None
        _check(lib().sptrsv_batch_create(arr, cnt, nr, F64, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value

    def close(self):
        if self.handle:
            lib().sptrsv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, bs, xs, *, stream=None, report=True):
        cnt = len(self.plans)
        lds = []
        for p, b, x, r in zip(self.plans, bs, xs, self.nrhs):
            nr, ld = _colmajor_info(b, p.n)
            if nr != r or b.dtype.itemsize != 8 or x.shape != b.shape or x.stride() != b.stride():
                raise ValueError("b/x must be float64 with the batch's nrhs and matching strides")
            lds.append(ld)
        barr = (ctypes.c_void_p * cnt)(*[b.data_ptr() for b in bs])
        xarr = (ctypes.c_void_p * cnt)(*[x.data_ptr() for x in xs])
        ldarr = (ctypes.c_int64 * cnt)(*lds)
        reps = (Report * cnt)() if report else None
        st = lib().sptrsv_batch_run(self.handle, barr, xarr, ldarr, _stream_handle(stream), reps)
        _check(st)
        return [r.as_dict() for r in reps] if report else None


class Server:
    """Continuous-batching server over resident plans (see include/sptrsv.h)."""

    def __init__(self, budget_bytes, mode="continuous", precision="f32_refine", device=0, **kw):
        o = ServeOpts()
        lib().sptrsv_serve_opts_default(ctypes.byref(o))
        o.mode = SERVE_CONTINUOUS if mode == "continuous" else SERVE_SERIAL_F64
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.device = int(device)
        for k, v in kw.items():
            setattr(o, k, v)
        h = ctypes.c_void_p()
        self.handle = None
        _check(lib().sptrsv_serve_create(int(budget_bytes), ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value
        self.plans = []

    def register(self, plan):
        fid = ctypes.c_int32()
        _check(lib().sptrsv_serve_register(self.handle, plan.handle, ctypes.byref(fid)))
        self.plans.append(plan)
        return fid.value

    def submit(self, fid, b, x):
        nrhs, ld = _colmajor_info(b, self.plans[fid].n)
        rid = ctypes.c_uint64()
        _check(lib().sptrsv_serve_submit(self.handle, int(fid), b.data_ptr(), x.data_ptr(), nrhs, ld,
                                         ctypes.byref(rid)))
        return rid.value

    def submit_host(self, fid, b, x):
        """Submit with host buffers: ``b`` and ``x`` are CPU tensors (float64, n or n x nrhs,
        column-major; pinned memory keeps the copies asynchronous).  ``x`` is written by the
        server; read it only after poll / wait reported the request done."""
        if b.is_cuda or x.is_cuda:
            raise TypeError("submit_host takes CPU tensors")
        nrhs, ldb = _colmajor_info(b, self.plans[fid].n)
        nx, ldx = _colmajor_info(x, self.plans[fid].n)
        if nx != nrhs:
            raise ValueError("b and x have different numbers of columns")
        rid = ctypes.c_uint64()
        _check(lib().sptrsv_serve_submit_host(self.handle, int(fid), b.data_ptr(), ldb, x.data_ptr(), ldx, nrhs,
                                              ctypes.byref(rid)))
        return rid.value

    def poll(self, rid):
        """None while pending, else the report dict (raises on a failed request)."""
        rep = Report()
        st = lib().sptrsv_serve_poll(self.handle, ctypes.c_uint64(rid), ctypes.byref(rep))
        if st == ERR_PENDING:
            return None
        _check(st)
        return rep.as_dict()

    def wait(self, rid, timeout=60.0):
        rep = Report()
        st = lib().sptrsv_serve_wait(self.handle, ctypes.c_uint64(rid), float(timeout), ctypes.byref(rep))
        _check(st)
        return rep.as_dict()

    def drain(self, timeout=600.0):
        _check(lib().sptrsv_serve_drain(self.handle, float(timeout)))

    def stats(self):
        s = ServeStats()
        _check(lib().sptrsv_serve_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if self.handle:
            lib().sptrsv_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
