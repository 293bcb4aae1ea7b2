"""Seeded synthetic lower-triangular factors and right-hand sides.

This module is shared *as input only* by the CPU oracle (``oracle/``) and by the
GPU library tests / benchmark.  It holds none of the triangular-solve
arithmetic: it draws sparsity patterns and values, and manufactures
``b = L @ x_star`` so that every solve has a known answer.

All matrices are returned in CSR with int32 indices and float64 values, rows
sorted by column, the diagonal stored last in each row, no explicit zeros.

Generators (shapes follow the workloads of the paper, Sec. 6.2, and the
configurations the library is measured on):

* ``laplace2d_lower(n, width)``  - lower triangle of the 5-point Laplacian on
  the first ``n`` nodes of a ``width``-wide grid in natural order
  (diagonal 4, off-diagonals -1).
* ``laplace3d_lower(n, width)``  - lower triangle of the 7-point Laplacian on
  the first ``n`` nodes of a ``width x width x inf`` brick (diagonal 6, -1).
* ``random_window_lower(n, per_row, window, seed)`` - row ``i`` holds
  ``min(i, per_row)`` distinct columns drawn uniformly from
  ``[max(0, i - window), i)``; off-diagonals N(0,1); diagonal
  ``1 + sum |off-diagonal|`` (strictly diagonally dominant).  With
  ``window = 64, per_row = 4`` this is the random banded factor.
* ``erdos_renyi_lower(n, p, seed)`` - Sec. 6.2.4: each strictly-lower entry is
  non-zero with probability ``p``; off-diagonals U[-2, 2]; |diagonal|
  log-uniform in [1/2, 2] with a random sign.
* ``narrow_band_lower(n, p, B, seed)`` - Sec. 6.2.5: entry ``(i, j)`` non-zero
  with probability ``p * exp((1 + j - i) / B)``; values as Erdos-Renyi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSR", "laplace2d_lower", "laplace3d_lower", "random_window_lower",
    "erdos_renyi_lower", "narrow_band_lower", "make_dominant", "from_pattern", "manufactured_rhs",
    "config_small_2d", "config_random_1m", "config_3d_160", "batch_factor",
    "serve_factor", "batch_sizes", "serve_sizes", "serve_requests",
]


@dataclass
class CSR:
    """Square triangular CSR factor (int32 indices, float64 values); lower unless built by ``transpose``."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _assemble(n, counts, offcols_flat, offvals_flat, diag, name, meta=None):
    """Pack per-row sorted off-diagonal columns plus a trailing diagonal."""
    counts = np.asarray(counts, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts + 1, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    diag_pos = rowptr[1:] - 1
    is_diag = np.zeros(nnz, dtype=bool)
    is_diag[diag_pos] = True
    col[~is_diag] = offcols_flat
    val[~is_diag] = offvals_flat
    col[diag_pos] = np.arange(n, dtype=np.int32)
    val[diag_pos] = diag
    if nnz >= 2**31:
        raise ValueError("factor too large for int32 row pointers")
    return CSR(n, rowptr.astype(np.int32), col, val, name, meta or {})


def _stencil_lower(n: int, width: int, dims: int, diag: float, off: float, name: str) -> CSR:
    idx = np.arange(n, dtype=np.int64)
    strides = [width ** d for d in range(dims)]          # 1, w, w^2
    parents = []
    for d in reversed(range(dims)):                      # farthest column first -> sorted
        s = strides[d]
        if d == dims - 1:
            has = idx - s >= 0                           # outermost axis is unbounded
        else:
            has = (idx // s) % width != 0
        parents.append(np.where(has, idx - s, -1))
    P = np.stack(parents, axis=1)                        # (n, dims), ascending where present
    mask = P >= 0
    counts = mask.sum(axis=1)
    offcols = P[mask].astype(np.int32)                   # row-major flatten keeps rows in order
    offvals = np.full(offcols.size, off, dtype=np.float64)
    return _assemble(n, counts, offcols, offvals, np.full(n, diag), name,
                     {"kind": f"laplace{dims}d", "width": width})


def laplace2d_lower(n: int, width: int | None = None, diag: float = 4.0, off: float = -1.0) -> CSR:
    """Lower triangle of the 5-point Laplacian, natural order, first ``n`` grid nodes."""
    if width is None:
        width = math.isqrt(n - 1) + 1 if n > 1 else 1
    return _stencil_lower(n, width, 2, diag, off, f"laplace2d_n{n}_w{width}")


def laplace3d_lower(n: int, width: int | None = None, diag: float = 6.0, off: float = -1.0) -> CSR:
    """Lower triangle of the 7-point Laplacian, natural order, first ``n`` brick nodes."""
    if width is None:
        width = max(1, round(n ** (1.0 / 3.0)))
        while width ** 3 < n:
            width += 1
    return _stencil_lower(n, width, 3, diag, off, f"laplace3d_n{n}_w{width}")


def _distinct_sorted_draws(rng, lo, width, per_row):
    """Per row: ``per_row`` distinct sorted integers in [lo, lo + width).

    Narrow windows (where a batch of independent draws would rarely be distinct)
    draw without replacement row by row; the rest use vectorised rejection.
    """
    m = lo.size
    out = np.empty((m, per_row), dtype=np.int64)
    narrow = np.nonzero(width < per_row * per_row)[0]
    for r in narrow:
        out[r] = np.sort(rng.choice(int(width[r]), size=per_row, replace=False))
    pending = np.nonzero(width >= per_row * per_row)[0]
    while pending.size:
        d = rng.integers(0, width[pending, None], size=(pending.size, per_row))
        d.sort(axis=1)
        ok = np.all(d[:, 1:] != d[:, :-1], axis=1) if per_row > 1 else np.ones(pending.size, bool)
        out[pending[ok]] = d[ok]
        pending = pending[~ok]
    return out + lo[:, None]


def random_window_lower(n: int, per_row: int, window: int, seed: int) -> CSR:
    """Random lower factor: ``min(i, per_row)`` distinct columns in ``[max(0,i-window), i)``."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.int64)
    counts = np.minimum(i, per_row)
    full = i >= per_row
    rows_f = i[full]
    lo = np.maximum(0, rows_f - window)
    width = rows_f - lo
    draws = _distinct_sorted_draws(rng, lo, width, per_row)      # (nf, per_row)
    small_rows = i[~full]
    # rows with i < per_row take every earlier column
    pieces_small = [np.arange(r, dtype=np.int64) for r in small_rows]
    offcols = np.concatenate(pieces_small + [draws.reshape(-1)]).astype(np.int32) \
        if n else np.zeros(0, np.int32)
    offvals = rng.standard_normal(offcols.size)
    # diagonal = 1 + sum |off| of the row (rows are contiguous in offvals)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    absum = np.add.reduceat(np.abs(offvals), rp[:-1]) if offvals.size else np.zeros(n)
    absum = np.where(counts > 0, absum, 0.0)
    diag = 1.0 + absum
    return _assemble(n, counts, offcols, offvals, diag,
                     f"random_n{n}_k{per_row}_w{window}_s{seed}",
                     {"kind": "random_window", "per_row": per_row, "window": window, "seed": seed})


def _er_values(rng, nnz_off, n):
    offvals = rng.uniform(-2.0, 2.0, size=nnz_off)
    mag = np.exp(rng.uniform(math.log(0.5), math.log(2.0), size=n))
    sign = np.where(rng.integers(0, 2, size=n) == 1, 1.0, -1.0)
    return offvals, mag * sign


def erdos_renyi_lower(n: int, p: float, seed: int) -> CSR:
    """Sec. 6.2.4 Erdos-Renyi lower factor (independent Bernoulli(p) per strictly-lower entry).

    Sampled as: number of entries in row i ~ Binomial(i, p), then that many
    distinct columns uniformly from [0, i) - the same distribution.
    """
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.int64)
    counts = rng.binomial(i, p).astype(np.int64)
    rows = []
    for r in np.nonzero(counts)[0]:
        c = np.sort(rng.choice(int(r), size=int(counts[r]), replace=False))
        rows.append(c)
    offcols = (np.concatenate(rows) if rows else np.zeros(0, np.int64)).astype(np.int32)
    offvals, diag = _er_values(rng, offcols.size, n)
    return _assemble(n, counts, offcols, offvals, diag, f"er_n{n}_p{p}_s{seed}",
                     {"kind": "erdos_renyi", "p": p, "seed": seed})


def narrow_band_lower(n: int, p: float, B: float, seed: int) -> CSR:
    """Sec. 6.2.5 narrow-bandwidth factor: P(A_ij != 0) = p * exp((1 + j - i) / B), j < i."""
    rng = np.random.default_rng(seed)
    dmax = int(math.ceil(B * math.log(max(p, 1e-300) * 1e12))) + 1   # prob < 1e-12 beyond
    dmax = max(1, min(dmax, n))
    i = np.arange(n, dtype=np.int64)
    hit = []
    for d in range(1, dmax + 1):
        prob = p * math.exp((1 - d) / B)
        h = (rng.random(n) < prob) & (i - d >= 0)
        hit.append(h)
    H = np.stack(hit, axis=1)[:, ::-1]                     # column order: offset dmax..1
    counts = H.sum(axis=1)
    offs = np.arange(dmax, 0, -1)
    rr, cc = np.nonzero(H)
    offcols = (rr - offs[cc]).astype(np.int32)
    offvals, diag = _er_values(rng, offcols.size, n)
    return _assemble(n, counts, offcols, offvals, diag, f"nb_n{n}_p{p}_B{B}_s{seed}",
                     {"kind": "narrow_band", "p": p, "B": B, "seed": seed})


def make_dominant(A: CSR) -> CSR:
    """Same pattern and off-diagonal values, diagonal replaced by 1 + sum |off-diagonal|
    (strictly diagonally dominant, so FP64 solves stay at rounding-level error)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag_pos = A.rowptr[1:] - 1
    off = np.ones(A.val.size, dtype=bool)
    off[diag_pos] = False
    absum = np.bincount(rows[off], weights=np.abs(A.val[off]), minlength=A.n)
    val = A.val.copy()
    val[diag_pos] = 1.0 + absum
    return CSR(A.n, A.rowptr, A.col, val, A.name + "_dom", dict(A.meta))


def from_pattern(n: int, entries, diag: float = 1.0, off: float = -1.0) -> CSR:
    """Build a factor from a list of 0-based (row, col) positions (diagonal added if absent)."""
    rows = [[] for _ in range(n)]
    for r, c in entries:
        if c < r:
            rows[r].append(c)
    counts = [len(set(x)) for x in rows]
    offcols = np.array([c for x in rows for c in sorted(set(x))], dtype=np.int32)
    return _assemble(n, counts, offcols, np.full(offcols.size, off), np.full(n, diag), "pattern")


def transpose(A: CSR) -> CSR:
    """A^T in CSR (columns sorted): the transpose of a lower factor is an upper
    factor whose rows start with the diagonal."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr))
    order = np.lexsort((rows, A.col))                   # by column, then row
    col_t = rows[order].astype(np.int32)
    val_t = np.asarray(A.val)[order]
    counts = np.bincount(A.col, minlength=A.n)
    rp_t = np.zeros(A.n + 1, dtype=np.int32)
    rp_t[1:] = np.cumsum(counts)
    return CSR(A.n, rp_t, col_t, val_t, name=(A.name + "^T") if A.name else "", meta=dict(A.meta))


def manufactured_rhs(A: CSR, nrhs: int = 1, seed: int = 0, dtype=np.float64):
    """Draw ``x_star ~ U[-1,1]^(n x nrhs)`` (column-major) and form ``b = A @ x_star`` in FP64."""
    rng = np.random.default_rng(seed)
    xs = rng.uniform(-1.0, 1.0, size=(nrhs, A.n))          # row j = column j of x_star
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    b = np.empty((nrhs, A.n), dtype=np.float64)
    for j in range(nrhs):
        b[j] = np.bincount(rows, weights=A.val * xs[j, A.col], minlength=A.n)
    return np.ascontiguousarray(xs.T.copy(order="F")), np.asfortranarray(b.T).astype(dtype)


# --------------------------------------------------------------------------- configurations
def config_small_2d():
    """2D 5-point Laplacian lower triangle on a 64x64 grid (n = 4096), x* seed 0, 1 RHS."""
    A = laplace2d_lower(4096, 64)
    xs, b = manufactured_rhs(A, 1, seed=0)
    return A, xs, b


def config_random_1m(n: int = 1_000_000, seed: int = 0):
    """Random factor n = 1M, min(i,6) columns in a 20000-wide window, x* seed ``seed + 1``."""
    A = random_window_lower(n, 6, 20000, seed)
    xs, b = manufactured_rhs(A, 1, seed=seed + 1)
    return A, xs, b


def config_3d_160(width: int = 160, nrhs: int = 1, seed: int = 0):
    """3D 7-point Laplacian lower triangle on a width^3 brick (n = 4,096,000 at 160)."""
    A = laplace3d_lower(width ** 3, width)
    xs, b = manufactured_rhs(A, nrhs, seed=seed)
    return A, xs, b


def _log_uniform_size(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def _mixed_factor(f: int, lo: int, hi: int, seed_base: int) -> CSR:
    rng = np.random.default_rng(seed_base + f)
    n = _log_uniform_size(rng, lo, hi)
    kind = f % 3
    if kind == 0:
        A = laplace2d_lower(n)
    elif kind == 1:
        A = laplace3d_lower(n)
    else:
        A = random_window_lower(n, 4, 64, seed_base + f)
    A.meta["factor"] = f
    return A


def batch_sizes(count: int = 256, lo: int = 1000, hi: int = 50000, seed_base: int = 3000):
    return [_log_uniform_size(np.random.default_rng(seed_base + f), lo, hi) for f in range(count)]


def batch_factor(f: int, lo: int = 1000, hi: int = 50000, seed_base: int = 3000) -> CSR:
    """Factor ``f`` of the batched workload: log-uniform n in [1k, 50k]; kinds cycle
    2D Laplacian, 3D Laplacian, random banded (bandwidth 64, 4 off-diagonals per row)."""
    return _mixed_factor(f, lo, hi, seed_base)


def serve_sizes(count: int = 64, lo: int = 10_000, hi: int = 2_000_000, seed_base: int = 4000):
    return [_log_uniform_size(np.random.default_rng(seed_base + f), lo, hi) for f in range(count)]


def serve_factor(f: int, lo: int = 10_000, hi: int = 2_000_000, seed_base: int = 4000) -> CSR:
    """Resident factor ``f`` of the serving workload: log-uniform n in [10k, 2M], mixed kinds."""
    return _mixed_factor(f, lo, hi, seed_base)


def serve_requests(count: int = 10_000, rate: float = 2000.0, nfactors: int = 64,
                   max_rhs: int = 16, seed: int = 1):
    """Poisson request stream: arrival times (s), factor ids, RHS counts (uniform 1..max_rhs)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrival = np.cumsum(gaps) - gaps[0]
    fid = rng.integers(0, nfactors, size=count)
    nrhs = rng.integers(1, max_rhs + 1, size=count)
    return arrival, fid.astype(np.int32), nrhs.astype(np.int32)
