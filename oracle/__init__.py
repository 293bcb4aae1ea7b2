"""CPU oracle for the superstep-scheduled sparse lower-triangular solve.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` -- never by the GPU library, which
fails loudly when its CUDA extension is missing instead of falling back here.
The oracle and the library share no code: only the seeded input generators in
``workloads/`` feed both.

What it computes (each function cites the passage it follows):

* ``solve``          forward substitution, Eq. 2.1, sequential FP64 (C)
* ``solve_upper``    backward substitution for upper-triangular U (diagonal first
  in each row), the other direction of the method (C)
* ``solve_transposed``  L^T x = b from L's rows, column-oriented backward
  substitution (C)
* ``levels_upper``   wavefronts of an upper factor's DAG (row i waits on its
  columns j > i), plain reverse pass
* ``spmv``           y = A x in FP64 (C), for residual checks
* ``levels``         wavefronts of the DAG of Sec. 2.2 / Fig. 1.1 (C)
* ``growlocal``      the GrowLocal scheduler, Sec. 3 / Algorithm 3.1 (C)
* ``growlocal_blocks``  block-parallel scheduling, Sec. 3.1: GrowLocal on each
  diagonal block's sub-DAG (full-row weights), block schedules concatenated
* ``triangle_reduce``, ``funnel_parts``, ``funnel_growlocal``  Sec. 4: the
  triangle transitive reduction, in-funnel coarsening (Algorithm 4.1) with a
  part weight cap, and GrowLocal on the coarsened DAG
* ``level_schedule`` sigma = wavefront, pi = 0 (the wavefront scheduler, Sec. 1)
* ``check_schedule`` Definition 2.1 plus the bookkeeping rules of a schedule
* ``permutation``    the reordering of Sec. 5: sort by (superstep, core, id)
* ``permute``        the symmetric permutation P A P^T of Sec. 5
* ``validate``       input rules: square, lower, sorted, unique, diagonal last
  and non-zero (Sec. 2.2 assumes a non-singular matrix)

Pins (tests/test_oracle.py): the Fig. 1.1 worked example, dense triangular
solves on tiny inputs, closed forms for diagonal and bidiagonal factors,
closed-form wavefront counts of natural-order stencils, manufactured
solutions, the hand-derived GrowLocal example on a diagonal matrix, a
hand-derived two-block schedule that only the full-row weights produce, the
closed form of one block per row, and brute force Definition 2.1 checks on
small random DAGs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sptrsv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_solve_fp64.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p,
                                              _f64p, ctypes.c_int64, _f64p, ctypes.c_int64]
            lib.oracle_solve_fp64.restype = None
            for name in ("oracle_solve_upper_fp64", "oracle_solve_lower_transposed_fp64"):
                fn = getattr(lib, name)
                fn.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p,
                               _f64p, ctypes.c_int64, _f64p, ctypes.c_int64]
                fn.restype = None
            lib.oracle_spmv_fp64.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
            lib.oracle_spmv_fp64.restype = None
            lib.oracle_levels.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
            lib.oracle_levels.restype = ctypes.c_int32
            lib.oracle_growlocal.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, _i32p, _i32p]
            lib.oracle_growlocal.restype = ctypes.c_int32
            lib.oracle_growlocal_weighted.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, ctypes.c_int32,
                                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_double, _i32p, _i32p]
            lib.oracle_growlocal_weighted.restype = ctypes.c_int32
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _arrays(A):
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    c = np.ascontiguousarray(A.col, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, c, v


class InvalidFactor(ValueError):
    pass


def validate(A) -> None:
    """Check the input rules of the problem (Sec. 2.2): lower-triangular CSR with
    strictly increasing columns and a non-zero diagonal stored last in every row."""
    n = A.n
    rp, c, v = _arrays(A)
    if rp.size != n + 1 or rp[0] != 0 or np.any(np.diff(rp) < 1) or rp[-1] != c.size:
        raise InvalidFactor("bad row pointers (every row needs at least its diagonal)")
    rows = np.repeat(np.arange(n), np.diff(rp))
    if np.any(c < 0) or np.any(c > rows):
        raise InvalidFactor("entry above the diagonal or out of range")
    same_row = rows[1:] == rows[:-1]
    if np.any(same_row & (c[1:] <= c[:-1])):
        raise InvalidFactor("columns not strictly increasing within a row")
    last = rp[1:] - 1
    if np.any(c[last] != np.arange(n)):
        raise InvalidFactor("diagonal missing")
    if np.any(v[last] == 0.0):
        raise InvalidFactor("zero diagonal")


def solve(A, b: np.ndarray) -> np.ndarray:
    """Eq. 2.1 forward substitution in FP64; ``b`` is (n,) or (n, nrhs)."""
    lib = _load()
    rp, c, v = _arrays(A)
    b2 = np.asfortranarray(np.asarray(b, dtype=np.float64).reshape(A.n, -1))
    x = np.empty_like(b2, order="F")
    lib.oracle_solve_fp64(A.n, b2.shape[1], _p(rp, _i32p), _p(c, _i32p), _p(v, _f64p),
                          _p(b2, _f64p), A.n, _p(x, _f64p), A.n)
    return x.reshape(np.shape(b)) if np.ndim(b) == 1 else x


def validate_upper(U) -> None:
    """Upper-triangular CSR: strictly increasing columns, the non-zero diagonal
    present and stored first in every row."""
    n = U.n
    rp, c, v = _arrays(U)
    if rp.size != n + 1 or rp[0] != 0 or np.any(np.diff(rp) < 1) or rp[-1] != c.size:
        raise InvalidFactor("bad row pointers (every row needs at least its diagonal)")
    rows = np.repeat(np.arange(n), np.diff(rp))
    if np.any(c < rows) or np.any(c >= n):
        raise InvalidFactor("entry below the diagonal or out of range")
    same_row = rows[1:] == rows[:-1]
    if np.any(same_row & (c[1:] <= c[:-1])):
        raise InvalidFactor("columns not strictly increasing within a row")
    first = rp[:-1]
    if np.any(c[first] != np.arange(n)):
        raise InvalidFactor("diagonal missing")
    if np.any(v[first] == 0.0):
        raise InvalidFactor("zero diagonal")


def _solve_with(fn, A, b):
    lib = _load()
    rp, c, v = _arrays(A)
    b2 = np.asfortranarray(np.asarray(b, dtype=np.float64).reshape(A.n, -1))
    x = np.empty_like(b2, order="F")
    getattr(lib, fn)(A.n, b2.shape[1], _p(rp, _i32p), _p(c, _i32p), _p(v, _f64p),
                     _p(b2, _f64p), A.n, _p(x, _f64p), A.n)
    return x.reshape(np.shape(b)) if np.ndim(b) == 1 else x


def solve_upper(U, b: np.ndarray) -> np.ndarray:
    """Backward substitution U x = b in FP64 (U upper-triangular, diagonal first)."""
    return _solve_with("oracle_solve_upper_fp64", U, b)


def solve_transposed(L, b: np.ndarray) -> np.ndarray:
    """L^T x = b in FP64 from L's rows (L lower-triangular, diagonal last)."""
    return _solve_with("oracle_solve_lower_transposed_fp64", L, b)


def levels_upper(U):
    """Wavefronts of an upper factor: row i waits on the rows j > i it references,
    so one pass from the last row: level(i) = 1 + max level over those j (0 if none)."""
    rp, c, _ = _arrays(U)
    lv = np.zeros(U.n, dtype=np.int32)
    for i in range(U.n - 1, -1, -1):
        js = c[rp[i] + 1:rp[i + 1]]
        if js.size:
            lv[i] = lv[js].max() + 1
    return lv, int(lv.max()) + 1 if U.n else 0


def spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x in FP64 (every stored entry, diagonal included)."""
    lib = _load()
    rp, c, v = _arrays(A)
    x2 = np.asfortranarray(np.asarray(x, dtype=np.float64).reshape(A.n, -1))
    y = np.empty_like(x2, order="F")
    for j in range(x2.shape[1]):
        xj = np.ascontiguousarray(x2[:, j])
        yj = np.empty(A.n)
        lib.oracle_spmv_fp64(A.n, _p(rp, _i32p), _p(c, _i32p), _p(v, _f64p),
                             _p(xj, _f64p), _p(yj, _f64p))
        y[:, j] = yj
    return y.reshape(np.shape(x)) if np.ndim(x) == 1 else y


def levels(A):
    """Wavefront index of every row (Fig. 1.1) and the number of wavefronts."""
    lib = _load()
    rp, c, _ = _arrays(A)
    lv = np.empty(A.n, dtype=np.int32)
    nlev = lib.oracle_levels(A.n, _p(rp, _i32p), _p(c, _i32p), _p(lv, _i32p))
    return lv, int(nlev)


def avg_wavefront(A) -> float:
    """n divided by the length of the longest path (Sec. 6.2), counted in vertices."""
    return A.n / max(1, levels(A)[1])


def level_schedule(A):
    """Wavefront schedule: superstep = wavefront, every vertex on core 0."""
    lv, nlev = levels(A)
    return lv, np.zeros(A.n, dtype=np.int32), nlev


def growlocal(A, k: int, alpha0: float = 20.0, growth: float = 1.5, L: float = 500.0,
              accept: float = 0.97):
    """GrowLocal schedule (Algorithm 3.1): returns (sigma, pi, supersteps), 0-based."""
    if k < 1:
        raise ValueError("k must be >= 1")
    lib = _load()
    rp, c, _ = _arrays(A)
    sigma = np.empty(A.n, dtype=np.int32)
    pi = np.empty(A.n, dtype=np.int32)
    S = lib.oracle_growlocal(A.n, _p(rp, _i32p), _p(c, _i32p), int(k), float(alpha0),
                             float(growth), float(L), float(accept), _p(sigma, _i32p),
                             _p(pi, _i32p))
    if S < 0:
        raise MemoryError("oracle_growlocal failed")
    return sigma, pi, int(S)


def block_subdag(A, r0: int, r1: int):
    """Sub-DAG of the diagonal block of rows r0..r1-1 (Sec. 3.1, Fig. 3.1): the
    block's rows renumbered from 0 with only the entries in the block's own
    columns (diagonal last), and every vertex's weight = its FULL row's entry
    count.  Returns (rowptr, col, weight)."""
    rp, c, _ = _arrays(A)
    m = r1 - r0
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp[r0:r1 + 1]))
    cols = c[rp[r0]:rp[r1]]
    keep = cols >= r0                           # entries inside the diagonal block
    sub_rp = np.zeros(m + 1, dtype=np.int32)
    sub_rp[1:] = np.cumsum(np.bincount(rows[keep], minlength=m))
    sub_col = np.ascontiguousarray(cols[keep] - r0, dtype=np.int32)
    weight = np.ascontiguousarray(np.diff(rp[r0:r1 + 1]), dtype=np.int64)
    return sub_rp, sub_col, weight


def growlocal_blocks(A, k: int, blocks: int, alpha0: float = 20.0, growth: float = 1.5,
                     L: float = 500.0, accept: float = 0.97):
    """Block-parallel scheduling (Sec. 3.1, Fig. 3.1), run one block after another.

    The rows are cut into ``blocks`` diagonal blocks, block b holding rows
    floor(b n / blocks) .. floor((b+1) n / blocks) - 1 (the figure's equal
    blocks).  Each block is scheduled by GrowLocal on its own sub-DAG: its rows,
    renumbered from 0, keep only the entries in the block's own columns (the
    edges from earlier blocks are met because those blocks run first), while
    every vertex keeps the weight of its full row.  The block schedules are
    concatenated: a vertex of block b gets its superstep plus the number of
    supersteps of blocks 0..b-1.  Returns (sigma, pi, supersteps)."""
    if blocks <= 1:
        return growlocal(A, k, alpha0, growth, L, accept)
    if k < 1:
        raise ValueError("k must be >= 1")
    lib = _load()
    n = A.n
    sigma = np.empty(n, dtype=np.int32)
    pi = np.empty(n, dtype=np.int32)
    offset = 0
    for b in range(blocks):
        r0, r1 = b * n // blocks, (b + 1) * n // blocks
        m = r1 - r0
        if m == 0:
            continue
        sub_rp, sub_col, weight = block_subdag(A, r0, r1)
        s_b = np.empty(m, dtype=np.int32)
        p_b = np.empty(m, dtype=np.int32)
        S = lib.oracle_growlocal_weighted(m, _p(sub_rp, _i32p), _p(sub_col, _i32p), _p(weight, _i64p),
                                          int(k), float(alpha0), float(growth), float(L), float(accept),
                                          _p(s_b, _i32p), _p(p_b, _i32p))
        if S < 0:
            raise MemoryError("oracle_growlocal_weighted failed")
        sigma[r0:r1] = s_b + offset
        pi[r0:r1] = p_b
        offset += int(S)
    return sigma, pi, offset


def triangle_reduce(A):
    """Approximate transitive reduction used before coarsening (Sec. 4.2): every
    edge (u, w) that is the long side of a triangle u -> v -> w of the DAG is
    removed, all decided on the original edge set.  Returns the kept parents of
    each vertex as a list of sorted int lists."""
    n = A.n
    par = [set(A.col[A.rowptr[i]:A.rowptr[i + 1] - 1].tolist()) for i in range(n)]
    kept = []
    for w in range(n):
        long_edges = set()
        for v in par[w]:
            long_edges |= par[w] & par[v]          # u -> v -> w with u -> w also present
        kept.append(sorted(par[w] - long_edges))
    return kept


def funnel_parts(n, parents, weight, max_weight):
    """In-funnel coarsening, Algorithm 4.1 (Sec. 4.2), with the part weight cap.

    Vertices are taken in reverse topological order (n-1 .. 0, the natural order
    of a lower factor being topological); an unvisited vertex starts a part and
    a priority queue (largest id first) grows it through parents all of whose
    children already joined the part.  A popped vertex joins only while the
    part's weight stays <= max_weight (a part's first vertex always joins).
    Returns part[v] and the parts' roots in increasing root id."""
    import heapq
    children_count = [0] * n
    outdeg = [0] * n
    for w in range(n):
        for u in parents[w]:
            outdeg[u] += 1
    visited = [False] * n
    members_of = []
    for v in range(n - 1, -1, -1):
        if visited[v]:
            continue
        U, total = [], 0
        touched = []
        heap = [-v]
        while heap:
            w = -heapq.heappop(heap)
            if U and total + weight[w] > max_weight:
                continue                            # stays outside; starts its own part later
            U.append(w)
            total += weight[w]
            for u in parents[w]:
                children_count[u] += 1
                touched.append(u)
                if children_count[u] == outdeg[u]:
                    heapq.heappush(heap, -u)
        for u in touched:                           # ChildrenCount reset for the next part
            children_count[u] = 0
        for u in U:
            visited[u] = True
        members_of.append(U)
    part = np.empty(n, dtype=np.int64)
    roots = sorted(max(U) for U in members_of)
    index = {r: i for i, r in enumerate(roots)}
    for U in members_of:
        part[U] = index[max(U)]
    return part, roots


def funnel_growlocal(A, k: int, max_weight: float = 500.0, reduce: bool = True, alpha0: float = 20.0,
                     growth: float = 1.5, L: float = 500.0, accept: float = 0.97):
    """Funnel + GrowLocal (Sec. 4): triangle reduction, in-funnel coarsening with
    the weight cap, GrowLocal on the coarsened DAG (parts numbered by root, a
    part weighing the sum of its rows' entries, an edge between two parts for
    every kept edge between their members) and every vertex taking its part's
    superstep and core.  Returns (sigma, pi, supersteps, part)."""
    n = A.n
    if n == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32), 0, np.zeros(0, np.int64)
    parents = triangle_reduce(A) if reduce else [A.col[A.rowptr[i]:A.rowptr[i + 1] - 1].tolist()
                                                  for i in range(n)]
    weight = np.diff(A.rowptr).astype(np.int64)
    part, roots = funnel_parts(n, parents, weight.tolist(), max_weight)
    m = len(roots)
    cpar = [set() for _ in range(m)]
    for w in range(n):
        for u in parents[w]:
            if part[u] != part[w]:
                cpar[part[w]].add(int(part[u]))
    crp = np.zeros(m + 1, dtype=np.int32)
    ccol = []
    for i in range(m):
        assert all(j < i for j in cpar[i])          # root order is topological
        ccol += sorted(cpar[i]) + [i]
        crp[i + 1] = len(ccol)
    ccol = np.array(ccol, dtype=np.int32)
    cw = np.bincount(part, weights=weight, minlength=m).astype(np.int64)
    s_c = np.empty(m, dtype=np.int32)
    p_c = np.empty(m, dtype=np.int32)
    lib = _load()
    S = lib.oracle_growlocal_weighted(m, _p(crp, _i32p), _p(ccol, _i32p), _p(cw, _i64p), int(k),
                                      float(alpha0), float(growth), float(L), float(accept),
                                      _p(s_c, _i32p), _p(p_c, _i32p))
    if S < 0:
        raise MemoryError("oracle_growlocal_weighted failed")
    return s_c[part].astype(np.int32), p_c[part].astype(np.int32), int(S), part


def edges(A):
    """DAG edges (j -> i) for every stored off-diagonal A_ij (Sec. 2.2)."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr))
    off = A.col != rows
    return A.col[off].astype(np.int64), rows[off]


def check_schedule(A, sigma, pi, k: int, strict: bool = False) -> list[str]:
    """Definition 2.1 and schedule bookkeeping; returns a list of violations.

    * every vertex has one superstep sigma >= 0 and one core 0 <= pi < k;
    * superstep numbers are contiguous 0..S-1;
    * every edge (u, v): sigma(u) <= sigma(v), and sigma(u) < sigma(v) when
      pi(u) != pi(v) (Def. 2.1); with ``strict`` every edge crosses a barrier
      (the wavefront schedule).
    """
    sigma = np.asarray(sigma)
    pi = np.asarray(pi)
    bad = []
    if sigma.shape != (A.n,) or pi.shape != (A.n,):
        return ["schedule arrays have the wrong length"]
    if A.n == 0:
        return bad
    if sigma.min() < 0:
        bad.append("negative superstep")
    if pi.min() < 0 or pi.max() >= k:
        bad.append("core index out of range")
    used = np.unique(sigma)
    if used.size != sigma.max() + 1:
        bad.append("superstep numbers not contiguous")
    u, v = edges(A)
    if np.any(sigma[u] > sigma[v]):
        bad.append("edge goes to an earlier superstep")
    cross = pi[u] != pi[v]
    if np.any(cross & (sigma[u] >= sigma[v])):
        bad.append("edge between cores inside a superstep")
    if strict and np.any(sigma[u] >= sigma[v]):
        bad.append("edge inside a superstep (wavefront schedule must be strict)")
    return bad


def permutation(sigma, pi) -> np.ndarray:
    """Sec. 5 reordering: new position -> old row, sorted by (superstep, core, id)."""
    sigma = np.asarray(sigma, dtype=np.int64)
    pi = np.asarray(pi, dtype=np.int64)
    ids = np.arange(sigma.size, dtype=np.int64)
    return np.lexsort((ids, pi, sigma)).astype(np.int32)


def permute(A, perm):
    """Symmetric permutation P A P^T (row/col r of the result = row/col perm[r] of A),
    returned as a dense-free (rows, cols, vals) triple in the new numbering."""
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr))
    return inv[rows], inv[A.col.astype(np.int64)], A.val.copy()


def rel_error(x, xref) -> float:
    """Normwise relative error max_i |x_i - xref_i| / max_i |xref_i| per right-hand-side
    column, worst column returned (the error metric of the parity checks).  A column whose
    reference is all zeros reports its absolute error; an empty system has error 0."""
    xr = np.asarray(xref, dtype=np.float64)
    n = xr.shape[0]
    cols = xr.size // n if n else (xr.shape[1] if xr.ndim > 1 else 1)
    xr = xr.reshape(n, cols)
    x = np.asarray(x, dtype=np.float64).reshape(n, cols)
    if x.size == 0:
        return 0.0                     # no entries: nothing differs
    num = np.max(np.abs(x - xr), axis=0)
    den = np.max(np.abs(xr), axis=0)
    den = np.where(den == 0, 1.0, den)
    return float(np.max(num / den))
