"""The allocation-free entry point (sptrsv_solve_csr_noalloc).

Callers that cannot let the library allocate device memory (their device bytes
come only from their own pool or budget, or an allocation inside a
latency-critical loop could synchronise the device) pass their own device CSR,
b and x; the entry point keeps its scratch in a fixed device array.  Its
results are checked against the CPU oracle and against the planned solve
(sptrsv_analyze + sptrsv_solve), on two calls in a row.  Malformed factors
must be refused with the documented status, and a valid call made right after
a refused one must still be correct (the status is cleared, the ready flags
move to a new epoch).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_05408_gb300")

pytestmark = pytest.mark.gpu

TOL = 1e-12          # the FP64 parity bound used by every GPU solve test


def _entry(L):
    f = L.sptrsv_solve_csr_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_int64] + [ctypes.c_void_p] * 6
    return f


def _noalloc(L, A_dev, n, nnz, b, x):
    return _entry(L)(n, nnz, *(t.data_ptr() for t in A_dev), b.data_ptr(), x.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)


def _to_dev(rowptr, col, val):
    return [torch.from_numpy(np.asarray(rowptr, dtype=np.int32)).cuda(),
            torch.from_numpy(np.asarray(col, dtype=np.int32)).cuda(),
            torch.from_numpy(np.asarray(val, dtype=np.float64)).cuda()]


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _solve_checked(L, A, A_dev, seed):
    """One allocation-free solve of A x = L x* (seeded), checked against the oracle; returns x and b."""
    _, b_np = W.manufactured_rhs(A, 1, seed=seed)
    b = torch.from_numpy(np.ascontiguousarray(b_np[:, 0])).cuda()
    x = torch.full_like(b, float("nan"))
    st = _noalloc(L, A_dev, A.n, A.nnz, b, x)
    assert st == 0, ctypes.c_char_p(L.sptrsv_last_error()).value
    torch.cuda.synchronize()
    x_np = x.cpu().numpy()
    assert oracle.rel_error(x_np, oracle.solve(A, b_np[:, 0])) <= TOL
    return x_np, b


@pytest.mark.parametrize("make", [
    lambda: W.config_random_1m(200_000)[0],
    lambda: W.laplace2d_lower(4096, 64),
    lambda: W.laplace3d_lower(40 ** 3, 40),
])
def test_noalloc_matches_oracle_and_plan_solve_twice(make):
    _need_gpu()
    L = sp.lib()
    A = make()
    A_dev = _to_dev(A.rowptr, A.col, A.val)
    plan = sp.Plan(A)
    for seed in (1, 2):                                  # two calls in a row
        x_np, b = _solve_checked(L, A, A_dev, seed)
        x_ref, _ = plan.solve(b)                         # the existing entry point
        assert oracle.rel_error(x_np, x_ref.cpu().numpy()) <= TOL


def test_noalloc_rejects_oversized_factor():
    _need_gpu()
    L = sp.lib()
    st = _entry(L)((1 << 20) + 1, (1 << 20) + 1, 1, 1, 1, 1, 1, 0)
    assert st == sp.ERR_ARG
    assert b"at most" in ctypes.c_char_p(L.sptrsv_last_error()).value


# Four rows; row 2 is the malformed one.  Every check fires before the row
# waits on anything, and the rows waiting on row 2 see the status word and stop.
_GOOD_ROWPTR = [0, 1, 3, 5, 7]
_GOOD_COL = [0, 0, 1, 1, 2, 2, 3]


@pytest.mark.parametrize("col2, expect", [
    ([3, 2], "ERR_NOT_LOWER"),      # a column above the diagonal (the diagonal itself is last)
    ([0, 1], "ERR_ARG"),            # no diagonal: the last entry of the row is not column 2
])
def test_noalloc_malformed_factor_then_valid_call(col2, expect):
    _need_gpu()
    L = sp.lib()
    col = list(_GOOD_COL)
    col[3:5] = col2
    val = [2.0, -1.0, 2.0, -1.0, 2.0, -1.0, 2.0]
    A_dev = _to_dev(_GOOD_ROWPTR, col, val)
    b = torch.ones(4, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st = _noalloc(L, A_dev, 4, 7, b, x)
    assert st == getattr(sp, expect), (st, ctypes.c_char_p(L.sptrsv_last_error()).value)
    # the next valid call in the same process: status cleared, new epoch, correct result
    A = W.laplace2d_lower(4096, 64)
    _solve_checked(L, A, _to_dev(A.rowptr, A.col, A.val), seed=3)
    # and the well-formed four-row factor itself (bidiagonal, diagonal 2, off-diagonal -1)
    good = _to_dev(_GOOD_ROWPTR, _GOOD_COL, val)
    assert _noalloc(L, good, 4, 7, b, x) == 0
    torch.cuda.synchronize()
    # x_i = (1 + x_{i-1}) / 2: 1/2, 3/4, 7/8, 15/16
    assert x.cpu().numpy().tolist() == [0.5, 0.75, 0.875, 0.9375]
