"""The allocation-free entry point (sptrsv_solve_csr_noalloc) against sptrsv_solve.

Callers that cannot let the library allocate device memory pass their own
device CSR, b and x; the entry point keeps its scratch in a fixed device array.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_05408_gb300")

pytestmark = pytest.mark.gpu

TOL = 1e-12          # the FP64 parity bound used by every GPU solve test


def _noalloc(L, A_dev, n, nnz, b, x):
    f = L.sptrsv_solve_csr_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_int64] + [ctypes.c_void_p] * 6
    return f(n, nnz, *(t.data_ptr() for t in A_dev), b.data_ptr(), x.data_ptr(),
             torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("make", [
    lambda: W.config_random_1m(200_000)[0],
    lambda: W.laplace2d_lower(4096, 64),
    lambda: W.laplace3d_lower(40 ** 3, 40),
])
def test_noalloc_matches_plan_solve_twice(make):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = sp.lib()
    A = make()
    A_dev = [torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda(),
             torch.from_numpy(A.val).cuda()]
    plan = sp.Plan(A)
    for seed in (1, 2):                                  # two calls in a row
        _, b_np = W.manufactured_rhs(A, 1, seed=seed)
        b = torch.from_numpy(np.ascontiguousarray(b_np[:, 0])).cuda()
        x_ref, _ = plan.solve(b)
        x = torch.full_like(b, float("nan"))
        st = _noalloc(L, A_dev, A.n, A.nnz, b, x)
        assert st == 0, L.sptrsv_last_error()
        torch.cuda.synchronize()
        xr = x_ref.cpu().numpy()
        err = np.max(np.abs(x.cpu().numpy() - xr)) / np.max(np.abs(xr))
        assert err <= TOL


def test_noalloc_rejects_oversized_factor():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = sp.lib()
    f = L.sptrsv_solve_csr_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_int64] + [ctypes.c_void_p] * 6
    st = f((1 << 20) + 1, (1 << 20) + 1, 1, 1, 1, 1, 1, 0)
    assert st == sp.ERR_ARG
    assert b"at most" in ctypes.c_char_p(L.sptrsv_last_error()).value
