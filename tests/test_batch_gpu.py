"""Batched persistent solve (one launch replayed from a CUDA graph) against the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_05408_gb300")

pytestmark = pytest.mark.gpu
F64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.lib()


def colmajor(b):
    b = np.asarray(b).reshape(b.shape[0], -1)
    t = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    return t.T if b.shape[1] > 1 else t[0].contiguous()


def run_batch(factors, nrhs, precision="f64", seed=0, runs=1, **opts):
    plans = [sp.Plan(A) for A in factors]
    batch = sp.Batch(plans, nrhs, precision=precision, **opts)
    results = []
    for run in range(runs):
        rhs = [W.manufactured_rhs(A, r, seed=seed + 97 * run + i) for i, (A, r) in enumerate(zip(factors, nrhs))]
        bs = [colmajor(b) for _, b in rhs]
        xs = [torch.full_like(b, float("nan")) for b in bs]
        reps = batch.run(bs, xs)
        torch.cuda.synchronize()
        results.append(([b for _, b in rhs], [x.cpu().numpy().reshape(A.n, -1) for x, A in zip(xs, factors)], reps))
    return results


MIXED = [W.batch_factor(f) for f in range(12)] + [W.make_dominant(W.erdos_renyi_lower(3000, 1e-3, 5)),
                                                   W.laplace2d_lower(1000, 10)]


@pytest.mark.parametrize("precision", ["f64", "f32_refine"])
@pytest.mark.parametrize("sync", ["auto", "cta"])
def test_batch_mixed_factors(precision, sync):
    nrhs = [1, 3, 8, 8, 2, 40, 8, 5, 16, 8, 1, 33, 8, 4]
    (bs, xs, reps), = run_batch(MIXED, nrhs, precision=precision, sync=sync)
    for A, b, x, rep in zip(MIXED, bs, xs, reps):
        assert rep["status"] == 0
        assert oracle.rel_error(x, oracle.solve(A, b)) <= F64_TOL
        if precision == "f32_refine":
            assert rep["sweeps"] >= 2


@pytest.mark.parametrize("values", ["f32", "f64|f32"])
def test_batch_refinement_residual_forms(values):
    # plans holding FP32 values only form the FP64 residual from the hi + lo split; plans
    # that also hold FP64 values use the scaled FP64 values: both reach the oracle at 1e-12
    v = sp.VALUES_F32 if values == "f32" else sp.VALUES_F64 | sp.VALUES_F32
    factors = MIXED[:8]
    nrhs = [1, 3, 8, 8, 2, 40, 8, 5]
    plans = [sp.Plan(A, values=v) for A in factors]
    batch = sp.Batch(plans, nrhs, precision="f32_refine")
    rhs = [W.manufactured_rhs(A, r, seed=300 + i)[1] for i, (A, r) in enumerate(zip(factors, nrhs))]
    bs = [colmajor(b) for b in rhs]
    xs = [torch.full_like(b, float("nan")) for b in bs]
    reps = batch.run(bs, xs)
    torch.cuda.synchronize()
    for A, b, x, rep in zip(factors, rhs, xs, reps):
        assert rep["status"] == 0 and rep["sweeps"] >= 2
        assert oracle.rel_error(x.cpu().numpy().reshape(A.n, -1), oracle.solve(A, b)) <= F64_TOL


def test_batch_graph_replay_new_vectors():
    factors = MIXED[:6]
    nrhs = [8] * 6
    res = run_batch(factors, nrhs, runs=3)
    for bs, xs, reps in res:
        for A, b, x in zip(factors, bs, xs):
            assert oracle.rel_error(x, oracle.solve(A, b)) <= F64_TOL


def test_batch_single_factor_matches_plain_solve():
    A = W.batch_factor(5)
    (bs, xs, reps), = run_batch([A], [8])
    plan = sp.Plan(A)
    x2, _ = plan.solve(colmajor(bs[0]))
    assert np.max(np.abs(x2.cpu().numpy().reshape(A.n, -1) - xs[0])) <= F64_TOL * np.max(np.abs(xs[0]))


def test_batch_rejects_bad_input():
    A = W.batch_factor(0)
    p = sp.Plan(A)
    with pytest.raises(sp.SptrsvError):
        sp.Batch([p], [0])
    host = sp.Plan(A, device=-1)
    with pytest.raises(sp.SptrsvError) as e:
        sp.Batch([host], [1])
    assert e.value.status == sp.ERR_NO_DEVICE


@pytest.mark.parametrize("precision", ["f64", "f32_refine"])
def test_batch_full_config_256x8(precision):
    factors = [W.batch_factor(f) for f in range(256)]
    (bs, xs, reps), = run_batch(factors, [8] * 256, precision=precision)
    worst = max(oracle.rel_error(x, oracle.solve(A, b)) for A, b, x in zip(factors, bs, xs))
    assert worst <= F64_TOL


def test_batch_mixes_lower_and_upper_plans():
    # a batch may hold plans of both directions; each item matches its own oracle
    import oracle as O
    facs = [W.batch_factor(f) for f in range(6)]
    plans, bs, xs_, refs = [], [], [], []
    for i, A in enumerate(facs):
        if i % 2:
            U = W.transpose(A)
            p = sp.Plan(U, triangle="upper")
            _, b = W.manufactured_rhs(U, 3, seed=400 + i)
            ref = O.solve_upper(U, b)
        else:
            p = sp.Plan(A)
            _, b = W.manufactured_rhs(A, 3, seed=400 + i)
            ref = O.solve(A, b)
        plans.append(p)
        bd = torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T
        bs.append(bd)
        xs_.append(torch.empty_strided(bd.shape, bd.stride(), dtype=bd.dtype, device=bd.device))
        refs.append(ref)
    batch = sp.Batch(plans, [3] * len(plans), precision="f64")
    batch.run(bs, xs_)
    torch.cuda.synchronize()
    for x, ref in zip(xs_, refs):
        assert O.rel_error(x.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("precision", ["f64", "f32_refine"])
def test_batch_over_device_analysed_plans(precision):
    # plans analysed on the device are the host plans bit for bit: the batch runs them the same way
    factors = [W.batch_factor(f) for f in range(12)]
    nrhs = [1, 3, 8, 2] * 3
    host = [sp.Plan(A) for A in factors]
    dev = [sp.Plan(A, analyze_on_device=True) for A in factors]
    rhs = [W.manufactured_rhs(A, r, seed=400 + i) for i, (A, r) in enumerate(zip(factors, nrhs))]
    out = []
    for plans in (host, dev):
        batch = sp.Batch(plans, nrhs, precision=precision)
        bs = [colmajor(b) for _, b in rhs]
        xs = [torch.full_like(b, float("nan")) for b in bs]
        reps = batch.run(bs, xs)
        torch.cuda.synchronize()
        assert all(r["status"] == 0 for r in reps)
        out.append([x.cpu().numpy().reshape(A.n, -1) for x, A in zip(xs, factors)])
    for A, (_, b), xh, xd in zip(factors, rhs, out[0], out[1]):
        xo = oracle.solve(A, b)
        assert oracle.rel_error(xd, xo) <= F64_TOL
        assert oracle.rel_error(xh, xo) <= F64_TOL
