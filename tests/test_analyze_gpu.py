"""Wavefront analysis on the device (analyze_on_device) against the host analysis
and the oracle.

The device path computes the wavefronts with a polled kernel, the Sec. 5 order
with a stable radix sort and the device layout with gathers; the plan must be
the host plan bit for bit: the same schedule exports (and the oracle's
wavefronts), the same statistics, and the same x bits from deterministic
executors (one thread per row, or one entry per lane)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_05408_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.lib()


def _chain(n):
    return W.from_pattern(n, [(i, i - 1) for i in range(1, n)], diag=2.0, off=-1.0)


CASES = {
    "one_row": lambda: W.from_pattern(1, []),
    "diag_3000": lambda: W.from_pattern(3000, []),
    "fig1_1": lambda: W.from_pattern(6, [(1, 0), (2, 1), (3, 1), (4, 2), (5, 3)]),
    "lap2d_64": lambda: W.laplace2d_lower(4096, 64),
    "lap3d_30_ragged": lambda: W.laplace3d_lower(30 ** 3 - 17, 30),
    "random_60k": lambda: W.random_window_lower(60_000, 6, 20000, 0),
    "dense_rows": lambda: W.random_window_lower(5_000, 40, 200, 4),
    "er_30k": lambda: W.make_dominant(W.erdos_renyi_lower(30_000, 3e-4, 2)),
    "chain_70k": lambda: _chain(70_000),          # 70,000 wavefronts: three radix passes
}

DETERMINISTIC = [dict(sync="grid", lanes=1), dict(sync="flags", lanes=32, eager_sum=2), dict(sync="cta", lanes=1)]


def _solve(plan, b_np, **o):
    b = torch.from_numpy(b_np[:, 0].copy()).cuda()
    x = torch.full_like(b, float("nan"))
    _, rep = plan.solve(b, x, **o)
    torch.cuda.synchronize()
    assert rep["status"] == 0
    return x.cpu().numpy()


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_analysis_equals_host_analysis(name):
    A = CASES[name]()
    host = sp.Plan(A, mode="levels")
    dev = sp.Plan(A, mode="levels", analyze_on_device=True)
    eh, ed = host.export(), dev.export()
    for f in ("level", "sigma", "pi", "perm"):
        assert np.array_equal(getattr(eh, f), getattr(ed, f)), f
    lv, nlev = oracle.levels(A)
    assert np.array_equal(ed.level, lv)
    assert np.array_equal(ed.perm, oracle.permutation(lv, np.zeros(A.n, np.int32)))
    sh, sd = host.stats(), dev.stats()
    for f in ("n", "nnz", "levels", "supersteps", "k", "max_level_rows", "phases", "ring_rows", "device_bytes",
              "sched_blocks", "coarse_vertices"):
        assert sh[f] == sd[f], f
    xs, b = W.manufactured_rhs(A, 1, seed=31)
    xo = oracle.solve(A, b)
    # one entry per lane keeps the 32-lane executor's sums in a fixed order
    cfgs = [o for o in DETERMINISTIC if o["lanes"] == 1 or int(np.diff(A.rowptr).max()) <= 32]
    for o in cfgs:
        xh = _solve(host, b, **o)
        xd = _solve(dev, b, **o)
        assert np.array_equal(xh, xd), o
        assert oracle.rel_error(xd[:, None], xo) <= 1e-12
    # refinement reads the FP32 splits and the row-sum norm: same sweeps, same bits
    xh = _solve(host, b, sync="grid", lanes=1, precision="f32_refine")
    xd = _solve(dev, b, sync="grid", lanes=1, precision="f32_refine")
    assert np.array_equal(xh, xd)


def test_device_analysis_full_size_random_1m():
    A, xs, b = W.config_random_1m()
    host = sp.Plan(A, mode="levels")
    dev = sp.Plan(A, mode="levels", analyze_on_device=True)
    eh, ed = host.export(), dev.export()
    assert np.array_equal(eh.level, ed.level) and np.array_equal(eh.perm, ed.perm)
    assert host.stats()["device_bytes"] == dev.stats()["device_bytes"]
    x1 = _solve(host, b, sync="local", lanes=32, threads=1024, eager_sum=2)
    x2 = _solve(dev, b, sync="local", lanes=32, threads=1024, eager_sum=2)
    assert np.array_equal(x1, x2)


def test_device_analysis_argument_errors():
    A = W.laplace2d_lower(256, 16)
    for kw in (dict(mode="growlocal", k=4), dict(mode="levels", device=-1)):
        with pytest.raises(sp.SptrsvError) as e:
            sp.Plan(A, analyze_on_device=True, **kw)
        assert e.value.status == sp.ERR_ARG
    # host validation still runs first: a zero diagonal is refused before any upload
    bad = W.CSR(A.n, A.rowptr, A.col, A.val.copy(), "bad")
    bad.val[A.rowptr[5 + 1] - 1] = 0.0
    with pytest.raises(sp.SptrsvError) as e:
        sp.Plan(bad, analyze_on_device=True)
    assert e.value.status == sp.ERR_ZERO_DIAG


def test_device_analysed_plan_saves_and_loads(tmp_path):
    A = W.random_window_lower(50_000, 6, 5000, 7)
    dev = sp.Plan(A, mode="levels", analyze_on_device=True)
    xs, b = W.manufactured_rhs(A, 1, seed=33)
    x1 = _solve(dev, b, sync="local", lanes=32, threads=1024, eager_sum=2)      # builds the partition
    dev.save(A, tmp_path / "d.plan")
    q = sp.Plan.load(tmp_path / "d.plan")
    for f in ("level", "sigma", "pi", "perm"):
        assert np.array_equal(getattr(dev.export(), f), getattr(q.export(), f)), f
    x2 = _solve(q, b, sync="local", lanes=32, threads=1024, eager_sum=2)
    assert np.array_equal(x1, x2)
    assert oracle.rel_error(x2[:, None], oracle.solve(A, b)) <= 1e-12


@pytest.mark.parametrize("name", ["lap3d_30_ragged", "random_60k", "dense_rows", "chain_70k"])
@pytest.mark.parametrize("tri", ["upper", "lower_transposed"])
def test_device_analysis_of_backward_substitution(name, tri):
    # the reversed factor L' is analysed on the device; ids and permutation come back in the
    # caller's numbering, exactly as the host analysis writes them
    L = CASES[name]()
    A = W.transpose(L) if tri == "upper" else L
    host = sp.Plan(A, mode="levels", triangle=tri)
    dev = sp.Plan(A, mode="levels", triangle=tri, analyze_on_device=True)
    eh, ed = host.export(), dev.export()
    for f in ("level", "sigma", "pi", "perm"):
        assert np.array_equal(getattr(eh, f), getattr(ed, f)), f
    sh, sd = host.stats(), dev.stats()
    for f in ("levels", "supersteps", "phases", "ring_rows", "device_bytes", "max_level_rows"):
        assert sh[f] == sd[f], f
    U = W.transpose(L)
    xs, b = W.manufactured_rhs(U, 1, seed=35)
    xo = oracle.solve_upper(U, b)
    for o in [dict(sync="grid", lanes=1), dict(sync="cta", lanes=1)]:
        xh = _solve(host, b, **o)
        xd = _solve(dev, b, **o)
        assert np.array_equal(xh, xd), o
        assert oracle.rel_error(xd[:, None], xo) <= 1e-12
