"""The resident one-block executor (SPTRSV_SYNC_RESIDENT) against the CPU oracle.

The whole factor sits in one thread block's shared memory and the block walks
the plan's phases with a barrier between them (Eq. 2.1 in the Sec. 5 order).
Checked: FP64 parity at 1e-12 on small factors with the wavefront and GrowLocal
schedules, lower, upper and transposed triangles; FP32 sweeps and FP32 + FP64
refinement; the same bits at every block size; and the refusals (several
right-hand sides, a factor larger than one SM's shared memory).
"""
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


def _solve(plan, b, dtype=torch.float64, **opts):
    bd = torch.from_numpy(np.ascontiguousarray(np.asarray(b).reshape(-1))).to("cuda", dtype)
    xd = torch.full_like(bd, float("nan"))
    _, rep = plan.solve(bd, xd, **opts)
    torch.cuda.synchronize()
    return xd.double().cpu().numpy(), rep


# every factor fits one SM's shared memory: 8 (2 n + m) + 4 (m + 2 n + phases + 2) bytes
CASES = {
    "lap2d_64x64": lambda: W.laplace2d_lower(4096, 64),          # the small FP64 configuration
    "lap3d_12": lambda: W.laplace3d_lower(12 ** 3, 12),
    "banded_2500": lambda: W.random_window_lower(2_500, 4, 64, 1),
    "random_2k": lambda: W.random_window_lower(2_000, 6, 1500, 0),
    "er_2k": lambda: W.make_dominant(W.erdos_renyi_lower(2_000, 2e-3, 2)),
    "dense_rows": lambda: W.random_window_lower(400, 40, 200, 4),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("threads", [128, 512, 1024])
def test_resident_f64_parity(name, threads):
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=61)
    plan = sp.Plan(A)
    x, rep = _solve(plan, b, sync="resident", threads=threads)
    assert rep["status"] == 0 and rep["sync_name"] == "resident" and rep["grid"] == 1
    assert rep["threads"] == threads and rep["cross_edges"] == -1
    assert oracle.rel_error(x, oracle.solve(A, b)[:, 0]) <= F64_TOL


@pytest.mark.parametrize("name", ["lap2d_64x64", "random_2k", "dense_rows"])
def test_resident_same_bits_every_run_and_block_size(name):
    # a row's entries are summed in stored order by one thread: no run-to-run variation
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=62)
    plan = sp.Plan(A)
    x1, _ = _solve(plan, b, sync="resident", threads=256)
    x2, _ = _solve(plan, b, sync="resident", threads=256)
    x3, _ = _solve(plan, b, sync="resident", threads=1024)
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)


@pytest.mark.parametrize("k", [8, 152])
@pytest.mark.parametrize("tri", ["lower", "upper", "lower_transposed"])
def test_resident_growlocal_and_triangles(k, tri):
    Lo = CASES["er_2k"]()
    if tri == "lower":
        A, xo_of = Lo, lambda b: oracle.solve(Lo, b)
    elif tri == "upper":
        A = W.transpose(Lo)
        xo_of = lambda b: oracle.solve_upper(A, b)
    else:
        A, xo_of = Lo, lambda b: oracle.solve_transposed(Lo, b)
    probe = W.transpose(Lo) if tri != "lower" else Lo
    xs, b = W.manufactured_rhs(probe, 1, seed=63)
    xo = xo_of(b)[:, 0]
    for plan in (sp.Plan(A, triangle=tri), sp.Plan(A, mode="growlocal", k=k, triangle=tri)):
        x, rep = _solve(plan, b, sync="resident")
        assert rep["status"] == 0 and oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("name", ["lap2d_64x64", "lap3d_12", "er_2k"])
def test_resident_f32_and_refinement(name):
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=64)
    xo = oracle.solve(A, b)[:, 0]
    plan = sp.Plan(A)
    x32, rep = _solve(plan, b, dtype=torch.float32, sync="resident")
    assert rep["status"] == 0 and oracle.rel_error(x32, xo) <= 1e-4
    x, rep = _solve(plan, b, sync="resident", precision="f32_refine")
    assert rep["status"] == 0 and rep["sweeps"] >= 2 and rep["berr"] <= 1e-13
    assert oracle.rel_error(x, xo) <= F64_TOL


def test_resident_refusals_leave_the_plan_usable():
    A = CASES["lap2d_64x64"]()
    xs, b = W.manufactured_rhs(A, 2, seed=65)
    plan = sp.Plan(A)
    b2 = torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T
    with pytest.raises(sp.SptrsvError) as e:
        plan.solve(b2, torch.empty_like(b2), sync="resident")
    assert e.value.status == sp.ERR_ARG
    big = W.laplace3d_lower(40 ** 3, 40)                              # 64,000 rows: ~1.5 MB
    bb = torch.ones(big.n, dtype=torch.float64, device="cuda")
    with pytest.raises(sp.SptrsvError) as e:
        sp.Plan(big).solve(bb, torch.empty_like(bb), sync="resident")
    assert e.value.status == sp.ERR_ARG and "shared memory" in str(e.value)
    x, rep = _solve(plan, b[:, 0], sync="resident")
    assert rep["status"] == 0 and oracle.rel_error(x, oracle.solve(A, b[:, :1])[:, 0]) <= F64_TOL


def test_resident_small_configuration():
    # the 64 x 64 configuration: one barrier per wavefront (127), x equal to the oracle's
    A, xs, b = W.config_small_2d()
    plan = sp.Plan(A)
    assert plan.stats()["levels"] == 127
    x, rep = _solve(plan, b, sync="resident")
    assert rep["status"] == 0 and oracle.rel_error(x, oracle.solve(A, b)[:, 0]) <= F64_TOL


def test_resident_degenerate_factors():
    # no off-diagonal entry at all (the bulk copies of columns and values are skipped)
    A = W.from_pattern(5_000, [])
    A.val[:] = np.linspace(0.5, 2.0, A.n)
    b = np.random.default_rng(1).standard_normal((A.n, 1))
    x, rep = _solve(sp.Plan(A), b, sync="resident")
    assert rep["status"] == 0
    assert np.max(np.abs(x - b[:, 0] / A.val) / np.abs(b[:, 0] / A.val)) <= 4.5e-16
    # a single row
    A1 = W.from_pattern(1, [])
    A1.val[:] = 4.0
    x1, rep = _solve(sp.Plan(A1), np.array([[2.0]]), sync="resident")
    assert rep["status"] == 0 and x1.tolist() == [0.5]
    # a chain: one row per phase (4096 phases, 32 walking threads)
    n = 4096
    Ab = W.from_pattern(n, [(i, i - 1) for i in range(1, n)], diag=2.0, off=-1.0)
    xb, rep = _solve(sp.Plan(Ab), np.ones((n, 1)), sync="resident", threads=256)
    assert rep["status"] == 0
    # x_i = (1 + x_{i-1}) / 2 = 1 - 2^-(i+1): exact in FP64 while representable
    assert np.allclose(xb, 1.0 - 2.0 ** -(np.arange(n) + 1.0), rtol=0, atol=1e-15)
