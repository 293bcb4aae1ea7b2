"""GPU parity of the superstep-scheduled solve against the CPU oracle.

Every case compares the library's x (CUDA kernels through the C ABI) with the
oracle's sequential FP64 forward substitution (Eq. 2.1) element by element:
normwise relative error <= 1e-12 in FP64 (the summation order differs from
the oracle's, so results are not bit-identical), and a bound derived from
FP32 rounding for FP32 solves.
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
    torch.cuda.init()


def to_dev(b, dtype=torch.float64, ld=None):
    """Column-major device copy of a (n, nrhs) array, optional padded leading dimension."""
    b = np.asarray(b).reshape(b.shape[0], -1)
    n, r = b.shape
    ld = ld or n
    buf = torch.zeros((r, ld), dtype=dtype, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(b.T)).to(dtype)
    return buf.T[:n] if ld == n else buf.T[:n, :]


def solve_gpu(plan, b_np, dtype=torch.float64, ld=None, **opts):
    b = to_dev(b_np, dtype, ld)
    x = to_dev(np.full(np.shape(b_np), np.nan).reshape(b.shape[0], -1), dtype, ld)
    x = x.reshape(b.shape) if b.dim() == 1 else x
    x, rep = plan.solve(b, x, **opts)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), rep


SMALL = {
    "lap2d_64x64": lambda: W.laplace2d_lower(4096, 64),
    "lap3d_24": lambda: W.laplace3d_lower(24 ** 3, 24),
    "random_60k": lambda: W.random_window_lower(60_000, 6, 20000, 0),
    "banded_20k": lambda: W.random_window_lower(20_000, 4, 64, 1),
    "er_30k": lambda: W.make_dominant(W.erdos_renyi_lower(30_000, 3e-4, 2)),
    "nb_20k": lambda: W.make_dominant(W.narrow_band_lower(20_000, 0.05, 20, 3)),
    "dense_rows": lambda: W.random_window_lower(5_000, 40, 200, 4),
}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("sync", ["grid", "flags", "cta", "cta_regs", "local", "chunks"])
@pytest.mark.parametrize("lanes", [1, 4, 32])
def test_f64_levels_parity(name, sync, lanes):
    A = SMALL[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=11)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A, mode="levels")
    x, rep = solve_gpu(plan, b, sync=sync, lanes=lanes)
    assert rep["status"] == 0
    assert oracle.rel_error(x, xo) <= F64_TOL
    if sync == "grid":
        assert rep["barriers"] == plan.stats()["supersteps"] - 1


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("lanes", [2, 8, 32])
@pytest.mark.parametrize("eager", [1, 2])
@pytest.mark.parametrize("threads", [128, 512])
@pytest.mark.parametrize("sync", ["flags", "local"])
def test_polled_eager_sum_parity(name, lanes, eager, threads, sync):
    # polled executors, entry-split lanes, with and without the eager group sum;
    # dense_rows (40 entries per row) also runs the non-blocking long-row tail
    A = SMALL[name]()
    nrhs = 2 if sync == "flags" else 1
    xs, b = W.manufactured_rhs(A, nrhs, seed=17)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A, mode="levels")
    x, rep = solve_gpu(plan, b, sync=sync, lanes=lanes, rhs_tile=1, eager_sum=eager, threads=threads,
                       blocks_per_sm=1)
    assert rep["status"] == 0 and rep["lanes"] == lanes
    assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("name", ["lap2d_64x64", "er_30k", "nb_20k", "banded_20k"])
@pytest.mark.parametrize("sync", ["grid", "flags", "cta", "cta_regs", "local", "chunks"])
@pytest.mark.parametrize("k", [1, 8, 152])
def test_f64_growlocal_parity(name, sync, k):
    A = SMALL[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=12)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A, mode="growlocal", k=k)
    ex = plan.export()
    s, pi, S = oracle.growlocal(A, k)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    x, rep = solve_gpu(plan, b, sync=sync)
    assert rep["status"] == 0
    assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("name", ["lap2d_64x64", "random_60k", "nb_20k"])
@pytest.mark.parametrize("sync", ["grid", "flags", "cta", "local", "chunks"])
@pytest.mark.parametrize("blocks", [2, 6, 22])
def test_f64_block_parallel_schedule_parity(name, sync, blocks):
    # block-parallel GrowLocal (Sec. 3.1): schedule bit-exact, solve within FP64 tolerance
    A = SMALL[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=14)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A, mode="growlocal", k=152, sched_blocks=blocks)
    ex = plan.export()
    s, pi, S = oracle.growlocal_blocks(A, 152, blocks)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    x, rep = solve_gpu(plan, b, sync=sync)
    assert rep["status"] == 0
    assert oracle.rel_error(x, xo) <= F64_TOL
    xr, rep = solve_gpu(plan, b, precision="f32_refine")
    assert rep["status"] == 0
    assert oracle.rel_error(xr, xo) <= F64_TOL


@pytest.mark.parametrize("name", ["er_30k", "nb_20k", "lap2d_64x64"])
@pytest.mark.parametrize("sync", ["grid", "flags", "cta", "local", "chunks"])
@pytest.mark.parametrize("max_weight", [40.0, 500.0])
def test_f64_funnel_schedule_parity(name, sync, max_weight):
    # Funnel + GrowLocal (Sec. 4): schedule bit-exact, solve within FP64 tolerance
    A = SMALL[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=15)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A, mode="growlocal", k=152, coarsen="funnel", coarsen_max_weight=max_weight)
    ex = plan.export()
    s, pi, S, part = oracle.funnel_growlocal(A, 152, max_weight=max_weight)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    x, rep = solve_gpu(plan, b, sync=sync)
    assert rep["status"] == 0
    assert oracle.rel_error(x, xo) <= F64_TOL
    if sync == "grid":
        assert rep["barriers"] <= S - 1


@pytest.mark.parametrize("tri", ["upper", "lower_transposed"])
@pytest.mark.parametrize("sched", [dict(coarsen="funnel"), dict(sched_blocks=5)])
@pytest.mark.parametrize("sync", ["grid", "flags", "local"])
def test_backward_substitution_with_funnel_and_blocks(tri, sched, sync):
    # the other direction (Sec. 2) under the Sec. 3.1 / Sec. 4 schedules of the reversed DAG
    L = W.make_dominant(W.narrow_band_lower(20_000, 0.05, 20, 5))
    A = W.transpose(L) if tri == "upper" else L
    xs, b = W.manufactured_rhs(W.transpose(L), 1, seed=16)
    xo = oracle.solve_upper(W.transpose(L), b)
    plan = sp.Plan(A, mode="growlocal", k=152, triangle=tri, **sched)
    x, rep = solve_gpu(plan, b, sync=sync)
    assert rep["status"] == 0
    assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("sync", ["grid", "flags", "cta", "cta_regs"])
@pytest.mark.parametrize("nrhs,ld_pad", [(2, 0), (5, 7), (32, 0), (37, 3)])
@pytest.mark.parametrize("rhs_tile", [0, 1, 4, 32])
def test_multi_rhs(sync, nrhs, ld_pad, rhs_tile):
    A = W.laplace3d_lower(20 ** 3, 20)
    xs, b = W.manufactured_rhs(A, nrhs, seed=13)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    x, rep = solve_gpu(plan, b, ld=A.n + ld_pad, sync=sync, lanes=1, rhs_tile=rhs_tile)
    assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("sync", ["grid", "flags", "cta"])
@pytest.mark.parametrize("rhs_tile", [1, 8])
def test_multi_rhs_random_rows(sync, rhs_tile):
    # rows longer than the 8-entry register tile exercise the on-demand tail
    A = W.random_window_lower(8_000, 12, 400, 6)
    xs, b = W.manufactured_rhs(A, 8, seed=16)
    plan = sp.Plan(A)
    x, rep = solve_gpu(plan, b, sync=sync, rhs_tile=rhs_tile)
    assert oracle.rel_error(x, oracle.solve(A, b)) <= F64_TOL


def test_f32_solve():
    # FP32 values and arithmetic: the error is bounded by ~n_levels * eps32 * growth;
    # these diagonally dominant factors stay far below 1e-4.
    for A in (W.laplace2d_lower(4096, 64), W.random_window_lower(40_000, 6, 20000, 5)):
        xs, b = W.manufactured_rhs(A, 1, seed=14)
        xo = oracle.solve(A, b)
        plan = sp.Plan(A)
        for sync in ("grid", "flags", "cta", "local", "chunks"):
            x, rep = solve_gpu(plan, b, dtype=torch.float32, sync=sync)
            assert oracle.rel_error(x, xo) <= 1e-4


@pytest.mark.parametrize("n", [1, 2, 33, 1000])
def test_edge_sizes(n):
    A = W.from_pattern(n, [(i, i - 1) for i in range(1, n)], diag=2.0, off=-1.0)
    b = np.ones((n, 1))
    plan = sp.Plan(A)
    for sync in ("grid", "flags", "cta", "cta_regs", "local", "chunks", "resident"):
        x, rep = solve_gpu(plan, b, sync=sync)
        assert np.allclose(x[:, 0], 1.0 - 2.0 ** -(np.arange(n) + 1.0), rtol=0, atol=1e-15)


def test_diagonal_only_is_one_superstep():
    A = W.from_pattern(100_000, [])
    A.val[:] = np.linspace(0.5, 2.0, A.n)
    b = np.random.default_rng(0).standard_normal((A.n, 1))
    plan = sp.Plan(A)
    for sync in ("grid", "flags", "cta", "local", "chunks"):
        x, rep = solve_gpu(plan, b, sync=sync)
        # x = b * (1/d): the reciprocal is rounded once on the host, so at most two roundings
        assert np.max(np.abs(x[:, 0] - b[:, 0] / A.val) / np.abs(b[:, 0] / A.val)) <= 4.5e-16
    assert rep["barriers"] == 0


def test_timeout_is_reported_and_context_survives():
    # A 1 ns wait limit makes every grid barrier give up: the kernel records
    # SPTRSV_ERR_TIMEOUT and returns (no trap); the next solve works normally.
    A = W.laplace2d_lower(4096 * 4, 128)
    xs, b = W.manufactured_rhs(A, 1, seed=15)
    plan = sp.Plan(A)
    with pytest.raises(sp.SptrsvError) as e:
        solve_gpu(plan, b, sync="grid", timeout_s=1e-9)
    assert e.value.status == sp.ERR_TIMEOUT
    x, rep = solve_gpu(plan, b, sync="grid")
    assert oracle.rel_error(x, oracle.solve(A, b)) <= F64_TOL


@pytest.mark.parametrize("cfg", ["small_2d", "random_1m", "lap3d_160"])
def test_full_size_configs_f64(cfg):
    if cfg == "small_2d":
        A, xs, b = W.config_small_2d()
    elif cfg == "random_1m":
        A, xs, b = W.config_random_1m()
    else:
        A, xs, b = W.config_3d_160()
    xo = oracle.solve(A, b)
    assert oracle.rel_error(xo, xs) < 1e-13
    plan = sp.Plan(A)
    for sync in ("grid", "flags", "local", "chunks"):
        x, rep = solve_gpu(plan, b, sync=sync)
        assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("lanes", [32, 8])
def test_local_executor_full_block(name, lanes):
    # 1024 threads per block (32 warps) on the block-local executor
    A = SMALL[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=19)
    plan = sp.Plan(A)
    x, rep = solve_gpu(plan, b, sync="local", lanes=lanes, threads=1024)
    assert rep["status"] == 0 and rep["threads"] == 1024
    assert oracle.rel_error(x, oracle.solve(A, b)) <= F64_TOL


def test_local_executor_rejects_several_rhs():
    A = W.laplace2d_lower(4096, 64)
    xs, b = W.manufactured_rhs(A, 2, seed=18)
    plan = sp.Plan(A)
    with pytest.raises(sp.SptrsvError) as e:
        solve_gpu(plan, b, sync="local")
    assert e.value.status == sp.ERR_ARG
    x, rep = solve_gpu(plan, b[:, :1], sync="local")            # the plan stays usable
    assert oracle.rel_error(x, oracle.solve(A, b[:, :1])) <= F64_TOL


# ------------------------------------------------------------ FP32 + FP64 refinement
REFINE_CASES = {
    "lap2d_64x64": lambda: W.laplace2d_lower(4096, 64),
    "random_60k": lambda: W.random_window_lower(60_000, 6, 20000, 0),   # N(0,1): not FP32-exact
    "banded_20k": lambda: W.random_window_lower(20_000, 4, 64, 1),
    "lap3d_24": lambda: W.laplace3d_lower(24 ** 3, 24),
    "er_30k": lambda: W.make_dominant(W.erdos_renyi_lower(30_000, 3e-4, 2)),
}


@pytest.mark.parametrize("name", sorted(REFINE_CASES))
@pytest.mark.parametrize("sync", ["grid", "flags", "cta", "cta_regs", "local", "chunks"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_refine_parity(name, sync, nrhs):
    if sync in ("local", "chunks") and nrhs > 1:
        pytest.skip("the block-local executors solve one right-hand side")
    A = REFINE_CASES[name]()
    xs, b = W.manufactured_rhs(A, nrhs, seed=21)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    x, rep = solve_gpu(plan, b, sync=sync, precision="f32_refine")
    assert rep["status"] == 0
    assert oracle.rel_error(x, xo) <= F64_TOL
    assert rep["sweeps"] >= 2            # at least one FP64-residual correction after the FP32 solve
    assert rep["berr"] <= 1e-13


def test_refine_needs_lo_part():
    # The FP32 solve alone is ~1e-7 off; refinement with the hi+lo split reaches FP64 accuracy
    # on values that FP32 cannot represent.
    A = W.random_window_lower(50_000, 6, 20000, 3)
    xs, b = W.manufactured_rhs(A, 1, seed=22)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    x32, _ = solve_gpu(plan, b, dtype=torch.float32, sync="flags")
    assert 1e-9 < oracle.rel_error(x32, xo) < 1e-4
    x, rep = solve_gpu(plan, b, sync="flags", precision="f32_refine")
    assert oracle.rel_error(x, xo) <= F64_TOL


def test_refine_not_converged_reports_and_returns_iterate():
    A = W.random_window_lower(30_000, 6, 20000, 4)
    xs, b = W.manufactured_rhs(A, 1, seed=23)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    bd = to_dev(b)
    xd = torch.empty_like(bd)
    with pytest.raises(sp.SptrsvError) as e:
        plan.solve(bd, xd, precision="f32_refine", max_iters=0, refine_tol=1e-15)
    assert e.value.status == sp.ERR_NOT_CONVERGED
    torch.cuda.synchronize()
    assert oracle.rel_error(xd.cpu().numpy(), xo) < 1e-4        # the FP32 iterate is still there


@pytest.mark.parametrize("nrhs", [1, 32])
def test_full_size_3d_refine(nrhs):
    A, xs, b = W.config_3d_160(nrhs=nrhs)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    x, rep = solve_gpu(plan, b, sync="flags", precision="f32_refine")
    assert oracle.rel_error(x, xo) <= F64_TOL
    assert oracle.rel_error(x, xs) <= F64_TOL


def test_full_size_3d_f64_r32():
    # 160^3 stencil, 32 right-hand sides (column-major), plain FP64: the explicit
    # polled and grid-barrier tiles and the launch shape the autotuner picks
    A, xs, b = W.config_3d_160(nrhs=32)
    xo = oracle.solve(A, b)
    assert oracle.rel_error(xo, xs) < 1e-13
    plan = sp.Plan(A, analyze_on_device=True)
    for sync in ("flags", "grid"):
        x, rep = solve_gpu(plan, b, sync=sync, rhs_tile=32)
        assert rep["status"] == 0
        assert oracle.rel_error(x, xo) <= F64_TOL
    bd = to_dev(b)
    xd = torch.empty_like(bd)
    opts = plan.autotune(bd, xd, precision="f64")
    x, rep = solve_gpu(plan, b, precision="f64", **opts)
    assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("name", ["random_60k", "er_30k", "lap3d_24"])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_refine_residual_from_split_values(name, nrhs):
    # a plan holding FP32 values only forms the FP64 residual from the hi + lo split;
    # with FP64 values it uses the scaled FP64 values: both reach the oracle at 1e-12
    A = SMALL[name]()
    xs, b = W.manufactured_rhs(A, nrhs, seed=25)
    xo = oracle.solve(A, b)
    for values in (sp.VALUES_F32, sp.VALUES_F64 | sp.VALUES_F32):
        plan = sp.Plan(A, values=values)
        x, rep = solve_gpu(plan, b, sync="flags", precision="f32_refine")
        assert rep["status"] == 0 and rep["berr"] <= 1e-13
        assert oracle.rel_error(x, xo) <= F64_TOL


def test_full_size_random_refine():
    A, xs, b = W.config_random_1m()
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    for sync in ("flags", "grid", "local", "chunks"):
        x, rep = solve_gpu(plan, b, sync=sync, precision="f32_refine")
        assert oracle.rel_error(x, xo) <= F64_TOL


def test_staged_walker_matches_register_walker():
    # same per-row arithmetic in the same order; only FMA contraction of the first
    # term may differ, so the two one-block walkers agree to rounding
    for A in (W.laplace2d_lower(4096, 64), W.random_window_lower(20_000, 4, 64, 8),
              W.make_dominant(W.narrow_band_lower(20_000, 0.05, 20, 9))):
        xs, b = W.manufactured_rhs(A, 3, seed=17)
        plan = sp.Plan(A)
        for tile in (1, 4):
            x1, r1 = solve_gpu(plan, b, sync="cta", rhs_tile=tile)
            x2, r2 = solve_gpu(plan, b, sync="cta_regs", rhs_tile=tile)
            assert np.max(np.abs(x1 - x2)) <= 1e-14 * np.max(np.abs(x2))


# ------------------------------------------------------------ upper and transposed systems
UPPER_CASES = ["lap2d_64x64", "lap3d_24", "random_60k", "banded_20k", "er_30k", "dense_rows"]


@pytest.mark.parametrize("name", UPPER_CASES)
@pytest.mark.parametrize("sync", ["grid", "flags", "cta", "cta_regs", "local", "chunks"])
@pytest.mark.parametrize("tri", ["upper", "lower_transposed"])
def test_upper_and_transposed_parity(name, sync, tri):
    Lo = SMALL[name]()
    U = W.transpose(Lo)
    xs, b = W.manufactured_rhs(U, 1, seed=31)
    xo = oracle.solve_upper(U, b)
    plan = sp.Plan(U if tri == "upper" else Lo, triangle=tri)
    x, rep = solve_gpu(plan, b, sync=sync)
    assert rep["status"] == 0
    assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("tri", ["upper", "lower_transposed"])
@pytest.mark.parametrize("nrhs,rhs_tile", [(5, 0), (5, 1), (32, 32)])
@pytest.mark.parametrize("sync", ["grid", "flags", "cta"])
def test_upper_multi_rhs(tri, nrhs, rhs_tile, sync):
    Lo = W.laplace3d_lower(20 ** 3, 20)
    U = W.transpose(Lo)
    xs, b = W.manufactured_rhs(U, nrhs, seed=32)
    plan = sp.Plan(U if tri == "upper" else Lo, triangle=tri)
    x, rep = solve_gpu(plan, b, sync=sync, rhs_tile=rhs_tile)
    assert oracle.rel_error(x, oracle.solve_transposed(Lo, b)) <= F64_TOL


@pytest.mark.parametrize("tri", ["upper", "lower_transposed"])
@pytest.mark.parametrize("sync", ["grid", "flags", "local", "chunks"])
def test_upper_refine_and_growlocal(tri, sync):
    Lo = W.make_dominant(W.erdos_renyi_lower(30_000, 3e-4, 2))
    U = W.transpose(Lo)
    xs, b = W.manufactured_rhs(U, 1, seed=33)
    xo = oracle.solve_upper(U, b)
    A = U if tri == "upper" else Lo
    x, rep = solve_gpu(sp.Plan(A, triangle=tri), b, sync=sync, precision="f32_refine")
    assert oracle.rel_error(x, xo) <= F64_TOL and rep["berr"] <= 1e-13
    x, rep = solve_gpu(sp.Plan(A, mode="growlocal", k=16, triangle=tri), b, sync=sync)
    assert oracle.rel_error(x, xo) <= F64_TOL


def test_upper_full_size_3d():
    Lo = W.laplace3d_lower(160 ** 3, 160)
    U = W.transpose(Lo)
    xs, b = W.manufactured_rhs(U, 1, seed=34)
    xo = oracle.solve_upper(U, b)
    assert oracle.rel_error(xo, xs) < 1e-13
    plan = sp.Plan(U, triangle="upper")
    for sync in ("flags", "local", "chunks"):
        x, rep = solve_gpu(plan, b, sync=sync)
        assert oracle.rel_error(x, xo) <= F64_TOL


@pytest.mark.parametrize("name", ["random_60k", "lap3d_24"])
@pytest.mark.parametrize("tri", ["lower", "upper"])
def test_saved_plan_with_local_partition(tmp_path, name, tri):
    # a block-local solve builds the partition; the saved plan carries it and the loaded
    # plan solves with it.  Same x bits with one entry per lane (32 lanes, rows of at most
    # 32 entries): then no lane's partial sum depends on the order its parents arrive in,
    # so equal bits mean the same partition and the same summation order.
    A = SMALL[name]()
    if tri == "upper":
        A = W.transpose(A)
    xs, b = W.manufactured_rhs(A, 1, seed=21)
    xo = oracle.solve_upper(A, b) if tri == "upper" else oracle.solve(A, b)
    plan = sp.Plan(A, mode="growlocal", k=152, sched_blocks=4, triangle=tri)
    det = dict(sync="local", lanes=32, threads=1024, eager_sum=2)
    x1, rep = solve_gpu(plan, b, **det)
    assert rep["status"] == 0 and oracle.rel_error(x1, xo) <= F64_TOL
    path = tmp_path / "p.plan"
    plan.save(A, path)
    n, nnz = A.n, A.nnz
    assert path.stat().st_size == 56 + (n + 1) * 4 + nnz * 12 + n * 8 + n * 8 + 8   # partition included
    loaded = sp.Plan.load(path)
    assert loaded.stats()["supersteps"] == plan.stats()["supersteps"]
    x2, rep = solve_gpu(loaded, b, **det)
    assert rep["status"] == 0
    assert np.array_equal(x1, x2)
    x4, rep = solve_gpu(loaded, b, sync="local")
    assert rep["status"] == 0 and oracle.rel_error(x4, xo) <= F64_TOL
    x3, rep = solve_gpu(loaded, b, sync="flags")
    assert rep["status"] == 0 and oracle.rel_error(x3, xo) <= F64_TOL


@pytest.mark.parametrize("sync", ["chunks", "resident", "flags", "cta"])
def test_solve_host_buffers_match_device_call(sync):
    # sptrsv_solve_host: b copied in, the solve, x copied out, all by the library
    A = SMALL["lap2d_64x64"]()
    xs, b = W.manufactured_rhs(A, 1, seed=71)
    plan = sp.Plan(A)
    bh = torch.from_numpy(np.ascontiguousarray(b[:, 0])).pin_memory()
    xh, rep = plan.solve_host(bh, sync=sync)
    assert rep["status"] == 0 and not xh.is_cuda
    assert oracle.rel_error(xh.numpy(), oracle.solve(A, b)[:, 0]) <= F64_TOL
    xd, _ = plan.solve(bh.cuda(), sync=sync)
    if sync == "flags":     # sums in arrival order: the last bits may differ from run to run
        assert oracle.rel_error(xh.numpy(), xd.cpu().numpy()) <= F64_TOL
    else:                   # a fixed order per row: the same bits as the device-buffer call
        assert np.array_equal(xh.numpy(), xd.cpu().numpy())


def test_solve_host_buffers_padded_pageable_and_refined():
    A = SMALL["random_60k"]()
    n, r, ld = A.n, 3, A.n + 5
    xs, b = W.manufactured_rhs(A, r, seed=72)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    buf = torch.zeros((r, ld), dtype=torch.float64)                    # pageable, padded
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(b.T))
    bh = buf.T[:n]
    xbuf = torch.full((r, ld), float("nan"), dtype=torch.float64)
    xh = xbuf.T[:n]
    _, rep = plan.solve_host(bh, xh, sync="flags", lanes=4)
    assert rep["status"] == 0 and oracle.rel_error(xh.numpy(), xo) <= F64_TOL
    assert torch.isnan(xbuf[:, n:]).all()                               # the padding is untouched
    x1 = torch.empty(n, dtype=torch.float64).pin_memory()
    _, rep = plan.solve_host(bh[:, 0].contiguous().pin_memory(), x1, precision="f32_refine")
    assert rep["status"] == 0 and rep["berr"] <= 1e-13
    assert oracle.rel_error(x1.numpy(), xo[:, 0]) <= F64_TOL
    x32, rep = plan.solve_host(bh[:, 0].contiguous().float())
    assert rep["status"] == 0 and oracle.rel_error(x32.double().numpy(), xo[:, 0]) <= 1e-4
    with pytest.raises(TypeError):
        plan.solve_host(bh.cuda())
