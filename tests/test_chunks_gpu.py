"""The chunked block-local executor (SPTRSV_SYNC_CHUNKS) against the CPU oracle.

One row per lane; a block's (wavefront, id) list cut into chunks of up to 32
rows of one wavefront; a chunk waits for all of its parents and then applies
Eq. 2.1 to every row at once, in a fixed order per row.  Checked: FP64 parity at
1e-12 on every small factor with both partitions and several block sizes, FP32
sweeps and FP32 + FP64 refinement, bit-identical results across runs, the
reported cross-block edge count against the host partition, and the full-size
configurations.
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


def _dev(b, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(b).reshape(-1))).to("cuda", dtype)


def _solve(plan, b, dtype=torch.float64, **opts):
    bd = _dev(b, dtype)
    xd = torch.full_like(bd, float("nan"))
    _, rep = plan.solve(bd, xd, **opts)
    torch.cuda.synchronize()
    return xd.double().cpu().numpy(), rep


CASES = {
    "lap2d_64x64": lambda: W.laplace2d_lower(4096, 64),
    "lap3d_24": lambda: W.laplace3d_lower(24 ** 3, 24),
    "lap3d_40": lambda: W.laplace3d_lower(40 ** 3, 40),
    "random_60k": lambda: W.random_window_lower(60_000, 6, 20000, 0),
    "banded_20k": lambda: W.random_window_lower(20_000, 4, 64, 1),
    "er_30k": lambda: W.make_dominant(W.erdos_renyi_lower(30_000, 3e-4, 2)),
    "nb_20k": lambda: W.make_dominant(W.narrow_band_lower(20_000, 0.05, 20, 3)),
    "dense_rows": lambda: W.random_window_lower(5_000, 40, 200, 4),       # chunks wider than 8: tail path
}


SYNCS = ["chunks"]


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("partition", ["parents", "ranges", "grid"])
@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("sync", SYNCS)
def test_chunks_f64_parity(name, partition, threads, sync):
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=41)
    xo = oracle.solve(A, b)
    plan = sp.Plan(A)
    x, rep = _solve(plan, b, sync=sync, partition=partition, threads=threads)
    assert rep["status"] == 0 and rep["sync_name"] == sync and rep["threads"] == threads
    assert oracle.rel_error(x, xo[:, 0]) <= F64_TOL


@pytest.mark.parametrize("name", ["lap2d_64x64", "lap3d_24", "lap3d_40"])
@pytest.mark.parametrize("partition", ["parents", "ranges", "grid"])
def test_chunks_768_threads_for_short_rows(name, partition):
    # rows of at most three off-diagonal entries: up to 768 threads per block
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=47)
    plan = sp.Plan(A)
    x, rep = _solve(plan, b, sync="chunks", partition=partition, threads=768)
    assert rep["status"] == 0 and rep["threads"] == 768
    assert oracle.rel_error(x, oracle.solve(A, b)[:, 0]) <= F64_TOL
    x2, _ = _solve(plan, b, sync="chunks", partition=partition, threads=512)
    assert np.array_equal(x, x2)                      # the same per-row order at any block size


def test_chunks_768_threads_rejected_for_longer_rows():
    A = CASES["banded_20k"]()                         # four off-diagonal entries per row
    xs, b = W.manufactured_rhs(A, 1, seed=48)
    plan = sp.Plan(A)
    bd = torch.from_numpy(np.ascontiguousarray(b[:, 0])).cuda()
    with pytest.raises(sp.SptrsvError) as e:
        plan.solve(bd, torch.empty_like(bd), sync="chunks", threads=768)
    assert e.value.status == sp.ERR_ARG
    x, rep = _solve(plan, b, sync="chunks", threads=512)
    assert rep["status"] == 0 and oracle.rel_error(x, oracle.solve(A, b)[:, 0]) <= F64_TOL


@pytest.mark.parametrize("name", ["lap2d_64x64", "lap3d_40", "random_60k", "banded_20k"])
def test_chunks_reproducible(name):
    # every row sums in a fixed order once its parents are in: the same bits on every run
    # and for every block size
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=42)
    plan = sp.Plan(A)
    x1, rep = _solve(plan, b, sync="chunks", threads=512)
    x2, _ = _solve(plan, b, sync="chunks", threads=512)
    x3, _ = _solve(plan, b, sync="chunks", threads=256)
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)
    assert oracle.rel_error(x1, oracle.solve(A, b)[:, 0]) <= F64_TOL


@pytest.mark.parametrize("name", ["lap2d_64x64", "lap3d_24", "random_60k", "nb_20k"])
def test_chunks_cross_edges_match_host_partition(name):
    # the report's cross-block edge count is the number of (parent, row) pairs the
    # host partition puts in different blocks
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=43)
    plan = sp.Plan(A)
    x, rep = _solve(plan, b, sync="chunks", partition="parents")
    # small factors: no block reaches its shared-memory row cap, so the cap does not matter
    blk, pos = sp.local_partition(A, rep["grid"])
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    off = A.col != rows
    cross = int(np.count_nonzero(blk[A.col[off]] != blk[rows[off]]))
    assert rep["cross_edges"] == cross
    assert rep["edges"] == A.nnz - A.n
    _, rep2 = _solve(plan, b, sync="flags")
    assert rep2["cross_edges"] == -1


@pytest.mark.parametrize("name", ["lap2d_64x64", "lap3d_24", "random_60k", "er_30k"])
@pytest.mark.parametrize("sync", SYNCS)
def test_chunks_f32_and_refinement(name, sync):
    A = CASES[name]()
    xs, b = W.manufactured_rhs(A, 1, seed=44)
    xo = oracle.solve(A, b)[:, 0]
    plan = sp.Plan(A)
    x32, rep = _solve(plan, b, dtype=torch.float32, sync=sync)
    assert rep["status"] == 0 and oracle.rel_error(x32, xo) <= 1e-4
    for partition in ("parents", "ranges", "grid"):
        x, rep = _solve(plan, b, sync=sync, partition=partition, precision="f32_refine")
        assert rep["status"] == 0 and rep["sweeps"] >= 2 and rep["berr"] <= 1e-13
        assert oracle.rel_error(x, xo) <= F64_TOL


def test_chunks_saved_partition_is_used(tmp_path):
    A = CASES["lap3d_24"]()
    xs, b = W.manufactured_rhs(A, 1, seed=45)
    plan = sp.Plan(A)
    x1, rep1 = _solve(plan, b, sync="chunks", partition="ranges")
    path = tmp_path / "p.plan"
    plan.save(A, path)
    loaded = sp.Plan.load(path)
    x2, rep2 = _solve(loaded, b, sync="chunks")              # AUTO: the saved partition
    assert np.array_equal(x1, x2) and rep2["cross_edges"] == rep1["cross_edges"]


@pytest.mark.parametrize("partition", ["parents", "ranges", "grid"])
@pytest.mark.parametrize("sync", SYNCS)
def test_chunks_full_size_3d_160(partition, sync):
    A, xs, b = W.config_3d_160()
    xo = oracle.solve(A, b)[:, 0]
    plan = sp.Plan(A, analyze_on_device=True)
    for threads in (384, 768):
        x, rep = _solve(plan, b, sync=sync, partition=partition, threads=threads)
        assert rep["status"] == 0 and oracle.rel_error(x, xo) <= F64_TOL
    xr, rep = _solve(plan, b, sync=sync, partition=partition, precision="f32_refine")
    assert rep["status"] == 0 and oracle.rel_error(xr, xo) <= F64_TOL


def test_chunks_full_size_random_1m():
    A, xs, b = W.config_random_1m()
    xo = oracle.solve(A, b)[:, 0]
    plan = sp.Plan(A, analyze_on_device=True)
    for partition in ("parents", "ranges", "grid"):
        for sync in SYNCS:
            x, rep = _solve(plan, b, sync=sync, partition=partition)
            assert rep["status"] == 0 and oracle.rel_error(x, xo) <= F64_TOL


def test_chunks_rejects_large_blocks_and_several_rhs():
    A = CASES["lap2d_64x64"]()
    xs, b = W.manufactured_rhs(A, 2, seed=46)
    plan = sp.Plan(A)
    bd = torch.from_numpy(np.ascontiguousarray(b[:, 0])).cuda()
    with pytest.raises(sp.SptrsvError) as e:
        plan.solve(bd, torch.empty_like(bd), sync="chunks", threads=1024)
    assert e.value.status == sp.ERR_ARG
    b2 = torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T
    with pytest.raises(sp.SptrsvError) as e:
        plan.solve(b2, torch.empty_like(b2), sync="chunks")
    assert e.value.status == sp.ERR_ARG
    x, rep = _solve(plan, b[:, 0], sync="chunks")              # the plan stays usable
    assert oracle.rel_error(x, oracle.solve(A, b[:, :1])[:, 0]) <= F64_TOL
