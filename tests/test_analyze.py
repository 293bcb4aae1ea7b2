"""Host-side analysis of the library against the oracle (CPU only, no GPU needed).

The library is loaded through its C ABI and asked for a host-only plan
(device = -1), so the schedules and permutations it exports can be compared
bit for bit with the oracle's on any machine.
"""
import networkx as nx
import numpy as np
import pytest

import oracle
import workloads as W

sp = pytest.importorskip("paper_2503_05408_gb300")


@pytest.fixture(scope="module")
def L():
    try:
        return sp.lib()
    except RuntimeError as e:
        pytest.skip(str(e))


def test_library_exports_every_declared_symbol(L):
    import re
    import os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "sptrsv.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)                     # drop comments
    names = set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(sptrsv_[a-z_0-9]+)\s*\(", hdr, re.M))
    assert names, "no declarations found"
    for name in sorted(names):
        assert hasattr(L, name), f"{name} declared in include/sptrsv.h but not exported"


def _host_plan(A, **kw):
    return sp.Plan(A, device=-1, **kw)


CASES = {
    "fig1_1": lambda: W.from_pattern(6, [(1, 0), (2, 1), (3, 1), (4, 2), (5, 3)]),
    "lap2d_64": lambda: W.laplace2d_lower(4096, 64),
    "lap3d_20": lambda: W.laplace3d_lower(8000, 20),
    "random_50k": lambda: W.random_window_lower(50_000, 6, 20000, 0),
    "banded_30k": lambda: W.random_window_lower(30_000, 4, 64, 2),
    "er_20k": lambda: W.erdos_renyi_lower(20_000, 2e-4, 1),
    "nb_20k": lambda: W.narrow_band_lower(20_000, 0.05, 20, 1),
    "diag_1000": lambda: W.from_pattern(1000, []),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_levels_and_level_schedule_bit_exact(L, name):
    A = CASES[name]()
    p = _host_plan(A, mode="levels")
    ex = p.export()
    lv, nlev = oracle.levels(A)
    assert np.array_equal(ex.level, lv)
    s, pi, S = oracle.level_schedule(A)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    assert np.array_equal(ex.perm, oracle.permutation(s, pi))
    st = p.stats()
    assert st["levels"] == nlev and st["supersteps"] == S and st["k"] == 1
    assert st["avg_wavefront"] == pytest.approx(A.n / nlev)
    assert oracle.check_schedule(A, ex.sigma, ex.pi, 1, strict=True) == []


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("k", [1, 2, 7, 22, 152])
def test_growlocal_bit_exact(L, name, k):
    A = CASES[name]()
    p = _host_plan(A, mode="growlocal", k=k)
    ex = p.export()
    s, pi, S = oracle.growlocal(A, k)
    assert np.array_equal(ex.sigma, s)
    assert np.array_equal(ex.pi, pi)
    assert np.array_equal(ex.perm, oracle.permutation(s, pi))
    assert p.stats()["supersteps"] == S
    assert oracle.check_schedule(A, ex.sigma, ex.pi, k) == []


@pytest.mark.parametrize("seed", range(60))
def test_growlocal_bit_exact_random_parameters(L, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 3000))
    kind = seed % 3
    if kind == 0:
        A = W.erdos_renyi_lower(n, float(rng.uniform(1e-4, 2e-2)), seed)
    elif kind == 1:
        A = W.narrow_band_lower(n, float(rng.uniform(0.02, 0.2)), float(rng.uniform(3, 40)), seed)
    else:
        A = W.random_window_lower(n, int(rng.integers(1, 8)), int(rng.integers(8, 2000)), seed)
    k = int(rng.integers(1, 40))
    kw = dict(alpha0=float(rng.choice([1.0, 2.0, 7.0, 20.0])), growth=float(rng.choice([1.2, 1.5, 2.0])),
              L=float(rng.choice([0.0, 10.0, 500.0, 5000.0])), accept=float(rng.choice([0.9, 0.97, 1.0])))
    p = _host_plan(A, mode="growlocal", k=k, **kw)
    ex = p.export()
    s, pi, S = oracle.growlocal(A, k, **kw)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    assert np.array_equal(ex.perm, oracle.permutation(s, pi))


def test_growlocal_bit_exact_er_100k(L):
    A = W.erdos_renyi_lower(100_000, 5e-4, 3)
    p = _host_plan(A, mode="growlocal", k=22)
    ex = p.export()
    s, pi, S = oracle.growlocal(A, 22)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)


@pytest.mark.parametrize("bad,code", [
    ("zero_diag", sp.ERR_ZERO_DIAG), ("upper", sp.ERR_NOT_LOWER), ("unsorted", sp.ERR_UNSORTED_OR_DUP),
    ("dup", sp.ERR_UNSORTED_OR_DUP), ("no_diag", sp.ERR_ZERO_DIAG), ("rowptr", sp.ERR_ARG),
])
def test_validation_errors(L, bad, code):
    A = W.laplace2d_lower(64, 8)
    rp, c, v = A.rowptr.copy(), A.col.copy(), A.val.copy()
    r = 20
    lo, hi = rp[r], rp[r + 1]
    if bad == "zero_diag":
        v[hi - 1] = 0.0
    elif bad == "upper":
        c[hi - 1] = r + 1
    elif bad == "unsorted":
        c[lo], c[lo + 1] = c[lo + 1], c[lo]
    elif bad == "dup":
        c[lo + 1] = c[lo]
    elif bad == "no_diag":
        c[hi - 1] = r - 2
        c[lo:hi - 1] = [r - 12, r - 5][: hi - 1 - lo]
    elif bad == "rowptr":
        rp[-1] += 1
    B = W.CSR(A.n, rp, c, v)
    with pytest.raises(sp.SptrsvError) as e:
        _host_plan(B)
    assert e.value.status == code


def test_host_only_plan_refuses_to_solve(L):
    A = W.laplace2d_lower(64, 8)
    p = _host_plan(A)
    o = sp.solve_opts()
    rep = sp.Report()
    st = L.sptrsv_solve(p.handle, 1, 1, 1, 64, sp.F64, None, 0, None)
    assert st == sp.ERR_NO_DEVICE
    assert b"host-only" in L.sptrsv_last_error()


def test_stats_on_configs(L):
    A = W.laplace3d_lower(160 ** 3, 160)
    p = _host_plan(A)
    st = p.stats()
    assert st["levels"] == 478 and st["n"] == 4_096_000 and st["nnz"] == 16_307_200


# ------------------------------------------------------------ block-local partition
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("blocks", [1, 3, 152])
def test_local_partition_invariants(L, name, blocks):
    """The executor's progress argument needs every block's list in (wavefront, id)
    order; balance needs at most ceil(1.25 * width / blocks) rows of a wavefront per block."""
    A = CASES[name]()
    blk, pos = sp.local_partition(A, blocks)
    lv, nlev = oracle.levels(A)
    lv = np.asarray(lv)
    assert blk.min() >= 0 and blk.max() < blocks
    width = np.bincount(lv, minlength=nlev)
    for b in range(blocks):
        rows = np.nonzero(blk == b)[0]
        if rows.size == 0:
            continue
        order = rows[np.argsort(pos[rows])]
        assert np.array_equal(np.sort(pos[rows]), np.arange(rows.size))          # positions 0..k-1
        key = lv[order].astype(np.int64) * A.n + order                              # (wavefront, id)
        assert np.all(np.diff(key) > 0)
        per_level = np.bincount(lv[rows], minlength=nlev)
        cap = np.maximum(1, np.ceil(width * 1.25 / blocks))
        assert np.all(per_level <= cap)


def test_local_partition_keeps_chains_in_one_block(L):
    # a bidiagonal factor is one dependency chain: every row follows its parent
    n = 200
    A = W.from_pattern(n, [(i, i - 1) for i in range(1, n)])
    blk, pos = sp.local_partition(A, 8)
    assert np.all(blk == blk[0]) and np.array_equal(pos, np.arange(n))


def test_local_partition_row_cap(L):
    A = W.laplace2d_lower(4096, 64)
    blk, pos = sp.local_partition(A, 4, row_cap=1024)
    assert np.bincount(blk, minlength=4).max() <= 1024
    with pytest.raises(sp.SptrsvError) as e:
        sp.local_partition(A, 4, row_cap=1000)          # 4 * 1000 < 4096 rows
    assert e.value.status == sp.ERR_ARG


def test_local_partition_locality_on_random_window(L):
    # most edges to a previous-wavefront parent stay inside a block (the executor's purpose)
    A = W.random_window_lower(60_000, 6, 20000, 0)
    blk, pos = sp.local_partition(A, 152)
    lv = np.asarray(oracle.levels(A)[0])
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    off = A.col != rows
    r, c = rows[off], A.col[off]
    prev = lv[c] == lv[r] - 1
    assert np.mean(blk[r][prev] == blk[c][prev]) > 0.5


def _lists_valid(A, blk, pos, blocks):
    """Every block's list is a permutation of 0..k-1 in (wavefront, id) order."""
    lv = np.asarray(oracle.levels(A)[0])
    assert blk.min() >= 0 and blk.max() < blocks
    for b in range(blocks):
        rows = np.nonzero(blk == b)[0]
        if rows.size == 0:
            continue
        order = rows[np.argsort(pos[rows])]
        assert np.array_equal(np.sort(pos[rows]), np.arange(rows.size))
        key = lv[order].astype(np.int64) * A.n + order
        assert np.all(np.diff(key) > 0)


def _block_graph_acyclic(A, blk, blocks):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    off = A.col != rows
    e = set(zip(blk[A.col[off]].tolist(), blk[rows[off]].tolist()))
    g = nx.DiGraph([(a, b) for a, b in e if a != b])
    g.add_nodes_from(range(blocks))
    return nx.is_directed_acyclic_graph(g), g


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("kind", ["parents", "ranges", "grid"])
@pytest.mark.parametrize("blocks", [1, 7, 152])
def test_block_partition_lists(L, name, kind, blocks):
    A = CASES[name]()
    blk, pos = sp.block_partition(A, blocks, kind)
    _lists_valid(A, blk, pos, blocks)


def test_parents_kind_is_the_local_partition(L):
    A = CASES["random_50k"]()
    for got, want in zip(sp.block_partition(A, 152, "parents"), sp.local_partition(A, 152)):
        assert np.array_equal(got, want)


@pytest.mark.parametrize("blocks", [3, 152])
def test_ranges_partition_is_contiguous(L, blocks):
    A = CASES["random_50k"]()
    blk, pos = sp.block_partition(A, blocks, "ranges")
    assert np.array_equal(blk, (np.arange(A.n, dtype=np.int64) * blocks // A.n).astype(np.int32))
    ok, _ = _block_graph_acyclic(A, blk, blocks)          # dependencies only to later ranges
    assert ok


@pytest.mark.parametrize("m,blocks", [(24, 152), (40, 152), (40, 12), (20, 6)])
def test_grid_partition_pencil_tiles(L, m, blocks):
    # the 3D 7-point stencil in natural order has strides 1 | m | m^2: blocks are unions of
    # whole x-lines forming (y, z) rectangles, the block graph is acyclic and a path crosses
    # at most TA + TB - 2 blocks
    A = W.laplace3d_lower(m ** 3, m)
    blk, pos = sp.block_partition(A, blocks, "grid")
    _lists_valid(A, blk, pos, blocks)
    v = np.arange(A.n)
    line = v // m
    assert np.all(blk == blk[line * m])                    # whole x-lines
    y, z = line % m, line // m
    used = np.unique(blk)
    assert 2 <= used.size <= blocks
    spans = []
    for b in used:
        ys, zs = y[blk == b], z[blk == b]
        # a rectangle of (y, z): its row count is the product of its extents (times m)
        ny, nz = ys.max() - ys.min() + 1, zs.max() - zs.min() + 1
        assert np.count_nonzero(blk == b) == ny * nz * m
        spans.append((ys.min(), zs.min()))
    TA, TB = len({s[0] for s in spans}), len({s[1] for s in spans})
    assert TA * TB == used.size
    ok, g = _block_graph_acyclic(A, blk, blocks)
    assert ok
    assert nx.dag_longest_path_length(g) <= TA + TB - 2


def test_grid_partition_falls_back_without_strides(L):
    A = CASES["random_50k"]()                              # offsets spread over a 20000-row window
    for got, want in zip(sp.block_partition(A, 152, "grid"), sp.local_partition(A, 152)):
        assert np.array_equal(got, want)
    A2 = W.laplace2d_lower(4096, 64)                       # two strides only: no (line, plane) tiling
    for got, want in zip(sp.block_partition(A2, 16, "grid"), sp.local_partition(A2, 16)):
        assert np.array_equal(got, want)


# ------------------------------------------------------------ upper and transposed systems
@pytest.mark.parametrize("name", ["lap2d_64", "lap3d_20", "random_50k", "banded_30k", "er_20k", "fig1_1"])
def test_upper_and_transposed_levels_bit_exact(L, name):
    Lo = CASES[name]()
    U = W.transpose(Lo)
    lv, nlev = oracle.levels_upper(U)
    for A, tri in ((U, "upper"), (Lo, "lower_transposed")):
        p = sp.Plan(A, device=-1, triangle=tri)
        ex = p.export()
        assert np.array_equal(ex.level, lv)
        assert p.stats()["levels"] == nlev
        # wavefront schedule: sigma = level, and the permutation lists rows by (sigma, id)
        # in the reversed numbering, i.e. by (level, descending id) here
        assert np.array_equal(ex.sigma, lv)
        key = ex.level[ex.perm].astype(np.int64) * A.n + (A.n - 1 - ex.perm)
        assert np.all(np.diff(key) > 0) and np.array_equal(np.sort(ex.perm), np.arange(A.n))


def test_upper_validation_errors(L):
    U = W.transpose(W.laplace2d_lower(64, 8))
    bad = W.CSR(U.n, U.rowptr.copy(), U.col.copy(), U.val.copy())
    bad.val[bad.rowptr[7]] = 0.0
    with pytest.raises(sp.SptrsvError) as e:
        sp.Plan(bad, device=-1, triangle="upper")
    assert e.value.status == sp.ERR_ZERO_DIAG
    with pytest.raises(sp.SptrsvError) as e:
        sp.Plan(W.laplace2d_lower(64, 8), device=-1, triangle="upper")   # a lower factor
    assert e.value.status in (sp.ERR_ZERO_DIAG, sp.ERR_NOT_LOWER)


# ------------------------------------------------- block-parallel GrowLocal (Sec. 3.1)
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("blocks", [2, 3, 8, 22])
def test_growlocal_blocks_bit_exact(L, name, blocks):
    A = CASES[name]()
    p = _host_plan(A, mode="growlocal", k=22, sched_blocks=blocks)
    ex = p.export()
    s, pi, S = oracle.growlocal_blocks(A, 22, blocks)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    assert np.array_equal(ex.perm, oracle.permutation(s, pi))
    st = p.stats()
    assert st["supersteps"] == S and st["sched_blocks"] == blocks
    assert 0.0 <= st["schedule_ms"] <= st["analyze_ms"]
    assert oracle.check_schedule(A, ex.sigma, ex.pi, 22) == []


@pytest.mark.parametrize("seed", range(24))
def test_growlocal_blocks_bit_exact_random_parameters(L, seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(1, 3000))
    A = (W.erdos_renyi_lower(n, float(rng.uniform(1e-4, 2e-2)), seed) if seed % 2 else
         W.narrow_band_lower(n, float(rng.uniform(0.02, 0.2)), float(rng.uniform(3, 40)), seed))
    k = int(rng.integers(1, 40))
    blocks = int(rng.integers(1, 40))
    threads = int(rng.integers(0, 6))
    kw = dict(alpha0=float(rng.choice([1.0, 2.0, 20.0])), growth=float(rng.choice([1.2, 1.5, 2.0])),
              L=float(rng.choice([0.0, 10.0, 500.0])), accept=float(rng.choice([0.9, 0.97, 1.0])))
    p = _host_plan(A, mode="growlocal", k=k, sched_blocks=blocks, sched_threads=threads, **kw)
    ex = p.export()
    s, pi, S = oracle.growlocal_blocks(A, k, blocks, **kw)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    assert p.stats()["supersteps"] == S


def test_growlocal_blocks_independent_of_threads(L):
    A = W.random_window_lower(200_000, 6, 20000, 3)
    ref = None
    for threads in (1, 2, 3, 6, 0):
        ex = _host_plan(A, mode="growlocal", k=152, sched_blocks=6, sched_threads=threads).export()
        if ref is None:
            ref = ex
        assert np.array_equal(ex.sigma, ref.sigma) and np.array_equal(ex.pi, ref.pi)
        assert np.array_equal(ex.perm, ref.perm)


def test_growlocal_blocks_upper_factor(L):
    # U = L^T is analysed as the reversed lower factor: its blocks cut the reversed rows
    A = W.random_window_lower(20_000, 5, 3000, 4)
    U = W.transpose(A)
    p = _host_plan(U, mode="growlocal", k=16, sched_blocks=4, triangle="upper")
    st = p.stats()
    assert st["sched_blocks"] == 4 and st["supersteps"] >= 4
    ex = p.export()
    # every edge of U (row i waits on its columns j > i) respects Definition 2.1
    rows = np.repeat(np.arange(U.n), np.diff(U.rowptr))
    off = U.col != rows
    u, v = U.col[off], rows[off]
    assert np.all(ex.sigma[u] <= ex.sigma[v])
    assert not np.any((ex.pi[u] != ex.pi[v]) & (ex.sigma[u] >= ex.sigma[v]))


def test_sched_blocks_argument_errors(L):
    A = W.laplace2d_lower(256, 16)
    with pytest.raises(sp.SptrsvError) as e:
        _host_plan(A, mode="levels", sched_blocks=4)
    assert e.value.status == sp.ERR_ARG
    for kw in (dict(sched_blocks=-1), dict(sched_threads=-2)):
        with pytest.raises(sp.SptrsvError) as e:
            _host_plan(A, mode="growlocal", k=4, **kw)
        assert e.value.status == sp.ERR_ARG
    # 0 and 1 both mean one schedule over the whole DAG
    a = _host_plan(A, mode="growlocal", k=4, sched_blocks=0).export()
    b = _host_plan(A, mode="growlocal", k=4, sched_blocks=1).export()
    assert np.array_equal(a.sigma, b.sigma) and np.array_equal(a.pi, b.pi)


# ------------------------------------------------------ Funnel coarsening (Sec. 4)
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("max_weight", [0.5, 40.0, 500.0])
def test_funnel_growlocal_bit_exact(L, name, max_weight):
    A = CASES[name]()
    p = _host_plan(A, mode="growlocal", k=22, coarsen="funnel", coarsen_max_weight=max_weight)
    ex = p.export()
    s, pi, S, part = oracle.funnel_growlocal(A, 22, max_weight=max_weight)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    assert np.array_equal(ex.perm, oracle.permutation(s, pi))
    st = p.stats()
    assert st["supersteps"] == S
    assert st["coarse_vertices"] == (int(part.max()) + 1 if A.n else 0)
    assert oracle.check_schedule(A, ex.sigma, ex.pi, 22) == []


@pytest.mark.parametrize("seed", range(24))
def test_funnel_growlocal_bit_exact_random_parameters(L, seed):
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.integers(1, 2500))
    A = (W.erdos_renyi_lower(n, float(rng.uniform(1e-4, 2e-2)), seed) if seed % 3 == 0 else
         W.narrow_band_lower(n, float(rng.uniform(0.02, 0.5)), float(rng.uniform(2, 40)), seed) if seed % 3 == 1
         else W.random_window_lower(n, int(rng.integers(1, 8)), int(rng.integers(4, 500)), seed))
    k = int(rng.integers(1, 40))
    cap = float(rng.choice([1.0, 7.0, 100.0, 500.0, 5000.0]))
    kw = dict(alpha0=float(rng.choice([1.0, 5.0, 20.0])), growth=float(rng.choice([1.2, 1.5])),
              L=float(rng.choice([0.0, 50.0, 500.0])), accept=float(rng.choice([0.9, 0.97])))
    p = _host_plan(A, mode="growlocal", k=k, coarsen="funnel", coarsen_max_weight=cap, **kw)
    ex = p.export()
    s, pi, S, part = oracle.funnel_growlocal(A, k, max_weight=cap, **kw)
    assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)
    assert p.stats()["supersteps"] == S


def test_funnel_default_weight_and_errors(L):
    A = W.erdos_renyi_lower(3000, 1e-3, 2)
    a = _host_plan(A, mode="growlocal", k=8, coarsen="funnel").export()
    b = _host_plan(A, mode="growlocal", k=8, coarsen="funnel", coarsen_max_weight=500.0).export()
    assert np.array_equal(a.sigma, b.sigma) and np.array_equal(a.pi, b.pi)
    for kw in (dict(mode="levels", coarsen="funnel"), dict(mode="growlocal", k=4, coarsen="funnel", sched_blocks=3),
               dict(mode="growlocal", k=4, coarsen=7)):
        with pytest.raises(sp.SptrsvError) as e:
            _host_plan(A, **kw)
        assert e.value.status == sp.ERR_ARG
    st = _host_plan(A, mode="growlocal", k=8).stats()
    assert st["coarse_vertices"] == A.n


def test_funnel_plan_round_trips_through_a_file(L, tmp_path):
    A = W.narrow_band_lower(6000, 0.05, 20, 3)
    p = _host_plan(A, mode="growlocal", k=16, coarsen="funnel")
    p.save(A, tmp_path / "f.plan")
    q = sp.Plan.load(tmp_path / "f.plan", device=-1)
    assert np.array_equal(p.export().sigma, q.export().sigma)
    assert q.stats()["coarse_vertices"] == p.stats()["coarse_vertices"] < A.n


def test_device_analysis_argument_errors_on_host(L):
    # refused before any device call: wrong schedule, wrong triangle, no device
    A = W.laplace2d_lower(256, 16)
    for B, kw in ((A, dict(mode="growlocal", k=4, device=-1)), (W.transpose(A), dict(triangle="upper", device=-1)),
                  (A, dict(device=-1))):
        with pytest.raises(sp.SptrsvError) as e:
            sp.Plan(B, analyze_on_device=True, **kw)
        assert e.value.status == sp.ERR_ARG


@pytest.mark.parametrize("kw", [dict(coarsen="funnel"), dict(sched_blocks=3), dict(sched_blocks=5, sched_threads=2)])
def test_new_schedules_on_degenerate_factors(L, kw):
    # empty factor: no supersteps; one row: one superstep; more blocks than rows allowed
    empty = _host_plan(W.from_pattern(0, []), mode="growlocal", k=4, **kw)
    assert empty.stats()["supersteps"] == 0 and empty.stats()["coarse_vertices"] == 0
    one = W.from_pattern(1, [])
    p = _host_plan(one, mode="growlocal", k=4, **kw)
    assert p.export().sigma.tolist() == [0] and p.stats()["supersteps"] == 1
    two = W.from_pattern(2, [(1, 0)])
    p = _host_plan(two, mode="growlocal", k=4, **kw)
    ex = p.export()
    if "coarsen" in kw:
        s, pi, S, _ = oracle.funnel_growlocal(two, 4)
    else:
        s, pi, S = oracle.growlocal_blocks(two, 4, kw["sched_blocks"])
    assert ex.sigma.tolist() == s.tolist() and ex.pi.tolist() == pi.tolist()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("max_weight", [5.0, 500.0])
def test_funnel_parts_bit_exact(L, name, max_weight):
    # the library's coarsening itself, not only the schedule, equals the oracle's
    A = CASES[name]()
    p = _host_plan(A, mode="growlocal", k=8, coarsen="funnel", coarsen_max_weight=max_weight)
    _, _, _, part = oracle.funnel_growlocal(A, 8, max_weight=max_weight)
    assert np.array_equal(p.funnel_parts(), part)


def test_funnel_parts_of_reversed_plans_group_the_same_rows(L):
    L_ = W.narrow_band_lower(3000, 0.1, 10, 6)
    U = W.transpose(L_)
    pu = _host_plan(U, mode="growlocal", k=8, coarsen="funnel", triangle="upper").funnel_parts()
    pt = _host_plan(L_, mode="growlocal", k=8, coarsen="funnel", triangle="lower_transposed").funnel_parts()
    assert np.array_equal(pu, pt)
    assert sorted(set(pu.tolist())) == list(range(int(pu.max()) + 1))
    with pytest.raises(sp.SptrsvError):
        _host_plan(L_, mode="growlocal", k=8).funnel_parts()        # not a Funnel plan


def test_funnel_independent_of_threads(L):
    A = W.erdos_renyi_lower(60_000, 5e-4, 9)
    ref = None
    for threads in (1, 2, 3, 0):
        p = _host_plan(A, mode="growlocal", k=64, coarsen="funnel", sched_threads=threads)
        got = (p.export().sigma, p.export().pi, p.funnel_parts())
        if ref is None:
            ref = got
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


def _reversed_lower(U):
    """L' with rows and columns numbered backwards: row i' of L' is row n-1-i' of U."""
    n = U.n
    cols, vals, rp = [], [], [0]
    for i2 in range(n):
        i = n - 1 - i2
        lo, hi = U.rowptr[i], U.rowptr[i + 1]
        cols.append((n - 1 - U.col[lo:hi])[::-1])
        vals.append(U.val[lo:hi][::-1])
        rp.append(rp[-1] + hi - lo)
    return W.CSR(n, np.array(rp, np.int32), np.concatenate(cols).astype(np.int32), np.concatenate(vals), "rev")


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("sched", ["funnel", "blocks"])
def test_reversed_plans_schedule_the_reversed_factor(L, seed, sched):
    # U x = b and L^T x = b are scheduled as L' (ids reversed): in the caller's numbering
    # the library's schedule is the oracle's schedule of L' read backwards
    rng = np.random.default_rng(8800 + seed)
    n = int(rng.integers(2, 900))
    Lo = (W.narrow_band_lower(n, float(rng.uniform(0.05, 0.5)), float(rng.uniform(2, 20)), seed) if seed % 2
          else W.erdos_renyi_lower(n, float(rng.uniform(2e-3, 0.03)), seed))
    U = W.transpose(Lo)
    Lr = _reversed_lower(U)
    oracle.validate(Lr)
    k = int(rng.integers(1, 30))
    if sched == "funnel":
        kw = dict(coarsen="funnel")
        s, pi = oracle.funnel_growlocal(Lr, k)[:2]
    else:
        kw = dict(sched_blocks=int(rng.integers(2, 9)))
        s, pi = oracle.growlocal_blocks(Lr, k, kw["sched_blocks"])[:2]
    for tri, A in (("upper", U), ("lower_transposed", Lo)):
        ex = _host_plan(A, mode="growlocal", k=k, triangle=tri, **kw).export()
        assert np.array_equal(ex.sigma, s[::-1]) and np.array_equal(ex.pi, pi[::-1])
