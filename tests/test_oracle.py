"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: every expectation is a value
printed in the paper (tests/golden), a closed form derived by hand, a library
routine (dense LAPACK triangular solve, networkx longest path) or a brute-force
enumeration on tiny inputs.
"""
import itertools

import networkx as nx
import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W
from conftest import golden


def _pattern_from_golden(g):
    n = int(g["n"])
    ents = [tuple(int(t) - 1 for t in e.split(",")) for e in g["entries"].split()]
    return n, ents


# ---------------------------------------------------------------- Fig. 1.1
def test_fig1_1_dag_and_wavefronts():
    g = golden("fig1_1.txt")
    n, ents = _pattern_from_golden(g)
    labels = g["labels"].split()
    A = W.from_pattern(n, ents)
    oracle.validate(A)
    u, v = oracle.edges(A)
    got = sorted((labels[a], labels[b]) for a, b in zip(u, v))
    want = sorted(tuple(e.split(",")) for e in g["edges"].split())
    assert got == want
    lv, nlev = oracle.levels(A)
    fronts = [set(f.split()) for f in g["wavefronts"].split("|")]
    assert nlev == len(fronts) == 4
    for w, members in enumerate(fronts):
        assert {labels[i] for i in range(n) if lv[i] == w} == members
    # Average wavefront size (Sec. 6.2): n / longest path (in vertices) = 6 / 4.
    assert oracle.avg_wavefront(A) == pytest.approx(1.5)


def test_fig1_1_solve_closed_form():
    # Unit diagonal, off-diagonals -1, b = 1: x_v = 1 + x_parent by Eq. 2.1, so
    # x_a = 1, x_b = 2, x_c = x_d = 3, x_e = x_f = 4 (one more per wavefront).
    g = golden("fig1_1.txt")
    n, ents = _pattern_from_golden(g)
    A = W.from_pattern(n, ents, diag=1.0, off=-1.0)
    x = oracle.solve(A, np.ones(n))
    assert x.tolist() == [1.0, 2.0, 3.0, 3.0, 4.0, 4.0]


# ---------------------------------------------------------------- Fig. 3.1
def test_fig3_1_blocks():
    g = golden("fig3_1.txt")
    n, ents = _pattern_from_golden(g)
    A = W.from_pattern(n, ents)
    oracle.validate(A)
    blocks = [tuple(int(t) - 1 for t in b.split("-")) for b in g["blocks"].split()]
    blk = np.empty(n, dtype=int)
    for bi, (lo, hi) in enumerate(blocks):
        blk[lo:hi + 1] = bi
    u, v = oracle.edges(A)
    intra = [sorted((a, b) for a, b in zip(u, v) if blk[a] == blk[b] == bi) for bi in range(3)]
    want = [sorted(tuple(int(t) - 1 for t in e.split(",")) for e in part.split())
            for part in g["intra"].split("|")]
    assert intra == want
    inter = {(int(blk[a]), int(blk[b])) for a, b in zip(u, v) if blk[a] != blk[b]}
    assert inter == {tuple(int(t) - 1 for t in e.split(",")) for e in g["inter"].split()}


# ------------------------------------------------------ solve vs LAPACK / closed forms
@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (33, 3), (64, 4)])
def test_solve_matches_dense_lapack(n, seed):
    rng = np.random.default_rng(seed)
    D = np.tril(rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.4), -1)
    D += np.diag(rng.uniform(1.0, 3.0, n) * np.where(rng.random(n) < 0.5, -1, 1))
    rows, cols = np.nonzero(D)
    A = W.from_pattern(n, list(zip(rows.tolist(), cols.tolist())))
    A.val[:] = D[np.repeat(np.arange(n), np.diff(A.rowptr)), A.col]
    oracle.validate(A)
    B = rng.standard_normal((n, 3))
    X = oracle.solve(A, B)
    Xref = scipy.linalg.solve_triangular(D, B, lower=True)
    assert oracle.rel_error(X, Xref) < 1e-12


def test_solve_diagonal_closed_form():
    rng = np.random.default_rng(5)
    n = 50
    d = rng.uniform(0.5, 2.0, n)
    A = W.from_pattern(n, [])
    A.val[:] = d
    b = rng.standard_normal(n)
    x = oracle.solve(A, b)
    assert np.array_equal(x, b / d)          # one IEEE division per row, nothing else
    assert oracle.levels(A)[1] == 1


def test_solve_bidiagonal_closed_form():
    # diag 2, sub-diagonal -1, b = 1: x_i = (1 + x_{i-1}) / 2 = 1 - 2^-(i+1), exact in FP64.
    n = 80
    A = W.from_pattern(n, [(i, i - 1) for i in range(1, n)], diag=2.0, off=-1.0)
    x = oracle.solve(A, np.ones(n))
    assert np.array_equal(x, 1.0 - 2.0 ** -(np.arange(n) + 1.0))
    assert oracle.levels(A)[1] == n


@pytest.mark.parametrize("make", [
    lambda: W.laplace2d_lower(4096, 64),
    lambda: W.laplace3d_lower(24 ** 3, 24),
    lambda: W.random_window_lower(30000, 6, 20000, 0),
    lambda: W.random_window_lower(20000, 4, 64, 3),
    lambda: W.erdos_renyi_lower(5000, 5e-4, 1),
])
def test_manufactured_solution(make):
    A = make()
    oracle.validate(A)
    xs, b = W.manufactured_rhs(A, 2, seed=7)
    x = oracle.solve(A, b)
    assert oracle.rel_error(x, xs) < 1e-13
    # and the residual it leaves is at rounding level
    r = b - oracle.spmv(A, x)
    assert np.max(np.abs(r)) < 1e-12 * np.max(np.abs(b))


def test_spmv_against_dense():
    A = W.random_window_lower(300, 6, 50, 9)
    D = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    D[rows, A.col] = A.val
    x = np.random.default_rng(0).standard_normal(A.n)
    assert np.allclose(oracle.spmv(A, x), D @ x, rtol=1e-14, atol=1e-12)


# ------------------------------------------------------------------- levels
def test_levels_stencil_closed_forms():
    # Natural-order 2D stencil: wavefront of node (i, j) is i + j -> 2*64-1 = 127 fronts.
    A = W.laplace2d_lower(4096, 64)
    lv, nlev = oracle.levels(A)
    i, j = np.arange(4096) % 64, np.arange(4096) // 64
    assert nlev == 127 and np.array_equal(lv, i + j)
    # 3D: wavefront of (i, j, k) is i + j + k -> 3*w - 2 fronts (478 at w = 160).
    w = 30
    A = W.laplace3d_lower(w ** 3, w)
    lv, nlev = oracle.levels(A)
    idx = np.arange(w ** 3)
    assert nlev == 3 * w - 2 and np.array_equal(lv, idx % w + (idx // w) % w + idx // (w * w))
    assert oracle.levels(W.laplace3d_lower(160 ** 3, 160))[1] == 478


@pytest.mark.parametrize("seed", range(6))
def test_levels_vs_networkx_longest_path(seed):
    A = W.erdos_renyi_lower(300, 0.02, seed)
    lv, nlev = oracle.levels(A)
    G = nx.DiGraph()
    G.add_nodes_from(range(A.n))
    u, v = oracle.edges(A)
    G.add_edges_from(zip(u.tolist(), v.tolist()))
    assert nlev == nx.dag_longest_path_length(G) + 1
    # level(v) = longest path ending at v (edges), computed independently
    depth = {}
    for node in nx.topological_sort(G):
        depth[node] = max((depth[p] + 1 for p in G.predecessors(node)), default=0)
    assert [depth[i] for i in range(A.n)] == lv.tolist()


# ---------------------------------------------------------------- validation
def test_validate_rejects_bad_inputs():
    A = W.laplace2d_lower(16, 4)
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.val[bad.rowptr[5] - 1] = 0.0
    with pytest.raises(oracle.InvalidFactor, match="zero diagonal"):
        oracle.validate(bad)
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[bad.rowptr[6] - 1] = 7                      # diagonal of row 5 moved above it
    with pytest.raises(oracle.InvalidFactor):
        oracle.validate(bad)
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    r = 10
    bad.col[bad.rowptr[r]], bad.col[bad.rowptr[r] + 1] = bad.col[bad.rowptr[r] + 1], bad.col[bad.rowptr[r]]
    with pytest.raises(oracle.InvalidFactor):
        oracle.validate(bad)


# ------------------------------------------------------------ schedule checker
def _brute_force_def21(A, sigma, pi):
    """Definition 2.1 by enumerating every ordered pair (u, v) against the dense pattern."""
    D = np.zeros((A.n, A.n), dtype=bool)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    D[rows, A.col] = True
    for v, u in itertools.product(range(A.n), repeat=2):
        if u < v and D[v, u]:                               # edge u -> v
            if sigma[u] > sigma[v]:
                return False
            if pi[u] != pi[v] and not sigma[u] < sigma[v]:
                return False
    return True


@pytest.mark.parametrize("seed", range(40))
def test_checker_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 13))
    A = W.erdos_renyi_lower(n, float(rng.uniform(0.1, 0.6)), seed)
    k = int(rng.integers(1, 4))
    sigma = rng.integers(0, 4, n)
    _, sigma = np.unique(sigma, return_inverse=True)        # contiguous superstep ids
    pi = rng.integers(0, k, n)
    ok_checker = oracle.check_schedule(A, sigma, pi, k) == []
    assert ok_checker == _brute_force_def21(A, sigma, pi)


def test_checker_catches_planted_violations():
    A = W.erdos_renyi_lower(400, 0.01, 3)
    sigma, pi, S = oracle.growlocal(A, 4)
    assert oracle.check_schedule(A, sigma, pi, 4) == []
    u, v = oracle.edges(A)
    e = int(np.argmax(sigma[v] > 0))
    s2 = sigma.copy()
    s2[v[e]] = sigma[u[e]] - 1 if sigma[u[e]] > 0 else 0
    s2[u[e]] = s2[v[e]] + 1
    assert oracle.check_schedule(A, s2, pi, 4) != []        # child before its parent
    p2 = pi.copy()
    s3 = sigma.copy()
    s3[v[e]] = s3[u[e]]
    p2[v[e]] = (pi[u[e]] + 1) % 4
    assert oracle.check_schedule(A, s3, p2, 4) != []        # cross-core edge in a superstep
    lv, zeros, _ = oracle.level_schedule(A)
    assert oracle.check_schedule(A, lv, zeros, 1, strict=True) == []


# ------------------------------------------------------------------ GrowLocal
def test_growlocal_diagonal_worked_example():
    # n = 40 isolated vertices (weights 1), k = 2, default parameters.
    # attempt alpha=20: core0 = {0..19}, core1 = {20..39}, beta = 40/520
    # attempt alpha=30: core0 = {0..29}, core1 = {30..39}, beta = 40/530 >= 0.97*40/520,
    #   worthy, and every vertex is assigned -> one superstep.
    A = W.from_pattern(40, [])
    sigma, pi, S = oracle.growlocal(A, 2)
    assert S == 1
    assert sigma.tolist() == [0] * 40
    assert pi.tolist() == [0] * 30 + [1] * 10


def test_growlocal_hand_example_two_supersteps():
    # Vertices 0,1 sources; 2 <- 0; 3 <- 1; 4 <- {2, 3}.  Weights 1,1,2,2,3.
    # alpha0 = 1, growth = 2, L = 1, accept = 0.97, k = 2:
    #  superstep 0, attempt 0 (limit 1): core0 {0}, core1 {1}; beta = 2/(1+1) = 1.0
    #               attempt 1 (limit 2): core0 {0,2}, core1 {1,3}; 4 has parents on two
    #                 cores -> blocked; beta = 6/(3+1) = 1.5 (worthy)
    #               attempt 2 (limit 4): core0 {0,2,1,3}, core1 {} ; beta = 6/7 < 0.97*1.5
    #                 -> unworthy, keep attempt 1
    #  superstep 1: R = {4}: core0 {4}.
    A = W.from_pattern(5, [(2, 0), (3, 1), (4, 2), (4, 3)])
    sigma, pi, S = oracle.growlocal(A, 2, alpha0=1.0, growth=2.0, L=1.0, accept=0.97)
    assert S == 2
    assert sigma.tolist() == [0, 0, 0, 0, 1]
    assert pi.tolist() == [0, 1, 0, 1, 0]
    assert oracle.permutation(sigma, pi).tolist() == [0, 2, 1, 3, 4]


@pytest.mark.parametrize("make", [
    lambda: W.laplace2d_lower(4096, 64),
    lambda: W.random_window_lower(3000, 6, 500, 1),
    lambda: W.erdos_renyi_lower(2000, 1e-3, 2),
])
def test_growlocal_single_core_is_one_superstep(make):
    A = make()
    sigma, pi, S = oracle.growlocal(A, 1)
    assert S == 1 and not sigma.any() and not pi.any()
    assert np.array_equal(oracle.permutation(sigma, pi), np.arange(A.n))


@pytest.mark.parametrize("seed", range(30))
def test_growlocal_valid_on_random_dags(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 400))
    A = W.erdos_renyi_lower(n, float(rng.uniform(0.001, 0.05)), seed)
    k = int(rng.integers(1, 9))
    a0 = float(rng.choice([1.0, 3.0, 20.0]))
    sigma, pi, S = oracle.growlocal(A, k, alpha0=a0, L=float(rng.choice([1.0, 50.0, 500.0])))
    assert oracle.check_schedule(A, sigma, pi, k) == []
    assert S == sigma.max() + 1 if n else S == 0


def test_growlocal_every_vertex_once_on_er_100k():
    A = W.erdos_renyi_lower(100_000, 1e-4, 0)
    sigma, pi, S = oracle.growlocal(A, 22)
    assert oracle.check_schedule(A, sigma, pi, 22) == []
    lv, nlev = oracle.levels(A)
    # GrowLocal merges wavefronts: never more supersteps than wavefronts here.
    assert 1 <= S <= nlev


# ------------------------------------------------- block-parallel GrowLocal (Sec. 3.1)
def test_block_subdags_match_fig3_1():
    # Three blocks of the 9x9 example: the equal-row cut reproduces the figure's blocks,
    # each sub-DAG holds exactly the figure's solid (intra-block) edges, the dropped
    # entries are its dashed (inter-block) dependencies, and weights stay full-row.
    g = golden("fig3_1.txt")
    n, ents = _pattern_from_golden(g)
    A = W.from_pattern(n, ents)
    blocks = [tuple(int(t) - 1 for t in b.split("-")) for b in g["blocks"].split()]
    want_intra = [sorted(tuple(int(t) - 1 for t in e.split(",")) for e in part.split())
                  for part in g["intra"].split("|")]
    dropped = set()
    for b, (lo, hi) in enumerate(blocks):
        r0, r1 = b * n // 3, (b + 1) * n // 3
        assert (r0, r1 - 1) == (lo, hi)
        rp, col, w = oracle.block_subdag(A, r0, r1)
        got = []
        for i in range(r1 - r0):
            assert col[rp[i + 1] - 1] == i                    # diagonal kept, last
            got += [(int(col[q]) + r0, i + r0) for q in range(rp[i], rp[i + 1] - 1)]
        assert sorted(got) == want_intra[b]
        assert w.tolist() == np.diff(A.rowptr)[r0:r1].tolist()
        for i in range(r0, r1):
            for q in range(A.rowptr[i], A.rowptr[i + 1] - 1):
                if A.col[q] < r0:
                    dropped.add((int(A.col[q]) // 3, b))
    assert dropped == {tuple(int(t) - 1 for t in e.split(",")) for e in g["inter"].split()}


def test_growlocal_blocks_hand_example_full_row_weights():
    # Rows 0..3: diagonal only (weight 1).  Row 4 <- {0,1,2,3} (weight 5), rows 5..7
    # diagonal only.  Two blocks {0..3}, {4..7}; k = 2, alpha0 = 1, growth = 2, L = 0.
    # Block 0 (all ready, weights 1): attempt limit 1: core0 {0}, core1 {1}, beta 2/1;
    #   limit 2: core0 {0,1}, core1 {2,3}, beta 4/2 (worthy); limit 4: core0 {0..3},
    #   beta 4/4 < 0.97*2 -> keep {0,1 | 2,3}: one superstep.
    # Block 1: the edges into row 4 come from block 0 and are dropped, but row 4 keeps
    #   weight 5.  limit 1: core0 {4} (Omega 5), core1 {5,6,7} (Omega 3), beta 8/5;
    #   limit 2: core0 {4,5} (6), core1 {6,7} (2), beta 8/6 < 0.97*1.6 -> keep the first.
    #   (Block-local weights would give core0 {4,5}, core1 {6,7} instead.)
    # Concatenation: block 1's superstep 0 becomes superstep 1.
    A = W.from_pattern(8, [(4, 0), (4, 1), (4, 2), (4, 3)])
    sigma, pi, S = oracle.growlocal_blocks(A, 2, 2, alpha0=1.0, growth=2.0, L=0.0, accept=0.97)
    assert S == 2
    assert sigma.tolist() == [0, 0, 0, 0, 1, 1, 1, 1]
    assert pi.tolist() == [0, 0, 1, 1, 0, 1, 1, 1]
    assert oracle.check_schedule(A, sigma, pi, 2) == []


@pytest.mark.parametrize("make", [
    lambda: W.laplace2d_lower(400, 20),
    lambda: W.random_window_lower(300, 6, 50, 4),
])
def test_growlocal_blocks_one_row_per_block_is_sequential(make):
    # Every block is one vertex: core 0, superstep 0 of its block -> sigma = id, pi = 0.
    A = make()
    sigma, pi, S = oracle.growlocal_blocks(A, 4, A.n)
    assert S == A.n
    assert sigma.tolist() == list(range(A.n)) and not pi.any()


def _block_diagonal(parts):
    rp, cols, vals, off = [0], [], [], 0
    for P in parts:
        for i in range(P.n):
            lo, hi = P.rowptr[i], P.rowptr[i + 1]
            cols += (P.col[lo:hi] + off).tolist()
            vals += P.val[lo:hi].tolist()
            rp.append(len(cols))
        off += P.n
    return W.CSR(off, np.array(rp, np.int32), np.array(cols, np.int32), np.array(vals), "blockdiag")


def test_growlocal_blocks_block_diagonal_matches_separate_schedules():
    # Three independent parts of 144 rows, cut into the same three blocks: no edge
    # crosses a block, nothing is dropped and every weight is the block's own, so
    # each block's schedule is GrowLocal of that part alone, shifted by the
    # supersteps of the parts before it.
    parts = [W.laplace2d_lower(144, 12), W.erdos_renyi_lower(144, 0.03, 7),
             W.random_window_lower(144, 5, 40, 8)]
    A = _block_diagonal(parts)
    sigma, pi, S = oracle.growlocal_blocks(A, 3, 3, alpha0=3.0, L=10.0)
    offset = 0
    for b, P in enumerate(parts):
        s_b, p_b, S_b = oracle.growlocal(P, 3, alpha0=3.0, L=10.0)
        r0 = 144 * b
        assert np.array_equal(sigma[r0:r0 + 144], s_b + offset)
        assert np.array_equal(pi[r0:r0 + 144], p_b)
        offset += S_b
    assert S == offset


@pytest.mark.parametrize("seed", range(12))
def test_growlocal_blocks_valid_and_block_ordered(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(1, 500))
    A = W.erdos_renyi_lower(n, float(rng.uniform(0.002, 0.05)), seed)
    k = int(rng.integers(1, 7))
    blocks = int(rng.integers(2, 9))
    sigma, pi, S = oracle.growlocal_blocks(A, k, blocks, alpha0=float(rng.choice([1.0, 5.0, 20.0])),
                                           L=float(rng.choice([0.0, 20.0, 500.0])))
    assert oracle.check_schedule(A, sigma, pi, k) == []
    # each block owns a contiguous superstep range, in block order, none shared
    lo = 0
    for b in range(blocks):
        r0, r1 = b * n // blocks, (b + 1) * n // blocks
        if r1 == r0:
            continue
        seg = sigma[r0:r1]
        assert seg.min() == lo
        lo = int(seg.max()) + 1
    assert S == lo


# -------------------------------------------------- Funnel coarsening (Sec. 4)
def _digraph(n, parents):
    G = nx.DiGraph()
    G.add_nodes_from(range(n))
    G.add_edges_from((u, w) for w in range(n) for u in parents[w])
    return G


@pytest.mark.parametrize("seed", range(25))
def test_triangle_reduce_brute_force(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 13))
    A = W.erdos_renyi_lower(n, float(rng.uniform(0.1, 0.7)), seed)
    full = [set(A.col[A.rowptr[i]:A.rowptr[i + 1] - 1].tolist()) for i in range(n)]
    kept = oracle.triangle_reduce(A)
    for w in range(n):
        want = {u for u in full[w] if not any(u in full[v] for v in full[w])}
        assert set(kept[w]) == want and kept[w] == sorted(kept[w])
    # the reduction keeps reachability: same transitive closure as the DAG
    G, R = _digraph(n, [sorted(f) for f in full]), _digraph(n, kept)
    assert set(nx.transitive_closure_dag(G).edges) == set(nx.transitive_closure_dag(R).edges)


def test_funnel_hand_examples():
    inf = float("inf")
    # diamond 0 -> {1, 2} -> 3: one in-funnel rooted at 3
    part, roots = oracle.funnel_parts(4, [[], [0], [0], [1, 2]], [1, 2, 2, 3], inf)
    assert part.tolist() == [0, 0, 0, 0] and roots == [3]
    # an in-tree is an in-funnel (Sec. 4.2 footnote): 0,1 -> 2; 3 -> 4; 2,4 -> 5
    part, roots = oracle.funnel_parts(6, [[], [], [0, 1], [], [3], [2, 4]], [1] * 6, inf)
    assert part.tolist() == [0] * 6 and roots == [5]
    # a vertex with children in two parts joins neither: 0 -> 1, 0 -> 2
    part, roots = oracle.funnel_parts(3, [[], [0], [0]], [1, 2, 2], inf)
    assert roots == [0, 1, 2] and part.tolist() == [0, 1, 2]
    # weight cap 4 on the chain 0 -> 1 -> 2 -> 3 (weights 1, 2, 2, 2): {2, 3} fills the
    # first part (1 would make it 6), {0, 1} the second; parts numbered by root
    part, roots = oracle.funnel_parts(4, [[], [0], [1], [2]], [1, 2, 2, 2], 4)
    assert part.tolist() == [0, 0, 1, 1] and roots == [1, 3]


@pytest.mark.parametrize("seed", range(10))
def test_funnel_single_sink_collapses_without_the_cap(seed):
    # Sec. 4.2: without the size constraint a DAG with a single sink coarsens to one vertex
    rng = np.random.default_rng(1500 + seed)
    n = int(rng.integers(2, 60))
    A = W.erdos_renyi_lower(n - 1, float(rng.uniform(0.02, 0.3)), seed)
    parents = [A.col[A.rowptr[i]:A.rowptr[i + 1] - 1].tolist() for i in range(n - 1)]
    has_child = set(u for p in parents for u in p)
    parents.append([v for v in range(n - 1) if v not in has_child])      # every sink -> vertex n-1
    part, roots = oracle.funnel_parts(n, parents, [1] * n, float("inf"))
    assert roots == [n - 1] and not part.any()
    part, roots = oracle.funnel_parts(n, parents, [1] * n, 3)            # the cap splits it again
    assert len(roots) >= (n + 2) // 3


@pytest.mark.parametrize("seed", range(25))
def test_funnel_parts_are_in_funnels_and_coarsening_is_acyclic(seed):
    rng = np.random.default_rng(1300 + seed)
    n = int(rng.integers(1, 40))
    A = (W.erdos_renyi_lower(n, float(rng.uniform(0.03, 0.4)), seed) if seed % 2 else
         W.narrow_band_lower(n, float(rng.uniform(0.2, 0.9)), float(rng.uniform(1, 4)), seed))
    kept = oracle.triangle_reduce(A)
    weight = np.diff(A.rowptr).tolist()
    cap = float(rng.choice([3, 8, 1e9]))
    part, roots = oracle.funnel_parts(n, kept, weight, cap)
    assert sorted(set(part.tolist())) == list(range(len(roots)))
    R = _digraph(n, kept)
    reach = nx.transitive_closure_dag(R)
    for i, r in enumerate(roots):
        U = set(np.nonzero(part == i)[0].tolist())
        assert max(U) == r
        out_cut = {u for u in U if any(w not in U for w in R.successors(u))}
        in_cut = {v for v in U if any(u not in U for u in R.predecessors(v))}
        assert out_cut <= {r}                                   # Def. in-funnel: one exit at most
        assert all(v == u or reach.has_edge(v, u) for v in in_cut for u in out_cut)   # cascade
        if len(U) > 1:
            assert sum(weight[u] for u in U) <= cap
    # Prop. (cascade coarsening): the ORIGINAL DAG coarsened along the parts is acyclic
    u, v = oracle.edges(A)
    C = nx.DiGraph()
    C.add_nodes_from(range(len(roots)))
    C.add_edges_from((int(part[a]), int(part[b])) for a, b in zip(u, v) if part[a] != part[b])
    assert nx.is_directed_acyclic_graph(C)


@pytest.mark.parametrize("seed", range(12))
def test_funnel_growlocal_schedule_valid(seed):
    rng = np.random.default_rng(1700 + seed)
    n = int(rng.integers(1, 600))
    A = W.erdos_renyi_lower(n, float(rng.uniform(0.002, 0.05)), seed)
    k = int(rng.integers(1, 9))
    sigma, pi, S, part = oracle.funnel_growlocal(A, k, max_weight=float(rng.choice([4.0, 50.0, 500.0])),
                                                 alpha0=float(rng.choice([1.0, 20.0])))
    assert oracle.check_schedule(A, sigma, pi, k) == []
    for i in range(int(part.max()) + 1 if n else 0):           # a part never straddles a block
        members = part == i
        assert len(set(sigma[members])) == 1 and len(set(pi[members])) == 1


@pytest.mark.parametrize("make", [
    lambda: W.erdos_renyi_lower(500, 0.01, 3),
    lambda: W.laplace2d_lower(400, 20),
    lambda: W.narrow_band_lower(500, 0.1, 8, 4),
])
def test_funnel_growlocal_without_coarsening_is_growlocal(make):
    # max_weight 0: every part is one vertex; without the reduction the coarsened DAG is
    # the DAG itself, so the schedule must be GrowLocal's
    A = make()
    sigma, pi, S, part = oracle.funnel_growlocal(A, 6, max_weight=0.0, reduce=False)
    s, p, S2 = oracle.growlocal(A, 6)
    assert np.array_equal(part, np.arange(A.n))
    assert np.array_equal(sigma, s) and np.array_equal(pi, p) and S == S2


# ---------------------------------------------------------------- permutation
@pytest.mark.parametrize("seed", range(5))
def test_permutation_is_bijection_and_keeps_lower(seed):
    A = W.erdos_renyi_lower(1500, 2e-3, seed)
    sigma, pi, S = oracle.growlocal(A, 5)
    perm = oracle.permutation(sigma, pi)
    assert np.array_equal(np.sort(perm), np.arange(A.n))
    r, c, _ = oracle.permute(A, perm)
    assert np.all(c <= r)                                     # P A P^T stays lower (Sec. 5)
    # blocks in (superstep, core) order, original order inside each block
    key = sigma[perm].astype(np.int64) * 64 + pi[perm]
    assert np.all(np.diff(key) >= 0)
    same = np.diff(key) == 0
    assert np.all(np.diff(perm)[same] > 0)
    # the permuted system has the permuted solution
    xs, b = W.manufactured_rhs(A, 1, seed=seed)
    x = oracle.solve(A, b)
    inv = np.empty(A.n, dtype=np.int64)
    inv[perm] = np.arange(A.n)
    B = W.CSR(A.n, *_csr_from_coo(A.n, r, c, A.val))
    xp = oracle.solve(B, b[perm])
    assert oracle.rel_error(xp, x[perm]) < 1e-13


def _csr_from_coo(n, r, c, v):
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), c.astype(np.int32), v


# ------------------------------------------------------ backward substitution (upper / L^T)
def _dense(A):
    D = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    D[rows, A.col] = A.val
    return D


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (33, 3), (64, 4)])
def test_solve_upper_and_transposed_match_dense_lapack(n, seed):
    rng = np.random.default_rng(100 + seed)
    D = np.tril(rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.4), -1)
    D += np.diag(rng.uniform(1.0, 3.0, n) * np.where(rng.random(n) < 0.5, -1, 1))
    rows, cols = np.nonzero(D)
    L = W.from_pattern(n, list(zip(rows.tolist(), cols.tolist())))
    L.val[:] = D[np.repeat(np.arange(n), np.diff(L.rowptr)), L.col]
    U = W.transpose(L)
    oracle.validate_upper(U)
    assert np.array_equal(_dense(U), D.T)
    B = rng.standard_normal((n, 3))
    Xref = scipy.linalg.solve_triangular(D.T, B, lower=False)
    assert oracle.rel_error(oracle.solve_upper(U, B), Xref) < 1e-12
    assert oracle.rel_error(oracle.solve_transposed(L, B), Xref) < 1e-12


def test_solve_upper_bidiagonal_closed_form():
    # diag 2, super-diagonal -1, b = 1: x_i = (1 + x_{i+1}) / 2 = 1 - 2^-(n-i), exact in FP64.
    n = 80
    U = W.transpose(W.from_pattern(n, [(i, i - 1) for i in range(1, n)], diag=2.0, off=-1.0))
    want = 1.0 - 2.0 ** -(n - np.arange(n, dtype=np.float64))
    assert np.array_equal(oracle.solve_upper(U, np.ones(n)), want)
    L = W.from_pattern(n, [(i, i - 1) for i in range(1, n)], diag=2.0, off=-1.0)
    assert np.array_equal(oracle.solve_transposed(L, np.ones(n)), want)
    lv, nl = oracle.levels_upper(U)
    assert nl == n and lv[0] == n - 1 and lv[-1] == 0


def test_solve_upper_diagonal_closed_form():
    rng = np.random.default_rng(6)
    n = 40
    d = rng.uniform(0.5, 2.0, n)
    L = W.from_pattern(n, [])
    L.val[:] = d
    b = rng.standard_normal(n)
    assert np.array_equal(oracle.solve_upper(W.transpose(L), b), b / d)
    assert np.array_equal(oracle.solve_transposed(L, b), b / d)


@pytest.mark.parametrize("make", [
    lambda: W.laplace2d_lower(4096, 64),
    lambda: W.random_window_lower(30000, 6, 20000, 0),
])
def test_upper_manufactured_solution_and_levels(make):
    L = make()
    U = W.transpose(L)
    xs, b = W.manufactured_rhs(U, 2, seed=8)
    x = oracle.solve_upper(U, b)
    assert oracle.rel_error(x, xs) < 1e-13
    assert oracle.rel_error(oracle.solve_transposed(L, b), xs) < 1e-13
    # the upper DAG is the lower one reversed: same number of wavefronts
    assert oracle.levels_upper(U)[1] == oracle.levels(L)[1]


def test_validate_upper_rejects_bad_inputs():
    U = W.transpose(W.laplace2d_lower(64, 8))
    oracle.validate_upper(U)
    bad = W.CSR(U.n, U.rowptr.copy(), U.col.copy(), U.val.copy())
    bad.val[bad.rowptr[5]] = 0.0
    with pytest.raises(oracle.InvalidFactor):
        oracle.validate_upper(bad)
    with pytest.raises(oracle.InvalidFactor):
        oracle.validate_upper(W.laplace2d_lower(64, 8))       # lower, diagonal last


# ---------------------------------------------------------------- error metric
def test_rel_error_hand_values():
    """The normwise relative error every parity test goes through (reading iv of
    the error metric: max_i |x_i - xref_i| / max_i |xref_i| per right-hand-side
    column, worst column reported), on values worked out by hand."""
    xref = np.array([[1.0, 10.0], [2.5, 20.0], [3.0, 28.0]])
    x = np.array([[1.0, 10.0], [2.0, 20.0], [3.0, 30.0]])
    # column 0: max |diff| = 0.5, max |xref| = 3  -> 1/6
    # column 1: max |diff| = 2.0, max |xref| = 28 -> 1/14
    assert oracle.rel_error(x, xref) == pytest.approx(1.0 / 6.0, rel=1e-15)
    # per-column denominators: one shared over both columns (28) would give 1/14
    assert oracle.rel_error(x[:, 1:], xref[:, 1:]) == pytest.approx(1.0 / 14.0, rel=1e-15)
    # the worst column decides, whichever position it holds
    assert oracle.rel_error(x[:, ::-1], xref[:, ::-1]) == pytest.approx(1.0 / 6.0, rel=1e-15)
    # absolute values in numerator and denominator: [1, 2, -4] vs [1, 2, -5] -> 1/5
    assert oracle.rel_error(np.array([1.0, 2.0, -4.0]), np.array([1.0, 2.0, -5.0])) == pytest.approx(0.2)
    # the reference is the second argument: |2 - 1| / 1 against |1 - 2| / 2
    assert oracle.rel_error(np.array([2.0]), np.array([1.0])) == 1.0
    assert oracle.rel_error(np.array([1.0]), np.array([2.0])) == 0.5
    # a vector and an n x 1 block are the same single column (no broadcasting)
    v, vr = np.array([1.0, 2.0, 4.0]), np.array([1.0, 2.5, 4.0])
    assert oracle.rel_error(v, vr.reshape(3, 1)) == pytest.approx(0.125)
    assert oracle.rel_error(v.reshape(3, 1), vr) == pytest.approx(0.125)
    # a zero reference column falls back to the absolute error of that column
    assert oracle.rel_error(np.array([[0.0, 1.0], [0.25, 1.0]]), np.array([[0.0, 1.0], [0.0, 1.0]])) == 0.25
    # exact agreement and empty inputs
    assert oracle.rel_error(xref, xref) == 0.0
    assert oracle.rel_error(np.zeros((0, 2)), np.zeros((0, 2))) == 0.0
