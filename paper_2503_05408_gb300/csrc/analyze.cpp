// Host analysis: input validation, the DAG of Sec. 2.2, wavefronts (Sec. 1),
// the superstep schedule (wavefronts or GrowLocal, Sec. 3), the Sec. 5
// reordering and the execution structure the device kernels walk.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.hpp"

namespace sptrsv {

namespace {
thread_local std::string g_last_error;
}

int fail(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}
void clear_error() { g_last_error.clear(); }
const char *last_error_cstr() { return g_last_error.c_str(); }

// Input rules (Sec. 2.2 assumes a non-singular lower-triangular factor):
// row pointers monotone from 0 to nnz, columns in [0, row], strictly
// increasing, the diagonal present, last and non-zero.
int validate_csr(const sptrsv_csr *A) {
    if (!A) return fail(SPTRSV_ERR_ARG, "csr is NULL");
    if (A->n < 0 || A->nnz < 0) return fail(SPTRSV_ERR_ARG, "negative size");
    if (A->n > 0 && (!A->rowptr || !A->col || !A->val))
        return fail(SPTRSV_ERR_ARG, "csr array is NULL");
    if (A->nnz > INT32_MAX) return fail(SPTRSV_ERR_ARG, "nnz exceeds int32 indexing");
    if (A->n == 0) return SPTRSV_OK;
    if (A->rowptr[0] != 0 || int64_t(A->rowptr[A->n]) != A->nnz)
        return fail(SPTRSV_ERR_ARG, "rowptr[0] must be 0 and rowptr[n] must equal nnz");
    for (int32_t i = 0; i < A->n; ++i) {
        const int32_t lo = A->rowptr[i], hi = A->rowptr[i + 1];
        if (hi < lo) return fail(SPTRSV_ERR_ARG, "rowptr decreases at row " + std::to_string(i));
        if (hi == lo) return fail(SPTRSV_ERR_ZERO_DIAG, "row " + std::to_string(i) + " is empty");
        for (int32_t q = lo; q < hi; ++q) {
            const int32_t c = A->col[q];
            if (c < 0 || c > i)
                return fail(SPTRSV_ERR_NOT_LOWER, "entry (" + std::to_string(i) + "," +
                                                      std::to_string(c) + ") outside the lower triangle");
            if (q > lo && c <= A->col[q - 1])
                return fail(SPTRSV_ERR_UNSORTED_OR_DUP,
                            "columns of row " + std::to_string(i) + " not strictly increasing");
        }
        if (A->col[hi - 1] != i)
            return fail(SPTRSV_ERR_ZERO_DIAG, "diagonal of row " + std::to_string(i) + " missing");
        if (A->val[hi - 1] == 0.0)
            return fail(SPTRSV_ERR_ZERO_DIAG, "zero diagonal in row " + std::to_string(i));
    }
    return SPTRSV_OK;
}

namespace {

// Wavefront of every row: 0 without parents, else 1 + deepest parent.  The
// natural order of a lower-triangular factor is topological.
int32_t compute_levels(const sptrsv_csr *A, std::vector<int32_t> &level) {
    level.assign(A->n, 0);
    int32_t deepest = -1;
    for (int32_t i = 0; i < A->n; ++i) {
        int32_t d = 0;
        const int32_t last = A->rowptr[i + 1] - 1;
        for (int32_t q = A->rowptr[i]; q < last; ++q) d = std::max(d, level[A->col[q]] + 1);
        level[i] = d;
        deepest = std::max(deepest, d);
    }
    return deepest + 1;
}

// Stable counting sort of `ids` by key[id] in [0, nkeys).
void stable_bucket(std::vector<int32_t> &ids, const std::vector<int32_t> &key, int32_t nkeys) {
    std::vector<int64_t> start(size_t(nkeys) + 1, 0);
    for (int32_t v : ids) start[size_t(key[v]) + 1]++;
    for (int32_t b = 0; b < nkeys; ++b) start[b + 1] += start[b];
    std::vector<int32_t> out(ids.size());
    for (int32_t v : ids) out[start[key[v]]++] = v;
    ids.swap(out);
}

// Shared-memory ring for the single-block walker: x[v] lives in slot
// v mod W from the phase that writes it until the last phase that reads it
// (its last child).  W is safe iff no two rows sharing a slot are live in the
// same phase; rows are visited in phase order, so comparing each row with the
// previous occupant of its slot suffices.
int32_t ring_window(const sptrsv_csr *A, const HostSchedule &h) {
    const int32_t n = h.n;
    if (n == 0) return 0;
    std::vector<int32_t> phase_of(n), last_use(n);
    const int32_t nph = int32_t(h.phase_row.size()) - 1;
    for (int32_t q = 0; q < nph; ++q)
        for (int32_t r = h.phase_row[q]; r < h.phase_row[q + 1]; ++r) phase_of[h.dev_perm[r]] = q;
    for (int32_t v = 0; v < n; ++v) last_use[v] = phase_of[v];
    for (int32_t v = 0; v < n; ++v)
        for (int32_t q = A->rowptr[v]; q < A->rowptr[v + 1] - 1; ++q) {
            const int32_t c = A->col[q];
            last_use[c] = std::max(last_use[c], phase_of[v]);
        }
    constexpr int32_t kMaxRingRows = 1 << 15;
    std::vector<int32_t> slot_last(kMaxRingRows);
    for (int32_t W = 32; W <= kMaxRingRows; W <<= 1) {
        std::fill(slot_last.begin(), slot_last.begin() + W, -1);
        bool ok = true;
        for (int32_t r = 0; r < n && ok; ++r) {
            const int32_t v = h.dev_perm[r];
            int32_t &prev = slot_last[v & (W - 1)];
            if (prev >= phase_of[v]) ok = false;
            prev = last_use[v];
        }
        if (ok) return W;
    }
    return 0;
}

// Upper-triangular input: columns strictly increasing, diagonal present, first
// and non-zero.  Mirrors validate_csr's rules for the other direction.
int validate_upper_csr(const sptrsv_csr *A) {
    if (!A || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!A->rowptr || !A->col || !A->val)))
        return fail(SPTRSV_ERR_ARG, "bad csr");
    if (A->nnz > INT32_MAX) return fail(SPTRSV_ERR_ARG, "nnz exceeds int32 indexing");
    if (A->n == 0) return SPTRSV_OK;
    const int32_t n = A->n;
    if (A->rowptr[0] != 0 || A->rowptr[n] != A->nnz) return fail(SPTRSV_ERR_ARG, "bad row pointers");
    for (int32_t i = 0; i < n; ++i) {
        const int32_t b = A->rowptr[i], e = A->rowptr[i + 1];
        if (e <= b || e > A->nnz) return fail(SPTRSV_ERR_ARG, "bad row pointers");
        if (A->col[b] != i) return fail(SPTRSV_ERR_ZERO_DIAG, "row " + std::to_string(i) + ": diagonal not first");
        if (A->val[b] == 0.0) return fail(SPTRSV_ERR_ZERO_DIAG, "row " + std::to_string(i) + ": zero diagonal");
        for (int32_t q = b + 1; q < e; ++q) {
            if (A->col[q] >= n) return fail(SPTRSV_ERR_ARG, "column out of range");
            if (A->col[q] <= A->col[q - 1])
                return fail(A->col[q] < i ? SPTRSV_ERR_NOT_LOWER : SPTRSV_ERR_UNSORTED_OR_DUP,
                            "row " + std::to_string(i) + ": entry below the diagonal, unsorted or duplicate");
        }
    }
    return SPTRSV_OK;
}

// L' with ids i' = n-1-i from an upper factor U: row i' lists U's row i
// backwards, so its columns n-1-j increase and the diagonal comes last.
void reverse_upper(const sptrsv_csr *U, std::vector<int32_t> &rp, std::vector<int32_t> &col,
                   std::vector<double> &val) {
    const int32_t n = U->n;
    rp.assign(size_t(n) + 1, 0);
    col.resize(size_t(U->nnz));
    val.resize(size_t(U->nnz));
    int64_t o = 0;
    for (int32_t ip = 0; ip < n; ++ip) {
        const int32_t i = n - 1 - ip;
        for (int32_t q = U->rowptr[i + 1] - 1; q >= U->rowptr[i]; --q, ++o) {
            col[size_t(o)] = n - 1 - U->col[q];
            val[size_t(o)] = U->val[q];
        }
        rp[size_t(ip) + 1] = int32_t(o);
    }
}

// L' with ids i' = n-1-i for L^T, from the rows of L: entry (k, j) of L is
// entry (j, k) of L^T, i.e. (n-1-j, n-1-k) of L'.  Rows of L taken from the last
// one append every L' row's columns in increasing order, the diagonal last.
void reverse_transpose(const sptrsv_csr *L, std::vector<int32_t> &rp, std::vector<int32_t> &col,
                       std::vector<double> &val) {
    const int32_t n = L->n;
    rp.assign(size_t(n) + 1, 0);
    for (int64_t q = 0; q < L->nnz; ++q) rp[size_t(n - 1 - L->col[q]) + 1]++;
    for (int32_t i = 0; i < n; ++i) rp[size_t(i) + 1] += rp[size_t(i)];
    std::vector<int32_t> fill(rp.begin(), rp.end() - 1);
    col.resize(size_t(L->nnz));
    val.resize(size_t(L->nnz));
    for (int32_t k = n - 1; k >= 0; --k)
        for (int32_t q = L->rowptr[k]; q < L->rowptr[k + 1]; ++q) {
            const int32_t r = n - 1 - L->col[q];
            col[size_t(fill[r])] = n - 1 - k;
            val[size_t(fill[r]++)] = L->val[q];
        }
}

}  // namespace

// Block-local partition (SPTRSV_SYNC_LOCAL; Sec. 3's locality applied to the
// thread blocks of a persistent grid).  Rows are taken in (wavefront, id)
// order.  A row goes to the block holding most of its parents of the two
// previous wavefronts (weight 4 for the previous wavefront, which holds its
// last-finishing parent, 1 for the one before), as long as that block has taken
// fewer than ceil(1.25 * width / nb) rows of the row's wavefront and has room;
// otherwise to the block with the fewest rows of this wavefront (then the
// fewest rows overall).  The cap keeps every wavefront spread over all blocks,
// the vote keeps dependency chains inside a block.  Rows join their block's
// list in (wavefront, id) order, which the executor's progress argument needs.
bool local_partition(int32_t n, int32_t nb, int32_t row_cap, const std::vector<int32_t> &level, int32_t nlevels,
                     const int32_t *rp, const int32_t *col, const int32_t *row_of, std::vector<int32_t> &blk,
                     std::vector<int32_t> &lidx, std::vector<int32_t> &load) {
    constexpr double kSlack = 1.25;
    if (nb < 1 || int64_t(row_cap) * nb < int64_t(n)) return false;
    std::vector<int32_t> lstart(size_t(nlevels) + 1, 0), ord(n);
    for (int32_t v = 0; v < n; ++v) lstart[level[v] + 1]++;
    for (int32_t l = 0; l < nlevels; ++l) lstart[l + 1] += lstart[l];
    {
        std::vector<int32_t> fill(lstart.begin(), lstart.end() - 1);
        for (int32_t v = 0; v < n; ++v) ord[fill[level[v]]++] = v;   // (wavefront, id) order
    }
    blk.assign(n, -1);
    lidx.assign(n, 0);
    load.assign(nb, 0);
    std::vector<int32_t> cnt(nb, 0);
    std::vector<std::pair<int32_t, int32_t>> tally;
    int32_t cur = -1, cap = 0;
    for (int32_t t = 0; t < n; ++t) {
        const int32_t v = ord[t], l = level[v];
        if (l != cur) {
            cur = l;
            std::fill(cnt.begin(), cnt.end(), 0);
            const double w = double(lstart[l + 1] - lstart[l]);
            cap = std::max<int32_t>(1, int32_t(std::ceil(w * kSlack / nb)));
        }
        tally.clear();
        const int32_t dr = row_of[v];
        for (int32_t q = rp[dr]; q < rp[dr + 1]; ++q) {
            const int32_t c = col[q], lc = level[c];
            if (lc < l - 2) continue;
            const int32_t w = lc == l - 1 ? 4 : 1, b = blk[c];
            bool found = false;
            for (auto &e : tally)
                if (e.first == b) {
                    e.second += w;
                    found = true;
                    break;
                }
            if (!found) tally.push_back({b, w});
        }
        int32_t best = -1, bestw = 0;
        for (const auto &e : tally)
            if (cnt[e.first] < cap && load[e.first] < row_cap &&
                (e.second > bestw || (e.second == bestw && cnt[e.first] < cnt[best]))) {
                best = e.first;
                bestw = e.second;
            }
        if (best < 0) {
            for (int32_t b = 0; b < nb; ++b)
                if (load[b] < row_cap &&
                    (best < 0 || cnt[b] < cnt[best] || (cnt[b] == cnt[best] && load[b] < load[best])))
                    best = b;
        }
        blk[v] = best;
        lidx[v] = load[best]++;
        cnt[best]++;
    }
    return true;
}


bool range_partition(int32_t n, int32_t nb, int32_t row_cap, const std::vector<int32_t> &level, int32_t nlevels,
                     std::vector<int32_t> &blk, std::vector<int32_t> &lidx, std::vector<int32_t> &load) {
    if (nb < 1 || int64_t(row_cap) * nb < int64_t(n)) return false;
    blk.assign(n, 0);
    lidx.assign(n, 0);
    load.assign(nb, 0);
    for (int32_t v = 0; v < n; ++v) {
        blk[v] = int32_t(int64_t(v) * nb / std::max<int32_t>(n, 1));
        if (++load[blk[v]] > row_cap) return false;
    }
    // positions in (wavefront, id) order inside every block
    std::vector<int32_t> lstart(size_t(nlevels) + 1, 0), ord(n);
    for (int32_t v = 0; v < n; ++v) lstart[level[v] + 1]++;
    for (int32_t l = 0; l < nlevels; ++l) lstart[l + 1] += lstart[l];
    for (int32_t v = 0; v < n; ++v) ord[lstart[level[v]]++] = v;
    std::vector<int32_t> fill(nb, 0);
    for (int32_t t = 0; t < n; ++t) {
        const int32_t v = ord[t];
        lidx[v] = fill[blk[v]]++;
    }
    return true;
}

bool grid_partition(int32_t n, int32_t nb, int32_t row_cap, const std::vector<int32_t> &level, int32_t nlevels,
                    const int32_t *rp, const int32_t *col, const int32_t *row_of, std::vector<int32_t> &blk,
                    std::vector<int32_t> &lidx, std::vector<int32_t> &load) {
    if (nb < 1 || n < 1 || int64_t(row_cap) * nb < int64_t(n)) return false;
    // offsets v - c of the off-diagonal entries, on every 16th row
    std::unordered_map<int64_t, int64_t> count;
    int64_t sampled = 0;
    for (int32_t v = 0; v < n; v += 16) {
        ++sampled;
        const int32_t dr = row_of[v];
        for (int32_t q = rp[dr]; q < rp[dr + 1]; ++q) count[int64_t(v) - col[q]]++;
    }
    std::vector<int64_t> dom;                        // offsets present in a quarter of the rows
    for (const auto &e : count)
        if (4 * e.second >= sampled) dom.push_back(e.first);
    std::sort(dom.begin(), dom.end());
    // nested strides 1 | s1 | s2: the largest three-term chain of dominant offsets
    int64_t s1 = 0, s2 = 0;
    if (dom.empty() || dom[0] != 1) return false;
    for (size_t a = 1; a < dom.size(); ++a)
        for (size_t b = a + 1; b < dom.size(); ++b)
            if (dom[b] % dom[a] == 0 && dom[b] / dom[a] >= 2 && dom[a] >= 2 && dom[b] > s2) {
                s1 = dom[a];
                s2 = dom[b];
            }
    if (s2 == 0) return false;
    const int64_t A = s2 / s1;                       // lines per plane
    const int64_t B = (int64_t(n) + s2 - 1) / s2;    // planes
    // tiles TA x TB <= nb, as many as possible, tile sides within a factor 3 of each other
    int64_t TA = 0, TB = 0;
    for (int64_t ta = 1; ta <= std::min<int64_t>(A, nb); ++ta) {
        const int64_t tb = std::min<int64_t>(B, nb / ta);
        const double side_a = double(A) / ta, side_b = double(B) / tb;
        if (side_a > 3 * side_b || side_b > 3 * side_a) continue;
        if (ta * tb > TA * TB || (ta * tb == TA * TB && std::abs(side_a - side_b) <
                                  std::abs(double(A) / TA - double(B) / TB)))
            TA = ta, TB = tb;
    }
    if (TA * TB < 2) return false;
    blk.assign(n, 0);
    load.assign(nb, 0);
    for (int32_t v = 0; v < n; ++v) {
        const int64_t a = (v / s1) % A, b = v / s2;
        const int64_t ta = a * TA / A, tb = b * TB / B;
        blk[v] = int32_t(tb * TA + ta);
        if (++load[blk[v]] > row_cap) return false;
    }
    std::vector<int32_t> lstart(size_t(nlevels) + 1, 0), ord(n);
    for (int32_t v = 0; v < n; ++v) lstart[level[v] + 1]++;
    for (int32_t l = 0; l < nlevels; ++l) lstart[l + 1] += lstart[l];
    for (int32_t v = 0; v < n; ++v) ord[lstart[level[v]]++] = v;
    lidx.assign(n, 0);
    std::vector<int32_t> fill(nb, 0);
    for (int32_t t = 0; t < n; ++t) lidx[ord[t]] = fill[blk[ord[t]]]++;
    return true;
}

// A saved schedule is accepted only if the executors can run it: supersteps
// 0..S-1 all used, cores in [0, k), every edge into a later superstep or inside
// one core's block (Def. 2.1); a wavefront schedule must be the wavefronts.
int check_given(const sptrsv_csr *A, const HostSchedule &h, const GivenSchedule &g) {
    const int32_t n = A->n;
    if (g.S < 0 || g.k < 1 || (n > 0 && g.S < 1) || !(g.sigma && g.pi) && n > 0)
        return fail(SPTRSV_ERR_ARG, "saved schedule: bad header");
    std::vector<char> used(size_t(std::max(g.S, 1)), 0);
    for (int32_t v = 0; v < n; ++v) {
        if (g.sigma[v] < 0 || g.sigma[v] >= g.S || g.pi[v] < 0 || g.pi[v] >= g.k)
            return fail(SPTRSV_ERR_ARG, "saved schedule: superstep or core out of range");
        used[size_t(g.sigma[v])] = 1;
    }
    for (int32_t s = 0; s < g.S; ++s)
        if (!used[size_t(s)]) return fail(SPTRSV_ERR_ARG, "saved schedule: supersteps not contiguous");
    if (g.mode == SPTRSV_SCHED_LEVELS) {
        if (g.S != h.nlevels) return fail(SPTRSV_ERR_ARG, "saved schedule: not the wavefronts");
        for (int32_t v = 0; v < n; ++v)
            if (g.sigma[v] != h.level[v] || g.pi[v] != 0)
                return fail(SPTRSV_ERR_ARG, "saved schedule: not the wavefronts");
        return SPTRSV_OK;
    }
    for (int32_t v = 0; v < n; ++v) {
        const int32_t last = A->rowptr[v + 1] - 1;
        for (int32_t q = A->rowptr[v]; q < last; ++q) {
            const int32_t u = A->col[q];
            if (g.sigma[u] > g.sigma[v] || (g.sigma[u] == g.sigma[v] && g.pi[u] != g.pi[v]))
                return fail(SPTRSV_ERR_ARG, "saved schedule: violates Def. 2.1 on edge " + std::to_string(u) +
                                                " -> " + std::to_string(v));
        }
    }
    return SPTRSV_OK;
}

bool partition_valid(int32_t n, int32_t nb, const int32_t *blk, const int32_t *lidx, const std::vector<int32_t> &level) {
    if (nb < 1 || (n > 0 && (!blk || !lidx))) return false;
    std::vector<int32_t> load(size_t(nb), 0);
    for (int32_t v = 0; v < n; ++v) {
        if (blk[v] < 0 || blk[v] >= nb || lidx[v] < 0) return false;
        load[size_t(blk[v])]++;
    }
    std::vector<int64_t> start(size_t(nb) + 1, 0);
    for (int32_t b = 0; b < nb; ++b) start[b + 1] = start[b] + load[b];
    std::vector<int32_t> at(size_t(n), -1);
    for (int32_t v = 0; v < n; ++v) {
        if (lidx[v] >= load[size_t(blk[v])]) return false;
        int32_t &slot = at[size_t(start[blk[v]] + lidx[v])];
        if (slot >= 0) return false;                        // two rows in one position
        slot = v;
    }
    for (int32_t b = 0; b < nb; ++b)                         // (wavefront, id) order in each list
        for (int64_t t = start[b] + 1; t < start[b + 1]; ++t) {
            const int32_t u = at[size_t(t - 1)], v = at[size_t(t)];
            if (level[u] > level[v] || (level[u] == level[v] && u > v)) return false;
        }
    return true;
}

int32_t ring_rows_of(const sptrsv_csr *A, const HostSchedule &h) { return ring_window(A, h); }

int32_t factor_levels(const sptrsv_csr *A, std::vector<int32_t> &level) {
    return A->n ? compute_levels(A, level) : (level.clear(), 0);
}

int lower_factor(const sptrsv_csr *csr, int32_t triangle, std::vector<int32_t> &rp, std::vector<int32_t> &col,
                 std::vector<double> &val, sptrsv_csr &lowered, const sptrsv_csr **use) {
    int st;
    if (triangle == SPTRSV_TRI_UPPER) {
        if ((st = validate_upper_csr(csr))) return st;
        reverse_upper(csr, rp, col, val);
    } else if (triangle == SPTRSV_TRI_LOWER_TRANSPOSED) {
        if ((st = validate_csr(csr))) return st;
        reverse_transpose(csr, rp, col, val);
    } else if (triangle != SPTRSV_TRI_LOWER) {
        return fail(SPTRSV_ERR_ARG, "unknown triangle");
    }
    *use = csr;
    if (triangle != SPTRSV_TRI_LOWER) {
        lowered.n = csr->n;
        lowered.nnz = csr->nnz;
        lowered.rowptr = rp.data();
        lowered.col = col.data();
        lowered.val = val.data();
        *use = &lowered;
    }
    return validate_csr(*use);
}

int build_schedule(const sptrsv_csr *A, const sptrsv_analyze_opts &o, HostSchedule &h, const GivenSchedule *given) {
    const int32_t n = A->n;
    h.n = n;
    h.nnz = A->nnz;
    h.mode = o.mode;
    const auto t0 = std::chrono::steady_clock::now();
    h.nlevels = n ? compute_levels(A, h.level) : 0;
    {
        std::vector<int32_t> width(size_t(h.nlevels), 0);
        for (int32_t v = 0; v < n; ++v) width[h.level[v]]++;
        h.max_level_rows = width.empty() ? 0 : *std::max_element(width.begin(), width.end());
    }
    h.sigma.assign(n, 0);
    h.pi.assign(n, 0);
    h.sched_blocks = 1;
    if (given) {
        const auto t1 = std::chrono::steady_clock::now();
        int st = check_given(A, h, *given);
        if (st) return st;
        h.mode = given->mode;
        h.k = given->mode == SPTRSV_SCHED_LEVELS ? 1 : given->k;
        h.S = given->S;
        h.sched_blocks = std::max(1, given->sched_blocks);
        h.coarse_vertices = given->coarse_vertices > 0 ? given->coarse_vertices : n;
        if (n) {
            std::memcpy(h.sigma.data(), given->sigma, size_t(n) * sizeof(int32_t));
            std::memcpy(h.pi.data(), given->pi, size_t(n) * sizeof(int32_t));
        }
        if (given->loc_nb > 0) {
            if (!partition_valid(n, given->loc_nb, given->loc_blk, given->loc_lidx, h.level))
                return fail(SPTRSV_ERR_ARG, "saved block-local partition is not valid for this factor");
            h.loc_nb = given->loc_nb;
            h.loc_blk.assign(given->loc_blk, given->loc_blk + n);
            h.loc_lidx.assign(given->loc_lidx, given->loc_lidx + n);
            h.loc_part = -1;
            ++h.loc_gen;
        }
        h.schedule_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    } else if (o.mode == SPTRSV_SCHED_LEVELS) {
        h.k = 1;
        h.sigma = h.level;
        h.S = h.nlevels;
        h.coarse_vertices = n;
        h.schedule_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    } else if (o.mode == SPTRSV_SCHED_GROWLOCAL) {
        h.k = o.k;
        h.sched_blocks = std::max(1, o.sched_blocks);
        const auto t1 = std::chrono::steady_clock::now();
        h.coarse_vertices = n;
        if (o.coarsen == SPTRSV_COARSEN_FUNNEL)
            h.S = funnel_growlocal(n, A->rowptr, A->col, o.k, o.alpha0, o.growth, o.L, o.accept,
                                   o.coarsen_max_weight > 0.0 ? o.coarsen_max_weight : 500.0, o.sched_threads,
                                   h.sigma.data(), h.pi.data(), &h.coarse_vertices, &h.coarse_part);
        else
            h.S = growlocal_blocks(n, A->rowptr, A->col, o.k, o.alpha0, o.growth, o.L, o.accept, h.sched_blocks,
                                   o.sched_threads, h.sigma.data(), h.pi.data());
        h.schedule_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    } else {
        return fail(SPTRSV_ERR_ARG, "unknown schedule mode");
    }

    // Sec. 5: order by superstep, then core, then original id (LSD: core, then superstep).
    h.perm.resize(n);
    for (int32_t v = 0; v < n; ++v) h.perm[v] = v;
    stable_bucket(h.perm, h.pi, h.k);
    stable_bucket(h.perm, h.sigma, std::max(h.S, 1));

    // Phases inside a (superstep, core) block: depth among same-block parents.
    // Rows are visited in original order, which is topological.
    std::vector<int32_t> sub(n, 0);
    int32_t max_sub = 0;
    if (h.mode != SPTRSV_SCHED_LEVELS) {
        for (int32_t v = 0; v < n; ++v) {
            int32_t d = 0;
            const int32_t last = A->rowptr[v + 1] - 1;
            for (int32_t q = A->rowptr[v]; q < last; ++q) {
                const int32_t u = A->col[q];
                if (h.sigma[u] == h.sigma[v] && h.pi[u] == h.pi[v]) d = std::max(d, sub[u] + 1);
            }
            sub[v] = d;
            max_sub = std::max(max_sub, d);
        }
    }
    // Device order: the Sec. 5 order refined by phase inside each block.
    h.dev_perm = h.perm;
    if (max_sub > 0) {
        size_t a = 0;
        std::vector<int32_t> tmp;
        while (a < size_t(n)) {
            size_t b = a;
            const int32_t s = h.sigma[h.dev_perm[a]], p = h.pi[h.dev_perm[a]];
            while (b < size_t(n) && h.sigma[h.dev_perm[b]] == s && h.pi[h.dev_perm[b]] == p) ++b;
            std::stable_sort(h.dev_perm.begin() + a, h.dev_perm.begin() + b,
                             [&](int32_t x, int32_t y) { return sub[x] < sub[y]; });
            a = b;
        }
    }
    // Walk the device order and cut supersteps, blocks and phases.
    h.step_blk.assign(1, 0);
    h.blk_phase.assign(1, 0);
    h.phase_row.assign(1, 0);
    h.max_phase_rows = 0;
    h.max_block_rows = 0;
    int32_t r = 0;
    while (r < n) {
        const int32_t s = h.sigma[h.dev_perm[r]];
        while (r < n && h.sigma[h.dev_perm[r]] == s) {            // blocks of superstep s
            const int32_t p = h.pi[h.dev_perm[r]];
            const int32_t blk_start = r;
            while (r < n && h.sigma[h.dev_perm[r]] == s && h.pi[h.dev_perm[r]] == p) {
                const int32_t d = sub[h.dev_perm[r]];
                const int32_t ph_start = r;
                while (r < n && h.sigma[h.dev_perm[r]] == s && h.pi[h.dev_perm[r]] == p &&
                       sub[h.dev_perm[r]] == d)
                    ++r;
                h.phase_row.push_back(r);
                h.max_phase_rows = std::max(h.max_phase_rows, r - ph_start);
            }
            h.blk_phase.push_back(int32_t(h.phase_row.size()) - 1);
            h.max_block_rows = std::max(h.max_block_rows, r - blk_start);
        }
        h.step_blk.push_back(int32_t(h.blk_phase.size()) - 1);
    }
    if (int32_t(h.step_blk.size()) - 1 != h.S)
        return fail(SPTRSV_ERR_ARG, "internal: superstep count mismatch");
    h.ring_rows = n <= (1 << 20) ? ring_window(A, h) : 0;
    return SPTRSV_OK;
}

}  // namespace sptrsv

using namespace sptrsv;

extern "C" {

const char *sptrsv_status_string(int status) {
    switch (status) {
        case SPTRSV_OK: return "SPTRSV_OK";
        case SPTRSV_ERR_ARG: return "SPTRSV_ERR_ARG";
        case SPTRSV_ERR_NOT_LOWER: return "SPTRSV_ERR_NOT_LOWER";
        case SPTRSV_ERR_UNSORTED_OR_DUP: return "SPTRSV_ERR_UNSORTED_OR_DUP";
        case SPTRSV_ERR_ZERO_DIAG: return "SPTRSV_ERR_ZERO_DIAG";
        case SPTRSV_ERR_OOM: return "SPTRSV_ERR_OOM";
        case SPTRSV_ERR_BUDGET: return "SPTRSV_ERR_BUDGET";
        case SPTRSV_ERR_CUDA: return "SPTRSV_ERR_CUDA";
        case SPTRSV_ERR_LAUNCH: return "SPTRSV_ERR_LAUNCH";
        case SPTRSV_ERR_TIMEOUT: return "SPTRSV_ERR_TIMEOUT";
        case SPTRSV_ERR_NOT_CONVERGED: return "SPTRSV_ERR_NOT_CONVERGED";
        case SPTRSV_ERR_PENDING: return "SPTRSV_ERR_PENDING";
        case SPTRSV_ERR_NO_DEVICE: return "SPTRSV_ERR_NO_DEVICE";
        case SPTRSV_ERR_IO: return "SPTRSV_ERR_IO";
        default: return "SPTRSV_ERR_UNKNOWN";
    }
}

const char *sptrsv_last_error(void) { return last_error_cstr(); }

int sptrsv_version(void) { return 10000; }

void sptrsv_analyze_opts_default(sptrsv_analyze_opts *o) {
    if (!o) return;
    o->mode = SPTRSV_SCHED_LEVELS;
    o->k = 0;
    o->alpha0 = 20.0;
    o->growth = 1.5;
    o->L = 500.0;
    o->accept = 0.97;
    o->values = SPTRSV_VALUES_F64 | SPTRSV_VALUES_F32;
    o->device = 0;
    o->triangle = SPTRSV_TRI_LOWER;
    o->sched_blocks = 0;
    o->sched_threads = 0;
    o->coarsen = SPTRSV_COARSEN_NONE;
    o->coarsen_max_weight = 0.0;
    o->analyze_on_device = 0;
}

int sptrsv_analyze(const sptrsv_csr *csr, const sptrsv_analyze_opts *opts, sptrsv_plan **out) {
    clear_error();
    if (!out) return fail(SPTRSV_ERR_ARG, "out is NULL");
    *out = nullptr;
    sptrsv_analyze_opts o;
    sptrsv_analyze_opts_default(&o);
    if (opts) o = *opts;
    return analyze_impl(csr, o, nullptr, out);
}

}  // extern "C"

int sptrsv::analyze_impl(const sptrsv_csr *csr, sptrsv_analyze_opts o, const GivenSchedule *given,
                         sptrsv_plan **out) {
    if (given) {
        o.mode = given->mode;
        o.k = given->k;
        o.sched_blocks = given->sched_blocks;
    }
    if (o.values == 0) o.values = SPTRSV_VALUES_F64 | SPTRSV_VALUES_F32;
    if (o.values & ~(SPTRSV_VALUES_F64 | SPTRSV_VALUES_F32)) return fail(SPTRSV_ERR_ARG, "bad values mask");
    if (o.device < -1) return fail(SPTRSV_ERR_ARG, "bad device");
    if (o.mode == SPTRSV_SCHED_GROWLOCAL) {
        if (!(o.alpha0 >= 1.0) || !(o.growth > 1.0) || !(o.L >= 0.0) || !(o.accept > 0.0))
            return fail(SPTRSV_ERR_ARG, "GrowLocal needs alpha0 >= 1, growth > 1, L >= 0, accept > 0");
    }
    if (o.sched_blocks < 0 || o.sched_threads < 0) return fail(SPTRSV_ERR_ARG, "negative sched_blocks/threads");
    if (o.sched_blocks > 1 && o.mode != SPTRSV_SCHED_GROWLOCAL)
        return fail(SPTRSV_ERR_ARG, "sched_blocks > 1 needs the GROWLOCAL schedule");
    if (o.coarsen != SPTRSV_COARSEN_NONE && o.coarsen != SPTRSV_COARSEN_FUNNEL)
        return fail(SPTRSV_ERR_ARG, "unknown coarsen value");
    if (o.coarsen == SPTRSV_COARSEN_FUNNEL && (o.mode != SPTRSV_SCHED_GROWLOCAL || o.sched_blocks > 1))
        return fail(SPTRSV_ERR_ARG, "Funnel coarsening needs the GROWLOCAL schedule on one block");
    if (o.analyze_on_device != 0 && o.analyze_on_device != 1) return fail(SPTRSV_ERR_ARG, "bad analyze_on_device");
    if (o.analyze_on_device && !given && (o.mode != SPTRSV_SCHED_LEVELS || o.device < 0))
        return fail(SPTRSV_ERR_ARG, "device analysis covers the wavefront schedule, on a device");
    const auto t0 = std::chrono::steady_clock::now();
    // UPPER and LOWER_TRANSPOSED: analyse the lower factor L' numbered backwards
    std::vector<int32_t> rrp, rcol;
    std::vector<double> rval;
    sptrsv_csr lowered;
    int st = lower_factor(csr, o.triangle, rrp, rcol, rval, lowered, &csr);
    if (st) return st;
    int32_t sms = 1;
    if (o.device >= 0) {
        st = device_sm_count(o.device, &sms);
        if (st) return st;
    }
    if (o.mode == SPTRSV_SCHED_GROWLOCAL && o.k <= 0) o.k = sms;
    if (o.mode == SPTRSV_SCHED_GROWLOCAL && o.k > (1 << 20)) return fail(SPTRSV_ERR_ARG, "k too large");

    sptrsv_plan *p = new (std::nothrow) sptrsv_plan();
    if (!p) return fail(SPTRSV_ERR_OOM, "host allocation failed");
    if (o.analyze_on_device && !given && csr->n > 0) {
        p->values = o.values;
        p->device = o.device;
        p->triangle = o.triangle;
        p->reversed = o.triangle != SPTRSV_TRI_LOWER;
        p->num_sms = sms;
        p->nnz_off = csr->nnz - csr->n;
        try {
            st = analyze_levels_device(p, csr, o.device, o.values, p->reversed);
        } catch (const std::bad_alloc &) {
            st = fail(SPTRSV_ERR_OOM, "host allocation failed during analysis");
        }
        if (st) {
            free_device(p);
            delete p;
            return st;
        }
        p->analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = p;
        return SPTRSV_OK;
    }
    try {
        st = build_schedule(csr, o, p->h, given);
    } catch (const std::bad_alloc &) {
        st = fail(SPTRSV_ERR_OOM, "host allocation failed during analysis");
    } catch (const std::exception &e) {           // e.g. a scheduling thread that could not start
        st = fail(SPTRSV_ERR_OOM, std::string("analysis failed: ") + e.what());
    }
    if (st) {
        delete p;
        return st;
    }
    p->values = o.values;
    p->device = o.device;
    p->reversed = o.triangle != SPTRSV_TRI_LOWER;
    p->triangle = o.triangle;
    for (int32_t i = 0; i < csr->n; ++i) {
        double rs = 0.0;
        for (int32_t q = csr->rowptr[i]; q < csr->rowptr[i + 1]; ++q) rs += std::abs(csr->val[q]);
        p->lnorm = std::max(p->lnorm, rs);
    }
    p->num_sms = sms;
    p->nnz_off = csr->nnz - csr->n;
    if (o.device >= 0) {
        st = upload_plan(p, csr);
        if (st) {
            free_device(p);
            delete p;
            return st;
        }
    }
    p->analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SPTRSV_OK;
}

extern "C" {

int sptrsv_plan_stats(const sptrsv_plan *p, sptrsv_stats *out) {
    if (!p || !out) return fail(SPTRSV_ERR_ARG, "NULL argument");
    out->n = p->h.n;
    out->nnz = p->h.nnz;
    out->levels = p->h.nlevels;
    out->supersteps = p->h.S;
    out->k = p->h.k;
    out->max_level_rows = p->h.max_level_rows;
    out->avg_wavefront = p->h.nlevels ? double(p->h.n) / p->h.nlevels : 0.0;
    out->device_bytes = p->device_bytes;
    out->analyze_ms = p->analyze_ms;
    out->phases = int32_t(p->h.phase_row.size()) - 1;
    out->ring_rows = p->h.ring_rows;
    out->schedule_ms = p->h.schedule_ms;
    out->sched_blocks = p->h.sched_blocks;
    out->coarse_vertices = p->h.coarse_vertices;
    return SPTRSV_OK;
}

int sptrsv_plan_export(const sptrsv_plan *p, int32_t *level, int32_t *sigma, int32_t *pi, int32_t *perm) {
    if (!p) return fail(SPTRSV_ERR_ARG, "plan is NULL");
    const int32_t n = p->h.n;
    const size_t bytes = size_t(n) * sizeof(int32_t);
    if (!p->reversed) {
        if (level && bytes) std::memcpy(level, p->h.level.data(), bytes);
        if (sigma && bytes) std::memcpy(sigma, p->h.sigma.data(), bytes);
        if (pi && bytes) std::memcpy(pi, p->h.pi.data(), bytes);
        if (perm && bytes) std::memcpy(perm, p->h.perm.data(), bytes);
        return SPTRSV_OK;
    }
    // reversed plans: row i of the caller's system is row n-1-i of L'
    for (int32_t i = 0; i < n; ++i) {
        if (level) level[i] = p->h.level[size_t(n - 1 - i)];
        if (sigma) sigma[i] = p->h.sigma[size_t(n - 1 - i)];
        if (pi) pi[i] = p->h.pi[size_t(n - 1 - i)];
        if (perm) perm[i] = n - 1 - p->h.perm[size_t(i)];
    }
    return SPTRSV_OK;
}

int sptrsv_plan_export_parts(const sptrsv_plan *p, int32_t *part) {
    if (!p || !part) return fail(SPTRSV_ERR_ARG, "NULL argument");
    const int32_t n = p->h.n;
    if (p->h.coarse_part.size() != size_t(n))
        return fail(SPTRSV_ERR_ARG, "the plan was not scheduled on a Funnel-coarsened DAG in this process");
    const int32_t m = p->h.coarse_vertices;
    for (int32_t i = 0; i < n; ++i) {
        // caller's numbering; for a reversed plan row i is row n-1-i of L', whose parts
        // are renumbered so that part ids still increase with their root's caller id
        part[i] = p->reversed ? m - 1 - p->h.coarse_part[size_t(n - 1 - i)] : p->h.coarse_part[size_t(i)];
    }
    return SPTRSV_OK;
}

int sptrsv_block_partition(const sptrsv_csr *A, int32_t kind, int32_t blocks, int32_t row_cap, int32_t *block_of_row,
                           int32_t *position) {
    clear_error();
    if (!A || blocks < 1 || row_cap < 0) return fail(SPTRSV_ERR_ARG, "bad arguments");
    if (kind != SPTRSV_PART_PARENTS && kind != SPTRSV_PART_RANGES && kind != SPTRSV_PART_GRID)
        return fail(SPTRSV_ERR_ARG, "kind must be SPTRSV_PART_PARENTS, RANGES or GRID");
    int st = validate_csr(A);
    if (st) return st;
    const int32_t n = A->n;
    if (n > 0 && (!block_of_row || !position)) return fail(SPTRSV_ERR_ARG, "output arrays are NULL");
    std::vector<int32_t> level;
    const int32_t nlevels = n ? compute_levels(A, level) : 0;
    // off-diagonal parents in original order (the diagonal is each row's last entry)
    std::vector<int32_t> rp(size_t(n) + 1, 0), col, row_of(n);
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1] - 1; ++q) col.push_back(A->col[q]);
        rp[i + 1] = int32_t(col.size());
        row_of[i] = i;
    }
    const int32_t cap = row_cap ? row_cap : std::max<int32_t>(n, 1);
    std::vector<int32_t> blk, lidx, load;
    bool ok = false;
    if (kind == SPTRSV_PART_RANGES) ok = range_partition(n, blocks, cap, level, nlevels, blk, lidx, load);
    if (kind == SPTRSV_PART_GRID)
        ok = grid_partition(n, blocks, cap, level, nlevels, rp.data(), col.data(), row_of.data(), blk, lidx, load);
    if (kind == SPTRSV_PART_PARENTS || (kind == SPTRSV_PART_GRID && !ok))
        ok = local_partition(n, blocks, cap, level, nlevels, rp.data(), col.data(), row_of.data(), blk, lidx, load);
    if (!ok) return fail(SPTRSV_ERR_ARG, "rows do not fit blocks * row_cap");
    if (n) {
        std::memcpy(block_of_row, blk.data(), size_t(n) * sizeof(int32_t));
        std::memcpy(position, lidx.data(), size_t(n) * sizeof(int32_t));
    }
    return SPTRSV_OK;
}

int sptrsv_local_partition(const sptrsv_csr *A, int32_t blocks, int32_t row_cap, int32_t *block_of_row,
                           int32_t *position) {
    return sptrsv_block_partition(A, SPTRSV_PART_PARENTS, blocks, row_cap, block_of_row, position);
}

void sptrsv_destroy(sptrsv_plan *p) {
    if (!p) return;
    free_device(p);
    delete p;
}

}  // extern "C"
