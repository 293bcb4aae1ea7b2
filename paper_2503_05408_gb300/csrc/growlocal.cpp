// GrowLocal superstep scheduler (Sec. 3, Algorithm 3.1) - library implementation.
//
// Data structures (chosen for O(|E| log |V|) work, Thm. 3.1):
//  * R, the vertices ready at the start of the superstep, is a sorted vector
//    read through a cursor: within an attempt vertices leave R only in
//    increasing id order (Rule I(ii)), so "the smallest remaining id" is the
//    element under the cursor and an attempt undoes by resetting the cursor.
//  * Attempt-local per-vertex state (parents still unassigned, the core of
//    this superstep's parents) is stamped with the attempt number and
//    re-initialised lazily on first touch, so undoing an attempt costs
//    nothing proportional to n.
//  * X_p (vertices only computable on core p) is a binary min-heap per core.
//
// Readings where the paper is silent (identical to the reference checker):
//  * core 0 receives up to floor(alpha) vertices, alpha a double multiplied by
//    `growth` after every attempt;
//  * cores 1..k-1, in order, add vertices while their weight is below core 0's
//    weight (the last vertex may overshoot), drawing from their own X_p first
//    and then from R;
//  * a vertex whose new parents lie on two or more cores waits for the next
//    superstep;
//  * beta (Eq. 3.1) is evaluated in double; attempt 0 is worthy, later ones iff
//    beta >= accept * best beta of the worthy attempts so far;
//  * the superstep keeps the last worthy attempt and ends at the first unworthy
//    one, or after a worthy attempt in which core 0 got fewer than floor(alpha)
//    vertices (a larger alpha would repeat that attempt exactly).
//
// Block-parallel scheduling (Sec. 3.1, Fig. 3.1): the rows are cut into
// diagonal blocks, GrowLocal runs on each block's sub-DAG on its own host
// thread, and the block schedules are concatenated.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <exception>
#include <functional>
#include <queue>
#include <system_error>
#include <thread>
#include <vector>

#include "plan.hpp"

namespace sptrsv {

namespace {

constexpr int32_t kNoCore = -1;
constexpr int32_t kManyCores = -2;

using MinHeap = std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>>;

struct Dag {
    int32_t n = 0;
    std::vector<int32_t> child_ptr, child;   // children of v: child[child_ptr[v] .. child_ptr[v+1])
    std::vector<int64_t> weight;             // omega(v) = stored entries of row v (Sec. 2.2)
    std::vector<int32_t> indeg;              // parents of v
};

// The sub-DAG of rows [r0, r1), numbered from 0.  Parents below r0 belong to
// earlier blocks, which finish before this block starts, so their edges are
// dropped; omega(v) stays the entry count of the full row (Sec. 3.1), unless
// `weight` gives the weights (a coarsened DAG, Sec. 4).
Dag make_dag(int32_t r0, int32_t r1, const int32_t *rowptr, const int32_t *col, const int64_t *weight) {
    Dag g;
    const int32_t n = r1 - r0;
    g.n = n;
    g.child_ptr.assign(size_t(n) + 1, 0);
    g.weight.resize(n);
    g.indeg.assign(n, 0);
    for (int32_t v = 0; v < n; ++v) {
        const int32_t lo = rowptr[r0 + v], hi = rowptr[r0 + v + 1];
        g.weight[v] = weight ? weight[r0 + v] : hi - lo;
        for (int32_t q = lo; q < hi - 1; ++q)     // every stored entry but the diagonal
            if (col[q] >= r0) {
                g.indeg[v]++;
                g.child_ptr[size_t(col[q] - r0) + 1]++;
            }
    }
    for (int32_t v = 0; v < n; ++v) g.child_ptr[v + 1] += g.child_ptr[v];
    g.child.resize(g.child_ptr[n]);
    std::vector<int32_t> pos(g.child_ptr.begin(), g.child_ptr.end() - 1);
    for (int32_t v = 0; v < n; ++v)               // ascending v -> children sorted by id
        for (int32_t q = rowptr[r0 + v]; q < rowptr[r0 + v + 1] - 1; ++q)
            if (col[q] >= r0) g.child[pos[col[q] - r0]++] = v;
    return g;
}

class Scheduler {
  public:
    Scheduler(const Dag &g, int32_t k) : g_(g), k_(k), excl_(size_t(k)), omega_(size_t(k)) {
        waiting_ = g.indeg;
        stamp_.assign(g.n, -1);
        left_.resize(g.n);
        owner_.resize(g.n);
        for (int32_t v = 0; v < g.n; ++v)
            if (waiting_[v] == 0) ready_.push_back(v);       // already ascending
    }

    // Try one attempt with core-0 budget `budget`; fills take_v_/take_p_.
    void attempt(int64_t budget) {
        ++attempt_id_;
        cursor_ = 0;
        take_v_.clear();
        take_p_.clear();
        for (int32_t p = 0; p < k_; ++p) {
            excl_[p] = MinHeap();
            omega_[p] = 0;
        }
        int32_t v;
        int64_t got = 0;
        while (got < budget && next(0, v)) {
            place(v, 0);
            ++got;
        }
        core0_ = got;
        for (int32_t p = 1; p < k_; ++p)
            while (omega_[p] < omega_[0] && next(p, v)) place(v, p);
    }

    double beta(double L) const {
        int64_t total = 0, heaviest = 0;
        for (int64_t w : omega_) {
            total += w;
            heaviest = std::max(heaviest, w);
        }
        return double(total) / (double(heaviest) + L);       // Eq. 3.1
    }

    int64_t core0() const { return core0_; }
    const std::vector<int32_t> &taken_v() const { return take_v_; }
    const std::vector<int32_t> &taken_p() const { return take_p_; }

    // Finalise a kept attempt as superstep `s`.
    void commit(const std::vector<int32_t> &kv, const std::vector<int32_t> &kp, int32_t s,
                int32_t *sigma, int32_t *pi, std::vector<char> &done) {
        for (size_t t = 0; t < kv.size(); ++t) {
            sigma[kv[t]] = s;
            pi[kv[t]] = kp[t];
            done[kv[t]] = 1;
        }
        std::vector<int32_t> released;
        for (int32_t v : kv)
            for (int32_t q = g_.child_ptr[v]; q < g_.child_ptr[v + 1]; ++q) {
                int32_t u = g_.child[q];
                if (--waiting_[u] == 0 && !done[u]) released.push_back(u);
            }
        std::vector<int32_t> keep;
        keep.reserve(ready_.size() + released.size());
        for (int32_t v : ready_)
            if (!done[v]) keep.push_back(v);
        std::sort(released.begin(), released.end());
        std::vector<int32_t> merged(keep.size() + released.size());
        std::merge(keep.begin(), keep.end(), released.begin(), released.end(), merged.begin());
        ready_.swap(merged);
    }

  private:
    void touch(int32_t u) {
        if (stamp_[u] != attempt_id_) {
            stamp_[u] = attempt_id_;
            left_[u] = waiting_[u];
            owner_[u] = kNoCore;
        }
    }

    // Rule I: core-exclusive vertices first, then the smallest id of R.
    bool next(int32_t p, int32_t &v) {
        if (!excl_[p].empty()) {
            v = excl_[p].top();
            excl_[p].pop();
            return true;
        }
        if (cursor_ < ready_.size()) {
            v = ready_[cursor_++];
            return true;
        }
        return false;
    }

    void place(int32_t v, int32_t p) {
        take_v_.push_back(v);
        take_p_.push_back(p);
        omega_[p] += g_.weight[v];
        for (int32_t q = g_.child_ptr[v]; q < g_.child_ptr[v + 1]; ++q) {
            int32_t u = g_.child[q];
            touch(u);
            if (owner_[u] == kNoCore) owner_[u] = p;
            else if (owner_[u] != p) owner_[u] = kManyCores;
            if (--left_[u] == 0 && owner_[u] == p) excl_[p].push(u);
        }
    }

    const Dag &g_;
    int32_t k_;
    std::vector<int32_t> waiting_;    // parents not in a finished superstep
    std::vector<int32_t> ready_;      // R, ascending
    size_t cursor_ = 0;
    int32_t attempt_id_ = -1;
    std::vector<int32_t> stamp_, left_, owner_;
    std::vector<MinHeap> excl_;
    std::vector<int64_t> omega_;
    std::vector<int32_t> take_v_, take_p_;
    int64_t core0_ = 0;
};

}  // namespace

namespace {

// GrowLocal on rows [r0, r1); sigma and pi are indexed by the block-local id.
int32_t growlocal_range(int32_t r0, int32_t r1, const int32_t *rowptr, const int32_t *col, const int64_t *weight,
                        int32_t k, double alpha0, double growth, double L, double accept, int32_t *sigma,
                        int32_t *pi) {
    const int32_t n = r1 - r0;
    if (n <= 0) return 0;
    Dag g = make_dag(r0, r1, rowptr, col, weight);
    Scheduler sch(g, k);
    std::vector<char> done(n, 0);
    std::vector<int32_t> keep_v, keep_p;
    int64_t placed = 0;
    int32_t s = 0;
    while (placed < n) {
        double alpha = alpha0;
        double best = 0.0;
        for (int a = 0;; ++a) {
            const int64_t budget = int64_t(std::floor(alpha));
            sch.attempt(budget);
            const double b = sch.beta(L);
            if (a > 0 && !(b >= accept * best)) break;        // unworthy: keep the last one
            best = std::max(best, b);
            keep_v = sch.taken_v();
            keep_p = sch.taken_p();
            if (sch.core0() < budget) break;                  // nothing left for a larger alpha
            alpha *= growth;
        }
        sch.commit(keep_v, keep_p, s, sigma, pi, done);
        placed += int64_t(keep_v.size());
        ++s;
    }
    return s;
}

}  // namespace

int32_t growlocal_schedule(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k,
                           double alpha0, double growth, double L, double accept,
                           int32_t *sigma, int32_t *pi) {
    return growlocal_range(0, n, rowptr, col, nullptr, k, alpha0, growth, L, accept, sigma, pi);
}

int32_t growlocal_weighted(int32_t n, const int32_t *rowptr, const int32_t *col, const int64_t *weight, int32_t k,
                           double alpha0, double growth, double L, double accept, int32_t *sigma, int32_t *pi) {
    return growlocal_range(0, n, rowptr, col, weight, k, alpha0, growth, L, accept, sigma, pi);
}

int32_t growlocal_blocks(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k,
                         double alpha0, double growth, double L, double accept,
                         int32_t blocks, int32_t threads, int32_t *sigma, int32_t *pi) {
    if (blocks <= 1) return growlocal_schedule(n, rowptr, col, k, alpha0, growth, L, accept, sigma, pi);
    auto bound = [&](int32_t b) { return int32_t(int64_t(b) * n / blocks); };
    std::vector<int32_t> S(size_t(blocks), 0);
    int32_t T = threads > 0 ? threads : int32_t(std::thread::hardware_concurrency());
    T = std::max(1, std::min(T, blocks));
    std::vector<std::exception_ptr> err(static_cast<size_t>(T));
    auto work = [&](int32_t t) {
        try {
            for (int32_t b = t; b < blocks; b += T) {
                const int32_t r0 = bound(b), r1 = bound(b + 1);
                S[b] = growlocal_range(r0, r1, rowptr, col, nullptr, k, alpha0, growth, L, accept, sigma + r0,
                                       pi + r0);
            }
        } catch (...) {
            err[t] = std::current_exception();
        }
    };
    std::vector<std::thread> pool;
    pool.reserve(size_t(T) - 1);
    int32_t started = 1;
    try {
        for (; started < T; ++started) pool.emplace_back(work, started);
    } catch (const std::system_error &) {
        // no more threads: this thread also takes the shares that found none
    }
    work(0);
    for (int32_t t = started; t < T; ++t) work(t);
    for (auto &th : pool) th.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
    // concatenate: block b's supersteps follow those of blocks 0..b-1
    int32_t offset = 0;
    for (int32_t b = 0; b < blocks; ++b) {
        for (int32_t v = bound(b); v < bound(b + 1); ++v) sigma[v] += offset;
        offset += S[b];
    }
    return offset;
}

}  // namespace sptrsv
