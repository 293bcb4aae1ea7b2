// Funnel coarsening before GrowLocal (Sec. 4).
//
//  1. Approximate transitive reduction: every edge (u, w) that is the long side
//     of a triangle u -> v -> w is dropped, all decided on the factor's own
//     edges ("remove all long edges in triangles", cited in Sec. 4.2).  The
//     reduction keeps reachability, so the coarsening below stays acyclic for
//     the full DAG too.
//  2. In-funnel coarsening (Algorithm 4.1): vertices in reverse topological
//     order (n-1 .. 0); an unvisited vertex roots a part that grows, largest id
//     first, through parents whose children (in the reduced DAG) all joined the
//     part; a vertex joins only while the part's weight stays <= max_weight
//     (the size constraint Sec. 4.2 adds; the root always joins).  Every part is
//     an in-funnel, hence a cascade, so the coarsened DAG is acyclic (the
//     cascade proposition of Sec. 4.1).
//  3. GrowLocal on the coarsened DAG: parts numbered by root id (a topological
//     order: only a part's root has edges leaving the part), a part weighing its
//     rows' entries, one edge per pair of parts joined by a kept edge.  Every
//     row takes its part's superstep and core.
// Work O(sum deg^2) for step 1 (rows split over host threads), O(|V| + |E|) for
// step 2 (Sec. 4.2).
#include <algorithm>
#include <cstdint>
#include <exception>
#include <queue>
#include <system_error>
#include <thread>
#include <vector>

#include "plan.hpp"

namespace sptrsv {

namespace {

// Kept parents of rows [r0, r1): every parent u of w except those with u -> v -> w
// for another parent v.  mark[] (n entries, this thread's) holds w for a parent
// of w and -(w + 2) once that parent is found to be the long side of a triangle.
void reduce_rows(int32_t r0, int32_t r1, const int32_t *rowptr, const int32_t *col, std::vector<int32_t> &mark,
                 std::vector<int32_t> &kept, int32_t *kept_count) {
    for (int32_t w = r0; w < r1; ++w) {
        const int32_t lo = rowptr[w], last = rowptr[w + 1] - 1;
        for (int32_t q = lo; q < last; ++q) mark[col[q]] = w;
        for (int32_t q = lo; q < last; ++q) {
            const int32_t v = col[q];
            for (int32_t t = rowptr[v]; t < rowptr[v + 1] - 1; ++t)
                if (mark[col[t]] == w) mark[col[t]] = -(w + 2);             // col[t] -> v -> w
        }
        int32_t c = 0;
        for (int32_t q = lo; q < last; ++q)
            if (mark[col[q]] == w) {
                kept.push_back(col[q]);
                ++c;
            }
        kept_count[w] = c;
    }
}

}  // namespace

int32_t funnel_growlocal(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k, double alpha0,
                         double growth, double L, double accept, double max_weight, int32_t threads, int32_t *sigma,
                         int32_t *pi, int32_t *parts, std::vector<int32_t> *part_of) {
    *parts = 0;
    if (n == 0) return 0;
    // 1. triangle reduction, rows split over host threads: kept parents in CSR (kp, kc)
    std::vector<int32_t> kp(size_t(n) + 1, 0), kc;
    {
        // a thread keeps one n-entry mark array: at most 1 GiB of them in all
        int32_t T = threads > 0 ? threads : int32_t(std::thread::hardware_concurrency());
        T = std::max(1, std::min({T, std::max(1, n / 16384), int32_t(std::max<int64_t>(1, (int64_t(1) << 28) / n))}));
        std::vector<std::vector<int32_t>> chunk(static_cast<size_t>(T));
        std::vector<std::exception_ptr> err(static_cast<size_t>(T));
        auto work = [&](int32_t t) {
            try {
                std::vector<int32_t> mark(static_cast<size_t>(n), -1);
                reduce_rows(int32_t(int64_t(t) * n / T), int32_t(int64_t(t + 1) * n / T), rowptr, col, mark,
                            chunk[t], kp.data() + 1);
            } catch (...) {
                err[t] = std::current_exception();
            }
        };
        std::vector<std::thread> pool;
        int32_t started = 1;
        try {
            for (; started < T; ++started) pool.emplace_back(work, started);
        } catch (const std::system_error &) {
        }
        work(0);
        for (int32_t t = started; t < T; ++t) work(t);
        for (auto &th : pool) th.join();
        for (auto &e : err)
            if (e) std::rethrow_exception(e);
        for (int32_t w = 0; w < n; ++w) kp[w + 1] += kp[w];
        kc.reserve(size_t(kp[n]));
        for (auto &c : chunk) kc.insert(kc.end(), c.begin(), c.end());
    }
    // 2. in-funnel parts
    std::vector<int32_t> outdeg(n, 0), count(n, 0), part(n, -1), roots, touched;
    for (int32_t c : kc) outdeg[c]++;
    std::vector<int64_t> weight(n);
    for (int32_t v = 0; v < n; ++v) weight[v] = rowptr[v + 1] - rowptr[v];
    std::priority_queue<int32_t> heap;                                  // largest id first
    for (int32_t v = n - 1; v >= 0; --v) {
        if (part[v] >= 0) continue;
        const int32_t id = int32_t(roots.size());                       // renumbered below
        roots.push_back(v);
        int64_t total = 0;
        bool empty = true;
        heap.push(v);
        while (!heap.empty()) {
            const int32_t w = heap.top();
            heap.pop();
            if (!empty && double(total + weight[w]) > max_weight) continue;   // starts its own part later
            empty = false;
            total += weight[w];
            part[w] = id;
            for (int32_t q = kp[w]; q < kp[w + 1]; ++q) {
                const int32_t u = kc[q];
                if (count[u]++ == 0) touched.push_back(u);
                if (count[u] == outdeg[u]) heap.push(u);
            }
        }
        for (int32_t u : touched) count[u] = 0;
        touched.clear();
    }
    // roots were found in decreasing id order: part index by increasing root
    const int32_t m = int32_t(roots.size());
    for (int32_t v = 0; v < n; ++v) part[v] = m - 1 - part[v];
    // 3. coarsened DAG in CSR (parents ascending and unique, diagonal last) and its
    //    weights: the kept edges between parts, bucketed by the child's part
    std::vector<int64_t> cstart(size_t(m) + 1, 0);
    for (int32_t w = 0; w < n; ++w)
        for (int32_t q = kp[w]; q < kp[w + 1]; ++q)
            if (part[kc[q]] != part[w]) cstart[size_t(part[w]) + 1]++;
    for (int32_t i = 0; i < m; ++i) cstart[i + 1] += cstart[i];
    std::vector<int32_t> cpar(static_cast<size_t>(cstart[m]));
    {
        std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
        for (int32_t w = 0; w < n; ++w)
            for (int32_t q = kp[w]; q < kp[w + 1]; ++q)
                if (part[kc[q]] != part[w]) cpar[size_t(fill[part[w]]++)] = part[kc[q]];
    }
    std::vector<int32_t> crp(size_t(m) + 1, 0), ccol;
    ccol.reserve(cpar.size() + size_t(m));
    for (int32_t i = 0; i < m; ++i) {
        auto b = cpar.begin() + cstart[i], e = cpar.begin() + cstart[i + 1];
        std::sort(b, e);
        ccol.insert(ccol.end(), b, std::unique(b, e));
        ccol.push_back(i);
        crp[i + 1] = int32_t(ccol.size());
    }
    std::vector<int64_t> cw(m, 0);
    for (int32_t v = 0; v < n; ++v) cw[part[v]] += weight[v];
    std::vector<int32_t> cs(m), cpi(m);
    const int32_t S = growlocal_weighted(m, crp.data(), ccol.data(), cw.data(), k, alpha0, growth, L, accept,
                                         cs.data(), cpi.data());
    for (int32_t v = 0; v < n; ++v) {
        sigma[v] = cs[part[v]];
        pi[v] = cpi[part[v]];
    }
    *parts = m;
    if (part_of) part_of->swap(part);
    return S;
}

}  // namespace sptrsv
