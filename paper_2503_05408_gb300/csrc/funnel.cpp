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
// Work O(sum deg^2) for step 1, O(|V| + |E|) for step 2 (Sec. 4.2).
#include <algorithm>
#include <cstdint>
#include <queue>
#include <utility>
#include <vector>

#include "plan.hpp"

namespace sptrsv {

int32_t funnel_growlocal(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k, double alpha0,
                         double growth, double L, double accept, double max_weight, int32_t *sigma, int32_t *pi,
                         int32_t *parts, std::vector<int32_t> *part_of) {
    *parts = 0;
    if (n == 0) return 0;
    // 1. triangle reduction: kept parents in CSR (kp, kc), ascending per row
    std::vector<int32_t> kp(size_t(n) + 1, 0), kc;
    kc.reserve(size_t(rowptr[n] - n));
    {
        std::vector<int32_t> is_parent(n, -1), is_long(n, -1);
        for (int32_t w = 0; w < n; ++w) {
            const int32_t lo = rowptr[w], last = rowptr[w + 1] - 1;
            for (int32_t q = lo; q < last; ++q) is_parent[col[q]] = w;
            for (int32_t q = lo; q < last; ++q) {
                const int32_t v = col[q];
                for (int32_t t = rowptr[v]; t < rowptr[v + 1] - 1; ++t)
                    if (is_parent[col[t]] == w) is_long[col[t]] = w;     // col[t] -> v -> w
            }
            for (int32_t q = lo; q < last; ++q)
                if (is_long[col[q]] != w) kc.push_back(col[q]);
            kp[w + 1] = int32_t(kc.size());
        }
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
    // 3. coarsened DAG in CSR (parents ascending, diagonal last) and its weights
    std::vector<std::pair<int32_t, int32_t>> e;                         // (child part, parent part)
    for (int32_t w = 0; w < n; ++w)
        for (int32_t q = kp[w]; q < kp[w + 1]; ++q)
            if (part[kc[q]] != part[w]) e.push_back({part[w], part[kc[q]]});
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    std::vector<int32_t> crp(size_t(m) + 1, 0), ccol;
    ccol.reserve(e.size() + size_t(m));
    size_t t = 0;
    for (int32_t i = 0; i < m; ++i) {
        for (; t < e.size() && e[t].first == i; ++t) ccol.push_back(e[t].second);
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
