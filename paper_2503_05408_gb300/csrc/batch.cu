// Batched persistent solve: many independent factors and right-hand-side
// blocks in one launch, replayed from a CUDA graph.
//
// Work items are (factor, block of right-hand-side columns).  Thread blocks of
// one persistent grid pull items from an atomic queue, longest critical path
// first, and each walks its item's phases alone (factors are independent, so
// there is no cross-block synchronisation at all).  In refinement mode a block
// runs the item's whole loop - FP32 sweep, FP64 residual, convergence test,
// correction sweep - before taking the next item.  Per factor the launch shape
// (lanes per row or right-hand-side tile, shared-memory ring) comes from a
// small autotuner that times the candidates once per factor class.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "kernels.cuh"
#include "plan.hpp"

namespace sptrsv {
namespace {

#define BCUDA_TRY(expr)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            (void)cudaGetLastError();                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA, \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));             \
        }                                                                                \
    } while (0)

template <typename T>
__device__ __forceinline__ SolveArgs<T> item_args(const BatchItem &it, const T *val, const T *dinv) {
    SolveArgs<T> a;
    a.n = it.n;
    a.S = 0;
    a.nrhs = it.nrhs;
    a.rp = it.rp;
    a.col = it.col;
    a.val = val;
    a.dinv = dinv;
    a.perm = it.perm;
    a.step_blk = nullptr;
    a.blk_phase = nullptr;
    a.phase_row = it.phase_row;
    a.blk_row = nullptr;
    a.b = nullptr;
    a.x = nullptr;
    a.ldb = a.ldx = 0;
    a.brs = a.xrs = 1;
    a.ctl = nullptr;
    a.flags = nullptr;
    a.epoch = 0;
    a.timeout_ns = 0;
    a.refine = 0;
    a.sweep = 0;
    a.x64 = nullptr;
    a.ldx64 = 0;
    a.x64rs = 1;
    a.rtol = 0.0;
    a.lnorm = it.lnorm;
    return a;
}

// One out-of-line function per variant: each gets its own register allocation
// instead of fourteen inlined walkers competing inside the persistent kernel.
template <typename T, int L, int U, bool RING, bool RP>
__device__ __noinline__ void walk_call(const SolveArgs<T> &a, int nphases, int win, T *xs, double &dm, double &xm) {
    walk_block<T, L, U, RING, RP>(a, nphases, win, xs, dm, xm);
}

template <typename T, int L, bool RING, bool RP>
__device__ __noinline__ bool staged_call(const SolveArgs<T> &a, const StageInfo &si, int nphases, int win,
                                         unsigned char *smem, double &dm, double &xm) {
    return walk_block_staged<T, L, RING, RP>(a, si, nphases, win, smem, dm, xm);
}

// Returns false if a bounded wait of the staged walk failed.
template <typename T>
__device__ __forceinline__ bool walk_variant(const SolveArgs<T> &a, const BatchItem &it, unsigned char *smem,
                                             double &dm, double &xm) {
    const bool ring = it.win > 0;
    if (it.staged) {
        StageInfo si = it.si;
        si.bdev = it.bdev;
#define SPTRSV_STAGED(L, RP)                                                                   \
    return ring ? staged_call<T, L, true, RP>(a, si, it.nphases, it.win, smem, dm, xm)         \
                : staged_call<T, L, false, RP>(a, si, it.nphases, 0, smem, dm, xm);
        switch (it.variant) {
            case V_L1: SPTRSV_STAGED(1, false)
            case V_L2: SPTRSV_STAGED(2, false)
            case V_L4: SPTRSV_STAGED(4, false)
            case V_T4: SPTRSV_STAGED(4, true)
            case V_T8: SPTRSV_STAGED(8, true)
            case V_T16: SPTRSV_STAGED(16, true)
            default: SPTRSV_STAGED(32, true)
        }
#undef SPTRSV_STAGED
    }
    T *xs = reinterpret_cast<T *>(smem);
#define SPTRSV_WALK(L, U, RP)                                                              \
    {                                                                                      \
        if (ring) walk_call<T, L, U, true, RP>(a, it.nphases, it.win, xs, dm, xm);         \
        else walk_call<T, L, U, false, RP>(a, it.nphases, 0, xs, dm, xm);                 \
        return true;                                                                       \
    }
    switch (it.variant) {
        case V_L1: SPTRSV_WALK(1, 4, false)
        case V_L2: SPTRSV_WALK(2, 4, false)
        case V_L4: SPTRSV_WALK(4, 2, false)
        case V_T4: SPTRSV_WALK(4, 4, true)
        case V_T8: SPTRSV_WALK(8, 4, true)
        case V_T16: SPTRSV_WALK(16, 4, true)
        default: SPTRSV_WALK(32, 4, true)
    }
#undef SPTRSV_WALK
}

// FP64 residual of one item, stored as FP32; returns max |r| (and max |b| through
// bm) over the block.  With the plan's FP64 scaled values v'_ij = A_ij / A_ii:
// r_i = b_i - A_ii (x_i + sum_j v'_ij x_j), one FP64 FMA per entry and right-hand
// side; from the FP32 split alone: r = b - (hi + lo) x, two.
__device__ double item_residual(const BatchItem &it, bool zero_x, double &bm, double *s_scratch) {
    const double *b = static_cast<const double *>(it.b);
    const double *x = static_cast<const double *>(it.x);
    double rm = 0.0, bmax = 0.0;
    // Four rows per thread and round, their row data and (rows of at most four entries)
    // columns and values read up front, so each right-hand side's gathers of x for the
    // four rows are in flight together: one block walks the whole factor here, and a
    // row at a time it waits a memory round trip per row.
    constexpr int RU = 4, EU = 4;
    const int nt = blockDim.x;
    for (int r0 = threadIdx.x; r0 < it.n; r0 += nt * RU) {
        int o[RU], beg[RU], len[RU];
        double dh[RU], dl[RU];
        int cc[RU][EU];
        double vv[RU][EU];
#pragma unroll
        for (int k = 0; k < RU; ++k) {
            const int r = r0 + k * nt;
            const bool has = r < it.n;
            o[k] = has ? __ldg(it.perm + r) : -1;
            beg[k] = has ? __ldg(it.rp + r) : 0;
            len[k] = has ? __ldg(it.rp + r + 1) - beg[k] : 0;
            dh[k] = has ? double(__ldg(it.dhi + r)) : 0.0;
            dl[k] = has ? double(__ldg(it.dlo + r)) : 0.0;
        }
        const bool fast = it.val != nullptr;
#pragma unroll
        for (int k = 0; k < RU; ++k)
#pragma unroll
            for (int u = 0; u < EU; ++u) {
                const bool e = fast && u < len[k] && len[k] <= EU;
                cc[k][u] = e ? __ldg(it.col + beg[k] + u) : 0;
                vv[k][u] = e ? __ldg(it.val + beg[k] + u) : 0.0;
            }
        for (int j = 0; j < it.nrhs; ++j) {
            const double *xj = x + (int64_t)j * it.ldx;
            double s[RU], sum[RU];
#pragma unroll
            for (int k = 0; k < RU; ++k) {
                s[k] = o[k] >= 0 ? b[o[k] + (int64_t)j * it.ldb] : 0.0;
                sum[k] = (!zero_x && fast && o[k] >= 0) ? xj[o[k]] : 0.0;
            }
            if (!zero_x) {
#pragma unroll
                for (int k = 0; k < RU; ++k) {
                    if (o[k] < 0) continue;
                    if (fast && len[k] <= EU) {
                        double xv[EU];
#pragma unroll
                        for (int u = 0; u < EU; ++u) xv[u] = u < len[k] ? xj[cc[k][u]] : 0.0;
#pragma unroll
                        for (int u = 0; u < EU; ++u)
                            if (u < len[k]) sum[k] = fma(vv[k][u], xv[u], sum[k]);
                        s[k] = fma(-(dh[k] + dl[k]), sum[k], s[k]);
                    } else if (fast) {
                        for (int q = beg[k]; q < beg[k] + len[k]; ++q)
                            sum[k] = fma(__ldg(it.val + q), xj[__ldg(it.col + q)], sum[k]);
                        s[k] = fma(-(dh[k] + dl[k]), sum[k], s[k]);
                    } else {                   // FP32 values only: the hi + lo split
                        for (int q = beg[k]; q < beg[k] + len[k]; ++q) {
                            const double xv = xj[__ldg(it.col + q)];
                            s[k] = fma(-double(__ldg(it.hi + q)), xv, s[k]);
                            s[k] = fma(-double(__ldg(it.lo + q)), xv, s[k]);
                        }
                        const double xo = xj[o[k]];
                        s[k] = fma(-dh[k], xo, s[k]);
                        s[k] = fma(-dl[k], xo, s[k]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < RU; ++k) {
                if (o[k] < 0) continue;
                bmax = max_abs_bits(bmax, b[o[k] + (int64_t)j * it.ldb]);
                it.r32[o[k] + (int64_t)j * it.n] = float(s[k]);
                rm = max_abs_bits(rm, s[k]);
            }
        }
    }
    bm = block_max(bmax, s_scratch);
    return block_max(rm, s_scratch);
}

__global__ void __launch_bounds__(512, 1) k_batch(const BatchItem *__restrict__ items, int count,
                                               ItemResult *res, unsigned int *cursor, BatchCfg cfg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ double s_scratch[32];
    while (true) {
        if (threadIdx.x == 0) s_item = int(atomicAdd(cursor, 1u));
        __syncthreads();
        const int i = s_item;
        __syncthreads();
        if (i >= count) break;
        const BatchItem it = items[i];
        ItemResult out = {0, 1, 0.0, 0.0};
        if (!cfg.refine) {
            SolveArgs<double> a = item_args<double>(it, it.val, it.dinv);
            a.b = static_cast<const double *>(it.b);
            a.x = static_cast<double *>(it.x);
            a.ldb = it.ldb;
            a.ldx = it.ldx;
            double dm = 0.0, xm = 0.0;
            if (!walk_variant<double>(a, it, smem_raw, dm, xm)) out.status = SPTRSV_ERR_TIMEOUT;
        } else {
            // FP32 sweeps with FP64 residual refinement, entirely inside this block
            SolveArgs<float> a = item_args<float>(it, it.s32, it.dinv32);
            a.b = it.r32;
            a.ldb = it.n;
            a.x = it.d32;
            a.ldx = it.n;
            a.x64 = static_cast<double *>(it.x);
            a.ldx64 = it.ldx;
            double bm = 0.0;
            item_residual(it, true, bm, s_scratch);              // r_0 = b
            __syncthreads();
            double dmax = 0.0, xmax = 0.0, berr = 0.0;
            int sweeps = 0;
            bool conv = false;
            for (int t = 0;; ++t) {
                a.refine = t == 0 ? 1 : 2;
                double dm = 0.0, xm = 0.0;
                if (!walk_variant<float>(a, it, smem_raw, dm, xm)) {
                    out.status = SPTRSV_ERR_TIMEOUT;
                    break;
                }
                ++sweeps;
                __syncthreads();
                dmax = block_max(dm, s_scratch);
                xmax = block_max(xm, s_scratch);
                if (dmax <= cfg.tol * xmax) { conv = true; }
                double bdummy;
                const double rm = item_residual(it, false, bdummy, s_scratch);
                __syncthreads();
                const double den = it.lnorm * xmax + bm;
                berr = den > 0.0 ? rm / den : 0.0;
                if (berr <= cfg.tol) conv = true;
                if (conv || t >= cfg.max_iters) break;
            }
            out.sweeps = sweeps;
            out.dnorm = xmax > 0.0 ? dmax / xmax : 0.0;
            out.berr = berr;
            if (!out.status) out.status = conv ? 0 : SPTRSV_ERR_NOT_CONVERGED;
        }
        if (threadIdx.x == 0) res[i] = out;
        __syncthreads();
    }
}

}  // namespace

int batch_occupancy(int threads, size_t smem, int *per_sm) {
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch, threads, smem);
    if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, cudaGetErrorString(e));
    return SPTRSV_OK;
}

int batch_launch(const BatchItem *d_items, int count, ItemResult *d_res, unsigned int *d_cursor,
                 const BatchCfg &cfg, int grid, int threads, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_cursor, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        k_batch<<<grid, threads, smem, s>>>(d_items, count, d_res, d_cursor, cfg);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    return SPTRSV_OK;
}

namespace {
}  // namespace
}  // namespace sptrsv

using namespace sptrsv;

struct sptrsv_batch {
    int device = -1;
    int32_t dtype = SPTRSV_F64;
    sptrsv_solve_opts opts{};
    bool refine = false;
    std::vector<sptrsv_plan *> plans;
    std::vector<int32_t> nrhs;
    std::vector<BatchItem> items;                  // host copy, b/x filled per run
    std::vector<int32_t> item_factor, item_col0;
    BatchItem *d_items = nullptr;
    ItemResult *d_res = nullptr;
    unsigned int *d_cursor = nullptr;
    void *d_work = nullptr;
    int threads = 256, grid = 0;
    size_t smem = 0;
    bool tuned = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double est_ms = 0.0;
};

namespace sptrsv {
namespace {

int default_variant_impl(const sptrsv_plan *p, int nrhs) {
    if (nrhs >= 3) return nrhs <= 4 ? V_T4 : nrhs <= 8 ? V_T8 : nrhs <= 16 ? V_T16 : V_T32;
    const double per_row = p->h.n ? double(p->nnz_off) / p->h.n : 0.0;
    return per_row <= 8.0 ? V_L1 : per_row <= 16.0 ? V_L2 : V_L4;
}

int item_win(const sptrsv_plan *p, int nrhs, size_t elem, size_t budget) {
    const int w = p->h.ring_rows;
    if (w <= 0) return 0;
    return size_t(w) * size_t(nrhs) * elem <= budget ? w : 0;
}

constexpr size_t kBatchRingBudget = 64 * 1024;     // per block: leaves room for 2-3 blocks per SM
constexpr size_t kBatchStageBudget = 96 * 1024;    // staged walk per block: 2 blocks per SM
}  // namespace

int batch_default_variant(const sptrsv_plan *p, int nrhs) { return default_variant_impl(p, nrhs); }

size_t batch_item_workspace(const BatchItem &it, bool refine) {
    const size_t es = refine ? sizeof(float) : sizeof(double);
    const size_t v = (size_t(it.n) * size_t(it.nrhs) * sizeof(float) + 255) & ~size_t(255);
    size_t w = refine ? 2 * v : 0;
    if (it.staged) w += (size_t(it.n) * size_t(it.nrhs) * es + 64 + 255) & ~size_t(255);
    return w;
}

void batch_bind_workspace(BatchItem &it, char *base, bool refine) {
    const size_t v = (size_t(it.n) * size_t(it.nrhs) * sizeof(float) + 255) & ~size_t(255);
    size_t off = 0;
    if (refine) {
        it.r32 = reinterpret_cast<float *>(base);
        it.d32 = reinterpret_cast<float *>(base + v);
        off = 2 * v;
    }
    it.bdev = it.staged ? static_cast<void *>(base + off) : nullptr;
}

size_t batch_item_smem(const BatchItem &it, bool refine) {
    const size_t es = refine ? sizeof(float) : sizeof(double);
    const size_t ring = size_t(it.win) * size_t(it.nrhs) * es;
    return it.staged ? stage_smem_bytes(it.si, ring) : ring;
}

void batch_fill_item(BatchItem &it, const sptrsv_plan *p, int nrhs, bool refine, size_t ring_budget) {
    it = BatchItem{};
    it.n = p->h.n;
    it.nphases = int32_t(p->h.phase_row.size()) - 1;
    it.nrhs = nrhs;
    it.win = item_win(p, nrhs, refine ? sizeof(float) : sizeof(double), ring_budget);
    it.variant = default_variant_impl(p, nrhs);
    it.rp = p->d.rp;
    it.col = p->d.col;
    it.perm = p->d.perm;
    it.phase_row = p->d.phase_row;
    it.val = p->d.val;
    it.dinv = p->d.dinv;
    it.dinv32 = p->d.dinv32;
    it.s32 = p->d.s32;
    it.hi = p->d.val_hi;
    it.lo = p->d.val_lo;
    it.dhi = p->d.diag_hi;
    it.dlo = p->d.diag_lo;
    it.lnorm = p->lnorm;
    // staged walk when the factor's largest phase fits the block's shared-memory budget
    const size_t es = refine ? sizeof(float) : sizeof(double);
    stage_slot_layout(size_t(p->h.max_phase_rows), size_t(p->h.max_phase_ents), nrhs, es, it.si);
    it.si.phase_ent = p->d.phase_ent;
    it.staged = stage_smem_bytes(it.si, size_t(it.win) * size_t(nrhs) * es) <= kBatchStageBudget ? 1 : 0;
}

namespace {

int build_graph(sptrsv_batch *B) {
    if (B->exec) return SPTRSV_OK;
    BatchCfg cfg{B->refine ? 1 : 0, B->opts.max_iters, B->opts.refine_tol};
    if (B->smem > 0) {
        BCUDA_TRY(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, int(B->smem)));
    }
    int per_sm = 0;
    BCUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, B->threads, B->smem));
    if (per_sm < 1) return fail(SPTRSV_ERR_LAUNCH, "batch kernel does not fit on an SM");
    int sms = 0;
    BCUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device));
    const int want = B->opts.blocks_per_sm ? std::min(B->opts.blocks_per_sm, per_sm) : per_sm;
    B->grid = std::max(1, std::min<int>(int(B->items.size()), want * sms));
    if (!B->cap_stream) BCUDA_TRY(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
    BCUDA_TRY(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(B->d_cursor, 0, sizeof(unsigned int), B->cap_stream);
    k_batch<<<B->grid, B->threads, B->smem, B->cap_stream>>>(B->d_items, int(B->items.size()), B->d_res,
                                                              B->d_cursor, cfg);
    cudaError_t le = cudaGetLastError();
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(B->cap_stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return fail(SPTRSV_ERR_CUDA, std::string("capturing the batch graph: ") +
                                         cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    B->graph = g;
    BCUDA_TRY(cudaGraphInstantiate(&B->exec, g, 0));
    return SPTRSV_OK;
}

void fill_vectors(sptrsv_batch *B, const void *const *b, void *const *x, const int64_t *ld) {
    const size_t es = B->dtype == SPTRSV_F32 ? sizeof(float) : sizeof(double);
    for (size_t i = 0; i < B->items.size(); ++i) {
        const int f = B->item_factor[i];
        const int64_t off = int64_t(B->item_col0[i]) * ld[f] * int64_t(es);
        B->items[i].b = static_cast<const char *>(b[f]) + off;
        B->items[i].x = static_cast<char *>(x[f]) + off;
        B->items[i].ldb = ld[f];
        B->items[i].ldx = ld[f];
    }
}

// Time each candidate variant on the first factor of every class (shape key)
// with a one-item graph-less launch, and give the class the fastest.
int autotune_batch(sptrsv_batch *B, const void *const *b, void *const *x, const int64_t *ld, cudaStream_t s) {
    fill_vectors(B, b, x, ld);
    std::map<std::tuple<int, int, int, int>, std::vector<size_t>> classes;
    for (size_t i = 0; i < B->items.size(); ++i) {
        const sptrsv_plan *p = B->plans[B->item_factor[i]];
        const int per_row10 = p->h.n ? int(10.0 * double(p->nnz_off) / p->h.n) : 0;
        int lg = 0;
        while ((1 << (lg + 1)) <= p->h.n) ++lg;
        classes[{per_row10, B->items[i].win > 0, lg, B->items[i].nrhs}].push_back(i);
    }
    BatchItem *d_one = nullptr;
    ItemResult *d_r = nullptr;
    unsigned int *d_c = nullptr;
    BCUDA_TRY(cudaMalloc(&d_one, sizeof(BatchItem)));
    BCUDA_TRY(cudaMalloc(&d_r, sizeof(ItemResult)));
    BCUDA_TRY(cudaMalloc(&d_c, sizeof(unsigned int)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    BatchCfg cfg{B->refine ? 1 : 0, B->opts.max_iters, B->opts.refine_tol};
    if (B->smem > 0) cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, int(B->smem));
    int st = SPTRSV_OK;
    for (auto &kv : classes) {
        const size_t i0 = kv.second.front();
        BatchItem probe = B->items[i0];
        std::vector<int> cands;
        if (probe.nrhs >= 2)
            for (int v : {V_T4, V_T8, V_T16, V_T32})
                if (kVariantLanes[v] / 2 < probe.nrhs) cands.push_back(v);
        for (int v : {V_L1, V_L2, V_L4}) cands.push_back(v);
        double best = 1e30;
        int best_v = probe.variant;
        for (int v : cands) {
            probe.variant = v;
            if (cudaMemcpyAsync(d_one, &probe, sizeof(probe), cudaMemcpyHostToDevice, s) != cudaSuccess) break;
            double t = 1e30;
            for (int rep = 0; rep < 3; ++rep) {
                cudaMemsetAsync(d_c, 0, sizeof(unsigned int), s);
                cudaEventRecord(e0, s);
                k_batch<<<1, B->threads, B->smem, s>>>(d_one, 1, d_r, d_c, cfg);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(SPTRSV_ERR_CUDA, "autotune launch"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t = std::min(t, double(ms));
            }
            if (st) break;
            if (t < best) {
                best = t;
                best_v = v;
            }
        }
        if (st) break;
        for (size_t i : kv.second) B->items[i].variant = best_v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_one);
    cudaFree(d_r);
    cudaFree(d_c);
    (void)cudaGetLastError();
    B->tuned = true;
    return st;
}

}  // namespace
}  // namespace sptrsv

extern "C" {

int sptrsv_batch_create(sptrsv_plan *const *plans, int32_t count, const int32_t *nrhs, int32_t dtype,
                        const sptrsv_solve_opts *opts, sptrsv_batch **out) {
    clear_error();
    if (!out) return fail(SPTRSV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || !nrhs || count <= 0) return fail(SPTRSV_ERR_ARG, "plans/nrhs/count");
    if (dtype != SPTRSV_F64) return fail(SPTRSV_ERR_ARG, "batched solves take FP64 b and x (dtype SPTRSV_F64)");
    sptrsv_solve_opts o;
    sptrsv_solve_opts_default(&o);
    if (opts) o = *opts;
    const bool refine = o.precision == SPTRSV_PREC_F32_REFINE;
    if (o.precision != SPTRSV_PREC_F64 && !refine) return fail(SPTRSV_ERR_ARG, "unknown precision");
    if (refine && (o.max_iters < 0 || o.max_iters > 14 || !(o.refine_tol > 0.0)))
        return fail(SPTRSV_ERR_ARG, "max_iters must be in [0, 14] and refine_tol positive");
    const int threads = o.threads ? o.threads : 256;
    if (threads < 32 || threads > 512 || threads % 32) return fail(SPTRSV_ERR_ARG, "threads in [32, 512], multiple of 32");
    int device = -1;
    for (int32_t f = 0; f < count; ++f) {
        const sptrsv_plan *p = plans[f];
        if (!p) return fail(SPTRSV_ERR_ARG, "plan " + std::to_string(f) + " is NULL");
        if (p->device < 0) return fail(SPTRSV_ERR_NO_DEVICE, "plan " + std::to_string(f) + " is host-only");
        if (device < 0) device = p->device;
        if (p->device != device) return fail(SPTRSV_ERR_ARG, "all plans of a batch must live on one device");
        if (nrhs[f] < 1) return fail(SPTRSV_ERR_ARG, "nrhs must be >= 1");
        if (!(p->values & (refine ? SPTRSV_VALUES_F32 : SPTRSV_VALUES_F64)))
            return fail(SPTRSV_ERR_ARG, "plan " + std::to_string(f) + " lacks the value copy this precision needs");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    sptrsv_batch *B = new sptrsv_batch();
    B->device = device;
    B->dtype = dtype;
    B->opts = o;
    B->refine = refine;
    B->threads = threads;
    B->plans.assign(plans, plans + count);
    B->nrhs.assign(nrhs, nrhs + count);
    size_t work = 0;
    for (int32_t f = 0; f < count; ++f) {
        const sptrsv_plan *p = plans[f];
        for (int32_t c0 = 0; c0 < nrhs[f]; c0 += 32) {       // items of at most 32 columns
            BatchItem it;
            batch_fill_item(it, p, std::min(32, nrhs[f] - c0), refine, kBatchRingBudget);
            B->smem = std::max(B->smem, batch_item_smem(it, refine));
            work += batch_item_workspace(it, refine);
            B->items.push_back(it);
            B->item_factor.push_back(f);
            B->item_col0.push_back(c0);
        }
    }
    // longest critical path first (phases dominate a block's walk time)
    std::vector<size_t> order(B->items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const double ca = double(B->items[a].nphases) * 4.0 + double(B->items[a].n) * B->items[a].nrhs / 4096.0;
        const double cb = double(B->items[b].nphases) * 4.0 + double(B->items[b].n) * B->items[b].nrhs / 4096.0;
        return ca > cb;
    });
    {
        std::vector<BatchItem> it2;
        std::vector<int32_t> f2, c2;
        for (size_t i : order) {
            it2.push_back(B->items[i]);
            f2.push_back(B->item_factor[i]);
            c2.push_back(B->item_col0[i]);
        }
        B->items.swap(it2);
        B->item_factor.swap(f2);
        B->item_col0.swap(c2);
    }
    int st = SPTRSV_OK;
    cudaError_t e = cudaMalloc(&B->d_items, B->items.size() * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_res, B->items.size() * sizeof(ItemResult));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_cursor, sizeof(unsigned int));
    if (e == cudaSuccess && work) e = cudaMalloc(&B->d_work, work);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        st = fail(e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA, cudaGetErrorString(e));
    }
    if (!st && work) {
        char *w = static_cast<char *>(B->d_work);
        for (BatchItem &it : B->items) {
            batch_bind_workspace(it, w, refine);
            w += batch_item_workspace(it, refine);
        }
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (st) {
        sptrsv_batch_destroy(B);
        return st;
    }
    *out = B;
    return SPTRSV_OK;
}

int sptrsv_batch_run(sptrsv_batch *B, const void *const *b, void *const *x, const int64_t *ld,
                     sptrsv_stream stream, sptrsv_report *reports) {
    clear_error();
    if (!B || !b || !x || !ld) return fail(SPTRSV_ERR_ARG, "NULL argument");
    for (size_t f = 0; f < B->plans.size(); ++f) {
        if (!b[f] || !x[f]) return fail(SPTRSV_ERR_ARG, "b/x of factor " + std::to_string(f) + " is NULL");
        if (ld[f] < std::max<int64_t>(B->plans[f]->h.n, 1)) return fail(SPTRSV_ERR_ARG, "ld too small");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != B->device) cudaSetDevice(B->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int st = SPTRSV_OK;
    if (!B->tuned && B->opts.sync == SPTRSV_SYNC_AUTO) st = autotune_batch(B, b, x, ld, s);
    if (!st) st = build_graph(B);
    if (!st) {
        fill_vectors(B, b, x, ld);
        // pageable source: the CUDA driver stages it, so the host copy may change right after the call
        cudaError_t e = cudaMemcpyAsync(B->d_items, B->items.data(), B->items.size() * sizeof(BatchItem),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            st = fail(SPTRSV_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
        }
    }
    if (!st && reports) {
        std::vector<ItemResult> r(B->items.size());
        cudaError_t e = cudaMemcpyAsync(r.data(), B->d_res, r.size() * sizeof(ItemResult), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = fail(SPTRSV_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(e));
        } else {
            for (size_t f = 0; f < B->plans.size(); ++f) {
                std::memset(&reports[f], 0, sizeof(sptrsv_report));
                reports[f].sync = SPTRSV_SYNC_CTA;
                reports[f].grid = B->grid;
                reports[f].threads = B->threads;
            }
            for (size_t i = 0; i < r.size(); ++i) {
                sptrsv_report &rp = reports[B->item_factor[i]];
                if (r[i].status && !rp.status) rp.status = r[i].status;
                rp.sweeps = std::max(rp.sweeps, r[i].sweeps);
                rp.dnorm = std::max(rp.dnorm, r[i].dnorm);
                rp.berr = std::max(rp.berr, r[i].berr);
                rp.lanes = kVariantLanes[B->items[i].variant];
            }
            for (size_t f = 0; f < B->plans.size(); ++f)
                if (reports[f].status) {
                    st = fail(reports[f].status, "factor " + std::to_string(f) + ": " +
                                                    sptrsv_status_string(reports[f].status));
                    break;
                }
        }
    }
    if (prev >= 0 && prev != B->device) cudaSetDevice(prev);
    return st;
}

void sptrsv_batch_destroy(sptrsv_batch *B) {
    if (!B) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (B->device >= 0 && prev != B->device) cudaSetDevice(B->device);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    if (B->d_items) cudaFree(B->d_items);
    if (B->d_res) cudaFree(B->d_res);
    if (B->d_cursor) cudaFree(B->d_cursor);
    if (B->d_work) cudaFree(B->d_work);
    if (prev >= 0 && B->device >= 0 && prev != B->device) cudaSetDevice(prev);
    delete B;
}

int sptrsv_batch_solve(sptrsv_plan *const *plans, int32_t count, const void *const *b, void *const *x,
                       const int32_t *nrhs, const int64_t *ld, int32_t dtype, const sptrsv_solve_opts *opts,
                       sptrsv_stream stream, sptrsv_report *reports) {
    sptrsv_batch *B = nullptr;
    int st = sptrsv_batch_create(plans, count, nrhs, dtype, opts, &B);
    if (st) return st;
    st = sptrsv_batch_run(B, b, x, ld, stream, reports);
    if (!st && !reports) {
        cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) st = fail(SPTRSV_ERR_CUDA, cudaGetErrorString(e));
    }
    sptrsv_batch_destroy(B);
    return st;
}

}  // extern "C"
