// Wavefront analysis on the device: one upload of the caller's lower CSR, then
//   k_levels         wavefront of every row (Sec. 1): rows claimed in increasing
//                    id by a persistent co-resident grid, each waiting on its
//                    parents' published wavefronts (value polling, bounded);
//   k_digit_hist /   a stable LSD radix sort of the row ids by wavefront, 8 bits
//   k_digit_scatter  a pass: the Sec. 5 order (superstep, id) for LEVELS;
//   k_layout         the device-order copy the solve kernels read, built by
//                    gathers from the uploaded CSR: the same arrays, bit for bit,
//                    as the host analysis uploads.
// Only small per-wavefront tables and the level / permutation arrays come back
// to the host (they back sptrsv_plan_export and the block-local partition).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "plan.hpp"

namespace sptrsv {
namespace {

#define ANA_TRY(expr)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA, \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));                \
    } while (0)

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;       // keys per sort / scan tile

struct AnaCtl {
    int32_t status;                 // 0, or SPTRSV_ERR_TIMEOUT from k_levels
    int32_t maxlevel;               // deepest wavefront
    uint32_t pad0;
    int32_t max_row_off;            // most off-diagonal entries in a row
    unsigned long long lnorm_bits;  // max row sum |A_ij| (non-negative double as bits)
    int32_t total;                  // scan total
    int32_t pad;
};

__device__ __forceinline__ int32_t ld_level(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_level(int32_t *p, int32_t v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// level[] starts at -1.  Rows are dealt round-robin to the warps of a co-resident
// grid and taken in increasing order; a warp's lanes wait on the row's parents and
// lane 0 publishes 1 + the deepest parent's wavefront.  Every wait ends: the
// warp owning the smallest unfinished row has finished its earlier rows, so it is
// at that row, whose parents (smaller ids) are all finished.
__global__ void __launch_bounds__(kThreads) k_levels(int32_t n, const int32_t *rp, const int32_t *col,
                                                     int32_t *level, AnaCtl *c, long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    int32_t deepest = -1;                            // this warp's deepest row, one atomic at the end
    for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < n; r += warps) {
        const int32_t row = int32_t(r);
        const int32_t lo = rp[row], last = rp[row + 1] - 1;
        int32_t d = 0;
        bool bad = false;
        for (int32_t q = lo + lane; q < last; q += 32) {
            const int32_t p = col[q];
            int32_t lv = ld_level(level + p);
            if (lv < 0) {
                const long long t0 = gtimer();
                unsigned spins = 0;
                while ((lv = ld_level(level + p)) < 0) {
                    if ((++spins & 63u) == 0 &&
                        (*reinterpret_cast<volatile int32_t *>(&c->status) != 0 || gtimer() - t0 > timeout_ns)) {
                        bad = true;
                        break;
                    }
                }
            }
            if (bad) break;
            d = max(d, lv + 1);
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) atomicCAS(&c->status, 0, SPTRSV_ERR_TIMEOUT);
            return;
        }
        d = __reduce_max_sync(0xffffffffu, d);
        if (lane == 0) st_level(level + row, d);
        deepest = max(deepest, d);
    }
    if (lane == 0 && deepest >= 0) atomicMax(&c->maxlevel, deepest);
}

// Histogram of one 8-bit digit per tile, stored digit-major: hist[digit * ntiles + tile].
__global__ void __launch_bounds__(kThreads) k_digit_hist(const int32_t *keys, int32_t n, int shift,
                                                         int32_t *hist, int32_t ntiles) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kTile;
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = base + i * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[int64_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile by one digit: keys move in rounds of 256 in index
// order; inside a round a key's place is the digit's running base for the tile,
// plus the same-digit keys of lower warps, plus those of lower lanes.
// vin == nullptr: the values are the indices (the first pass).
__global__ void __launch_bounds__(kThreads) k_digit_scatter(const int32_t *kin, const int32_t *vin, int32_t n,
                                                            int shift, const int32_t *off, int32_t ntiles,
                                                            int32_t *kout, int32_t *vout) {
    __shared__ int32_t base[256];
    __shared__ int32_t wcnt[kThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = off[int64_t(tid) * ntiles + blockIdx.x];
    for (int w = 0; w < kThreads / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int64_t t0 = int64_t(blockIdx.x) * kTile;
    for (int round = 0; round < kItems; ++round) {
        const int64_t idx = t0 + round * kThreads + tid;
        const bool valid = idx < n;
        int32_t key = 0, val = 0;
        int dig = 256;                                   // invalid lanes group apart
        if (valid) {
            key = kin[idx];
            val = vin ? vin[idx] : int32_t(idx);
            dig = (key >> shift) & 255;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        int before = 0, total = 0;
        if (valid) {
            for (int w = 0; w < kThreads / 32; ++w) {
                const int cw = wcnt[w][dig];
                if (w < warp) before += cw;
                total += cw;
            }
            const int32_t pos = base[dig] + before + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        if (valid && before + rank == total - 1) base[dig] += total;     // the round's last key of the digit
        if (valid && rank == 0) wcnt[warp][dig] = 0;
        __syncthreads();
    }
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int32_t block_exclusive(int32_t v, int32_t *s_warp, int32_t &excl) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) s_warp[lane] = w;                 // inclusive warp totals
    }
    __syncthreads();
    const int32_t warp_base = warp ? s_warp[warp - 1] : 0;
    const int32_t total = s_warp[nw - 1];
    excl = warp_base + inc - v;
    __syncthreads();
    return total;
}

// Exclusive scan, phase 1: every tile scanned locally, its total kept.
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const int32_t *in, int32_t *out, int64_t m,
                                                         int32_t *tile_sum) {
    __shared__ int32_t s_warp[32];
    const int64_t base = int64_t(blockIdx.x) * kTile + int64_t(threadIdx.x) * kItems;
    int32_t v[kItems], sum = 0;
    for (int i = 0; i < kItems; ++i) {
        v[i] = base + i < m ? in[base + i] : 0;
        sum += v[i];
    }
    int32_t excl = 0;
    const int32_t total = block_exclusive(sum, s_warp, excl);
    for (int i = 0; i < kItems; ++i) {
        if (base + i < m) out[base + i] = excl;
        excl += v[i];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// Phase 2: one block scans the tile totals in chunks, carrying the running sum.
__global__ void __launch_bounds__(1024) k_scan_sums(int32_t *sums, int32_t count, AnaCtl *c) {
    __shared__ int32_t s_warp[32];
    int32_t carry = 0;
    for (int32_t b = 0; b < count; b += 1024) {
        const int32_t i = b + int32_t(threadIdx.x);
        const int32_t v = i < count ? sums[i] : 0;
        int32_t excl = 0;
        const int32_t total = block_exclusive(v, s_warp, excl);
        if (i < count) sums[i] = carry + excl;
        carry += total;
    }
    if (threadIdx.x == 0) c->total = carry;
}

// Phase 3: add every tile's offset.
__global__ void __launch_bounds__(kThreads) k_scan_add(int32_t *out, int64_t m, const int32_t *sums) {
    const int64_t base = int64_t(blockIdx.x) * kTile;
    const int32_t add = sums[blockIdx.x];
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = base + i * kThreads + threadIdx.x;
        if (idx < m) out[idx] += add;
    }
}

// First row of every wavefront in the sorted order (every wavefront is non-empty).
__global__ void k_starts(const int32_t *keys, int32_t n, int32_t *start) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
        if (r == 0 || keys[r] != keys[r - 1]) start[keys[r]] = int32_t(r);
    if (blockIdx.x == 0 && threadIdx.x == 0) start[keys[n - 1] + 1] = n;
}

// Off-diagonal entries of every device row.
__global__ void k_row_counts(const int32_t *rp, const int32_t *perm, int32_t n, int32_t *cnt) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
        const int32_t v = perm[r];
        cnt[r] = rp[v + 1] - rp[v] - 1;
    }
}

__global__ void k_set(int32_t *p, const AnaCtl *c) { *p = c->total; }

struct LayoutOut {
    int32_t flip;                   // 0, or n - 1 for a factor analysed with its ids reversed
    int32_t *col;
    double *val, *dinv;
    float *hi, *lo, *dhi, *dlo, *dinv32, *s32;
};

// One warp per device row r = row perm[r] of the factor: its off-diagonal entries
// scaled by the reciprocal diagonal (one IEEE division, as on the host), the FP32
// splits, and the row sum of |A_ij| (sequential, in column order, as on the host).
__global__ void __launch_bounds__(kThreads) k_layout(int32_t n, const int32_t *rp, const int32_t *col,
                                                     const double *val, const int32_t *perm, const int32_t *drp,
                                                     LayoutOut o, AnaCtl *c) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    unsigned long long norm_bits = 0;               // this warp's maxima, one atomic each at the end
    int32_t widest = 0;
    for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < n; r += warps) {
        const int32_t v = perm[r];
        const int32_t lo = rp[v], last = rp[v + 1] - 1, dst = drp[r];
        const double d = val[last];
        const double dinv = __ddiv_rn(1.0, d);
        for (int32_t j = lane; j < last - lo; j += 32) {
            const double a = val[lo + j];
            const double s = __dmul_rn(a, dinv);
            o.col[dst + j] = o.flip ? o.flip - col[lo + j] : col[lo + j];
            if (o.val) o.val[dst + j] = s;
            if (o.hi) {
                const float h = __double2float_rn(a);
                o.hi[dst + j] = h;
                o.lo[dst + j] = __double2float_rn(__dsub_rn(a, double(h)));
                o.s32[dst + j] = __double2float_rn(s);
            }
        }
        if (lane == 0) {
            if (o.dinv) o.dinv[r] = dinv;
            if (o.dhi) {
                const float h = __double2float_rn(d);
                o.dhi[r] = h;
                o.dlo[r] = __double2float_rn(__dsub_rn(d, double(h)));
                o.dinv32[r] = __double2float_rn(dinv);
            }
            double rs = 0.0;
            for (int32_t q = lo; q <= last; ++q) rs = __dadd_rn(rs, fabs(val[q]));
            norm_bits = max(norm_bits, static_cast<unsigned long long>(__double_as_longlong(rs)));
            widest = max(widest, last - lo);
        }
    }
    if (lane == 0) {
        atomicMax(&c->lnorm_bits, norm_bits);
        atomicMax(&c->max_row_off, widest);
    }
}

// Device row -> row of the caller's numbering (ids reversed for UPPER / LOWER_TRANSPOSED).
__global__ void k_perm_out(const int32_t *perm, int32_t n, int32_t flip, int32_t *out) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
        out[r] = flip ? flip - perm[r] : perm[r];
}

__global__ void k_phase_ent(const int32_t *start, int32_t count, const int32_t *drp, int32_t *pent) {
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
        pent[q] = drp[start[q]];
}

// Device arrays of a plan carry 64 zeroed bytes past their end (see upload_plan).
template <typename T>
int alloc_zeroed(T **d, size_t count, int64_t *bytes) {
    const size_t nb = count * sizeof(T) + 64;
    ANA_TRY(cudaMalloc((void **)d, nb));
    ANA_TRY(cudaMemset(*d, 0, nb));
    *bytes += int64_t(nb);
    return SPTRSV_OK;
}

struct Temps {
    std::vector<void *> ptrs;
    ~Temps() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    int get(T **p, size_t count) {
        ANA_TRY(cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(T)));
        ptrs.push_back(*p);
        return SPTRSV_OK;
    }
};

// Exclusive scan of m int32 (in place allowed); the total lands in c->total.
int scan(const int32_t *in, int32_t *out, int64_t m, int32_t *tile_sum, AnaCtl *c) {
    const int32_t tiles = int32_t((m + kTile - 1) / kTile);
    if (tiles > 0) k_scan_tiles<<<tiles, kThreads>>>(in, out, m, tile_sum);
    k_scan_sums<<<1, 1024>>>(tile_sum, tiles, c);
    if (tiles > 0) k_scan_add<<<tiles, kThreads>>>(out, m, tile_sum);
    ANA_TRY(cudaGetLastError());
    return SPTRSV_OK;
}

// Block-local layout values: entry q of the block-local order is device-order
// entry src[q], row t is device row rsrc[t].
template <typename T>
__global__ void k_local_values(int64_t nnz_off, int32_t n, const int32_t *src, const int32_t *rsrc, const T *val,
                               const T *dinv, T *lval, T *ldinv) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nnz_off; q += stride) lval[q] = val[src[q]];
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += stride) ldinv[t] = dinv[rsrc[t]];
}

struct SetDevice {
    int prev = -1;
    explicit SetDevice(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~SetDevice() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

int analyze_levels_device(sptrsv_plan *p, const sptrsv_csr *A, int device, int32_t values, bool reversed) {
    SetDevice guard(device);
    HostSchedule &h = p->h;
    DeviceBuffers &d = p->d;
    const int32_t n = A->n;
    const int64_t nnz = A->nnz, nnz_off = nnz - n;
    const auto t0 = std::chrono::steady_clock::now();
    Temps tmp;
    int32_t *g_rp, *g_col, *level, *k1, *k2, *v1, *v2, *hist, *tsum, *start;
    double *g_val;
    AnaCtl *c;
    const int32_t ntiles = int32_t((int64_t(n) + kTile - 1) / kTile);
    const int64_t hist_len = int64_t(256) * ntiles;
    const int32_t sum_len = int32_t(std::max<int64_t>((std::max<int64_t>(hist_len, n) + kTile - 1) / kTile, 1));
    int st;
    if ((st = tmp.get(&g_rp, size_t(n) + 1)) || (st = tmp.get(&g_col, size_t(nnz))) ||
        (st = tmp.get(&g_val, size_t(nnz))) || (st = tmp.get(&level, size_t(n))) || (st = tmp.get(&k1, size_t(n))) ||
        (st = tmp.get(&k2, size_t(n))) || (st = tmp.get(&v1, size_t(n))) || (st = tmp.get(&v2, size_t(n))) ||
        (st = tmp.get(&hist, size_t(hist_len))) || (st = tmp.get(&tsum, size_t(sum_len))) ||
        (st = tmp.get(&start, size_t(n) + 1)) || (st = tmp.get(&c, 1)))
        return st;
    ANA_TRY(cudaMemcpy(g_rp, A->rowptr, (size_t(n) + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    ANA_TRY(cudaMemcpy(g_col, A->col, size_t(nnz) * sizeof(int32_t), cudaMemcpyHostToDevice));
    ANA_TRY(cudaMemcpy(g_val, A->val, size_t(nnz) * sizeof(double), cudaMemcpyHostToDevice));
    ANA_TRY(cudaMemset(level, 0xff, size_t(n) * sizeof(int32_t)));
    ANA_TRY(cudaMemset(c, 0, sizeof(AnaCtl)));
    const auto t1 = std::chrono::steady_clock::now();
    // wavefronts: a co-resident persistent grid (cooperative launch: co-residency or an error)
    int per_sm = 0, sms = 0;
    ANA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels, kThreads, 0));
    ANA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(std::max(1, per_sm) * sms));
        cfg.blockDim = dim3(kThreads);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const long long timeout_ns = 2000000000LL;
        ANA_TRY(cudaLaunchKernelEx(&cfg, k_levels, n, (const int32_t *)g_rp, (const int32_t *)g_col, level, c,
                                   timeout_ns));
    }
    AnaCtl hc;
    ANA_TRY(cudaMemcpy(&hc, c, sizeof(hc), cudaMemcpyDeviceToHost));
    if (hc.status) return fail(hc.status, "device wavefront analysis: a bounded wait expired");
    const int32_t S = hc.maxlevel + 1;
    // stable radix sort of the ids by wavefront, 8 bits a pass
    const int32_t *kin = level, *vin = nullptr;
    int32_t *kout = k1, *vout = v1;
    for (int shift = 0; shift == 0 || (shift < 31 && (hc.maxlevel >> shift) != 0); shift += 8) {
        k_digit_hist<<<ntiles, kThreads>>>(kin, n, shift, hist, ntiles);
        if ((st = scan(hist, hist, hist_len, tsum, c))) return st;
        k_digit_scatter<<<ntiles, kThreads>>>(kin, vin, n, shift, hist, ntiles, kout, vout);
        ANA_TRY(cudaGetLastError());
        kin = kout;
        vin = vout;
        kout = kout == k1 ? k2 : k1;
        vout = vout == v1 ? v2 : v1;
    }
    const int32_t *keys = kin, *perm = vin;
    k_starts<<<std::max(1, std::min(ntiles * kItems, 4096)), kThreads>>>(keys, n, start);
    ANA_TRY(cudaGetLastError());
    ANA_TRY(cudaDeviceSynchronize());
    const auto t2 = std::chrono::steady_clock::now();
    // device layout
    int64_t bytes = 0;
    if ((st = alloc_zeroed(&d.rp, size_t(n) + 1, &bytes)) || (st = alloc_zeroed(&d.col, size_t(nnz_off), &bytes)) ||
        (st = alloc_zeroed(&d.perm, size_t(n), &bytes)) || (st = alloc_zeroed(&d.phase_row, size_t(S) + 1, &bytes)) ||
        (st = alloc_zeroed(&d.phase_ent, size_t(S) + 1, &bytes)))
        return st;
    k_row_counts<<<std::max(1, std::min(ntiles * kItems, 4096)), kThreads>>>(g_rp, perm, n, d.rp);
    if ((st = scan(d.rp, d.rp, n, tsum, c))) return st;
    k_set<<<1, 1>>>(d.rp + n, c);
    const int32_t flip = reversed ? n - 1 : 0;
    LayoutOut o{flip, d.col, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (values & SPTRSV_VALUES_F64) {
        if ((st = alloc_zeroed(&d.val, size_t(nnz_off), &bytes)) || (st = alloc_zeroed(&d.dinv, size_t(n), &bytes)))
            return st;
        o.val = d.val;
        o.dinv = d.dinv;
    }
    if (values & SPTRSV_VALUES_F32) {
        if ((st = alloc_zeroed(&d.val_hi, size_t(nnz_off), &bytes)) ||
            (st = alloc_zeroed(&d.val_lo, size_t(nnz_off), &bytes)) ||
            (st = alloc_zeroed(&d.s32, size_t(nnz_off), &bytes)) || (st = alloc_zeroed(&d.diag_hi, size_t(n), &bytes)) ||
            (st = alloc_zeroed(&d.diag_lo, size_t(n), &bytes)) || (st = alloc_zeroed(&d.dinv32, size_t(n), &bytes)))
            return st;
        o.hi = d.val_hi;
        o.lo = d.val_lo;
        o.s32 = d.s32;
        o.dhi = d.diag_hi;
        o.dlo = d.diag_lo;
        o.dinv32 = d.dinv32;
    }
    k_layout<<<std::max(1, std::min((n + 7) / 8, sms * 8)), kThreads>>>(n, g_rp, g_col, g_val, perm, d.rp, o, c);
    k_phase_ent<<<std::max(1, std::min((S + 1 + 255) / 256, 1024)), 256>>>(start, S + 1, d.rp, d.phase_ent);
    ANA_TRY(cudaGetLastError());
    k_perm_out<<<std::max(1, std::min(ntiles * kItems, 4096)), kThreads>>>(perm, n, flip, d.perm);
    ANA_TRY(cudaGetLastError());
    ANA_TRY(cudaMemcpy(d.phase_row, start, (size_t(S) + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice));
    // host side of the plan: the schedule arrays and the per-wavefront tables
    h.level.resize(n);
    h.perm.resize(n);
    h.phase_row.resize(size_t(S) + 1);
    std::vector<int32_t> pent(size_t(S) + 1);
    ANA_TRY(cudaMemcpy(h.level.data(), level, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    ANA_TRY(cudaMemcpy(h.perm.data(), perm, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    ANA_TRY(cudaMemcpy(h.phase_row.data(), start, (size_t(S) + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    ANA_TRY(cudaMemcpy(pent.data(), d.phase_ent, (size_t(S) + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    ANA_TRY(cudaMemcpy(&hc, c, sizeof(hc), cudaMemcpyDeviceToHost));
    h.n = n;
    h.nnz = nnz;
    h.mode = SPTRSV_SCHED_LEVELS;
    h.k = 1;
    h.S = S;
    h.nlevels = S;
    h.sched_blocks = 1;
    h.coarse_vertices = n;
    h.sigma = h.level;
    h.pi.assign(n, 0);
    h.dev_perm = h.perm;
    h.step_blk.resize(size_t(S) + 1);
    h.blk_phase.resize(size_t(S) + 1);
    for (int32_t s = 0; s <= S; ++s) h.step_blk[s] = h.blk_phase[s] = s;
    h.max_phase_rows = h.max_block_rows = h.max_level_rows = 0;
    h.max_phase_ents = 0;
    for (int32_t s = 0; s < S; ++s) {
        h.max_level_rows = std::max(h.max_level_rows, h.phase_row[s + 1] - h.phase_row[s]);
        h.max_phase_ents = std::max(h.max_phase_ents, pent[s + 1] - pent[s]);
    }
    h.max_phase_rows = h.max_block_rows = h.max_level_rows;
    h.ring_rows = n <= (1 << 20) ? ring_rows_of(A, h) : 0;
    h.schedule_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    p->max_row_off = hc.max_row_off;
    double ln = 0.0;
    std::memcpy(&ln, &hc.lnorm_bits, sizeof(ln));
    p->lnorm = ln;
    // the small per-superstep tables and the solve's control words, as upload_plan
    {
        int32_t *sb = nullptr, *bp = nullptr;
        if ((st = alloc_zeroed(&sb, size_t(S) + 1, &bytes))) return st;
        d.step_blk = sb;
        if ((st = alloc_zeroed(&bp, size_t(S) + 1, &bytes))) return st;
        d.blk_phase = bp;
        ANA_TRY(cudaMemcpy(d.step_blk, h.step_blk.data(), (size_t(S) + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
        ANA_TRY(cudaMemcpy(d.blk_phase, h.blk_phase.data(), (size_t(S) + 1) * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
    }
    ANA_TRY(cudaMalloc((void **)&d.counters, sizeof(Ctl)));
    ANA_TRY(cudaMemset(d.counters, 0, sizeof(Ctl)));
    bytes += sizeof(Ctl);
    ANA_TRY(cudaMalloc((void **)&d.flags, std::max<size_t>(size_t(n), 1) * sizeof(uint32_t)));
    ANA_TRY(cudaMemset(d.flags, 0, std::max<size_t>(size_t(n), 1) * sizeof(uint32_t)));
    bytes += int64_t(std::max<size_t>(size_t(n), 1) * sizeof(uint32_t));
    p->device_bytes = bytes;
    (void)t0;
    return SPTRSV_OK;
}

int local_values_device(sptrsv_plan *p, const std::vector<int32_t> &src, const std::vector<int32_t> &rsrc,
                        int64_t *bytes) {
    DeviceBuffers &d = p->d;
    const int64_t nnz_off = int64_t(src.size());
    const int32_t n = int32_t(rsrc.size());
    Temps tmp;
    int32_t *g_src, *g_rsrc;
    int st;
    if ((st = tmp.get(&g_src, size_t(nnz_off))) || (st = tmp.get(&g_rsrc, size_t(n)))) return st;
    if (nnz_off) ANA_TRY(cudaMemcpy(g_src, src.data(), size_t(nnz_off) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (n) ANA_TRY(cudaMemcpy(g_rsrc, rsrc.data(), size_t(n) * sizeof(int32_t), cudaMemcpyHostToDevice));
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((std::max<int64_t>(nnz_off, n) + 255) / 256, 4096)));
    if (d.val) {
        if ((st = alloc_zeroed(&d.l_val, size_t(nnz_off), bytes)) || (st = alloc_zeroed(&d.l_dinv, size_t(n), bytes)))
            return st;
        k_local_values<double><<<grid, 256>>>(nnz_off, n, g_src, g_rsrc, d.val, d.dinv, d.l_val, d.l_dinv);
    }
    if (d.s32) {
        if ((st = alloc_zeroed(&d.l_s32, size_t(nnz_off), bytes)) ||
            (st = alloc_zeroed(&d.l_dinv32, size_t(n), bytes)))
            return st;
        k_local_values<float><<<grid, 256>>>(nnz_off, n, g_src, g_rsrc, d.s32, d.dinv32, d.l_s32, d.l_dinv32);
    }
    ANA_TRY(cudaGetLastError());
    ANA_TRY(cudaDeviceSynchronize());                  // the temporaries are freed on return
    return SPTRSV_OK;
}

}  // namespace sptrsv
