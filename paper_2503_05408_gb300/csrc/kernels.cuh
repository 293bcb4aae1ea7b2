// Device kernels of the superstep-scheduled forward substitution (Eq. 2.1).
//
// The factor is stored in "device order": superstep-contiguous (Sec. 5),
// and inside a superstep grouped by block (core) and phase (depth among
// same-block parents).  Column ids stay ORIGINAL row ids, so every gather
// reads the caller's x (original order) directly and every row writes its
// result to x[perm[r]]: no un-permute pass and no internal copy of x.
//
// Three executors walk the same structure:
//  * k_grid   persistent grid; a superstep with a single wide phase is spread
//             over every warp of the grid, a superstep with several blocks
//             gives each block to one thread block (the paper's core) which
//             steps through the block's phases with __syncthreads; one
//             grid-wide barrier separates supersteps (Sec. 2.2 BSP model).
//  * k_flags  persistent grid without barriers: rows are taken in device
//             order and every row waits on per-row ready flags of its
//             parents (the flag holds the solve's epoch, so flags never need
//             resetting).
//  * k_cta    one thread block walks all supersteps, phases separated by
//             __syncthreads (small factors; also the batched executor's unit).
//
// Every wait is bounded (%globaltimer); on expiry the kernel records
// SPTRSV_ERR_TIMEOUT in the status word and returns - it never traps.
#pragma once

#include <cstdint>

#include "sptrsv.h"

namespace sptrsv {

struct Ctl {                         // per-plan control block in device memory
    unsigned long long barrier;      // grid barrier arrivals (zeroed per launch)
    unsigned long long barriers;     // barriers completed (written by block 0)
    unsigned long long flag_waits;   // flag waits that had to spin
    unsigned long long cursor;       // spare work cursor
    double norms[4];                 // refinement: max |d|, max |x|
    int32_t status;                  // 0 or SPTRSV_ERR_*
    int32_t pad[7];
};

template <typename T>
struct SolveArgs {
    int32_t n, S, nrhs;
    const int32_t *__restrict__ rp;
    const int32_t *__restrict__ col;
    const T *__restrict__ val;
    const T *__restrict__ diag;
    const int32_t *__restrict__ perm;
    const int32_t *__restrict__ step_blk;
    const int32_t *__restrict__ blk_phase;
    const int32_t *__restrict__ phase_row;
    const T *b;
    T *x;
    int64_t ldb, ldx;
    Ctl *ctl;
    uint32_t *flags;
    uint32_t epoch;
    long long timeout_ns;
};

__device__ __forceinline__ long long gtimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_status(const Ctl *c) {
    return *reinterpret_cast<const volatile int32_t *>(&c->status);
}
__device__ __forceinline__ void raise_status(Ctl *c, int32_t code) { atomicCAS(&c->status, 0, code); }

// Grid-wide barrier: one arrival per thread block on a monotonically growing
// counter; `target` is the arrival count that completes this barrier.
// Returns false (for the whole block) if the status word is set or the wait
// timed out.
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, unsigned long long target, long long timeout_ns,
                                             int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->barrier, 1ULL);
        int ok = 1;
        const long long t0 = gtimer();
        unsigned spins = 0;
        while (ld_acquire(&ctl->barrier) < target) {
            if ((++spins & 63u) == 1) {
                if (ld_status(ctl) != 0) { ok = 0; break; }
                if (gtimer() - t0 > timeout_ns) { raise_status(ctl, SPTRSV_ERR_TIMEOUT); ok = 0; break; }
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

template <int LANES>
__device__ __forceinline__ unsigned group_mask(int lane32) {
    if constexpr (LANES == 32) return 0xffffffffu;
    else return ((1u << LANES) - 1u) << (lane32 & ~(LANES - 1));
}

template <typename T, int LANES>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
    for (int off = LANES / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, LANES);
    return v;
}

// Eq. 2.1 for device row r: x[perm[r]] = (b[perm[r]] - sum_q val[q] x[col[q]]) / diag[r],
// LANES lanes cooperating on the row, looping over the right-hand sides.
template <typename T, int LANES>
__device__ __forceinline__ void row_solve(const SolveArgs<T> &a, int r, int lane, unsigned mask) {
    const int beg = a.rp[r], end = a.rp[r + 1];
    const int orow = a.perm[r];
    const T dg = a.diag[r];
    for (int j = 0; j < a.nrhs; ++j) {
        const T *xj = a.x + (int64_t)j * a.ldx;
        T acc = T(0);
        for (int q = beg + lane; q < end; q += LANES) acc += a.val[q] * xj[a.col[q]];
        acc = group_sum<T, LANES>(acc, mask);
        if (lane == 0) a.x[orow + (int64_t)j * a.ldx] = (a.b[orow + (int64_t)j * a.ldb] - acc) / dg;
    }
}

// Rows [r0, r1) spread over `nw` warps (this warp is `w`), 32/LANES rows per warp pass.
template <typename T, int LANES>
__device__ __forceinline__ void rows_span(const SolveArgs<T> &a, int r0, int r1, int w, int nw) {
    constexpr int RPW = 32 / LANES;
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    for (int base = r0 + w * RPW; base < r1; base += nw * RPW) {
        const int r = base + grp;
        if (r < r1) row_solve<T, LANES>(a, r, lane, mask);
    }
}

template <typename T, int LANES>
__global__ void __launch_bounds__(1024, 1) k_grid(SolveArgs<T> a) {
    __shared__ int s_flag;
    const int wpb = blockDim.x >> 5;
    const int w_in_b = threadIdx.x >> 5;
    const int gw = blockIdx.x * wpb + w_in_b;
    const int nw = gridDim.x * wpb;
    unsigned long long target = 0;
    for (int s = 0; s < a.S; ++s) {
        const int b0 = a.step_blk[s], b1 = a.step_blk[s + 1];
        if (b1 - b0 == 1 && a.blk_phase[b0 + 1] - a.blk_phase[b0] == 1) {
            const int q = a.blk_phase[b0];
            rows_span<T, LANES>(a, a.phase_row[q], a.phase_row[q + 1], gw, nw);
        } else {
            for (int blk = b0 + blockIdx.x; blk < b1; blk += gridDim.x) {
                const int q1 = a.blk_phase[blk + 1];
                for (int q = a.blk_phase[blk]; q < q1; ++q) {
                    rows_span<T, LANES>(a, a.phase_row[q], a.phase_row[q + 1], w_in_b, wpb);
                    __syncthreads();
                }
            }
        }
        if (s + 1 < a.S) {
            target += gridDim.x;
            if (!grid_barrier(a.ctl, target, a.timeout_ns, &s_flag)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->barriers = a.S > 0 ? a.S - 1 : 0;
}

template <typename T, int LANES>
__global__ void __launch_bounds__(1024, 1) k_cta(SolveArgs<T> a) {
    const int wpb = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    for (int s = 0; s < a.S; ++s) {
        const int b1 = a.step_blk[s + 1];
        for (int blk = a.step_blk[s]; blk < b1; ++blk) {
            const int q1 = a.blk_phase[blk + 1];
            for (int q = a.blk_phase[blk]; q < q1; ++q) {
                rows_span<T, LANES>(a, a.phase_row[q], a.phase_row[q + 1], w, wpb);
                __syncthreads();
            }
        }
    }
}

// Per-row ready flags.  Rows are dealt to (warp, group) slots round-robin in
// device order; each slot handles its rows in increasing order, so the
// smallest unfinished row always has its parents done and its owner at it:
// with every block co-resident the walk cannot deadlock.  Groups use their
// own shuffle masks so one group's wait never stalls another's reduction.
template <typename T, int LANES>
__global__ void __launch_bounds__(1024, 1) k_flags(SolveArgs<T> a) {
    constexpr int RPW = 32 / LANES;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int nw = gridDim.x * wpb;
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    unsigned long long waits = 0;
    bool alive = true;
    for (int base = gw * RPW; base < a.n && alive; base += nw * RPW) {
        const int r = base + grp;
        if (r >= a.n) break;
        const int beg = a.rp[r], end = a.rp[r + 1];
        // wait for this lane's parents
        for (int q = beg + lane; q < end; q += LANES) {
            const uint32_t *f = a.flags + a.col[q];
            if (ld_acquire(f) != a.epoch) {
                ++waits;
                const long long t0 = gtimer();
                unsigned spins = 0;
                while (ld_acquire(f) != a.epoch) {
                    if ((++spins & 63u) == 1) {
                        if (ld_status(a.ctl) != 0) { alive = false; break; }
                        if (gtimer() - t0 > a.timeout_ns) {
                            raise_status(a.ctl, SPTRSV_ERR_TIMEOUT);
                            alive = false;
                            break;
                        }
                    }
                }
                if (!alive) break;
            }
        }
        // all lanes of the group must agree before the reduction
        alive = __all_sync(mask, alive);
        if (!alive) break;
        const int orow = a.perm[r];
        const T dg = a.diag[r];
        for (int j = 0; j < a.nrhs; ++j) {
            const T *xj = a.x + (int64_t)j * a.ldx;
            T acc = T(0);
            for (int q = beg + lane; q < end; q += LANES) acc += a.val[q] * xj[a.col[q]];
            acc = group_sum<T, LANES>(acc, mask);
            if (lane == 0) a.x[orow + (int64_t)j * a.ldx] = (a.b[orow + (int64_t)j * a.ldb] - acc) / dg;
        }
        if (lane == 0) st_release(a.flags + orow, a.epoch);
        __syncwarp(mask);
    }
    if (waits) atomicAdd(&a.ctl->flag_waits, waits);
}

}  // namespace sptrsv
