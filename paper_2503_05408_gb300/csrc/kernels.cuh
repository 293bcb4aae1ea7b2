// Device kernels of the superstep-scheduled forward substitution (Eq. 2.1).
//
// The factor is stored in "device order": superstep-contiguous (Sec. 5),
// and inside a superstep grouped by block (core) and phase (depth among
// same-block parents).  Column ids stay ORIGINAL row ids, so every gather
// reads x in original order directly and every row writes its result to
// x[perm[r]]: no un-permute pass.
//
// The executors:
//  * k_walk<GRID>  persistent grid; every warp of the grid takes a share of a
//             superstep's rows, one grid-wide barrier separates supersteps
//             (Sec. 2.2 BSP model).  k_blocks: a superstep with several blocks
//             gives each block to one thread block (the paper's core), which
//             steps through its phases with __syncthreads.
//  * k_flags  persistent grid without barriers: rows are dealt to warps in
//             device order and every row polls its parents' values (x starts
//             as an all-ones NaN; a published value is the ready signal).
//  * k_local  persistent grid, rows partitioned over the blocks for locality;
//             parents of the same block are polled in shared memory.
//  * k_chunks the block-local partition with one row per lane: a block's rows
//             are cut into chunks of up to 32 rows of one wavefront, each
//             chunk is one warp's unit of work and its FP64 arithmetic runs
//             as full-warp instructions (sliced ELL entries, coalesced).
//  * k_stage / k_walk<CTA>  one thread block walks all supersteps, phases
//             separated by __syncthreads, the phases staged by bulk copies
//             (small factors; also the batched executor's unit).
// Right-hand-side tiles may run on internal row-major copies of b and x
// (k_to_rows / k_to_cols change the layout at the ends).
//
// Every wait is bounded (%globaltimer); on expiry the kernel records
// SPTRSV_ERR_TIMEOUT in the status word and returns - it never traps.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstring>

#include "sptrsv.h"

namespace sptrsv {

constexpr int kMaxSweeps = 16;        // refinement sweeps tracked in the control block

struct Ctl {                         // per-plan control block in device memory
    unsigned long long barrier;      // grid barrier arrivals (zeroed per launch)
    unsigned long long barriers;     // barriers completed (written by block 0)
    unsigned long long flag_waits;   // polled gathers that had to spin
    unsigned long long cursor;       // spare work cursor
    // refinement, per sweep t: max |d_t|, max |x_{t+1}|, max |r_t| (non-negative
    // doubles stored as their bit patterns, which order like unsigned integers)
    unsigned long long dmax[kMaxSweeps], xmax[kMaxSweeps], rmax[kMaxSweeps + 1];
    unsigned long long bmax;         // max |b|
    int32_t done;                    // refinement converged: later kernels return at once
    int32_t last_solve;              // index of the last FP32 sweep that ran
    int32_t conv;                    // 1: correction test met, 2: backward-error test met
    int32_t pad0;
    int32_t status;                  // 0 or SPTRSV_ERR_*; kept across launches until read
    int32_t pad[7];
};

template <typename T>
struct SolveArgs {
    int32_t n, S, nrhs;
    const int32_t *__restrict__ rp;
    const int32_t *__restrict__ col;
    const T *__restrict__ val;       // off-diagonal values scaled by 1 / diagonal
    const T *__restrict__ dinv;      // reciprocal of the diagonal (scales b)
    const int32_t *__restrict__ perm;
    const int32_t *__restrict__ step_blk;
    const int32_t *__restrict__ blk_phase;
    const int32_t *__restrict__ phase_row;
    const int32_t *__restrict__ blk_row;   // block-local executor: rows of thread block b
                                           // (chunked executor: its chunks)
    const int4 *__restrict__ chunk;        // chunked executor: per chunk {entry offset, width, rows, first slot}
    T *bdc;                                // chunked executor: b_i / A_ii in chunk-lane order (plan workspace)
    const T *b;
    T *x;
    int64_t ldb, ldx;
    int64_t brs, xrs;   // row strides of b and x: 1 = column-major; nrhs = row-major (tiles only)
    Ctl *ctl;
    uint32_t *flags;
    uint32_t epoch;
    long long timeout_ns;
    // FP32 correction sweeps of the refinement (refine != 0, T = float): the
    // solved value is the correction d; its epilogue applies x64 += d in FP64
    // (refine == 1: first sweep, x64 = d) and tracks max |d| and max |x64|.
    int32_t refine, sweep;
    double *x64;
    int64_t ldx64, x64rs;   // column and row strides of x64
    double rtol, lnorm;              // backward-error test: r <= rtol * (lnorm |x| + |b|)
};

__host__ __device__ __forceinline__ double bits_to_d(unsigned long long u) {
    double d;
    memcpy(&d, &u, sizeof(d));
    return d;
}

// Skip test at the start of a correction sweep: already converged, failed, or
// the residual of the current iterate passes the backward-error test.
template <typename T>
__device__ __forceinline__ bool refine_skip(const SolveArgs<T> &a) {
    if (!a.refine) return false;
    const volatile Ctl *c = a.ctl;
    if (c->done || c->status) return true;
    if (a.sweep > 0) {
        const double r = bits_to_d(c->rmax[a.sweep]);
        const double x = bits_to_d(c->xmax[a.sweep - 1]);
        const double b = bits_to_d(c->bmax);
        if (r <= a.rtol * (a.lnorm * x + b)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.ctl->done = 1;
                a.ctl->conv = 2;
            }
            return true;
        }
    }
    return false;
}

// Epilogue of a correction: x64 += d in FP64 (lane 0 of the row's group).
// The running maxima compare bit patterns of non-negative doubles as integers
// (same order), keeping FP64-pipe work to the conversion and the update.
__device__ __forceinline__ double max_abs_bits(double m, double v) {
    const unsigned long long a = __double_as_longlong(m), b = __double_as_longlong(v) & 0x7fffffffffffffffULL;
    return __longlong_as_double(a > b ? a : b);
}

template <typename T>
__device__ __forceinline__ void refine_apply(const SolveArgs<T> &a, int orow, int j, T d, double &dm, double &xm) {
    double *px = a.x64 + (int64_t)orow * a.x64rs + (int64_t)j * a.ldx64;
    const double dd = double(d);
    const double xn = (a.refine == 1 ? 0.0 : *px) + dd;
    *px = xn;
    dm = max_abs_bits(dm, dd);
    xm = max_abs_bits(xm, xn);
}

// Block-reduce the per-thread maxima and fold them into the sweep's slots.
__device__ __forceinline__ void refine_flush(Ctl *ctl, int sweep, double dm, double xm) {
    __shared__ double s_d[32], s_x[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, off));
        xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, off));
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_d[w] = dm;
        s_x[w] = xm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < nw; ++i) {
            dm = fmax(dm, s_d[i]);
            xm = fmax(xm, s_x[i]);
        }
        dm = fmax(dm, s_d[0]);
        xm = fmax(xm, s_x[0]);
        atomicMax(&ctl->dmax[sweep], (unsigned long long)__double_as_longlong(dm));
        atomicMax(&ctl->xmax[sweep], (unsigned long long)__double_as_longlong(xm));
        if (blockIdx.x == 0) ctl->last_solve = sweep;
    }
}

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
    __syncthreads();                 // the block's writes happen-before thread 0's release
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(&ctl->barrier) : "memory");
        int ok = 1;
        const long long t0 = gtimer();
        unsigned spins = 0;
        while (ld_acquire(&ctl->barrier) < target) {   // acquire: later reads see every block's writes
            if ((++spins & 63u) == 1) {
                if (ld_status(ctl) != 0) { ok = 0; break; }
                if (gtimer() - t0 > timeout_ns) { raise_status(ctl, SPTRSV_ERR_TIMEOUT); ok = 0; break; }
            }
        }
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

// Sum over the first `width` lanes of the group only (lanes >= width hold zeros):
// ceil(log2(width)) shuffle steps instead of log2(LANES) on the critical path.
template <typename T, int LANES>
__device__ __forceinline__ T group_sum_width(T v, unsigned mask, int width) {
#pragma unroll
    for (int off = LANES / 2; off > 0; off >>= 1)
        if (off < width) v += __shfl_xor_sync(mask, v, off, LANES);
    return v;
}

// Lanes of every LANES-wide group of the warp in which no lane is set in
// `blocking` (a warp-uniform mask): bit 0 of each group collects the OR of its
// group, then the group leaders' bits are spread back over their groups.
template <int LANES>
__device__ __forceinline__ unsigned groups_clear(unsigned blocking) {
    unsigned m = blocking;
#pragma unroll
    for (int s = 1; s < LANES; s <<= 1) m |= m >> s;
    unsigned lead = 0;
#pragma unroll
    for (int g = 0; g < 32; g += LANES) lead |= 1u << g;
    lead &= ~m;
    if constexpr (LANES == 32) return lead ? 0xffffffffu : 0u;
    else return lead * ((1u << LANES) - 1u);
}

// Eq. 2.1 for device row r: x[perm[r]] = (b[perm[r]] - sum_q val[q] x[col[q]]) / diag[r],
// LANES lanes cooperating on the row, looping over the right-hand sides.
template <typename T, int LANES>
__device__ __forceinline__ void row_solve(const SolveArgs<T> &a, int r, int lane, unsigned mask, double &dm,
                                          double &xm) {
    const int beg = a.rp[r], end = a.rp[r + 1];
    const int orow = a.perm[r];
    const T dv = a.dinv[r];
    for (int j = 0; j < a.nrhs; ++j) {
        const T *xj = a.x + (int64_t)j * a.ldx;
        T acc = T(0);
        for (int q = beg + lane; q < end; q += LANES) acc += a.val[q] * xj[a.col[q]];
        acc = group_sum<T, LANES>(acc, mask);
        if (lane == 0) {
            const T y = a.b[orow + (int64_t)j * a.ldb] * dv - acc;
            a.x[orow + (int64_t)j * a.ldx] = y;
            if (a.refine) refine_apply(a, orow, j, y, dm, xm);
        }
    }
}

// Rows [r0, r1) spread over `nw` warps (this warp is `w`), 32/LANES rows per warp pass.
template <typename T, int LANES>
__device__ __forceinline__ void rows_span(const SolveArgs<T> &a, int r0, int r1, int w, int nw, double &dm,
                                          double &xm) {
    constexpr int RPW = 32 / LANES;
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    for (int base = r0 + w * RPW; base < r1; base += nw * RPW) {
        const int r = base + grp;
        if (r < r1) row_solve<T, LANES>(a, r, lane, mask, dm, xm);
    }
}

// ----------------------------------------------------------------------------
// Row registers and the value-polling protocol.
//
// Rows are pre-scaled by the analysis: the device keeps v'_ij = A_ij / A_ii and
// 1 / A_ii, so Eq. 2.1 becomes x_i = b_i / A_ii - sum_j v'_ij x_j: one FMA per
// parent and no division or trailing multiply on the dependency chain (FP64
// arithmetic has long latency on this part, so the chain is kept short).
//
// A row's structure (row pointers, original id, diagonal, right-hand side,
// columns and values) does not depend on x, so every executor loads it ahead
// of time into registers; only the gathers of x sit on the dependency chain.
//
// Ready values: before a polled solve the output x is filled with an all-ones
// NaN (SENTINEL).  A producer publishes x[i] with one relaxed 4/8-byte store
// (a computed value that happens to equal SENTINEL is replaced by the
// canonical NaN), and a consumer polls x[c] itself with relaxed loads until it
// differs from SENTINEL.  Aligned 4/8-byte accesses are single-copy atomic, so
// the polled value IS the result: one round trip per dependency hop, no flag
// array, no fences.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ bool is_sentinel(T v);
template <>
__device__ __forceinline__ bool is_sentinel<double>(double v) { return __double_as_longlong(v) == -1LL; }
template <>
__device__ __forceinline__ bool is_sentinel<float>(float v) { return __float_as_int(v) == -1; }

template <typename T>
__device__ __forceinline__ T all_ones();
template <>
__device__ __forceinline__ double all_ones<double>() { return __longlong_as_double(-1LL); }
template <>
__device__ __forceinline__ float all_ones<float>() { return __int_as_float(-1); }

template <typename T>
__device__ __forceinline__ T publishable(T v) {
    return is_sentinel(v) ? T(__int_as_float(0x7fc00000)) : v;
}

__device__ __forceinline__ double ld_poll(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float ld_poll(const float *p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
// Prefetch loads pinned where they are written: the compiler may otherwise sink
// a read-only load to its use (re-issuing it instead of holding the register),
// which puts a DRAM round trip on the dependency chain.  ld_pin_nc for data that
// no thread writes during the kernel, ld_pin for data this block wrote earlier.
__device__ __forceinline__ int ld_pin_nc(const int *p) {
    int v;
    asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_pin_nc(const float *p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_pin_nc(const double *p) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int4 ld_pin_nc(const int4 *p) {
    int4 v;
    asm volatile("ld.global.nc.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_pin(const float *p) {
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double ld_pin(const double *p) {
    double v;
    asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_pub(double *p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_pub(float *p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}


template <typename T, int U>
struct RowRegs {
    int beg, end, orow;
    T dinv;
    T b0;          // right-hand side of column 0 (lane 0), prefetched with the entries
    int c[U];
    T v[U];
};

template <typename T, int U>
__device__ __forceinline__ void load_meta(const SolveArgs<T> &a, int r, RowRegs<T, U> &m) {
    m.beg = __ldg(a.rp + r);
    m.end = __ldg(a.rp + r + 1);
    m.orow = __ldg(a.perm + r);
    m.dinv = __ldg(a.dinv + r);
}

// The scaled right-hand side b_i / A_ii of column 0 (lane 0 of the group)
template <typename T, int U>
__device__ __forceinline__ T scaled_b0(const SolveArgs<T> &, const RowRegs<T, U> &m) {
    return m.b0 * m.dinv;
}

// RP (right-hand-side parallel tile): every lane of the group holds the same U
// entries (broadcast loads) and lane l works on right-hand sides l, l+LANES, ...
// Otherwise lanes split the row's entries and one lane owns the result.
template <typename T, int LANES, int U, bool RP = false>
__device__ __forceinline__ void load_entries(const SolveArgs<T> &a, int lane, RowRegs<T, U> &m) {
    if constexpr (RP) m.b0 = (lane < a.nrhs) ? a.b[(int64_t)m.orow * a.brs + (int64_t)lane * a.ldb] : T(0);
    else m.b0 = (lane == 0) ? a.b[m.orow] : T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int q = RP ? m.beg + u : m.beg + lane + u * LANES;
        if (q < m.end) {
            m.c[u] = __ldg(a.col + q);
            m.v[u] = __ldg(a.val + q);
        } else {
            m.c[u] = -1;
            m.v[u] = T(0);
        }
    }
}

// Spin until *p is no longer SENTINEL; bounded by the status word and the timeout.
template <typename T>
__device__ __forceinline__ bool poll_wait(const T *p, T &v, const SolveArgs<T> &a, unsigned long long &waits) {
    ++waits;
    const long long t0 = gtimer();
    unsigned spins = 0;
    do {
        v = ld_poll(p);
        if (!is_sentinel(v)) return true;
        if ((++spins & 63u) == 1) {
            if (ld_status(a.ctl) != 0) return false;
            if (gtimer() - t0 > a.timeout_ns) {
                raise_status(a.ctl, SPTRSV_ERR_TIMEOUT);
                return false;
            }
        }
    } while (true);
}

// One row (Eq. 2.1) from registers.  MODE 0: gathers are plain loads (every
// parent is finished, separated by a barrier); MODE 1: polled gathers; MODE 2:
// gathers from the shared-memory ring `xs` (slot = original id & wmask).
// Returns false if a bounded wait failed.
template <typename T, int LANES, int U, int MODE>
__device__ __forceinline__ bool row_exec_rp(const SolveArgs<T> &a, const RowRegs<T, U> &m, int lane,
                                            unsigned mask, T *xs, int win, unsigned long long &waits,
                                            double &dm, double &xm) {
    bool ok = true;
    for (int j = lane; j < a.nrhs && ok; j += LANES) {
        const T *xj = a.x + (int64_t)j * a.ldx;
        const T bj = (j == lane) ? m.b0 : a.b[(int64_t)m.orow * a.brs + (int64_t)j * a.ldb];
        T xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (m.c[u] >= 0) {
                if constexpr (MODE == 2) xv[u] = xs[(m.c[u] & (win - 1)) + j * win];
                else if constexpr (MODE == 1) xv[u] = ld_poll(xj + (int64_t)m.c[u] * a.xrs);
                else xv[u] = xj[(int64_t)m.c[u] * a.xrs];
            } else {
                xv[u] = T(0);
            }
        }
        if constexpr (MODE == 1) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok && m.c[u] >= 0 && is_sentinel(xv[u]))
                    ok = poll_wait(xj + (int64_t)m.c[u] * a.xrs, xv[u], a, waits);
        }
        T acc = bj * m.dinv;
        // the group shares the row's entries, so `cnt` is uniform: FP64 instructions
        // (whole-warp pipe cost) are issued for the row's entries only
        const int cnt = m.end - m.beg;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u >= cnt) break;
            acc -= m.v[u] * xv[u];
        }
        for (int q = m.beg + U; ok && q < m.end; ++q) {
            const int c = __ldg(a.col + q);
            T xc;
            if constexpr (MODE == 2) xc = xs[(c & (win - 1)) + j * win];
            else if constexpr (MODE == 1) {
                xc = ld_poll(xj + (int64_t)c * a.xrs);
                if (is_sentinel(xc)) ok = poll_wait(xj + (int64_t)c * a.xrs, xc, a, waits);
            } else xc = xj[(int64_t)c * a.xrs];
            acc -= __ldg(a.val + q) * xc;
        }
        if (!ok) break;
        const T y = acc;
        T *dst = a.x + (int64_t)m.orow * a.xrs + (int64_t)j * a.ldx;
        if constexpr (MODE == 1) st_pub(dst, publishable(y));
        else *dst = y;
        if constexpr (MODE == 2) xs[(m.orow & (win - 1)) + j * win] = y;
        if (a.refine) refine_apply(a, m.orow, j, y, dm, xm);
    }
    if constexpr (MODE == 1) return __all_sync(mask, ok);
    return true;
}

template <typename T, int LANES, int U, int MODE, bool RP = false>
__device__ __forceinline__ bool row_exec(const SolveArgs<T> &a, const RowRegs<T, U> &m, int lane,
                                         unsigned mask, T *xs, int win, unsigned long long &waits,
                                         double &dm, double &xm) {
    if constexpr (RP) return row_exec_rp<T, LANES, U, MODE>(a, m, lane, mask, xs, win, waits, dm, xm);
    bool ok = true;
    for (int j = 0; j < a.nrhs; ++j) {
        const T *xj = a.x + (int64_t)j * a.ldx;
        const T bj = (lane != 0) ? T(0) : (j == 0 ? m.b0 : a.b[m.orow + (int64_t)j * a.ldb]);
        T xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (m.c[u] >= 0) {
                if constexpr (MODE == 2) xv[u] = xs[(m.c[u] & (win - 1)) + j * win];
                else if constexpr (MODE == 1) xv[u] = ld_poll(xj + m.c[u]);
                else xv[u] = xj[m.c[u]];
            } else {
                xv[u] = T(0);
            }
        }
        // lane 0 carries the scaled right-hand side, every lane subtracts its parents
        T acc = (lane == 0) ? bj * m.dinv : T(0);
        if constexpr (MODE == 1) {
            // accumulate each parent as soon as its value lands: after the last
            // arrival only one FMA remains on the dependency chain (the order, and so
            // the last-bit rounding, follows arrival order)
            unsigned pend = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (m.c[u] >= 0) {
                    if (is_sentinel(xv[u])) pend |= 1u << u;
                    else acc -= m.v[u] * xv[u];
                }
            }
            if (pend) {
                ++waits;
                long long t0 = 0;
                unsigned spins = 0;
                while (pend) {
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (pend & (1u << u)) xv[u] = ld_poll(xj + m.c[u]);
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if ((pend & (1u << u)) && !is_sentinel(xv[u])) {
                            acc -= m.v[u] * xv[u];
                            pend &= ~(1u << u);
                        }
                    if (pend && (++spins & 63u) == 1) {
                        if (spins == 1) t0 = gtimer();
                        else if (ld_status(a.ctl) != 0) { ok = false; break; }
                        else if (gtimer() - t0 > a.timeout_ns) {
                            raise_status(a.ctl, SPTRSV_ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) acc -= m.v[u] * xv[u];
        }
        // entries beyond the register tile (long rows)
        for (int q = m.beg + lane + U * LANES; ok && q < m.end; q += LANES) {
            const int c = __ldg(a.col + q);
            T xc;
            if constexpr (MODE == 2) xc = xs[(c & (win - 1)) + j * win];
            else if constexpr (MODE == 1) {
                xc = ld_poll(xj + c);
                if (is_sentinel(xc)) ok = poll_wait(xj + c, xc, a, waits);
            } else xc = xj[c];
            acc -= __ldg(a.val + q) * xc;
        }
        if constexpr (MODE == 1) {
            if (!__all_sync(mask, ok)) return false;
        }
        acc = group_sum_width<T, LANES>(acc, mask, m.end - m.beg + 1);
        if (lane == 0) {
            const T y = acc;
            T *dst = a.x + m.orow + (int64_t)j * a.ldx;
            if constexpr (MODE == 1) st_pub(dst, publishable(y));
            else *dst = y;
            if constexpr (MODE == 2) xs[(m.orow & (win - 1)) + j * win] = y;
            if (a.refine) refine_apply(a, m.orow, j, y, dm, xm);
        }
    }
    return true;
}

// ----------------------------------------------------------------------------
// Polled row, entry-split lanes, driven by a warp-uniform loop.  Every group of
// the warp publishes its row in the poll round in which its last parent
// arrives, independently of the other groups: a warp holding 32/LANES rows
// never makes a finished row wait for a slower sibling.  `has_row` is false for
// groups past the end of the factor; they only take part in the votes.
//
// PRE (eager group sum): while a row waits, each poll round also reduces the
// group's partial sum (the shuffles overlap the poll loads).  When a single
// lane receives the row's last parents, that lane publishes presum - v*x: one
// FMA after the arrival instead of FMA + log2(width) shuffle-adds.  It pays off
// when a row's last parent arrives alone (rows with parents spread over many
// wavefronts) and costs issue slots when all parents arrive together (stencils).
//
// LOCAL (block-local executor): a column id c <= -2 names a parent owned by
// this thread block, whose value is polled in the block's shared-memory copy
// xs[-c - 2] instead of global memory; -1 marks an empty register slot.  The
// row's own value goes to xs[lrow] before the global store.
// ----------------------------------------------------------------------------
template <bool LOCAL>
__device__ __forceinline__ bool has_entry(int c) { return LOCAL ? c != -1 : c >= 0; }



template <typename T, bool LOCAL>
__device__ __forceinline__ T fetch_polled(const T *xj, const T *xs, int c) {
    if constexpr (LOCAL) {
        if (c < 0) return reinterpret_cast<const volatile T *>(xs)[-c - 2];
    }
    return ld_poll(xj + c);
}

// Entries beyond the register tile (rows longer than U * LANES), consumed in
// order while their values are ready.  Out of line: inlined into the poll loop,
// its column/value loads were hoisted into every poll round.
template <typename T, int LANES, bool PRE, bool LOCAL>
__device__ __noinline__ void tail_step(const SolveArgs<T> &a, const T *xj, const T *xs, int end, int &q, T &acc,
                                       T &ylast, bool &got) {
    while (q < end) {
        const int c = __ldg(a.col + q);
        const T xc = fetch_polled<T, LOCAL>(xj, xs, c);
        if (is_sentinel(xc)) break;
        const T vq = __ldg(a.val + q);
        acc -= vq * xc;
        if constexpr (PRE) {
            ylast -= vq * xc;
            got = true;
        }
        q += LANES;
    }
}

// ----------------------------------------------------------------------------
// One row per warp, lanes split its entries (one right-hand side).  FP64
// instructions are few and late: on this part a warp-wide FP64 instruction
// holds the SM's FP64 pipe for about 19 cycles however few lanes are active, so
// the parents' values are collected first (integer tests only) and the row is
// finished with one FMA per lane and the group reduction.
//   publish_row: shared-memory copy (block-local executor), then the global value.
// ----------------------------------------------------------------------------
template <typename T, bool LOCAL>
__device__ __forceinline__ void publish_row(const SolveArgs<T> &a, int orow, T y, T *xs, int lrow, double &dm,
                                            double &xm) {
    if constexpr (LOCAL) reinterpret_cast<volatile T *>(xs)[lrow] = publishable(y);
    st_pub(a.x + orow, publishable(y));
    if (a.refine) refine_apply(a, orow, 0, y, dm, xm);
}

// Bounded-wait bookkeeping shared by the polled loops: every 64 rounds, give up
// if another block recorded an error or the wait exceeded the limit.  The
// clock starts at the 64th round, not the first: most waits end within a few
// rounds, and a timer read at their start would sit on the dependency chain.
__device__ __forceinline__ bool wait_ok(const Ctl *ctl, long long timeout_ns, unsigned &spins, long long &t0,
                                        int lane) {
    if ((++spins & 63u) != 0) return true;
    if (spins == 64) {
        t0 = gtimer();
        return true;
    }
    const bool expired = gtimer() - t0 > timeout_ns;
    if (__any_sync(0xffffffffu, ld_status(ctl) != 0 || expired)) {
        if (expired && lane == 0) raise_status(const_cast<Ctl *>(ctl), SPTRSV_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// Polled form (flags executor, and the block-local executor without row
// barriers): every pending parent is polled each round.  PRE: once a single
// lane still waits, the others' sum is reduced; when its value lands that lane
// publishes presum - v*x without the reduction.
template <typename T, bool PRE, bool LOCAL>
__device__ __forceinline__ bool row_exec_lean(const SolveArgs<T> &a, const RowRegs<T, 1> &m, bool has_row, int lane,
                                              unsigned long long &waits, double &dm, double &xm, T *xs, int lrow) {
    constexpr unsigned kAll = 0xffffffffu;
    int width = has_row ? m.end - m.beg + 1 : 1;
    width = __reduce_max_sync(kAll, width);
    const int c = m.c[0];
    T acc = (has_row && lane == 0) ? scaled_b0(a, m) : T(0);
    T x = T(0);
    bool pend = false;
    int q = has_row ? m.beg + lane + 32 : 0;
    bool tail = has_row && q < m.end;
    if (has_row && has_entry<LOCAL>(c)) {
        x = fetch_polled<T, LOCAL>(a.x, xs, c);
        pend = is_sentinel(x);
        if (pend) ++waits;
    }
    bool single = false, last = false;
    T presum = T(0);
    unsigned spins = 0;
    long long t0 = 0;
    while (__any_sync(kAll, pend || tail)) {
        if constexpr (PRE) {
            if (!single) {
                const unsigned pl = __ballot_sync(kAll, pend || tail);
                if (__popc(pl) == 1 && !__any_sync(kAll, tail)) {
                    // reduce everything but the last outstanding parent while it is awaited
                    const T part = pend ? acc : acc - m.v[0] * x;
                    presum = group_sum_width<T, 32>(part, kAll, width);
                    single = true;
                    last = pend;
                }
            }
        }
        if (pend) {
            const T t = fetch_polled<T, LOCAL>(a.x, xs, c);
            if (!is_sentinel(t)) {
                x = t;
                pend = false;
            }
        } else if (tail) {
            T unused = T(0);
            bool g = false;
            tail_step<T, 32, false, LOCAL>(a, a.x, xs, m.end, q, acc, unused, g);
            tail = q < m.end;
        }
        if (!wait_ok(a.ctl, a.timeout_ns, spins, t0, lane)) return false;
    }
    if (!has_row) return true;
    if (single) {
        if (last) publish_row<T, LOCAL>(a, m.orow, presum - m.v[0] * x, xs, lrow, dm, xm);
    } else {
        const T y = group_sum_width<T, 32>(acc - m.v[0] * x, kAll, width);
        if (lane == 0) publish_row<T, LOCAL>(a, m.orow, y, xs, lrow, dm, xm);
    }
    return true;
}

template <typename T, int LANES, int U, bool PRE, bool LOCAL = false>
__device__ __forceinline__ bool row_exec_polled(const SolveArgs<T> &a, const RowRegs<T, U> &m, bool has_row,
                                                int lane, unsigned gmask, unsigned long long &waits,
                                                double &dm, double &xm, T *xs = nullptr, int lrow = 0) {
    if constexpr (LANES == 32 && U == 1 && !LOCAL) {
        if (a.nrhs == 1) return row_exec_lean<T, PRE, LOCAL>(a, m, has_row, lane, waits, dm, xm, xs, lrow);
    }
    constexpr unsigned kAll = 0xffffffffu;
    // the widest row of the warp sets the (warp-uniform) shuffle depth
    int width = has_row ? m.end - m.beg + 1 : 1;
    if constexpr (LANES > 1) width = __reduce_max_sync(kAll, width);
    for (int j = 0; j < a.nrhs; ++j) {
        const T *xj = a.x + (int64_t)j * a.ldx;
        T acc = T(0);
        unsigned pend = 0;
        int q = has_row ? m.beg + lane + U * LANES : 0;     // next entry beyond the register tile
        bool tail = has_row && q < m.end;
        if (has_row) {
            if (lane == 0) acc = j == 0 ? scaled_b0(a, m) : a.b[m.orow + (int64_t)j * a.ldb] * m.dinv;
            T xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = has_entry<LOCAL>(m.c[u]) ? fetch_polled<T, LOCAL>(xj, xs, m.c[u]) : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (has_entry<LOCAL>(m.c[u])) {
                    if (is_sentinel(xv[u])) pend |= 1u << u;
                    else acc -= m.v[u] * xv[u];
                }
            }
            if (pend) ++waits;
        }
        if constexpr (LANES == 32) {
            // one row per warp: poll until every parent landed, then reduce and publish
            unsigned spins = 0;
            long long t0 = 0;
            while (__any_sync(kAll, pend != 0 || tail)) {
                if (pend) {
                    T xv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (pend & (1u << u)) xv[u] = fetch_polled<T, LOCAL>(xj, xs, m.c[u]);
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if ((pend & (1u << u)) && !is_sentinel(xv[u])) {
                            acc -= m.v[u] * xv[u];
                            pend &= ~(1u << u);
                        }
                } else if (tail) {
                    T unused = T(0);
                    bool g = false;
                    tail_step<T, LANES, false, LOCAL>(a, xj, xs, m.end, q, acc, unused, g);
                    tail = q < m.end;
                }
                if ((++spins & 63u) == 1) {
                    if (spins == 1) {
                        t0 = gtimer();
                    } else {
                        const bool expired = gtimer() - t0 > a.timeout_ns;
                        if (__any_sync(kAll, ld_status(a.ctl) != 0 || expired)) {
                            if (expired && lane == 0) raise_status(a.ctl, SPTRSV_ERR_TIMEOUT);
                            return false;
                        }
                    }
                }
            }
            if (has_row) {
                const T y = group_sum_width<T, LANES>(acc, kAll, width);
                if (lane == 0) {
                    if constexpr (LOCAL) reinterpret_cast<volatile T *>(xs)[lrow] = publishable(y);
                    st_pub(a.x + m.orow + (int64_t)j * a.ldx, publishable(y));
                    if (a.refine) refine_apply(a, m.orow, j, y, dm, xm);
                }
            }
            continue;
        }
        // warp-uniform bookkeeping: `done` holds the lanes of groups that have
        // published (or hold no row); one vote per poll round
        const int lane32 = threadIdx.x & 31;
        unsigned done = __ballot_sync(kAll, !has_row);
        unsigned spins = 0;
        long long t0 = 0;
        // PRE: `presum` is the group's sum of everything accumulated before the
        // last round (reduced once per round in which values landed, after the
        // round's publications); `ylast` = presum minus this lane's arrivals of
        // the last round, the row's value if this lane alone received some.
        T presum = T(0), ylast = T(0);
        bool got = false, refresh = false;
        if constexpr (PRE && LANES > 1) presum = group_sum_width<T, LANES>(acc, kAll, width);
        // No lane ever blocks inside an iteration: a parent may be a row of this
        // same warp, published only at the vote below.
        while (true) {
            const unsigned busy = __ballot_sync(kAll, pend != 0 || tail);
            const unsigned fin = groups_clear<LANES>(busy | done);    // groups finishing now
            if (fin) {
                const bool mine = (fin >> lane32) & 1u;
                if constexpr (LANES > 1) {
                    bool single = false;
                    T y = acc;
                    if constexpr (PRE) {
                        single = __popc(__ballot_sync(kAll, got) & gmask) == 1;
                        if (__any_sync(kAll, mine && !single)) y = group_sum_width<T, LANES>(y, kAll, width);
                    } else {
                        y = group_sum_width<T, LANES>(y, kAll, width);
                    }
                    if (mine && (single ? got : lane == 0)) {
                        if (single) y = ylast;
                        if constexpr (LOCAL) reinterpret_cast<volatile T *>(xs)[lrow] = publishable(y);
                        st_pub(a.x + m.orow + (int64_t)j * a.ldx, publishable(y));
                        if (a.refine) refine_apply(a, m.orow, j, y, dm, xm);
                    }
                } else {
                    if (mine) {
                        if constexpr (LOCAL) reinterpret_cast<volatile T *>(xs)[lrow] = publishable(acc);
                        st_pub(a.x + m.orow + (int64_t)j * a.ldx, publishable(acc));
                        if (a.refine) refine_apply(a, m.orow, j, acc, dm, xm);
                    }
                }
                done |= fin;
            }
            if constexpr (PRE && LANES > 1) {
                if (refresh) presum = group_sum_width<T, LANES>(acc, kAll, width);
                refresh = false;
            }
            if (busy == 0) break;
            T xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (pend & (1u << u)) xv[u] = fetch_polled<T, LOCAL>(xj, xs, m.c[u]);
            // which parents landed: integer tests only
            unsigned arrived = 0;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if ((pend & (1u << u)) && !is_sentinel(xv[u])) arrived |= 1u << u;
            pend &= ~arrived;
            // An FP64 instruction holds the SM's FP64 pipe for the whole warp however
            // few lanes are active, so a spinning warp issues none: the FP64 work of a
            // round runs only when some lane's value landed.
            const bool landed = __any_sync(kAll, arrived != 0);
            if constexpr (PRE) {
                got = arrived != 0;
                ylast = presum;
            }
            if (landed) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (arrived & (1u << u)) {
                        acc -= m.v[u] * xv[u];
                        if constexpr (PRE) ylast -= m.v[u] * xv[u];
                    }
            }
            if (!pend && tail) {
                tail_step<T, LANES, PRE, LOCAL>(a, xj, xs, m.end, q, acc, ylast, got);
                tail = q < m.end;
            }
            if constexpr (PRE) refresh = __any_sync(kAll, got);
            if ((++spins & 63u) == 1) {                      // warp-uniform bound on the wait
                if (spins == 1) {
                    t0 = gtimer();
                } else {
                    const bool expired = gtimer() - t0 > a.timeout_ns;
                    if (__any_sync(kAll, ld_status(a.ctl) != 0 || expired)) {
                        if (expired && lane == 0) raise_status(a.ctl, SPTRSV_ERR_TIMEOUT);
                        return false;
                    }
                }
            }
        }
    }
    return true;
}

// ----------------------------------------------------------------------------
// Polled executor (SPTRSV_SYNC_FLAGS).  Rows are dealt to groups round-robin
// in device order and each group handles its rows in increasing order: the
// smallest unfinished row always has finished parents and an owner at it, so
// with every block co-resident the walk cannot deadlock.  Two-stage software
// pipeline: metadata two rows ahead, columns/values one row ahead.  Entry-split
// warps advance together (warp-uniform loop, per-group publication); right-hand-
// side tiles run one row per group.
// ----------------------------------------------------------------------------
// FP32 right-hand-side tiles of short rows fit 64 registers: two blocks of 512 per SM.
template <typename T, int LANES, int U, bool RP, bool PRE = false>
__global__ void __launch_bounds__(512, (RP && U <= 4 && sizeof(T) == 4) ? 2 : 1) k_flags(SolveArgs<T> a) {
    constexpr int RPW = 32 / LANES;
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    const int wbase = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW;     // the warp's first row
    const int G = ((gridDim.x * blockDim.x) >> 5) * RPW;
    if (refine_skip(a)) return;
    unsigned long long waits = 0;
    double dm = 0.0, xm = 0.0;
    RowRegs<T, U> cur, nxt, nn;
    int r = wbase + grp;
    if (r < a.n) {
        load_meta(a, r, cur);
        load_entries<T, LANES, U, RP>(a, lane, cur);
    }
    if (r + G < a.n) load_meta(a, r + G, nxt);
    if constexpr (RP) {
        for (; r < a.n; r += G) {
            if (r + 2 * G < a.n) load_meta(a, r + 2 * G, nn);
            if (r + G < a.n) load_entries<T, LANES, U, RP>(a, lane, nxt);
            if (!row_exec<T, LANES, U, 1, RP>(a, cur, lane, mask, nullptr, 0, waits, dm, xm)) break;
            cur = nxt;
            nxt = nn;
        }
    } else {
        for (int rb = wbase; rb < a.n; rb += G) {                                // warp-uniform
            r = rb + grp;
            if (r + 2 * G < a.n) load_meta(a, r + 2 * G, nn);
            if (r + G < a.n) load_entries<T, LANES, U, RP>(a, lane, nxt);
            if (!row_exec_polled<T, LANES, U, PRE>(a, cur, r < a.n, lane, mask, waits, dm, xm)) break;
            cur = nxt;
            nxt = nn;
        }
    }
    if (waits) atomicAdd(&a.ctl->flag_waits, waits);
    if (a.refine) refine_flush(a.ctl, a.sweep, dm, xm);
}

// ----------------------------------------------------------------------------
// Block-local executor (SPTRSV_SYNC_LOCAL).  The plan's rows are partitioned
// over the thread blocks of a persistent grid so that most dependency edges,
// in particular the edge to each row's last-finishing parent, join rows of the
// same block (the locality GrowLocal seeks for CPU cores, Sec. 3).  A block
// keeps the values of all of its rows in shared memory (all-ones NaN until
// written): parents owned by the block are polled there (tens of cycles), the
// others in global memory (an L2 round trip).  Rows are listed per block in
// (wavefront, id) order and dealt round-robin to the block's row groups, so the
// smallest unfinished (wavefront, id) row always has its owner at it: with all
// blocks co-resident (cooperative launch) the walk cannot deadlock.
// ----------------------------------------------------------------------------
template <typename T, int LANES, int U, bool PRE>
__global__ void __launch_bounds__(1024, 1) k_local(SolveArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    constexpr int RPW = 32 / LANES;
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    const int r0 = a.blk_row[blockIdx.x], nr = a.blk_row[blockIdx.x + 1] - r0;
    if (refine_skip(a)) return;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) xs[i] = all_ones<T>();
    __syncthreads();
    unsigned long long waits = 0;
    double dm = 0.0, xm = 0.0;
    const int wbase = (threadIdx.x >> 5) * RPW;                 // the warp's first block row
    const int G = (blockDim.x >> 5) * RPW;
    RowRegs<T, U> cur, nxt, nn;
    int lr = wbase + grp;
    if (lr < nr) {
        load_meta(a, r0 + lr, cur);
        load_entries<T, LANES, U, false>(a, lane, cur);
    }
    if (lr + G < nr) load_meta(a, r0 + lr + G, nxt);
    for (int rb = wbase; rb < nr; rb += G) {                    // warp-uniform
        lr = rb + grp;
        if (lr + 2 * G < nr) load_meta(a, r0 + lr + 2 * G, nn);
        if (lr + G < nr) load_entries<T, LANES, U, false>(a, lane, nxt);
        if (!row_exec_polled<T, LANES, U, PRE, true>(a, cur, lr < nr, lane, mask, waits, dm, xm, xs, lr)) break;
        cur = nxt;
        nxt = nn;
    }
    if (waits) atomicAdd(&a.ctl->flag_waits, waits);
    if (a.refine) refine_flush(a.ctl, a.sweep, dm, xm);
}

// ----------------------------------------------------------------------------
// Chunked block-local executor (SPTRSV_SYNC_CHUNKS).  Same partition as the
// block-local executor (rows of a thread block in (wavefront, id) order, their
// values kept in shared memory), but a warp works on a CHUNK: up to 32 rows of
// one wavefront, one row per lane.  The chunk's entries are stored sliced
// (entry u of lane l at offset + 32 u + l, a coalesced 128/256-byte load per u),
// so a chunk of width U costs U + 1 warp-wide FP64 instructions for up to 32
// rows: on this part a warp FP64 instruction holds the SM's FP64 pipe for about
// 19 cycles however few lanes are active, so packing rows into full warps is
// what lets a wavefront of a few hundred rows per SM finish in a few hundred
// cycles.  A chunk waits until the parents of all its rows have landed
// (integer tests on the polled values only), then runs Eq. 2.1 for every lane
// at once: x_i = b_i / A_ii - sum_u v'_iu x_c(iu).
// Chunks of a block are dealt round-robin to its warps in list order; every
// chunk holds a single wavefront, so the lowest unfinished chunk has finished
// parents and its warp is either at it or at an earlier chunk of the same
// wavefront (which cannot wait): with all blocks co-resident the walk cannot
// deadlock.  Column ids: c >= 0 an original row id polled in global memory,
// c <= -2 the parent in slot -c - 2 of this block's shared memory, -1 an empty
// entry (value 0).
// ----------------------------------------------------------------------------
// info.y packs the chunk's width (entries per lane, low 16 bits) and whether
// any of its entries names a parent of another block (bit 16).
constexpr int kChunkRemote = 1 << 16;
__device__ __forceinline__ int chunk_width(const int4 &info) { return info.y & 0xffff; }

template <typename T, int UMAX>
struct ChunkRegs {
    int4 info;        // entry offset, width | remote flag, rows, first shared-memory slot
    int orow;         // original row of this lane, -1 for none
    T bd;             // b_orow / A_ii (0 for lanes without a row)
    int c[UMAX];
    T v[UMAX];
};

// Two-stage prefetch: the chunk's descriptor and row ids are loaded two chunks
// ahead, its right-hand side and entries (whose addresses need them) one chunk
// ahead, so no load at the top of an iteration waits for another load.
struct ChunkHead {
    int4 info;
    int orow;
};

template <typename T>
__device__ __forceinline__ void chunk_head(const SolveArgs<T> &a, int ck, int lane, ChunkHead &h) {
    h.info = ld_pin_nc(a.chunk + ck);
    h.orow = ld_pin_nc(a.perm + int64_t(ck) * 32 + lane);
}

template <typename T, int UMAX>
__device__ __forceinline__ void chunk_body(const SolveArgs<T> &a, const ChunkHead &h, int ck, int lane,
                                           ChunkRegs<T, UMAX> &m) {
    m.info = h.info;
    m.orow = h.orow;
    m.bd = ld_pin(a.bdc + int64_t(ck) * 32 + lane);   // gathered by this block at launch: no dependent load
    const int width = chunk_width(h.info);
#pragma unroll
    for (int u = 0; u < UMAX; ++u) {
        if (u < width) {
            const int64_t q = int64_t(h.info.x) + int64_t(u) * 32 + lane;
            m.c[u] = ld_pin_nc(a.col + q);
            m.v[u] = ld_pin_nc(a.val + q);
        } else {
            m.c[u] = -1;
            m.v[u] = T(0);
        }
    }
}

template <typename T, int UMAX>
__device__ __forceinline__ void chunk_load(const SolveArgs<T> &a, int ck, int lane, ChunkRegs<T, UMAX> &m) {
    ChunkHead h;
    chunk_head(a, ck, lane, h);
    chunk_body(a, h, ck, lane, m);
}

// Entries u >= UMAX of a wide chunk, one poll loop per entry (rare: the
// autotuner keeps factors with long rows on the other executors).
template <typename T, int UMAX>
__device__ __noinline__ bool chunk_tail(const SolveArgs<T> &a, const ChunkRegs<T, UMAX> &m, int lane, const T *xs,
                                        T &acc) {
    const int width = chunk_width(m.info);
    for (int u = UMAX; u < width; ++u) {
        const int64_t q = int64_t(m.info.x) + int64_t(u) * 32 + lane;
        const int c = __ldg(a.col + q);
        const T v = __ldg(a.val + q);
        T xv = T(0);
        bool pend = false;
        if (c != -1) {
            xv = fetch_polled<T, true>(a.x, xs, c);
            pend = is_sentinel(xv);
        }
        unsigned spins = 0;
        long long t0 = 0;
        while (__any_sync(0xffffffffu, pend)) {
            if (pend) {
                xv = fetch_polled<T, true>(a.x, xs, c);
                pend = is_sentinel(xv);
            }
            if (!wait_ok(a.ctl, a.timeout_ns, spins, t0, lane)) return false;
        }
        acc -= v * xv;
    }
    return true;
}

// A row's entries are stored parents-of-other-blocks first (they usually land
// first: an upstream block runs ahead of its consumers), then the block's own
// parents in column order.  Every parent value is requested at once (global
// loads for other blocks, shared-memory loads for this block); then entry by
// entry, each is awaited if it was still missing - one load per wait-loop
// iteration: measured on GB300, re-testing several pending entries per
// iteration costs 3-4x more cycles per iteration - and folded into the sum
// right away, so only the last parent's FMA follows its arrival.
template <typename T, int UMAX>
__device__ __forceinline__ bool chunk_exec(const SolveArgs<T> &a, const ChunkRegs<T, UMAX> &m, int lane, T *xs,
                                           unsigned long long &waits, double &dm, double &xm) {
    constexpr unsigned kAll = 0xffffffffu;
    const volatile T *vxs = reinterpret_cast<const volatile T *>(xs);
    const int width = chunk_width(m.info);
    const bool remote = (m.info.y & kChunkRemote) != 0;     // warp-uniform
    T xv[UMAX];
#pragma unroll
    for (int u = 0; u < UMAX; ++u) {
        if (remote && m.c[u] >= 0) xv[u] = ld_poll(a.x + m.c[u]);
        else xv[u] = m.c[u] != -1 ? vxs[m.c[u] < -1 ? -m.c[u] - 2 : 0] : T(0);
    }
    T acc = m.bd;
    unsigned spins = 0;
    long long t0 = 0;
    bool waited = false;
#pragma unroll
    for (int u = 0; u < UMAX; ++u) {
        if (u < width) {                  // warp-uniform
            const int c = m.c[u];
            bool pend = c != -1 && is_sentinel(xv[u]);
            if (__any_sync(kAll, pend)) {
                waited = true;
                const bool glob = remote && c >= 0;
                const int slot = c < -1 ? -c - 2 : m.info.w;   // lanes without one read a valid slot
                do {
                    T t;
                    if (glob) t = pend ? ld_poll(a.x + c) : xv[u];
                    else t = vxs[slot];
                    if (pend && !is_sentinel(t)) {
                        xv[u] = t;
                        pend = false;
                    }
                    if (!wait_ok(a.ctl, a.timeout_ns, spins, t0, lane)) return false;
                } while (__any_sync(kAll, pend));
                // The later entries' parents mostly sit in the chunk that just published
                // this one: re-read the still-missing shared-memory ones once, so that
                // they usually need no wait loop of their own.
#pragma unroll
                for (int v = u + 1; v < UMAX; ++v)
                    if (v < width && m.c[v] < -1 && is_sentinel(xv[v]))
                        xv[v] = vxs[-m.c[v] - 2];
            }
            acc -= m.v[u] * xv[u];
        }
    }
    if (waited && lane == 0) ++waits;
    if (width > UMAX && !chunk_tail<T, UMAX>(a, m, lane, xs, acc)) return false;
    if (m.orow >= 0) {
        const T y = publishable(acc);
        reinterpret_cast<volatile T *>(xs)[m.info.w + lane] = y;
        st_pub(a.x + m.orow, y);
        if (a.refine) refine_apply(a, m.orow, 0, acc, dm, xm);
    }
    return true;
}

// Threads per block: a lane keeps its row, the next chunk's row and its parents'
// values in registers (more than the 64 a 1024-thread block allows).  Chunks of
// at most three entries per lane fit 768 threads; more warps per block mean each
// warp takes its next chunk further ahead of that chunk's parents, so the chunk's
// first reads (those of other blocks' parents are L2 round trips) are back before
// its parents land.
template <int UMAX>
constexpr int chunk_threads_max() { return UMAX <= 3 ? 768 : 512; }

template <typename T, int UMAX>
__global__ void __launch_bounds__(chunk_threads_max<UMAX>(), 1) k_chunks(SolveArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c0 = a.blk_row[blockIdx.x], c1 = a.blk_row[blockIdx.x + 1];
    if (refine_skip(a)) return;
    int nslots = 0;
    if (c1 > c0) {
        const int4 last = __ldg(a.chunk + c1 - 1);
        nslots = last.w + last.z;
    }
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) xs[i] = all_ones<T>();
    // b_i / A_ii of this block's rows in chunk-lane order: the gather of b through the
    // row ids (a dependent load) and the multiply run once here, off every step
    for (int64_t q = int64_t(c0) * 32 + threadIdx.x; q < int64_t(c1) * 32; q += blockDim.x) {
        const int orow = __ldg(a.perm + q);
        a.bdc[q] = orow >= 0 ? a.b[orow] * __ldg(a.dinv + q) : T(0);
    }
    __syncthreads();
    unsigned long long waits = 0;
    double dm = 0.0, xm = 0.0;
    ChunkRegs<T, UMAX> cur, nxt;
    ChunkHead h1, h2;
    int ck = c0 + w;
    if (ck < c1) chunk_load(a, ck, lane, cur);
    if (ck + nw < c1) chunk_head(a, ck + nw, lane, h1);
    for (; ck < c1; ck += nw) {                      // warp-uniform
        if (ck + 2 * nw < c1) chunk_head(a, ck + 2 * nw, lane, h2);
        if (ck + nw < c1) chunk_body(a, h1, ck + nw, lane, nxt);
        if (!chunk_exec<T, UMAX>(a, cur, lane, xs, waits, dm, xm)) break;
        cur = nxt;
        h1 = h2;
    }
    if (waits) atomicAdd(&a.ctl->flag_waits, waits);
    if (a.refine) refine_flush(a.ctl, a.sweep, dm, xm);
}

// ----------------------------------------------------------------------------
// One thread block walks every phase of a factor (phases separated by
// __syncthreads).  Shared by the single-block executor and the batched
// executor, where each block walks one independent factor.  Same pipeline as
// the grid walker: e0 executes, m1's entries and m2's metadata are in flight.
// ----------------------------------------------------------------------------
template <typename T, int LANES, int U, bool RING, bool RP>
__device__ __forceinline__ void walk_block(const SolveArgs<T> &a, int nphases, int win, T *xs, double &dm,
                                           double &xm) {
    constexpr int RPW = 32 / LANES;
    constexpr int MODE = RING ? 2 : 0;
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    const int g = (threadIdx.x >> 5) * RPW + grp;
    const int G = (blockDim.x >> 5) * RPW;
    unsigned long long waits = 0;
    auto bound = [&](int i) { return i <= nphases ? __ldg(a.phase_row + i) : a.phase_row[nphases]; };
    int pb0 = bound(0), pb1 = bound(1), pb2 = bound(2), pb3 = bound(3);
    RowRegs<T, U> e0, m1, m2;
    bool h0 = nphases > 0 && pb0 + g < pb1;
    bool h1 = nphases > 1 && pb1 + g < pb2;
    if (h0) {
        load_meta(a, pb0 + g, e0);
        load_entries<T, LANES, U, RP>(a, lane, e0);
    }
    if (h1) load_meta(a, pb1 + g, m1);
    for (int q = 0; q < nphases; ++q) {
        const int pb4 = bound(q + 4);
        const bool h2 = (q + 2 < nphases) && (pb2 + g < pb3);
        if (h2) load_meta(a, pb2 + g, m2);
        if (h1) load_entries<T, LANES, U, RP>(a, lane, m1);
        if (h0) row_exec<T, LANES, U, MODE, RP>(a, e0, lane, mask, xs, win, waits, dm, xm);
        for (int r = pb0 + g + G; r < pb1; r += G) {
            RowRegs<T, U> t;
            load_meta(a, r, t);
            load_entries<T, LANES, U, RP>(a, lane, t);
            row_exec<T, LANES, U, MODE, RP>(a, t, lane, mask, xs, win, waits, dm, xm);
        }
        __syncthreads();
        e0 = m1;
        h0 = h1;
        m1 = m2;
        h1 = h2;
        pb0 = pb1;
        pb1 = pb2;
        pb2 = pb3;
        pb3 = pb4;
    }
}

// ----------------------------------------------------------------------------
// Staged single-block walker.  Each phase's rows are contiguous in device order,
// and so are their row pointers, original ids, reciprocal diagonals, columns,
// values and - after the block has copied b into device order once - their
// right-hand sides.  One elected thread copies those six slices with TMA bulk
// copies (cp.async.bulk, completion counted on an mbarrier) three phases ahead
// into a four-slot shared-memory ring; the phase boundaries it needs arrive
// through a small cp.async FIFO.  A phase then costs one mbarrier wait, the
// rows' arithmetic out of shared memory and one block barrier: no dependent
// global load remains on the chain except the gathers of x when no
// shared-memory x ring is available.  Every wait is bounded; a failed wait
// ends the walk for the whole block.
// ----------------------------------------------------------------------------
struct StageInfo {
    const int32_t *phase_ent;        // entry offset of every phase boundary (rp[phase_row[q]])
    void *bdev;                      // workspace: b in device order, row-major (n x nrhs), 16-byte aligned
    int32_t rows_cap, ents_cap;      // largest phase of the plan
    int32_t slot_bytes;              // bytes of one ring slot (16-byte multiple)
    int32_t off_perm, off_dinv, off_col, off_val, off_b;   // slot layout
};

// Host: slot layout for phases of at most `rows` rows / `ents` entries and nrhs
// right-hand sides of `elem` bytes; returns the slot size.
inline size_t stage_slot_layout(size_t rows, size_t ents, int nrhs, size_t elem, StageInfo &si) {
    auto a16 = [](size_t v) { return (v + 15) & ~size_t(15); };
    size_t off = a16((rows + 8) * 4);                       // row pointers
    si.off_perm = int32_t(off);
    off += a16((rows + 8) * 4);
    si.off_dinv = int32_t(off);
    off += a16((rows + 8) * elem);
    si.off_col = int32_t(off);
    off += a16((ents + 8) * 4);
    si.off_val = int32_t(off);
    off += a16((ents + 8) * elem);
    si.off_b = int32_t(off);
    off += a16((rows * size_t(nrhs) + 8) * elem);
    si.slot_bytes = int32_t(off);
    si.rows_cap = int32_t(rows);
    si.ents_cap = int32_t(ents);
    si.bdev = nullptr;
    return off;
}
// Dynamic shared memory of a staged walk: 4 mbarriers, 4 slots, optional x ring.
inline size_t stage_smem_bytes(const StageInfo &si, size_t ring_bytes) { return 64 + 4 * size_t(si.slot_bytes) + ring_bytes; }

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_4() { asm volatile("cp.async.wait_group 4;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// 16-byte aligned superset [lo, hi) of element range [a, b) for elements of `esz` bytes.
__device__ __forceinline__ int align_lo(int a, int esz) { return a & ~(16 / esz - 1); }
__device__ __forceinline__ int align_hi(int b, int esz) { return (b + 16 / esz - 1) & ~(16 / esz - 1); }

template <typename T>
struct StageSlot {
    int32_t *rp, *perm, *col;
    T *dinv, *val, *b;
    int srp, sperm, sdinv, scol, sval, sb;  // first element of each copied slice
};

template <typename T>
__device__ __forceinline__ StageSlot<T> stage_slot(unsigned char *base, const StageInfo &si, int p0, int e0,
                                                   int nrhs) {
    StageSlot<T> s;
    s.rp = reinterpret_cast<int32_t *>(base);
    s.perm = reinterpret_cast<int32_t *>(base + si.off_perm);
    s.dinv = reinterpret_cast<T *>(base + si.off_dinv);
    s.col = reinterpret_cast<int32_t *>(base + si.off_col);
    s.val = reinterpret_cast<T *>(base + si.off_val);
    s.b = reinterpret_cast<T *>(base + si.off_b);
    s.srp = align_lo(p0, 4);
    s.sperm = align_lo(p0, 4);
    s.sdinv = align_lo(p0, sizeof(T));
    s.scol = align_lo(e0, 4);
    s.sval = align_lo(e0, sizeof(T));
    s.sb = align_lo(p0 * nrhs, sizeof(T));
    return s;
}

// Producer side: bulk-copy phase [p0, p1) with entries [e0, e1) into the slot.
template <typename T>
__device__ __forceinline__ void stage_issue(const SolveArgs<T> &a, unsigned char *base, const StageInfo &si,
                                            uint64_t *bar, int p0, int p1, int e0, int e1) {
    const StageSlot<T> s = stage_slot<T>(base, si, p0, e0, a.nrhs);
    const uint32_t nrp = uint32_t(align_hi(p1 + 1, 4) - s.srp) * 4u;
    const uint32_t nperm = uint32_t(align_hi(p1, 4) - s.sperm) * 4u;
    const uint32_t ndinv = uint32_t(align_hi(p1, sizeof(T)) - s.sdinv) * uint32_t(sizeof(T));
    const uint32_t ncol = e1 > e0 ? uint32_t(align_hi(e1, 4) - s.scol) * 4u : 0u;
    const uint32_t nval = e1 > e0 ? uint32_t(align_hi(e1, sizeof(T)) - s.sval) * uint32_t(sizeof(T)) : 0u;
    const uint32_t nb = uint32_t(align_hi(p1 * a.nrhs, sizeof(T)) - s.sb) * uint32_t(sizeof(T));
    // the slot's previous readers finished before the block barrier that precedes this issue
    mbar_expect_tx(bar, nrp + nperm + ndinv + ncol + nval + nb);
    bulk_g2s(s.rp, a.rp + s.srp, nrp, bar);
    bulk_g2s(s.perm, a.perm + s.sperm, nperm, bar);
    bulk_g2s(s.dinv, a.dinv + s.sdinv, ndinv, bar);
    if (ncol) bulk_g2s(s.col, a.col + s.scol, ncol, bar);
    if (nval) bulk_g2s(s.val, a.val + s.sval, nval, bar);
    bulk_g2s(s.b, static_cast<const T *>(si.bdev) + s.sb, nb, bar);
}

// Bounded wait on a slot's mbarrier; returns false on timeout (status recorded when ctl is set).
template <typename T>
__device__ __forceinline__ bool stage_wait(const SolveArgs<T> &a, uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > (a.timeout_ns > 0 ? a.timeout_ns : 2000000000LL)) {
            if (a.ctl) raise_status(a.ctl, SPTRSV_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// ----------------------------------------------------------------------------
// One thread block with the whole factor resident in shared memory (small
// factors, one right-hand side).  One thread bulk-copies (cp.async.bulk,
// completion counted on an mbarrier) the plan's row pointers, row ids,
// reciprocal diagonals, columns and scaled values into shared memory; the block
// then forms b_i / A_ii and keeps x by original row id.  The first `nact`
// threads (the widest phase, rounded up to a warp) walk the phases one row per
// thread with a barrier of their own between phases, so a step costs a few
// shared-memory loads, the row's FMAs and one small barrier - no global memory
// on the dependency chain.  Regions are 16-byte aligned and rounded up to 16
// bytes (the plan's arrays carry spare bytes past their end); their sum is
// resident_smem_bytes on the host.
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ size_t round16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_resident(SolveArgs<T> a, int nphases, int nact) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    if (refine_skip(a)) return;
    const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
    if (n <= 0) return;
    const int m = __ldg(a.rp + n);
    const uint32_t nb_t = uint32_t(round16(size_t(n) * sizeof(T))), nb_v = uint32_t(round16(size_t(m) * sizeof(T)));
    const uint32_t nb_c = uint32_t(round16(size_t(m) * 4)), nb_r = uint32_t(round16(size_t(n + 1) * 4));
    const uint32_t nb_p = uint32_t(round16(size_t(n) * 4));
    unsigned char *q = smem_raw;
    T *xs = reinterpret_cast<T *>(q);       q += nb_t;      // x by original row id
    T *bd = reinterpret_cast<T *>(q);       q += nb_t;      // 1 / A_ii, then b_i / A_ii, by device row
    T *vs = reinterpret_cast<T *>(q);       q += nb_v;      // A_ij / A_ii
    int *cs = reinterpret_cast<int *>(q);   q += nb_c;      // original column ids
    int *rps = reinterpret_cast<int *>(q);  q += nb_r;      // row pointers (n + 1)
    int *pms = reinterpret_cast<int *>(q);  q += nb_p;      // device row -> original row
    int *phs = reinterpret_cast<int *>(q);                  // phase bounds (nphases + 1)
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(&s_bar, nb_t + (m ? nb_v + nb_c : 0u) + nb_r + nb_p);
        bulk_g2s(bd, a.dinv, nb_t, &s_bar);
        if (m) {
            bulk_g2s(vs, a.val, nb_v, &s_bar);
            bulk_g2s(cs, a.col, nb_c, &s_bar);
        }
        bulk_g2s(rps, a.rp, nb_r, &s_bar);
        bulk_g2s(pms, a.perm, nb_p, &s_bar);
    }
    for (int i = tid; i <= nphases; i += nt) phs[i] = __ldg(a.phase_row + i);
    __syncthreads();                                   // the barrier's initialisation is visible
    const bool ok = stage_wait(a, &s_bar, 0);          // bounded; records a timeout in the status
    if (__syncthreads_or(!ok)) return;
    for (int i = tid; i < n; i += nt) bd[i] = a.b[int64_t(pms[i]) * a.brs] * bd[i];
    __syncthreads();
    if (tid < nact) {
        for (int ph = 0; ph < nphases; ++ph) {
            const int r1 = phs[ph + 1];
            for (int r = phs[ph] + tid; r < r1; r += nact) {
                T acc = bd[r];
                const int q1 = rps[r + 1];
                for (int e = rps[r]; e < q1; ++e) acc -= vs[e] * xs[cs[e]];
                xs[pms[r]] = acc;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(nact) : "memory");   // the walking warps only
        }
    }
    __syncthreads();
    double dm = 0.0, xm = 0.0;
    for (int o = tid; o < n; o += nt) {
        const T y = xs[o];
        a.x[int64_t(o) * a.xrs] = y;
        if (a.refine) refine_apply(a, o, 0, y, dm, xm);
    }
    if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&s_bar)) : "memory");
    if (a.refine) refine_flush(a.ctl, a.sweep, dm, xm);
}

// Rows of one staged phase (MODE 0: x from global, MODE 2: x from the shared ring).
template <typename T, int LANES, int MODE, bool RP>
__device__ __forceinline__ void stage_rows(const SolveArgs<T> &a, const StageSlot<T> &s, int p0, int p1, int g, int G,
                                           int lane, unsigned mask, T *xs, int win, double &dm, double &xm) {
    const int R = a.nrhs;
    for (int lr = g; lr < p1 - p0; lr += G) {
        const int r = p0 + lr;
        const int beg = s.rp[r - s.srp], end = s.rp[r + 1 - s.srp];
        const int orow = s.perm[r - s.sperm];
        const T dv = s.dinv[r - s.sdinv];
        const T *bb = s.b + (r * R - s.sb);
        if constexpr (RP) {
            for (int j = lane; j < R; j += LANES) {
                const T *xj = a.x + (int64_t)j * a.ldx;
                T acc = bb[j] * dv;
                for (int q = beg; q < end; ++q) {
                    const int c = s.col[q - s.scol];
                    const T xc = MODE == 2 ? xs[(c & (win - 1)) + j * win] : xj[c];
                    acc -= s.val[q - s.sval] * xc;
                }
                a.x[orow + (int64_t)j * a.ldx] = acc;
                if constexpr (MODE == 2) xs[(orow & (win - 1)) + j * win] = acc;
                if (a.refine) refine_apply(a, orow, j, acc, dm, xm);
            }
        } else {
            for (int j = 0; j < R; ++j) {
                const T *xj = a.x + (int64_t)j * a.ldx;
                T acc = (lane == 0) ? bb[j] * dv : T(0);
                for (int q = beg + lane; q < end; q += LANES) {
                    const int c = s.col[q - s.scol];
                    const T xc = MODE == 2 ? xs[(c & (win - 1)) + j * win] : xj[c];
                    acc -= s.val[q - s.sval] * xc;
                }
                acc = group_sum_width<T, LANES>(acc, mask, end - beg + 1);
                if (lane == 0) {
                    a.x[orow + (int64_t)j * a.ldx] = acc;
                    if constexpr (MODE == 2) xs[(orow & (win - 1)) + j * win] = acc;
                    if (a.refine) refine_apply(a, orow, j, acc, dm, xm);
                }
            }
        }
    }
}

// smem: [4 mbarriers (64 B)] [4 slots of si.slot_bytes] [x ring of win * nrhs * sizeof(T)]
template <typename T, int LANES, bool RING, bool RP>
__device__ __forceinline__ bool walk_block_staged(const SolveArgs<T> &a, const StageInfo &si, int nphases, int win,
                                                  unsigned char *smem, double &dm, double &xm) {
    constexpr int RPW = 32 / LANES;
    constexpr int MODE = RING ? 2 : 0;
    constexpr int NS = 4, NQ = 8;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    unsigned char *slots = smem + 64;
    T *xs = reinterpret_cast<T *>(slots + NS * si.slot_bytes);
    __shared__ int s_b[NS][4];          // p0, p1, e0, e1 of the phase held by each slot
    __shared__ __align__(16) int s_q[NQ][2];   // producer FIFO: phase_row, phase_ent of future boundaries
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    // the last warp only produces (bulk copies, boundary FIFO) so that its issue
    // work overlaps the other warps' rows instead of delaying a computing warp
    const int nwarps = blockDim.x >> 5;
    const bool producer = (threadIdx.x >> 5) == nwarps - 1;
    const int pthread = (nwarps - 1) * 32;
    const int g = (threadIdx.x >> 5) * RPW + grp;
    const int G = (nwarps - 1) * RPW;
    const int R = a.nrhs;
    // b in device order, row-major, written by this block for the bulk copies (async proxy)
    T *bdev = static_cast<T *>(si.bdev);
    const int n_rows = a.phase_row[nphases];
    for (int i = threadIdx.x; i < n_rows * R; i += blockDim.x) {
        const int r = i / R, j = i - r * R;
        bdev[i] = a.b[__ldg(a.perm + r) + (int64_t)j * a.ldb];
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (threadIdx.x == pthread) {
        for (int i = 0; i < NS; ++i) mbar_init(bars + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == pthread) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        for (int q = 0; q < 3 && q < nphases; ++q) {
            const int p0 = a.phase_row[q], p1 = a.phase_row[q + 1];
            const int e0 = si.phase_ent[q], e1 = si.phase_ent[q + 1];
            s_b[q][0] = p0; s_b[q][1] = p1; s_b[q][2] = e0; s_b[q][3] = e1;
            stage_issue<T>(a, slots + q * si.slot_bytes, si, bars + q, p0, p1, e0, e1);
        }
        // FIFO: boundary i (i = 3 .. 3 + NQ - 1) in entry i % NQ, one cp.async group each
        for (int i = 3; i < 3 + NQ; ++i) {
            if (i <= nphases) {
                cp_async<4>(&s_q[i % NQ][0], a.phase_row + i);
                cp_async<4>(&s_q[i % NQ][1], si.phase_ent + i);
            }
            cp_async_commit();
        }
    }
    __syncthreads();
    // one block barrier per phase: it also carries the readiness of the next slot
    bool ok = nphases == 0 || stage_wait(a, bars, 0);
    bool stop = __syncthreads_or(!ok);
    for (int q = 0; q < nphases && !stop; ++q) {
        const int slot = q & (NS - 1);
        if (producer) {
            // phase q+3 (boundaries q+3, q+4 from the FIFO) into the slot phase q-1
            // released at the last barrier; overlaps the other warps' rows
            if (threadIdx.x == pthread && q + 3 < nphases) {
                cp_async_wait_4();          // boundaries up to q + 4 have landed
                const int sl = (q + 3) & (NS - 1);
                const int p0 = s_q[(q + 3) % NQ][0], e0 = s_q[(q + 3) % NQ][1];
                const int p1 = s_q[(q + 4) % NQ][0], e1 = s_q[(q + 4) % NQ][1];
                s_b[sl][0] = p0; s_b[sl][1] = p1; s_b[sl][2] = e0; s_b[sl][3] = e1;
                stage_issue<T>(a, slots + sl * si.slot_bytes, si, bars + sl, p0, p1, e0, e1);
                const int i = q + 3 + NQ;  // refill the FIFO entry of boundary q + 3
                if (i <= nphases) {
                    cp_async<4>(&s_q[i % NQ][0], a.phase_row + i);
                    cp_async<4>(&s_q[i % NQ][1], si.phase_ent + i);
                }
                cp_async_commit();
            }
        } else {
            const int p0 = s_b[slot][0], p1 = s_b[slot][1];
            const StageSlot<T> s = stage_slot<T>(slots + slot * si.slot_bytes, si, p0, s_b[slot][2], R);
            stage_rows<T, LANES, MODE, RP>(a, s, p0, p1, g, G, lane, mask, xs, win, dm, xm);
        }
        if (q + 1 < nphases) ok = stage_wait(a, bars + ((q + 1) & (NS - 1)), ((q + 1) / NS) & 1);
        stop = __syncthreads_or(!ok);
    }
    if (threadIdx.x == pthread) {
        cp_async_wait_0();
        if (ok)                            // every barrier phase has completed: retire them
            for (int i = 0; i < NS; ++i)
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bars + i)) : "memory");
    }
    __syncthreads();
    return ok;
}

template <typename T, int LANES, bool RING, bool RP>
__global__ void __launch_bounds__(512, 1) k_stage(SolveArgs<T> a, StageInfo si, int nphases, int win) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (refine_skip(a)) return;
    double dm = 0.0, xm = 0.0;
    walk_block_staged<T, LANES, RING, RP>(a, si, nphases, win, smem_raw, dm, xm);
    if (a.refine) refine_flush(a.ctl, a.sweep, dm, xm);
}

// Maximum over the thread block (every thread gets the result).
__device__ __forceinline__ double block_max(double v, double *s_scratch) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    v = s_scratch[0];
    for (int i = 1; i < int(blockDim.x >> 5); ++i) v = fmax(v, s_scratch[i]);
    return v;
}

// ----------------------------------------------------------------------------
// Phase walker for schedules whose supersteps are single wide phases (the
// wavefront schedule) or, with GRID == false, any schedule walked by one
// thread block.  GRID: rows of a phase are spread over every group of the
// grid and a grid barrier separates phases.  CTA: rows of a phase are spread
// over the block's groups, __syncthreads separates phases, and, when `win`
// is non-zero, x is also kept in a shared-memory ring of `win` rows (the host
// proved that no two rows sharing a slot are live at once).  The first row
// each group owns in the next phase is prefetched: metadata at the start of
// the current phase, columns/values before the barrier.
// ----------------------------------------------------------------------------
template <typename T, int LANES, int U, bool GRID, bool RING, bool RP>
__global__ void __launch_bounds__(512, 1) k_walk(SolveArgs<T> a, int nphases, int win) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    __shared__ int s_flag;
    if (refine_skip(a)) return;
    constexpr int RPW = 32 / LANES;
    constexpr int MODE = RING ? 2 : 0;
    const int lane32 = threadIdx.x & 31;
    const int grp = lane32 / LANES, lane = lane32 % LANES;
    const unsigned mask = group_mask<LANES>(lane32);
    const int wid = GRID ? ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) : (threadIdx.x >> 5);
    const int g = wid * RPW + grp;
    const int G = ((GRID ? gridDim.x * blockDim.x : blockDim.x) >> 5) * RPW;
    unsigned long long waits = 0, target = 0;
    double dm = 0.0, xm = 0.0;
    // Three-stage pipeline over this group's first row of each phase:
    //   e0 - phase q:   entries in registers, executed now
    //   m1 - phase q+1: metadata arrived; its entries are requested during phase q
    //   m2 - phase q+2: metadata requested during phase q
    // Phase boundaries run one phase further ahead (pb3 is known at phase q).
    auto bound = [&](int i) { return i <= nphases ? __ldg(a.phase_row + i) : a.phase_row[nphases]; };
    int pb0 = bound(0), pb1 = bound(1), pb2 = bound(2), pb3 = bound(3);
    RowRegs<T, U> e0, m1, m2;
    bool h0 = nphases > 0 && pb0 + g < pb1;
    bool h1 = nphases > 1 && pb1 + g < pb2;
    if (h0) {
        load_meta(a, pb0 + g, e0);
        load_entries<T, LANES, U, RP>(a, lane, e0);
    }
    if (h1) load_meta(a, pb1 + g, m1);
    for (int q = 0; q < nphases; ++q) {
        const int pb4 = bound(q + 4);
        const bool h2 = (q + 2 < nphases) && (pb2 + g < pb3);
        if (h2) load_meta(a, pb2 + g, m2);
        if (h1) load_entries<T, LANES, U, RP>(a, lane, m1);
        if (h0) row_exec<T, LANES, U, MODE, RP>(a, e0, lane, mask, xs, win, waits, dm, xm);
        for (int r = pb0 + g + G; r < pb1; r += G) {          // rows beyond the first per group
            RowRegs<T, U> t;
            load_meta(a, r, t);
            load_entries<T, LANES, U, RP>(a, lane, t);
            row_exec<T, LANES, U, MODE, RP>(a, t, lane, mask, xs, win, waits, dm, xm);
        }
        if (q + 1 < nphases) {
            if constexpr (GRID) {
                target += gridDim.x;
                if (!grid_barrier(a.ctl, target, a.timeout_ns, &s_flag)) return;
            } else {
                __syncthreads();
            }
        }
        e0 = m1;
        h0 = h1;
        m1 = m2;
        h1 = h2;
        pb0 = pb1;
        pb1 = pb2;
        pb2 = pb3;
        pb3 = pb4;
    }
    if (GRID && blockIdx.x == 0 && threadIdx.x == 0) a.ctl->barriers = nphases > 0 ? nphases - 1 : 0;
    if (a.refine) refine_flush(a.ctl, a.sweep, dm, xm);
}

// Block-per-core executor for schedules whose supersteps hold several blocks
// (GrowLocal): each block is walked by one thread block phase by phase with
// __syncthreads, a grid barrier separates supersteps.  Kept on on-demand
// loads: a block's rows are contiguous and its phases are short.
template <typename T, int LANES>
__global__ void __launch_bounds__(512, 1) k_blocks(SolveArgs<T> a) {
    __shared__ int s_flag;
    if (refine_skip(a)) return;
    const int wpb = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    unsigned long long target = 0;
    double dm = 0.0, xm = 0.0;
    for (int s = 0; s < a.S; ++s) {
        const int b1 = a.step_blk[s + 1];
        for (int blk = a.step_blk[s] + blockIdx.x; blk < b1; blk += gridDim.x) {
            const int q1 = a.blk_phase[blk + 1];
            for (int q = a.blk_phase[blk]; q < q1; ++q) {
                rows_span<T, LANES>(a, a.phase_row[q], a.phase_row[q + 1], w, wpb, dm, xm);
                __syncthreads();
            }
        }
        if (s + 1 < a.S) {
            target += gridDim.x;
            if (!grid_barrier(a.ctl, target, a.timeout_ns, &s_flag)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->barriers = a.S > 0 ? a.S - 1 : 0;
    if (a.refine) refine_flush(a.ctl, a.sweep, dm, xm);
}

// ----------------------------------------------------------------------------
// FP64 residual of the refinement, r = b - L x, computed from the FP32 split
// L = hi + lo (each product formed in FP64), stored rounded to FP32 as the
// right-hand side of the next FP32 correction sweep.  No dependencies: a plain
// grid-stride pass over device rows.  Sweep 0 has x = 0, so r = b.  At the
// start of sweep t >= 1 the kernel stops the refinement if the last correction
// was small: max |d_{t-1}| <= dtol * max |x_t|.
// ----------------------------------------------------------------------------
// ----------------------------------------------------------------------------
// Layout change of a block of right-hand sides between the caller's
// column-major n x R (leading dimension ld) and an internal row-major copy
// (R consecutive values per row): with one row's R values in one or two cache
// lines, a right-hand-side tile gathers each parent in one coalesced load
// instead of R separate sectors.  32 x 32 tiles through shared memory keep
// both sides coalesced.  k_to_rows also fills `fill` (row-major, n x R) with
// the all-ones NaN of not-yet-computed values.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_to_rows(const T *__restrict__ src, int64_t ld, T *__restrict__ dst,
                                                 T *__restrict__ fill, int n, int R) {
    __shared__ T tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {          // column c0 + k, rows r0 + threadIdx.x
        const int r = r0 + threadIdx.x, c = c0 + k;
        if (r < n && c < R) tile[k][threadIdx.x] = src[(int64_t)c * ld + r];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {          // row r0 + k, columns c0 + threadIdx.x
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < n && c < R) {
            dst[(int64_t)r * R + c] = tile[threadIdx.x][k];
            if (fill) fill[(int64_t)r * R + c] = all_ones<T>();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_to_cols(const T *__restrict__ src, T *__restrict__ dst, int64_t ld, int n,
                                                 int R) {
    __shared__ T tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {          // row r0 + k, columns c0 + threadIdx.x
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < n && c < R) tile[k][threadIdx.x] = src[(int64_t)r * R + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {          // column c0 + k, rows r0 + threadIdx.x
        const int r = r0 + threadIdx.x, c = c0 + k;
        if (r < n && c < R) dst[(int64_t)c * ld + r] = tile[threadIdx.x][k];
    }
}

struct ResidualArgs {
    int32_t n, nrhs, sweep;
    const int32_t *__restrict__ rp;
    const int32_t *__restrict__ col;
    const float *__restrict__ hi;
    const float *__restrict__ lo;
    const double *__restrict__ v64;  // A_ij / A_ii in FP64 when the plan holds FP64 values, else null
    const float *__restrict__ dhi;
    const float *__restrict__ dlo;
    const int32_t *__restrict__ perm;
    const double *b;
    int64_t ldb, b_rs;               // column and row strides of b
    const double *x;
    int64_t ldx, x_rs;               // column and row strides of x
    float *r32;                      // n x nrhs: element (row, j) at r32[row * r_rs + j * r_cs]
    int64_t r_rs, r_cs;
    Ctl *ctl;
    double dtol;
};

// Convergence bookkeeping at the start of a residual pass: true if the
// refinement already converged (the correction test of the previous sweep).
__device__ __forceinline__ bool residual_skip(const ResidualArgs &a) {
    if (a.sweep == 0) return false;
    const volatile Ctl *c = a.ctl;
    if (c->done || c->status) return true;
    const double d = bits_to_d(c->dmax[a.sweep - 1]);
    const double x = bits_to_d(c->xmax[a.sweep - 1]);
    if (d <= a.dtol * x) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->done = 1;
            a.ctl->conv = 1;
        }
        return true;
    }
    return false;
}

__device__ __forceinline__ void residual_flush(const ResidualArgs &a, double rm, double bm) {
    __shared__ double s_r[32], s_b[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        rm = max_abs_bits(rm, __shfl_xor_sync(0xffffffffu, rm, off));
        bm = max_abs_bits(bm, __shfl_xor_sync(0xffffffffu, bm, off));
    }
    if ((threadIdx.x & 31) == 0) {
        s_r[threadIdx.x >> 5] = rm;
        s_b[threadIdx.x >> 5] = bm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < int(blockDim.x >> 5); ++i) {
            rm = max_abs_bits(rm, s_r[i]);
            bm = max_abs_bits(bm, s_b[i]);
        }
        atomicMax(&a.ctl->rmax[a.sweep], (unsigned long long)__double_as_longlong(rm));
        if (a.sweep == 0) atomicMax(&a.ctl->bmax, (unsigned long long)__double_as_longlong(bm));
    }
}

// Residual from the FP64 scaled values v'_ij = A_ij / A_ii (plans holding FP64
// values): r_i = b_i - A_ii (x_i + sum_j v'_ij x_j), one FP64 FMA per entry and
// right-hand side for every row length, plus one per row for A_ii = hi + lo.
// Same bytes per entry as the hi/lo split (8-byte value + 4-byte column);
// v'_ij carries one rounding, so r keeps FP64 accuracy.  Thread per row; short
// rows keep their columns and values in registers for all right-hand sides.
static __global__ void __launch_bounds__(256) k_residual_scaled(ResidualArgs a) {
    if (residual_skip(a)) return;
    double rm = 0.0, bm = 0.0;
    const int stride = gridDim.x * blockDim.x;
    constexpr int kRes = 8;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += stride) {
        const int o = __ldg(a.perm + r);
        const int beg = __ldg(a.rp + r), end = __ldg(a.rp + r + 1);
        const double d = double(__ldg(a.dhi + r)) + double(__ldg(a.dlo + r));
        const bool short_row = end - beg <= kRes;
        int c8[kRes];
        double v8[kRes];
        if (short_row && a.sweep > 0) {
#pragma unroll
            for (int u = 0; u < kRes; ++u) {
                const int q = beg + u;
                c8[u] = q < end ? __ldg(a.col + q) : 0;
                v8[u] = q < end ? __ldg(a.v64 + q) : 0.0;
            }
        }
        for (int j = 0; j < a.nrhs; ++j) {
            const double bj = a.b[(int64_t)o * a.b_rs + (int64_t)j * a.ldb];
            bm = max_abs_bits(bm, bj);
            double rj = bj;
            if (a.sweep > 0) {
                const double *xj = a.x + (int64_t)j * a.ldx;
                double sum = xj[(int64_t)o * a.x_rs];
                if (short_row) {
#pragma unroll
                    for (int u = 0; u < kRes; ++u)
                        if (beg + u < end) sum = fma(v8[u], xj[(int64_t)c8[u] * a.x_rs], sum);
                } else {
                    for (int q = beg; q < end; ++q) sum = fma(__ldg(a.v64 + q), xj[(int64_t)__ldg(a.col + q) * a.x_rs], sum);
                }
                rj = fma(-d, sum, bj);
            }
            a.r32[(int64_t)o * a.r_rs + (int64_t)j * a.r_cs] = float(rj);
            rm = max_abs_bits(rm, rj);
        }
    }
    residual_flush(a, rm, bm);
}

// Thread per row.  Short rows with several right-hand sides form the row's
// values hi + lo once in FP64 and keep them for all right-hand sides (one FP64
// FMA per entry and right-hand side instead of two).
static __global__ void __launch_bounds__(256) k_residual(ResidualArgs a) {
    if (residual_skip(a)) return;
    double rm = 0.0, bm = 0.0;
    const int stride = gridDim.x * blockDim.x;
    constexpr int kRes = 8;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += stride) {
        const int o = __ldg(a.perm + r);
        const int beg = __ldg(a.rp + r), end = __ldg(a.rp + r + 1);
        const double dh = __ldg(a.dhi + r), dl = __ldg(a.dlo + r);
        const bool short_row = a.nrhs > 1 && end - beg <= kRes;
        int c8[kRes];
        double v8[kRes];
        if (short_row && a.sweep > 0) {
#pragma unroll
            for (int u = 0; u < kRes; ++u) {
                const int q = beg + u;
                c8[u] = q < end ? __ldg(a.col + q) : 0;
                v8[u] = q < end ? double(__ldg(a.hi + q)) + double(__ldg(a.lo + q)) : 0.0;
            }
        }
        for (int j = 0; j < a.nrhs; ++j) {
            double s = a.b[(int64_t)o * a.b_rs + (int64_t)j * a.ldb];
            bm = max_abs_bits(bm, s);
            if (a.sweep > 0) {
                const double *xj = a.x + (int64_t)j * a.ldx;
                if (short_row) {
#pragma unroll
                    for (int u = 0; u < kRes; ++u)
                        if (beg + u < end) s = fma(-v8[u], xj[(int64_t)c8[u] * a.x_rs], s);
                    s = fma(-(dh + dl), xj[(int64_t)o * a.x_rs], s);
                } else {
                    for (int q = beg; q < end; ++q) {
                        const double xv = xj[(int64_t)__ldg(a.col + q) * a.x_rs];
                        s = fma(-double(__ldg(a.hi + q)), xv, s);
                        s = fma(-double(__ldg(a.lo + q)), xv, s);
                    }
                    const double xo = xj[(int64_t)o * a.x_rs];
                    s = fma(-dh, xo, s);
                    s = fma(-dl, xo, s);
                }
            }
            a.r32[(int64_t)o * a.r_rs + (int64_t)j * a.r_cs] = float(s);
            rm = max_abs_bits(rm, s);
        }
    }
    residual_flush(a, rm, bm);
}

}  // namespace sptrsv
