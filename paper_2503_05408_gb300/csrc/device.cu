// Device residency of a plan and the single-factor solve entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "plan.hpp"

namespace sptrsv {

#define CUDA_TRY(expr)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA, \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));            \
    } while (0)

int device_sm_count(int device, int32_t *out) {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device >= count)
        return fail(SPTRSV_ERR_CUDA, std::string("no CUDA device ") + std::to_string(device) + ": " +
                                         cudaGetErrorString(e));
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    *out = sms;
    return SPTRSV_OK;
}

namespace {

// Every device array carries 64 zeroed bytes past its end: the staged walker's
// 16-byte aligned bulk copies may round a slice up by up to 12 bytes.
template <typename T>
int upload(const std::vector<T> &h, T **d, int64_t *bytes) {
    const size_t nb = h.size() * sizeof(T) + 64;
    CUDA_TRY(cudaMalloc((void **)d, nb));
    CUDA_TRY(cudaMemset(*d, 0, nb));
    if (!h.empty()) CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *bytes += int64_t(nb);
    return SPTRSV_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

int upload_plan(sptrsv_plan *p, const sptrsv_csr *A) {
    DeviceGuard g(p->device);
    const HostSchedule &h = p->h;
    const int32_t n = h.n;
    // gather the factor in device order, off-diagonals and diagonal apart
    std::vector<int32_t> rp(size_t(n) + 1, 0), col;
    std::vector<double> val, diag(n);
    col.reserve(size_t(p->nnz_off));
    val.reserve(size_t(p->nnz_off));
    for (int32_t r = 0; r < n; ++r) {
        const int32_t v = h.dev_perm[r];
        const int32_t lo = A->rowptr[v], last = A->rowptr[v + 1] - 1;
        for (int32_t q = lo; q < last; ++q) {
            // reversed plans: the kernels address b and x in the caller's numbering
            col.push_back(p->reversed ? n - 1 - A->col[q] : A->col[q]);
            val.push_back(A->val[q]);
        }
        diag[r] = A->val[last];
        rp[r + 1] = int32_t(col.size());
    }
    int64_t bytes = 0;
    int st;
    DeviceBuffers &d = p->d;
    p->max_row_off = 0;
    for (int32_t r = 0; r < n; ++r) p->max_row_off = std::max(p->max_row_off, rp[r + 1] - rp[r]);
    if ((st = upload(rp, &d.rp, &bytes))) return st;
    if ((st = upload(col, &d.col, &bytes))) return st;
    // rows scaled by their diagonal: x_i = b_i / A_ii - sum_j (A_ij / A_ii) x_j
    std::vector<double> dinv(n), scaled(val.size());
    for (int32_t i = 0; i < n; ++i) dinv[i] = 1.0 / diag[i];
    for (int32_t r = 0; r < n; ++r)
        for (int32_t q = rp[r]; q < rp[r + 1]; ++q) scaled[q] = val[q] * dinv[r];
    if (p->values & SPTRSV_VALUES_F64) {
        if ((st = upload(scaled, &d.val, &bytes))) return st;
        if ((st = upload(dinv, &d.dinv, &bytes))) return st;
    }
    if (p->values & SPTRSV_VALUES_F32) {
        // hi = fp32(v), lo = fp32(v - hi): hi + lo carries ~48 bits of v for the
        // FP64 residual, hi alone drives the FP32 sweeps.
        std::vector<float> hi(val.size()), lo(val.size()), dhi(n), dlo(n);
        for (size_t i = 0; i < val.size(); ++i) {
            hi[i] = float(val[i]);
            lo[i] = float(val[i] - double(hi[i]));
        }
        for (int32_t i = 0; i < n; ++i) {
            dhi[i] = float(diag[i]);
            dlo[i] = float(diag[i] - double(dhi[i]));
        }
        if ((st = upload(hi, &d.val_hi, &bytes))) return st;
        if ((st = upload(lo, &d.val_lo, &bytes))) return st;
        std::vector<float> dinv32(n), s32(val.size());
        for (int32_t i = 0; i < n; ++i) dinv32[i] = float(dinv[i]);
        for (size_t q = 0; q < val.size(); ++q) s32[q] = float(scaled[q]);
        if ((st = upload(dhi, &d.diag_hi, &bytes))) return st;
        if ((st = upload(dlo, &d.diag_lo, &bytes))) return st;
        if ((st = upload(dinv32, &d.dinv32, &bytes))) return st;
        if ((st = upload(s32, &d.s32, &bytes))) return st;
    }
    {
        std::vector<int32_t> perm(h.dev_perm);
        if (p->reversed)
            for (auto &v : perm) v = n - 1 - v;
        if ((st = upload(perm, &d.perm, &bytes))) return st;
    }
    if ((st = upload(h.step_blk, &d.step_blk, &bytes))) return st;
    if ((st = upload(h.blk_phase, &d.blk_phase, &bytes))) return st;
    if ((st = upload(h.phase_row, &d.phase_row, &bytes))) return st;
    {
        std::vector<int32_t> pent(h.phase_row.size());
        int32_t mx = 0;
        for (size_t q = 0; q < pent.size(); ++q) pent[q] = rp[h.phase_row[q]];
        for (size_t q = 0; q + 1 < pent.size(); ++q) mx = std::max(mx, pent[q + 1] - pent[q]);
        p->h.max_phase_ents = mx;
        if ((st = upload(pent, &d.phase_ent, &bytes))) return st;
    }
    CUDA_TRY(cudaMalloc((void **)&d.counters, sizeof(Ctl)));
    CUDA_TRY(cudaMemset(d.counters, 0, sizeof(Ctl)));
    bytes += sizeof(Ctl);
    CUDA_TRY(cudaMalloc((void **)&d.flags, std::max<size_t>(size_t(n), 1) * sizeof(uint32_t)));
    CUDA_TRY(cudaMemset(d.flags, 0, std::max<size_t>(size_t(n), 1) * sizeof(uint32_t)));
    bytes += int64_t(std::max<size_t>(size_t(n), 1) * sizeof(uint32_t));
    p->device_bytes = bytes;
    return SPTRSV_OK;
}

void free_device(sptrsv_plan *p) {
    if (!p || p->device < 0) return;
    DeviceGuard g(p->device);
    DeviceBuffers &d = p->d;
    void *ptrs[] = {d.rp,       d.col,      d.val,       d.dinv,      d.val_hi,    d.val_lo, d.diag_hi,
                    d.diag_lo,  d.dinv32,   d.s32,       d.perm,      d.step_blk,  d.blk_phase, d.phase_row,
                    d.phase_ent,
                    d.counters, d.flags,    d.work,      d.io,
                    d.l_rp,     d.l_col,    d.l_perm,    d.l_blk_row, d.l_val,     d.l_dinv, d.l_s32,
                    d.l_dinv32,
                    d.ck_info,  d.ck_blk,   d.ck_col,    d.ck_orow,   d.ck_val,    d.ck_dinv, d.ck_s32,
                    d.ck_dinv32, d.ck_bd};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    d = DeviceBuffers();
}

// ------------------------------------------------------------------ launch
namespace {

template <typename T>
using Kern = void (*)(SolveArgs<T>);
template <typename T>
using WalkKern = void (*)(SolveArgs<T>, int, int);

// Register tile per lane for each supported lanes-per-row value; the
// right-hand-side-parallel tiles (rp) keep 8 entries of every row in registers.
constexpr int tile_for(int lanes) { return lanes == 1 ? 8 : lanes == 2 ? 4 : lanes == 4 ? 2 : 1; }
constexpr int kRpTile = 8;

bool lanes_ok(int lanes) { return lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32; }
bool rp_ok(int tile) { return tile == 4 || tile == 8 || tile == 16 || tile == 32; }

template <typename T, bool RP>
Kern<T> flags_kernel(int lanes, bool pre, bool short_rows = false) {
    if constexpr (RP) {
        // rows of at most 4 off-diagonal entries: a 4-entry register tile, fewer
        // registers, twice the resident warps
        if (short_rows) {
            switch (lanes) {
                case 4: return k_flags<T, 4, 4, true>;
                case 8: return k_flags<T, 8, 4, true>;
                case 16: return k_flags<T, 16, 4, true>;
                case 32: return k_flags<T, 32, 4, true>;
                default: return nullptr;
            }
        }
        switch (lanes) {
            case 4: return k_flags<T, 4, kRpTile, true>;
            case 8: return k_flags<T, 8, kRpTile, true>;
            case 16: return k_flags<T, 16, kRpTile, true>;
            case 32: return k_flags<T, 32, kRpTile, true>;
            default: return nullptr;
        }
    } else {
        switch (lanes) {
            case 1: return k_flags<T, 1, tile_for(1), false>;
            case 2: return pre ? k_flags<T, 2, tile_for(2), false, true> : k_flags<T, 2, tile_for(2), false>;
            case 4: return pre ? k_flags<T, 4, tile_for(4), false, true> : k_flags<T, 4, tile_for(4), false>;
            case 8: return pre ? k_flags<T, 8, tile_for(8), false, true> : k_flags<T, 8, tile_for(8), false>;
            case 16: return pre ? k_flags<T, 16, tile_for(16), false, true> : k_flags<T, 16, tile_for(16), false>;
            case 32: return pre ? k_flags<T, 32, tile_for(32), false, true> : k_flags<T, 32, tile_for(32), false>;
            default: return nullptr;
        }
    }
}
template <typename T>
Kern<T> local_kernel(int lanes, bool pre) {
    switch (lanes) {
        case 1: return k_local<T, 1, tile_for(1), false>;
        case 2: return pre ? k_local<T, 2, tile_for(2), true> : k_local<T, 2, tile_for(2), false>;
        case 4: return pre ? k_local<T, 4, tile_for(4), true> : k_local<T, 4, tile_for(4), false>;
        case 8: return pre ? k_local<T, 8, tile_for(8), true> : k_local<T, 8, tile_for(8), false>;
        case 16: return pre ? k_local<T, 16, tile_for(16), true> : k_local<T, 16, tile_for(16), false>;
        case 32: return pre ? k_local<T, 32, tile_for(32), true> : k_local<T, 32, tile_for(32), false>;
        default: return nullptr;
    }
}
// Shared memory of the resident one-block executor for a plan (bytes).
size_t resident_smem_bytes(const sptrsv_plan *p, size_t es) {
    const size_t n = size_t(p->h.n), m = size_t(p->nnz_off), nph = p->h.phase_row.size();
    return 2 * round16(n * es) + round16(m * es) + round16(m * 4) + round16((n + 1) * 4) + round16(n * 4) +
           round16(nph * 4);
}
template <typename T>
Kern<T> chunks_kernel(int umax) {
    return umax <= 3 ? k_chunks<T, 3> : umax <= 4 ? k_chunks<T, 4> : k_chunks<T, 8>;
}
template <typename T>
Kern<T> blocks_kernel(int lanes) {
    switch (lanes) {
        case 1: return k_blocks<T, 1>;
        case 2: return k_blocks<T, 2>;
        case 4: return k_blocks<T, 4>;
        case 8: return k_blocks<T, 8>;
        case 16: return k_blocks<T, 16>;
        case 32: return k_blocks<T, 32>;
        default: return nullptr;
    }
}
template <typename T, bool GRID, bool RING, bool RP>
WalkKern<T> walk_kernel(int lanes) {
    if constexpr (RP) {
        switch (lanes) {
            case 4: return k_walk<T, 4, kRpTile, GRID, RING, true>;
            case 8: return k_walk<T, 8, kRpTile, GRID, RING, true>;
            case 16: return k_walk<T, 16, kRpTile, GRID, RING, true>;
            case 32: return k_walk<T, 32, kRpTile, GRID, RING, true>;
            default: return nullptr;
        }
    } else {
        switch (lanes) {
            case 1: return k_walk<T, 1, tile_for(1), GRID, RING, false>;
            case 2: return k_walk<T, 2, tile_for(2), GRID, RING, false>;
            case 4: return k_walk<T, 4, tile_for(4), GRID, RING, false>;
            case 8: return k_walk<T, 8, tile_for(8), GRID, RING, false>;
            case 16: return k_walk<T, 16, tile_for(16), GRID, RING, false>;
            case 32: return k_walk<T, 32, tile_for(32), GRID, RING, false>;
            default: return nullptr;
        }
    }
}

template <typename T>
using StageKern = void (*)(SolveArgs<T>, StageInfo, int, int);

template <typename T, bool RING, bool RP>
StageKern<T> stage_kernel(int lanes) {
    if constexpr (RP) {
        switch (lanes) {
            case 4: return k_stage<T, 4, RING, true>;
            case 8: return k_stage<T, 8, RING, true>;
            case 16: return k_stage<T, 16, RING, true>;
            case 32: return k_stage<T, 32, RING, true>;
            default: return nullptr;
        }
    } else {
        switch (lanes) {
            case 1: return k_stage<T, 1, RING, false>;
            case 2: return k_stage<T, 2, RING, false>;
            case 4: return k_stage<T, 4, RING, false>;
            case 8: return k_stage<T, 8, RING, false>;
            case 32: return k_stage<T, 32, RING, false>;
            default: return nullptr;
        }
    }
}

// Shared-memory slot layout of the staged walker for this plan and RHS count;
// returns the slot size in bytes.
template <typename T>
size_t stage_layout(const sptrsv_plan *p, int nrhs, StageInfo &si) {
    const size_t b = stage_slot_layout(size_t(p->h.max_phase_rows), size_t(p->h.max_phase_ents), nrhs, sizeof(T), si);
    si.phase_ent = p->d.phase_ent;
    return b;
}
constexpr size_t kStageSmemMax = 200 * 1024;

struct LaunchCfg {
    int sync, lanes, threads, grid;
    int kind;          // 0 flags, 1 walk (grid barrier), 2 blocks (grid barrier), 3 walk (one CTA),
                       // 4 staged walk (one CTA, TMA-staged phases), 5 block-local (polled),
                       // 6 chunked block-local (polled, one row per lane),
                       // 7 resident one CTA (whole factor in shared memory)
    int umax;          // chunked executor: entries per lane kept in registers (3, 4 or 8)
    StageInfo si;
    int win;           // shared-memory ring rows for kind 3 (0 = gather from global x)
    bool rp;           // lanes map to right-hand sides (multi-RHS tile) instead of entries
    bool eager;        // polled executor: eager group sum (SPTRSV_EAGER_ON)
    bool short_rows;   // every row has at most 4 off-diagonal entries
    size_t smem;
};

int auto_lanes(const sptrsv_plan *p) {
    const double per_row = p->h.n ? double(p->nnz_off) / p->h.n : 0.0;
    if (per_row <= 4.0) return 1;
    if (per_row <= 8.0) return 2;
    if (per_row <= 16.0) return 8;
    return 32;
}

bool wide_phases(const sptrsv_plan *p) {
    // every superstep is one block with one phase (the wavefront schedule)
    return int32_t(p->h.phase_row.size()) - 1 == p->h.S;
}

constexpr size_t kRingBytesMax = 200 * 1024;

int tune_slot(int32_t dtype, int32_t precision, int32_t nrhs) {
    const int r = nrhs <= 1 ? 0 : nrhs <= 4 ? 1 : nrhs <= 16 ? 2 : 3;
    return (dtype == SPTRSV_F32 ? 1 : 0) * 8 + (precision ? 4 : 0) + r;
}

template <typename T, bool RP>
const void *kernel_ptr_rp(const LaunchCfg &c) {
    if (c.kind == 4)
        return c.win ? reinterpret_cast<const void *>(stage_kernel<T, true, RP>(c.lanes))
                     : reinterpret_cast<const void *>(stage_kernel<T, false, RP>(c.lanes));
    switch (c.kind) {
        case 0: return reinterpret_cast<const void *>(flags_kernel<T, RP>(c.lanes, c.eager, c.short_rows));
        case 5: return RP ? nullptr : reinterpret_cast<const void *>(local_kernel<T>(c.lanes, c.eager));
        case 6: return RP ? nullptr : reinterpret_cast<const void *>(chunks_kernel<T>(c.umax));
        case 7: return RP ? nullptr : reinterpret_cast<const void *>(k_resident<T>);
        case 1: return reinterpret_cast<const void *>(walk_kernel<T, true, false, RP>(c.lanes));
        case 2: return RP ? nullptr : reinterpret_cast<const void *>(blocks_kernel<T>(c.lanes));
        default:
            return c.win ? reinterpret_cast<const void *>(walk_kernel<T, false, true, RP>(c.lanes))
                         : reinterpret_cast<const void *>(walk_kernel<T, false, false, RP>(c.lanes));
    }
}
template <typename T>
const void *kernel_ptr(const LaunchCfg &c) {
    return c.rp ? kernel_ptr_rp<T, true>(c) : kernel_ptr_rp<T, false>(c);
}

// ------------------------------------------------------------------ block-local layout
void free_local(DeviceBuffers &d) {
    void *ptrs[] = {d.l_rp, d.l_col, d.l_perm, d.l_blk_row, d.l_val, d.l_dinv, d.l_s32, d.l_dinv32};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    d.l_rp = d.l_col = d.l_perm = d.l_blk_row = nullptr;
    d.l_val = d.l_dinv = nullptr;
    d.l_s32 = d.l_dinv32 = nullptr;
    d.loc_nb = 0;
    d.loc_smem = 0;
    d.loc_bytes = 0;
}

template <typename T>
int download(const T *dptr, size_t count, std::vector<T> &h) {
    h.resize(count);
    if (count) CUDA_TRY(cudaMemcpy(h.data(), dptr, count * sizeof(T), cudaMemcpyDeviceToHost));
    return SPTRSV_OK;
}

// The device-order structure back from the device (the caller's CSR is not
// kept), column ids in the analysed numbering, and device row of every row.
int download_structure(sptrsv_plan *p, std::vector<int32_t> &rp, std::vector<int32_t> &col,
                       std::vector<int32_t> &dev_of) {
    const int32_t n = p->h.n;
    int st;
    if ((st = download(p->d.rp, size_t(n) + 1, rp)) || (st = download(p->d.col, size_t(p->nnz_off), col))) return st;
    if (p->reversed)                                   // back to the analysed factor's numbering
        for (auto &c : col) c = n - 1 - c;
    dev_of.assign(n, 0);
    for (int32_t r = 0; r < n; ++r) dev_of[p->h.dev_perm[r]] = r;
    return SPTRSV_OK;
}

// Rows one block may keep in shared memory (FP64 slots if the plan holds FP64 values).
int local_row_cap(const sptrsv_plan *p, int32_t *cap) {
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    *cap = int32_t((int64_t(optin) - 1024) / ((p->values & SPTRSV_VALUES_F64) ? 8 : 4));
    return SPTRSV_OK;
}

// The plan's row -> block partition for nb blocks of kind `part` (SPTRSV_PART_*;
// AUTO keeps whatever partition the plan holds for nb blocks, else PARENTS).
int ensure_partition(sptrsv_plan *p, int nb, int part) {
    HostSchedule &h = p->h;
    const int32_t n = h.n;
    // kept (a saved partition too: the launch checks that its blocks fit shared memory)
    if (h.loc_nb == nb && h.loc_blk.size() == size_t(n) && (part == SPTRSV_PART_AUTO || part == h.loc_part))
        return SPTRSV_OK;
    int32_t row_cap = 0;
    int st;
    if ((st = local_row_cap(p, &row_cap))) return st;
    if (part == SPTRSV_PART_AUTO || part == -1) part = SPTRSV_PART_PARENTS;
    std::vector<int32_t> blk, lidx, load;
    bool ok;
    if (part == SPTRSV_PART_RANGES) {
        ok = range_partition(n, nb, row_cap, h.level, h.nlevels, blk, lidx, load);
    } else if (part == SPTRSV_PART_PARENTS || part == SPTRSV_PART_GRID) {
        std::vector<int32_t> rp, col, dev_of;
        if ((st = download_structure(p, rp, col, dev_of))) return st;
        ok = part == SPTRSV_PART_GRID &&
             grid_partition(n, nb, row_cap, h.level, h.nlevels, rp.data(), col.data(), dev_of.data(), blk, lidx, load);
        if (!ok)      // no grid structure: the parents partition (recorded as asked, so it is not rebuilt)
            ok = local_partition(n, nb, row_cap, h.level, h.nlevels, rp.data(), col.data(), dev_of.data(), blk,
                                 lidx, load);
    } else {
        return fail(SPTRSV_ERR_ARG, "partition must be SPTRSV_PART_AUTO, PARENTS, RANGES or GRID");
    }
    if (!ok)
        return fail(SPTRSV_ERR_ARG, "block-local executor: " + std::to_string(n) + " rows do not fit the "
                                        "shared memory of " + std::to_string(nb) + " blocks");
    h.loc_nb = nb;
    h.loc_blk.swap(blk);
    h.loc_lidx.swap(lidx);
    h.loc_part = part;
    ++h.loc_gen;
    return SPTRSV_OK;
}

// The layouts are kept while the plan's partition is the one asked for: the
// checks below are O(1), so a solve pays no host work once they are built.
bool partition_kept(const sptrsv_plan *p, int nb, int part) {
    return p->h.loc_nb == nb && (part == SPTRSV_PART_AUTO || part == p->h.loc_part);
}

int ensure_local(sptrsv_plan *p, int nb, int part) {
    DeviceBuffers &d = p->d;
    if (d.loc_nb == nb && d.loc_gen == p->h.loc_gen && partition_kept(p, nb, part)) return SPTRSV_OK;
    DeviceGuard g(p->device);
    int st;
    if ((st = ensure_partition(p, nb, part))) return st;
    if (d.loc_nb == nb && d.loc_gen == p->h.loc_gen) return SPTRSV_OK;
    p->device_bytes -= d.loc_bytes;
    free_local(d);
    const HostSchedule &h = p->h;
    const int32_t n = h.n;
    const size_t nnz = size_t(p->nnz_off);
    std::vector<int32_t> rp, col, dev_of;
    if ((st = download_structure(p, rp, col, dev_of))) return st;
    const std::vector<int32_t> &blk = h.loc_blk, &lidx = h.loc_lidx;
    std::vector<int32_t> load(size_t(nb), 0);
    for (int32_t v = 0; v < n; ++v) load[size_t(blk[v])]++;
    std::vector<int32_t> bstart(size_t(nb) + 1, 0);
    for (int32_t b = 0; b < nb; ++b) bstart[b + 1] = bstart[b] + load[b];
    // column ids in the block-local order: a parent of the same block -> its
    // shared-memory slot -(position + 2), any other -> its original id
    std::vector<int32_t> lperm(n), lrp(size_t(n) + 1, 0), lcol(nnz), src(nnz);
    int32_t maxrows = 0;
    for (int32_t v = 0; v < n; ++v) lperm[bstart[blk[v]] + lidx[v]] = v;
    for (int32_t b = 0; b < nb; ++b) maxrows = std::max(maxrows, load[b]);
    int64_t cross = 0;
    for (int32_t t = 0; t < n; ++t) {
        const int32_t v = lperm[t], dr = dev_of[v];
        int32_t o = lrp[t];
        for (int32_t q = rp[dr]; q < rp[dr + 1]; ++q, ++o) {
            const int32_t c = col[q];
            const bool same = blk[c] == blk[v];
            cross += !same;
            lcol[o] = same ? -(lidx[c] + 2) : (p->reversed ? n - 1 - c : c);
            src[o] = q;
        }
        lrp[t + 1] = o;
    }
    int64_t bytes = 0;
    std::vector<int32_t> lperm_out(lperm);
    if (p->reversed)
        for (auto &v : lperm_out) v = n - 1 - v;
    if ((st = upload(lrp, &d.l_rp, &bytes)) || (st = upload(lcol, &d.l_col, &bytes)) ||
        (st = upload(lperm_out, &d.l_perm, &bytes)) || (st = upload(bstart, &d.l_blk_row, &bytes)))
        return st;
    // values: gathered on the device from the device-order arrays into the block-local order
    {
        std::vector<int32_t> rsrc(n);
        for (int32_t t = 0; t < n; ++t) rsrc[t] = dev_of[lperm[t]];
        if ((st = local_values_device(p, src, rsrc, &bytes))) return st;
    }
    d.loc_nb = nb;
    d.loc_gen = h.loc_gen;
    d.loc_smem = size_t(maxrows) * size_t((p->values & SPTRSV_VALUES_F64) ? 8 : 4);
    d.loc_bytes = bytes;
    d.cross_edges = cross;
    d.edges = int64_t(nnz);
    p->device_bytes += bytes;
    return SPTRSV_OK;
}

void free_chunks(DeviceBuffers &d) {
    void *ptrs[] = {d.ck_info, d.ck_blk, d.ck_col, d.ck_orow, d.ck_val, d.ck_dinv, d.ck_s32, d.ck_dinv32, d.ck_bd};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    d.ck_info = d.ck_blk = d.ck_col = d.ck_orow = nullptr;
    d.ck_bd = nullptr;
    d.ck_val = d.ck_dinv = nullptr;
    d.ck_s32 = d.ck_dinv32 = nullptr;
    d.ck_gen = -1;
    d.ck_nb = 0;
    d.ck_width = 0;
    d.ck_slots = 0;
    d.ck_bytes = 0;
}

// out[i] = in[src[i]], 0 where src[i] < 0 (values into the chunked layout)
template <typename T>
__global__ void __launch_bounds__(256) k_gather(int64_t count, const int32_t *__restrict__ src,
                                                const T *__restrict__ in, T *__restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t q = src[i];
        out[i] = q >= 0 ? in[q] : T(0);
    }
}

template <typename T>
int gather_values(const std::vector<int32_t> &src, const T *in, T **out, int64_t *bytes) {
    const size_t count = src.size();
    const size_t nb = count * sizeof(T) + 64;
    CUDA_TRY(cudaMalloc((void **)out, nb));
    CUDA_TRY(cudaMemset(*out, 0, nb));
    *bytes += int64_t(nb);
    if (!count) return SPTRSV_OK;
    int32_t *g_src = nullptr;
    CUDA_TRY(cudaMalloc((void **)&g_src, count * sizeof(int32_t)));
    cudaError_t e = cudaMemcpy(g_src, src.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int grid = int(std::min<size_t>((count + 255) / 256, 8192));
        k_gather<T><<<grid, 256>>>(int64_t(count), g_src, in, *out);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(g_src);
    if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, std::string("chunk values: ") + cudaGetErrorString(e));
    return SPTRSV_OK;
}

// Chunked layout of the plan's partition for nb blocks: every block's
// (wavefront, id) list cut into chunks of up to 32 rows of one wavefront.
int ensure_chunks(sptrsv_plan *p, int nb, int part) {
    DeviceBuffers &d = p->d;
    if (d.ck_nb == nb && d.ck_gen == p->h.loc_gen && partition_kept(p, nb, part)) return SPTRSV_OK;
    DeviceGuard g(p->device);
    int st;
    if ((st = ensure_partition(p, nb, part))) return st;
    if (d.ck_nb == nb && d.ck_gen == p->h.loc_gen) return SPTRSV_OK;
    p->device_bytes -= d.ck_bytes;
    free_chunks(d);
    const HostSchedule &h = p->h;
    const int32_t n = h.n;
    std::vector<int32_t> rp, col, dev_of;
    if ((st = download_structure(p, rp, col, dev_of))) return st;
    const std::vector<int32_t> &blk = h.loc_blk, &lidx = h.loc_lidx;
    std::vector<int32_t> load(size_t(nb), 0);
    for (int32_t v = 0; v < n; ++v) load[size_t(blk[v])]++;
    std::vector<int32_t> bstart(size_t(nb) + 1, 0);
    for (int32_t b = 0; b < nb; ++b) bstart[b + 1] = bstart[b] + load[b];
    std::vector<int32_t> lperm(n);
    for (int32_t v = 0; v < n; ++v) lperm[bstart[blk[v]] + lidx[v]] = v;
    std::vector<int32_t> info, cblk(size_t(nb) + 1, 0), ccol, csrc, corow, crsrc;
    int64_t ent = 0, cross = 0;
    int32_t width_max = 0, slots_max = 0;
    for (int32_t b = 0; b < nb; ++b) {
        cblk[b] = int32_t(info.size() / 4);
        slots_max = std::max(slots_max, load[b]);
        for (int32_t t = bstart[b]; t < bstart[b + 1];) {
            const int32_t l = h.level[lperm[t]];
            int32_t k = 0, width = 0;
            while (t + k < bstart[b + 1] && k < 32 && h.level[lperm[t + k]] == l) {
                const int32_t dr = dev_of[lperm[t + k]];
                width = std::max(width, rp[dr + 1] - rp[dr]);
                ++k;
            }
            if (ent + int64_t(width) * 32 > int64_t(INT32_MAX) || width > 0xffff)
                return fail(SPTRSV_ERR_ARG, "chunked executor: too many entries for 32-bit offsets");
            // every row's entries: parents of other blocks first, then this block's, each in column order
            std::vector<int32_t> order(size_t(width) * 32, -1);
            bool remote = false;
            for (int32_t lane = 0; lane < k; ++lane) {
                const int32_t dr = dev_of[lperm[t + lane]];
                int32_t o = 0;
                for (int pass = 0; pass < 2; ++pass)
                    for (int32_t q = rp[dr]; q < rp[dr + 1]; ++q)
                        if ((blk[col[q]] != b) == (pass == 0)) order[size_t(o++) * 32 + lane] = q;
                remote = remote || (rp[dr + 1] > rp[dr] && blk[col[order[size_t(lane)]]] != b);
            }
            info.insert(info.end(), {int32_t(ent), width | (remote ? (1 << 16) : 0), k, t - bstart[b]});
            for (int32_t u = 0; u < width; ++u)
                for (int32_t lane = 0; lane < 32; ++lane) {
                    int32_t c_out = -1, s_out = -1;
                    const int32_t q = order[size_t(u) * 32 + lane];
                    if (q >= 0) {
                        const int32_t c = col[q];
                        const bool same = blk[c] == b;
                        cross += !same;
                        c_out = same ? -(lidx[c] + 2) : (p->reversed ? n - 1 - c : c);
                        s_out = q;
                    }
                    ccol.push_back(c_out);
                    csrc.push_back(s_out);
                }
            for (int32_t lane = 0; lane < 32; ++lane) {
                const int32_t v = lane < k ? lperm[t + lane] : -1;
                corow.push_back(v < 0 ? -1 : (p->reversed ? n - 1 - v : v));
                crsrc.push_back(v < 0 ? -1 : dev_of[v]);
            }
            ent += int64_t(width) * 32;
            width_max = std::max(width_max, width);
            t += k;
        }
    }
    cblk[nb] = int32_t(info.size() / 4);
    int64_t bytes = 0;
    if ((st = upload(info, &d.ck_info, &bytes)) || (st = upload(cblk, &d.ck_blk, &bytes)) ||
        (st = upload(ccol, &d.ck_col, &bytes)) || (st = upload(corow, &d.ck_orow, &bytes)))
        return st;
    if (d.val && ((st = gather_values<double>(csrc, d.val, &d.ck_val, &bytes)) ||
                  (st = gather_values<double>(crsrc, d.dinv, &d.ck_dinv, &bytes))))
        return st;
    if (d.s32 && ((st = gather_values<float>(csrc, d.s32, &d.ck_s32, &bytes)) ||
                  (st = gather_values<float>(crsrc, d.dinv32, &d.ck_dinv32, &bytes))))
        return st;
    {
        const size_t bdb = corow.size() * sizeof(double) + 64;
        CUDA_TRY(cudaMalloc(&d.ck_bd, bdb));
        bytes += int64_t(bdb);
    }
    d.ck_nb = nb;
    d.ck_gen = h.loc_gen;
    d.ck_width = width_max;
    d.ck_slots = size_t(slots_max);
    d.ck_bytes = bytes;
    d.cross_edges = cross;
    d.edges = p->nnz_off;
    p->device_bytes += bytes;
    return SPTRSV_OK;
}

template <typename T>
void use_chunks(sptrsv_plan *p, SolveArgs<T> &a) {
    a.col = p->d.ck_col;
    a.perm = p->d.ck_orow;
    a.blk_row = p->d.ck_blk;
    a.chunk = reinterpret_cast<const int4 *>(p->d.ck_info);
    a.bdc = static_cast<T *>(p->d.ck_bd);
    if constexpr (std::is_same<T, double>::value) {
        a.val = p->d.ck_val;
        a.dinv = p->d.ck_dinv;
    } else {
        a.val = p->d.ck_s32;
        a.dinv = p->d.ck_dinv32;
    }
}

template <typename T>
void use_local(sptrsv_plan *p, SolveArgs<T> &a) {
    a.rp = p->d.l_rp;
    a.col = p->d.l_col;
    a.perm = p->d.l_perm;
    a.blk_row = p->d.l_blk_row;
    if constexpr (std::is_same<T, double>::value) {
        a.val = p->d.l_val;
        a.dinv = p->d.l_dinv;
    } else {
        a.val = p->d.l_s32;
        a.dinv = p->d.l_dinv32;
    }
}

template <typename T>
int choose(const sptrsv_plan *p, const sptrsv_solve_opts &o_in, int32_t nrhs, LaunchCfg &c) {
    sptrsv_solve_opts o = o_in;
    if (o.sync == SPTRSV_SYNC_AUTO && p->tuned_slot >= 0) {
        const TunedCfg &t = p->tuned[p->tuned_slot];
        if (t.valid) {
            o.sync = t.sync;
            if (!o.lanes) o.lanes = t.lanes;
            if (!o.threads) o.threads = t.threads;
            if (!o.blocks_per_sm) o.blocks_per_sm = t.blocks_per_sm;
            if (!o.rhs_tile) o.rhs_tile = t.rhs_tile;
            if (!o.eager_sum) o.eager_sum = t.eager_sum;
            if (!o.partition) o.partition = t.partition;
        }
    }
    c.sync = o.sync;
    if (c.sync == SPTRSV_SYNC_AUTO) {
        if (p->h.n <= 8192) c.sync = SPTRSV_SYNC_CTA;
        else c.sync = SPTRSV_SYNC_FLAGS;
    }
    // multi-RHS: lanes map to right-hand sides (tile of 4..32 columns) unless rhs_tile == 1
    int tile = o.rhs_tile;
    if (tile == 0) {
        tile = 1;
        if (nrhs >= 3) {
            tile = 4;
            while (tile < nrhs && tile < 32) tile <<= 1;
        }
    }
    c.rp = tile > 1;
    if (c.rp) {
        if (!rp_ok(tile)) return fail(SPTRSV_ERR_ARG, "rhs_tile must be 0, 1, 4, 8, 16 or 32");
        c.lanes = tile;
    } else {
        c.lanes = o.lanes ? o.lanes : auto_lanes(p);
        if (!lanes_ok(c.lanes)) return fail(SPTRSV_ERR_ARG, "lanes must be 1, 2, 4, 8, 16 or 32");
    }
    if (o.eager_sum < 0 || o.eager_sum > 2) return fail(SPTRSV_ERR_ARG, "eager_sum must be 0, 1 or 2");
    c.eager = o.eager_sum != SPTRSV_EAGER_OFF;
    c.threads = o.threads ? o.threads : 256;
    const bool chunked = c.sync == SPTRSV_SYNC_CHUNKS;
    const bool resident = c.sync == SPTRSV_SYNC_RESIDENT;
    const bool one_per_sm = c.sync == SPTRSV_SYNC_LOCAL || chunked || resident;
    if (chunked && !o.threads) c.threads = 512;
    const int max_threads = one_per_sm ? 1024 : 512;
    if (c.threads < 32 || c.threads > max_threads || c.threads % 32)
        return fail(SPTRSV_ERR_ARG, "threads must be a multiple of 32 in [32, 512] ([32, 1024] for LOCAL, CHUNKS, RESIDENT)");
    c.win = 0;
    c.smem = 0;
    c.short_rows = p->max_row_off <= 4;
    if (c.sync == SPTRSV_SYNC_LOCAL) {
        if (nrhs != 1 || c.rp) return fail(SPTRSV_ERR_ARG, "the block-local executor solves one right-hand side");
        if (o.blocks_per_sm > 1) return fail(SPTRSV_ERR_ARG, "the block-local executor runs one block per SM");
        int st = ensure_local(const_cast<sptrsv_plan *>(p), p->num_sms, o.partition);
        if (st) return st;
        c.kind = 5;
        c.smem = std::max<size_t>(16, p->d.loc_smem);   // sized for FP64 values (FP32 uses part)
        int optin = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
        if (c.smem > size_t(optin))
            return fail(SPTRSV_ERR_ARG, "block-local executor: " + std::to_string(p->d.loc_smem) +
                                            " bytes per block exceed the shared memory of one SM");
    } else if (chunked) {
        if (nrhs != 1 || c.rp) return fail(SPTRSV_ERR_ARG, "the chunked executor solves one right-hand side");
        if (o.blocks_per_sm > 1) return fail(SPTRSV_ERR_ARG, "the chunked executor runs one block per SM");
        int st = ensure_chunks(const_cast<sptrsv_plan *>(p), p->num_sms, o.partition);
        if (st) return st;
        c.kind = 6;
        c.lanes = 1;
        c.umax = p->d.ck_width <= 3 ? 3 : p->d.ck_width <= 4 ? 4 : 8;
        const int tmax = c.umax <= 3 ? 768 : 512;
        if (c.threads > tmax)
            return fail(SPTRSV_ERR_ARG, "the chunked executor runs at most " + std::to_string(tmax) +
                                            " threads per block for this factor");
        c.smem = std::max<size_t>(16, p->d.ck_slots * sizeof(T));
        int optin = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
        if (c.smem > size_t(optin))
            return fail(SPTRSV_ERR_ARG, "chunked executor: " + std::to_string(c.smem) +
                                            " bytes per block exceed the shared memory of one SM");
    } else if (resident) {
        if (nrhs != 1 || c.rp) return fail(SPTRSV_ERR_ARG, "the resident executor solves one right-hand side");
        c.kind = 7;
        c.lanes = 1;
        c.smem = resident_smem_bytes(p, sizeof(T));
        // walking threads: the widest phase rounded up to a warp, at most the block
        c.win = std::max(32, std::min(c.threads, (p->h.max_phase_rows + 31) / 32 * 32));
        int optin = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
        if (c.smem + 1024 > size_t(optin))       // 1 KB of static shared memory (refinement reduction)
            return fail(SPTRSV_ERR_ARG, "resident executor: the factor needs " + std::to_string(c.smem) +
                                            " bytes of shared memory, more than one SM has");
    } else if (c.sync == SPTRSV_SYNC_FLAGS) c.kind = 0;
    else if (c.sync == SPTRSV_SYNC_GRID) {
        c.kind = wide_phases(p) ? 1 : 2;
        if (c.kind == 2 && c.rp) c.rp = false, c.lanes = auto_lanes(p);   // block executor: entry lanes
    }
    else if (c.sync == SPTRSV_SYNC_CTA || c.sync == SPTRSV_SYNC_CTA_REGS) {
        c.kind = 3;
        const int w = p->h.ring_rows;
        const size_t ring = size_t(w) * size_t(nrhs) * sizeof(T);
        if (w > 0 && ring <= kRingBytesMax) {
            c.win = w;
            c.smem = ring;
        }
        if (c.sync == SPTRSV_SYNC_CTA) {
            const size_t slot = stage_layout<T>(p, nrhs, c.si);
            (void)slot;
            const size_t need = stage_smem_bytes(c.si, c.win ? ring : 0);
            if (need <= kStageSmemMax && c.threads >= 64) {   // one warp of the block only produces
                c.kind = 4;
                c.smem = need;
            }
        }
    } else {
        return fail(SPTRSV_ERR_ARG, "unknown sync mode");
    }
    const void *k = kernel_ptr<T>(c);
    if (c.smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(c.smem));
        if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    }
    if (c.kind == 3 || c.kind == 4 || c.kind == 7) {
        c.grid = 1;
        return SPTRSV_OK;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, c.threads, c.smem);
    if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, cudaGetErrorString(e));
    int want = o.blocks_per_sm ? o.blocks_per_sm : std::min(per_sm, c.sync == SPTRSV_SYNC_FLAGS ? 2 : 1);
    if (want > per_sm || want < 1)
        return fail(SPTRSV_ERR_LAUNCH, "persistent grid of " + std::to_string(want) +
                                           " blocks/SM cannot be co-resident (max " +
                                           std::to_string(per_sm) + ")");
    c.grid = std::max(1, want * p->num_sms);
    return SPTRSV_OK;
}

template <typename T>
int launch(sptrsv_plan *p, const LaunchCfg &c, const SolveArgs<T> &args, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.grid);
    cfg.blockDim = dim3(c.threads);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = (c.kind == 3 || c.kind == 4 || c.kind == 7) ? 0 : 1;   // co-residency or error
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    const int nph = int(p->h.phase_row.size()) - 1;
    const void *k = kernel_ptr<T>(c);
    if (c.kind == 0 || c.kind == 2 || c.kind == 5 || c.kind == 6) {
        e = cudaLaunchKernelEx(&cfg, reinterpret_cast<Kern<T>>(const_cast<void *>(k)), args);
    } else if (c.kind == 4) {
        e = cudaLaunchKernelEx(&cfg, reinterpret_cast<StageKern<T>>(const_cast<void *>(k)), args, c.si, nph, c.win);
    } else {
        e = cudaLaunchKernelEx(&cfg, reinterpret_cast<WalkKern<T>>(const_cast<void *>(k)), args, nph,
                               (c.kind == 3 || c.kind == 7) ? c.win : 0);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(e == cudaErrorCooperativeLaunchTooLarge ? SPTRSV_ERR_LAUNCH : SPTRSV_ERR_CUDA,
                    std::string("launch: ") + cudaGetErrorString(e));
    }
    return SPTRSV_OK;
}

template <typename T>
SolveArgs<T> base_args(sptrsv_plan *p, const T *val, const T *dinv) {
    SolveArgs<T> a;
    a.n = p->h.n;
    a.S = p->h.S;
    a.nrhs = 0;
    a.rp = p->d.rp;
    a.col = p->d.col;
    a.val = val;
    a.dinv = dinv;
    a.perm = p->d.perm;
    a.step_blk = p->d.step_blk;
    a.blk_phase = p->d.blk_phase;
    a.phase_row = p->d.phase_row;
    a.blk_row = nullptr;
    a.chunk = nullptr;
    a.bdc = nullptr;
    a.b = nullptr;
    a.x = nullptr;
    a.ldb = a.ldx = 0;
    a.brs = a.xrs = 1;
    a.ctl = reinterpret_cast<Ctl *>(p->d.counters);
    a.flags = p->d.flags;
    a.epoch = 0;
    a.timeout_ns = 0;
    a.refine = 0;
    a.sweep = 0;
    a.x64 = nullptr;
    a.ldx64 = 0;
    a.x64rs = 1;
    a.rtol = 0.0;
    a.lnorm = p->lnorm;
    return a;
}

// Device workspace owned by the plan, grown on demand (refinement vectors).
int ensure_work(sptrsv_plan *p, size_t bytes) {
    if (p->d.work_bytes >= bytes) return SPTRSV_OK;
    if (p->d.work) {
        cudaError_t e = cudaFree(p->d.work);
        p->d.work = nullptr;
        p->d.work_bytes = 0;
        if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, std::string("cudaFree: ") + cudaGetErrorString(e));
    }
    CUDA_TRY(cudaMalloc(&p->d.work, bytes));
    p->d.work_bytes = bytes;
    return SPTRSV_OK;
}

int check_solve_args(const sptrsv_plan *p, const void *b, const void *x, int32_t nrhs, int64_t ld,
                     int32_t dtype, const sptrsv_solve_opts &o) {
    if (!p) return fail(SPTRSV_ERR_ARG, "plan is NULL");
    if (p->device < 0) return fail(SPTRSV_ERR_NO_DEVICE, "plan was analysed host-only");
    if (nrhs < 0 || (p->h.n > 0 && nrhs > 0 && (!b || !x)) || ld < std::max<int64_t>(p->h.n, 1))
        return fail(SPTRSV_ERR_ARG, "bad b/x/nrhs/ld");
    if (dtype != SPTRSV_F64 && dtype != SPTRSV_F32) return fail(SPTRSV_ERR_ARG, "dtype must be SPTRSV_F64 or SPTRSV_F32");
    if (!(o.timeout_s > 0.0)) return fail(SPTRSV_ERR_ARG, "timeout_s must be positive");
    if (o.precision != SPTRSV_PREC_F64 && o.precision != SPTRSV_PREC_F32_REFINE)
        return fail(SPTRSV_ERR_ARG, "unknown precision mode");
    return SPTRSV_OK;
}

template <typename T>
int plain_solve(sptrsv_plan *p, const T *val, const T *dinv, const void *b, void *x, int32_t nrhs, int64_t ld,
                const sptrsv_solve_opts &o, cudaStream_t s, LaunchCfg &c) {
    int st = choose<T>(p, o, nrhs, c);
    if (st) return st;
    SolveArgs<T> a = base_args<T>(p, val, dinv);
    a.nrhs = nrhs;
    a.b = static_cast<const T *>(b);
    a.x = static_cast<T *>(x);
    a.ldb = a.ldx = ld;
    a.timeout_ns = (long long)(o.timeout_s * 1e9);
    if (c.kind == 4) {      // staged walk: b in device order, row-major, in the plan workspace
        if ((st = ensure_work(p, size_t(p->h.n) * size_t(nrhs) * sizeof(T) + 256))) return st;
        c.si.bdev = p->d.work;
    }
    if (c.kind == 5) use_local(p, a);
    if (c.kind == 6) use_chunks(p, a);
    // right-hand-side tiles on the grid executors: internal row-major copies of b
    // and x (original row order), so a tile gathers a parent's values in one load
    const bool rows = c.rp && nrhs > 1 && (c.kind == 0 || c.kind == 1) && p->h.n > 0;
    T *xr = nullptr;
    const dim3 tgrid((p->h.n + 31) / 32, (nrhs + 31) / 32), tblock(32, 8);
    if (rows) {
        const size_t vec = (size_t(p->h.n) * size_t(nrhs) * sizeof(T) + 255) & ~size_t(255);
        if ((st = ensure_work(p, 2 * vec + 256))) return st;
        T *br = static_cast<T *>(p->d.work);
        xr = reinterpret_cast<T *>(static_cast<char *>(p->d.work) + vec);
        k_to_rows<T><<<tgrid, tblock, 0, s>>>(static_cast<const T *>(b), ld, br, c.kind == 0 ? xr : nullptr,
                                               p->h.n, nrhs);
        CUDA_TRY(cudaGetLastError());
        a.b = br;
        a.x = xr;
        a.ldb = a.ldx = 1;
        a.brs = a.xrs = nrhs;
    } else if (c.kind == 0 || c.kind == 5 || c.kind == 6) {   // polled solve: x starts as all-ones NaN
        CUDA_TRY(cudaMemset2DAsync(x, size_t(ld) * sizeof(T), 0xFF, size_t(p->h.n) * sizeof(T), size_t(nrhs), s));
    }
    // zero the counters but keep the status word: a device error of an
    // asynchronous solve stays visible until a report reads and clears it
    CUDA_TRY(cudaMemsetAsync(p->d.counters, 0, offsetof(Ctl, status), s));
    if ((st = launch<T>(p, c, a, s))) return st;
    if (rows) {
        k_to_cols<T><<<tgrid, tblock, 0, s>>>(xr, static_cast<T *>(x), ld, p->h.n, nrhs);
        CUDA_TRY(cudaGetLastError());
    }
    return SPTRSV_OK;
}


// FP32 sweeps with FP64 residual refinement, all decisions taken on the device:
// for t = 0..M: r_t = b - L x_t (FP64; r_0 = b), d_t = solve32(L32, fp32(r_t)),
// x_{t+1} = x_t + d_t (FP64, in the sweep's epilogue); then one last residual.
// A sweep returns at once when the refinement has converged, so the whole
// sequence is enqueued without host synchronisation.
int refine_solve(sptrsv_plan *p, const double *b, double *x, int32_t nrhs, int64_t ld, const sptrsv_solve_opts &o,
                 cudaStream_t s, LaunchCfg &c) {
    if (!(p->values & SPTRSV_VALUES_F32)) return fail(SPTRSV_ERR_ARG, "plan has no FP32 values");
    if (o.max_iters < 0 || o.max_iters > kMaxSweeps - 2) return fail(SPTRSV_ERR_ARG, "max_iters must be in [0, 14]");
    if (!(o.refine_tol > 0.0)) return fail(SPTRSV_ERR_ARG, "refine_tol must be positive");
    int st = choose<float>(p, o, nrhs, c);
    if (st) return st;
    const int32_t n = p->h.n;
    const size_t vec = size_t(n) * size_t(nrhs) * sizeof(float);
    const size_t vpad = (vec + 255) & ~size_t(255);
    // right-hand-side tiles on the grid executors: residual, correction, b and the
    // FP64 iterate all kept row-major in internal buffers (a row's right-hand
    // sides in one or two lines; b and x change layout once, at the ends)
    const bool rows = c.rp && nrhs > 1 && (c.kind == 0 || c.kind == 1) && n > 0;
    const size_t dpad = rows ? ((size_t(n) * size_t(nrhs) * sizeof(double) + 255) & ~size_t(255)) : 0;
    if ((st = ensure_work(p, 3 * vpad + 2 * dpad + 256))) return st;
    char *wk = static_cast<char *>(p->d.work);
    float *r32 = reinterpret_cast<float *>(wk);
    float *d32 = reinterpret_cast<float *>(wk + vpad);
    c.si.bdev = wk + 2 * vpad;                                   // staged walk: b in device order
    double *br = rows ? reinterpret_cast<double *>(wk + 3 * vpad) : nullptr;
    double *xr = rows ? reinterpret_cast<double *>(wk + 3 * vpad + dpad) : nullptr;
    const dim3 tgrid((n + 31) / 32, (nrhs + 31) / 32), tblock(32, 8);
    CUDA_TRY(cudaMemsetAsync(p->d.counters, 0, offsetof(Ctl, status), s));
    if (rows) {
        k_to_rows<double><<<tgrid, tblock, 0, s>>>(b, ld, br, nullptr, n, nrhs);
        CUDA_TRY(cudaGetLastError());
    }
    ResidualArgs ra;
    ra.n = n;
    ra.nrhs = nrhs;
    ra.rp = p->d.rp;
    ra.col = p->d.col;
    ra.hi = p->d.val_hi;
    ra.lo = p->d.val_lo;
    ra.v64 = p->d.val;                 // FP64 values held: one FMA per entry (else the hi/lo split)
    ra.dhi = p->d.diag_hi;
    ra.dlo = p->d.diag_lo;
    ra.perm = p->d.perm;
    ra.b = rows ? br : b;
    ra.ldb = rows ? 1 : ld;
    ra.b_rs = rows ? nrhs : 1;
    ra.x = rows ? xr : x;
    ra.ldx = rows ? 1 : ld;
    ra.x_rs = rows ? nrhs : 1;
    ra.r32 = r32;
    ra.r_rs = rows ? nrhs : 1;
    ra.r_cs = rows ? 1 : n;
    ra.ctl = reinterpret_cast<Ctl *>(p->d.counters);
    ra.dtol = o.refine_tol;
    const int rgrid = std::max(1, std::min(4 * p->num_sms, (n + 255) / 256));
    SolveArgs<float> a = base_args<float>(p, p->d.s32, p->d.dinv32);
    a.nrhs = nrhs;
    a.b = r32;
    a.x = d32;
    if (rows) {
        a.ldb = a.ldx = 1;
        a.brs = a.xrs = nrhs;
        a.x64 = xr;
        a.ldx64 = 1;
        a.x64rs = nrhs;
    } else {
        a.ldb = a.ldx = n;
        a.x64 = x;
        a.ldx64 = ld;
    }
    a.timeout_ns = (long long)(o.timeout_s * 1e9);
    a.rtol = o.refine_tol;
    if (c.kind == 5) use_local(p, a);
    if (c.kind == 6) use_chunks(p, a);
    const int M = o.max_iters;
    for (int t = 0; t <= M + 1; ++t) {
        ra.sweep = t;
        if (ra.v64) k_residual_scaled<<<rgrid, 256, 0, s>>>(ra);
        else k_residual<<<rgrid, 256, 0, s>>>(ra);
        CUDA_TRY(cudaGetLastError());
        if (t > M) break;
        if (c.kind == 0 || c.kind == 5 || c.kind == 6) CUDA_TRY(cudaMemsetAsync(d32, 0xFF, vec, s));   // polled
        else CUDA_TRY(cudaMemsetAsync(p->d.counters, 0, sizeof(unsigned long long), s));  // fresh barrier count
        a.refine = t == 0 ? 1 : 2;
        a.sweep = t;
        if ((st = launch<float>(p, c, a, s))) return st;
    }
    if (rows) {
        k_to_cols<double><<<tgrid, tblock, 0, s>>>(xr, x, ld, n, nrhs);
        CUDA_TRY(cudaGetLastError());
    }
    return SPTRSV_OK;
}

int solve_impl(sptrsv_plan *p, const void *b, void *x, int32_t nrhs, int64_t ld, int32_t dtype,
               const sptrsv_solve_opts &o, cudaStream_t s, LaunchCfg &c) {
    p->tuned_slot = tune_slot(dtype, o.precision, nrhs);
    if (dtype == SPTRSV_F64) {
        if (o.precision == SPTRSV_PREC_F64) {
            if (!(p->values & SPTRSV_VALUES_F64)) return fail(SPTRSV_ERR_ARG, "plan has no FP64 values");
            return plain_solve<double>(p, p->d.val, p->d.dinv, b, x, nrhs, ld, o, s, c);
        }
        return refine_solve(p, static_cast<const double *>(b), static_cast<double *>(x), nrhs, ld, o, s, c);
    }
    if (!(p->values & SPTRSV_VALUES_F32)) return fail(SPTRSV_ERR_ARG, "plan has no FP32 values");
    return plain_solve<float>(p, p->d.s32, p->d.dinv32, b, x, nrhs, ld, o, s, c);
}

int read_report(sptrsv_plan *p, const LaunchCfg &c, cudaStream_t s, sptrsv_report *report, bool refine,
                const sptrsv_solve_opts &o) {
    Ctl ctl;
    CUDA_TRY(cudaMemcpyAsync(&ctl, p->d.counters, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    std::memset(report, 0, sizeof(*report));
    report->status = ctl.status;
    report->sweeps = 1;
    if (refine && !ctl.status) {
        const int last = std::max(0, ctl.last_solve);
        report->sweeps = last + 1;
        const double xm = bits_to_d(ctl.xmax[last]);
        report->dnorm = xm > 0 ? bits_to_d(ctl.dmax[last]) / xm : 0.0;
        // backward error of the final iterate (residual index last + 1), if it was formed
        const double rm = bits_to_d(ctl.rmax[last + 1]);
        const double den = p->lnorm * xm + bits_to_d(ctl.bmax);
        report->berr = den > 0 ? rm / den : 0.0;
        const bool converged = ctl.done || report->dnorm <= o.refine_tol || report->berr <= o.refine_tol;
        if (!converged) report->status = SPTRSV_ERR_NOT_CONVERGED;
    }
    report->barriers = int64_t(ctl.barriers);
    report->flag_waits = int64_t(ctl.flag_waits);
    report->sync = c.sync;
    report->lanes = c.lanes;
    report->grid = c.grid;
    report->threads = c.threads;
    report->cross_edges = (c.kind == 5 || c.kind == 6) ? p->d.cross_edges : -1;
    report->edges = p->nnz_off;
    if (ctl.status) {
        CUDA_TRY(cudaMemsetAsync(&reinterpret_cast<Ctl *>(p->d.counters)->status, 0, sizeof(int32_t), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return fail(ctl.status, "device reported " + std::string(sptrsv_status_string(ctl.status)));
    }
    if (report->status == SPTRSV_ERR_NOT_CONVERGED)
        return fail(SPTRSV_ERR_NOT_CONVERGED, "refinement did not converge within max_iters (x is the last iterate)");
    return SPTRSV_OK;
}
}  // namespace
}  // namespace sptrsv

using namespace sptrsv;

extern "C" {

void sptrsv_solve_opts_default(sptrsv_solve_opts *o) {
    if (!o) return;
    o->sync = SPTRSV_SYNC_AUTO;
    o->lanes = 0;
    o->precision = SPTRSV_PREC_F64;
    o->max_iters = 6;
    o->refine_tol = 1e-13;
    o->blocks_per_sm = 0;
    o->threads = 0;
    o->timeout_s = 2.0;
    o->rhs_tile = 0;
    o->eager_sum = SPTRSV_EAGER_AUTO;
    o->partition = SPTRSV_PART_AUTO;
}

int sptrsv_solve(sptrsv_plan *p, const void *b, void *x, int32_t nrhs, int64_t ld, int32_t dtype,
                 const sptrsv_solve_opts *opts, sptrsv_stream stream, sptrsv_report *report) {
    clear_error();
    sptrsv_solve_opts o;
    sptrsv_solve_opts_default(&o);
    if (opts) o = *opts;
    int st = check_solve_args(p, b, x, nrhs, ld, dtype, o);
    if (st) return st;
    DeviceGuard g(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->h.n == 0 || nrhs == 0) {
        if (report) std::memset(report, 0, sizeof(*report));
        return SPTRSV_OK;
    }
    LaunchCfg c{};
    st = solve_impl(p, b, x, nrhs, ld, dtype, o, s, c);
    if (st) return st;
    if (report) return read_report(p, c, s, report, dtype == SPTRSV_F64 && o.precision == SPTRSV_PREC_F32_REFINE, o);
    return SPTRSV_OK;
}

int sptrsv_solve_host(sptrsv_plan *p, const void *b_host, void *x_host, int32_t nrhs, int64_t ld, int32_t dtype,
                      const sptrsv_solve_opts *opts, sptrsv_stream stream, sptrsv_report *report) {
    clear_error();
    if (!b_host || !x_host) return fail(SPTRSV_ERR_ARG, "host buffers must not be NULL");
    if (!p) return fail(SPTRSV_ERR_ARG, "plan is NULL");
    if (dtype != SPTRSV_F64 && dtype != SPTRSV_F32) return fail(SPTRSV_ERR_ARG, "dtype must be F64 or F32");
    if (nrhs < 0 || (nrhs > 0 && ld < std::max<int64_t>(p->h.n, 1)))
        return fail(SPTRSV_ERR_ARG, "nrhs must be >= 0 and ld >= n");
    if (p->device < 0) return fail(SPTRSV_ERR_NO_DEVICE, "plan has no device copy");
    if (p->h.n == 0 || nrhs == 0) {
        if (report) std::memset(report, 0, sizeof(*report));
        return SPTRSV_OK;
    }
    DeviceGuard g(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = dtype == SPTRSV_F64 ? sizeof(double) : sizeof(float);
    const size_t n = size_t(p->h.n), vec = (n * size_t(nrhs) * es + 255) & ~size_t(255);
    if (p->d.io_bytes < 2 * vec) {
        if (p->d.io) {
            CUDA_TRY(cudaFree(p->d.io));
            p->device_bytes -= int64_t(p->d.io_bytes);
            p->d.io = nullptr;
            p->d.io_bytes = 0;
        }
        CUDA_TRY(cudaMalloc(&p->d.io, 2 * vec));
        p->d.io_bytes = 2 * vec;
        p->device_bytes += int64_t(2 * vec);
    }
    char *bd = static_cast<char *>(p->d.io), *xd = bd + vec;
    CUDA_TRY(cudaMemcpy2DAsync(bd, n * es, b_host, size_t(ld) * es, n * es, size_t(nrhs), cudaMemcpyHostToDevice, s));
    sptrsv_solve_opts o;
    sptrsv_solve_opts_default(&o);
    if (opts) o = *opts;
    int st = check_solve_args(p, bd, xd, nrhs, int64_t(n), dtype, o);
    if (st) return st;
    LaunchCfg c{};
    st = solve_impl(p, bd, xd, nrhs, int64_t(n), dtype, o, s, c);
    if (st) return st;
    CUDA_TRY(cudaMemcpy2DAsync(x_host, size_t(ld) * es, xd, n * es, n * es, size_t(nrhs), cudaMemcpyDeviceToHost, s));
    if (report) return read_report(p, c, s, report, dtype == SPTRSV_F64 && o.precision == SPTRSV_PREC_F32_REFINE, o);
    return SPTRSV_OK;
}

int sptrsv_autotune(sptrsv_plan *p, const void *b, void *x, int32_t nrhs, int64_t ld, int32_t dtype,
                    const sptrsv_solve_opts *base, sptrsv_stream stream, sptrsv_solve_opts *best,
                    double *best_ms) {
    clear_error();
    sptrsv_solve_opts o;
    sptrsv_solve_opts_default(&o);
    if (base) o = *base;
    int st = check_solve_args(p, b, x, nrhs, ld, dtype, o);
    if (st) return st;
    if (p->h.n == 0 || nrhs == 0) return fail(SPTRSV_ERR_ARG, "nothing to tune");
    DeviceGuard g(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<sptrsv_solve_opts> cands;
    const bool small = int64_t(p->h.n) * nrhs <= 400000;
    // row mappings: (rhs_tile, lanes); entry-split lanes, plus right-hand-side tiles for nrhs >= 2
    std::vector<std::pair<int, int>> maps;
    for (int lanes : {1, 2, 4, 8, 16, 32}) maps.push_back({1, lanes});
    if (nrhs >= 2)
        for (int tile : {4, 8, 16, 32})
            if (tile / 2 < nrhs) maps.push_back({tile, 0});
    for (int sync : {SPTRSV_SYNC_CTA, SPTRSV_SYNC_CTA_REGS, SPTRSV_SYNC_GRID, SPTRSV_SYNC_FLAGS, SPTRSV_SYNC_LOCAL}) {
        if ((sync == SPTRSV_SYNC_CTA || sync == SPTRSV_SYNC_CTA_REGS) && !small) continue;
        if (sync == SPTRSV_SYNC_LOCAL && nrhs != 1) continue;
        for (auto [tile, lanes] : maps) {
            if (sync == SPTRSV_SYNC_LOCAL && tile != 1) continue;
            for (int t : {128, 256, 512, 1024})
                for (int bps : {1, 2}) {
                    if (t > 512 && sync != SPTRSV_SYNC_LOCAL) continue;
                    const bool one_block = sync == SPTRSV_SYNC_CTA || sync == SPTRSV_SYNC_CTA_REGS;
                    if ((one_block || sync == SPTRSV_SYNC_LOCAL) && bps > 1) continue;
                    sptrsv_solve_opts c = o;
                    c.sync = sync; c.rhs_tile = tile; c.lanes = lanes; c.threads = t;
                    c.blocks_per_sm = one_block ? 0 : bps;
                    c.eager_sum = SPTRSV_EAGER_ON;
                    if (sync == SPTRSV_SYNC_LOCAL) c.partition = SPTRSV_PART_PARENTS;
                    cands.push_back(c);
                    if ((sync == SPTRSV_SYNC_FLAGS || sync == SPTRSV_SYNC_LOCAL) && tile == 1 && lanes > 1) {
                        c.eager_sum = SPTRSV_EAGER_OFF;
                        cands.push_back(c);
                    }
                }
        }
    }
    // chunked executor: both partitions (all candidates of one partition in a row,
    // so the partition is built once per kind)
    if (nrhs == 1)
        for (int part : {SPTRSV_PART_PARENTS, SPTRSV_PART_RANGES, SPTRSV_PART_GRID})
            for (int t : {256, 384, 512, 640, 768}) {  // 640, 768: chunks of at most three entries
                sptrsv_solve_opts c = o;
                c.sync = SPTRSV_SYNC_CHUNKS;
                c.rhs_tile = 1;
                c.lanes = 1;
                c.threads = t;
                c.blocks_per_sm = 1;
                c.partition = part;
                cands.push_back(c);
            }
    // resident one-block executor: small factors that fit one SM's shared memory
    if (nrhs == 1)
        for (int t : {128, 256, 512, 1024}) {
            sptrsv_solve_opts c = o;
            c.sync = SPTRSV_SYNC_RESIDENT;
            c.rhs_tile = 1;
            c.lanes = 1;
            c.threads = t;
            c.blocks_per_sm = 0;
            cands.push_back(c);
        }
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    double best_t = 1e30;
    sptrsv_solve_opts best_o = o;
    for (const sptrsv_solve_opts &c : cands) {
        LaunchCfg lc{};
        if (solve_impl(p, b, x, nrhs, ld, dtype, c, s, lc)) continue;     // e.g. not co-resident
        sptrsv_report rep;
        if (read_report(p, lc, s, &rep, dtype == SPTRSV_F64 && c.precision == SPTRSV_PREC_F32_REFINE, c)) continue;
        double t = 1e30;
        for (int rep_i = 0; rep_i < 3; ++rep_i) {
            cudaEventRecord(e0, s);
            if (solve_impl(p, b, x, nrhs, ld, dtype, c, s, lc)) break;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, double(ms));
            if (t > 4.0 * best_t) break;
        }
        if (t < best_t) {
            best_t = t;
            best_o = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    clear_error();
    if (best_t >= 1e30) return fail(SPTRSV_ERR_LAUNCH, "no candidate configuration ran");
    TunedCfg &m = p->tuned[tune_slot(dtype, o.precision, nrhs)];
    m.valid = true;
    m.sync = best_o.sync;
    m.lanes = best_o.lanes;
    m.threads = best_o.threads;
    m.blocks_per_sm = best_o.blocks_per_sm;
    m.rhs_tile = best_o.rhs_tile;
    m.eager_sum = best_o.eager_sum;
    m.partition = best_o.partition;
    m.ms = best_t;
    if (best) *best = best_o;
    if (best_ms) *best_ms = best_t;
    return SPTRSV_OK;
}

}  // extern "C"
