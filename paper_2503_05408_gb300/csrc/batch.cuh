// Internal interface of the batched executor, shared by the batch and the
// serving loop (work items, per-item results, launch helpers).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "plan.hpp"

namespace sptrsv {

// Row mappings a block can use for an item (variant id -> kernel shape).
enum Variant : int32_t {
    V_L1 = 0, V_L2, V_L4,              // lanes split each row's entries
    V_T4, V_T8, V_T16, V_T32,          // right-hand-side tiles
    V_COUNT
};
constexpr int kVariantLanes[V_COUNT] = {1, 2, 4, 4, 8, 16, 32};

struct BatchItem {
    int32_t n, nphases, win, variant, nrhs;
    int32_t staged;                                 // 1: TMA-staged walk (the item's phases fit)
    StageInfo si;                                   // staged layout (bdev points into the workspace)
    const int32_t *rp, *col, *perm, *phase_row;
    const double *val, *dinv;                       // FP64 values, reciprocal diagonal
    const float *hi, *lo, *dhi, *dlo;               // FP32 split (FP64 residual)
    const float *s32, *dinv32;                      // FP32 sweep: scaled values, reciprocal diagonal
    double lnorm;
    const void *b;
    void *x;
    int64_t ldb, ldx;
    float *r32, *d32;                               // refinement workspace, leading dimension n
    void *bdev;                                     // staged walk: b (or r) in device order
};

struct ItemResult {
    int32_t status, sweeps;
    double dnorm, berr;
};

struct BatchCfg {
    int32_t refine, max_iters;
    double tol;
};

int batch_default_variant(const sptrsv_plan *p, int nrhs);
// Fill the factor part of an item (vectors and workspace are set by the caller).
void batch_fill_item(BatchItem &it, const sptrsv_plan *p, int nrhs, bool refine, size_t ring_budget);
// Device workspace an item needs (refinement vectors, staged right-hand sides), bytes.
size_t batch_item_workspace(const BatchItem &it, bool refine);
// Carve an item's workspace out of `base` (at least batch_item_workspace bytes, 256-aligned).
void batch_bind_workspace(BatchItem &it, char *base, bool refine);
// Shared memory one block of the batched executor needs for this item.
size_t batch_item_smem(const BatchItem &it, bool refine);
// Blocks of k_batch that fit on one SM for this block size and dynamic shared memory.
int batch_occupancy(int threads, size_t smem, int *per_sm);
// Enqueue one batch launch over `count` device items (cursor is zeroed first).
int batch_launch(const BatchItem *d_items, int count, ItemResult *d_res, unsigned int *d_cursor,
                 const BatchCfg &cfg, int grid, int threads, size_t smem, cudaStream_t s);

}  // namespace sptrsv
