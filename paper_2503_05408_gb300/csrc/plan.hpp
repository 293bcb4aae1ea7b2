// Internal definitions shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "sptrsv.h"

namespace sptrsv {

// Thread-local error message + status helper.
int fail(int status, const std::string &msg);
void clear_error();

// Host-side result of the analysis (Sec. 2.2 DAG, Sec. 1 wavefronts, Sec. 3
// schedule, Sec. 5 reordering) plus the execution structure the kernels walk.
//
// Execution structure: superstep s owns blocks [step_blk[s], step_blk[s+1]);
// block b (one core's share of a superstep, Def. 2.1) owns phases
// [blk_phase[b], blk_phase[b+1]); phase q owns device rows
// [phase_row[q], phase_row[q+1]).  Rows of one phase are mutually
// independent once every earlier phase of the block and every earlier
// superstep is finished.  For the wavefront schedule every superstep is one
// block with one phase.
struct HostSchedule {
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t nlevels = 0;
    int32_t max_level_rows = 0;
    int32_t mode = SPTRSV_SCHED_LEVELS;
    int32_t k = 1;
    int32_t S = 0;
    int32_t sched_blocks = 1;        // diagonal blocks GrowLocal was run on (Sec. 3.1)
    int32_t coarse_vertices = 0;     // vertices of the scheduled DAG (Funnel parts, else n)
    std::vector<int32_t> coarse_part; // Funnel plans: the part of every row (analysed numbering)
    double schedule_ms = 0.0;        // host wall time of the superstep schedule alone
    // block-local executor partition, once built (or read from a saved plan):
    // loc_blk[v] = block of row v, loc_lidx[v] = its position in the block's list
    int32_t loc_nb = 0;
    std::vector<int32_t> loc_blk, loc_lidx;
    int32_t loc_part = 0;            // SPTRSV_PART_* that built it; -1 read from a saved plan
    int32_t loc_gen = 0;             // bumped whenever the partition changes
    std::vector<int32_t> level, sigma, pi;
    std::vector<int32_t> perm;       // Sec. 5 order: position -> original row
    std::vector<int32_t> dev_perm;   // device order: device row -> original row
    std::vector<int32_t> step_blk, blk_phase, phase_row;
    int32_t max_phase_rows = 0;
    int32_t max_block_rows = 0;
    int32_t max_phase_ents = 0;   // largest number of off-diagonal entries in one phase
    // Smallest power-of-two ring (rows) that can hold x in shared memory when one
    // thread block walks the phases in order (0 = none up to kMaxRingRows).
    int32_t ring_rows = 0;
};

struct DeviceBuffers {
    // matrix in device-row order; column ids stay ORIGINAL row ids
    int32_t *rp = nullptr;        // n + 1, off-diagonal entries only
    int32_t *col = nullptr;       // nnz_off
    double *val = nullptr;        // nnz_off (VALUES_F64): A_ij / A_ii
    double *dinv = nullptr;       // n: 1 / diagonal, rounded once on the host
    float *val_hi = nullptr, *val_lo = nullptr;    // nnz_off (VALUES_F32)
    float *diag_hi = nullptr, *diag_lo = nullptr;  // n: FP32 split of the diagonal (residual)
    float *dinv32 = nullptr;      // n: fp32(1 / diagonal) for the FP32 sweeps
    float *s32 = nullptr;         // nnz_off: fp32(A_ij / A_ii), the FP32 sweeps' scaled values
    int32_t *perm = nullptr;      // n: device row -> original row
    int32_t *step_blk = nullptr, *blk_phase = nullptr, *phase_row = nullptr;
    int32_t *phase_ent = nullptr; // entry offset (device-order row pointer) of every phase boundary
    // scratch
    unsigned long long *counters = nullptr;  // [0] barrier, [1] barriers done, [2] flag waits,
                                             // [3] work cursor, [4..] refinement norms
    int32_t *status = nullptr;    // device status word (0 ok, else SPTRSV_ERR_*)
    uint32_t *flags = nullptr;    // n ready flags holding the solve epoch
    void *work = nullptr;         // refinement / internal vectors (grown on demand)
    size_t work_bytes = 0;
    void *io = nullptr;           // host-buffer solves: device copies of b and x (grown on demand)
    size_t io_bytes = 0;
    // block-local executor layout (built on first use for loc_nb thread blocks):
    // rows block-major, each block's rows in (wavefront, id) order; a column id
    // c >= 0 is an original row id (parent of another block), c <= -2 names the
    // parent at position -c - 2 of the same block
    int32_t loc_nb = 0;           // 0 = not built
    size_t loc_smem = 0;          // shared memory of the largest block (its rows' values)
    int64_t loc_bytes = 0;
    int32_t *l_rp = nullptr, *l_col = nullptr, *l_perm = nullptr, *l_blk_row = nullptr;
    double *l_val = nullptr, *l_dinv = nullptr;
    float *l_s32 = nullptr, *l_dinv32 = nullptr;
    int32_t loc_gen = -1;         // partition generation the l_* arrays were built from
    // chunked executor layout (same partition, cut into chunks of <= 32 rows of
    // one wavefront): ck_info holds 4 int32 per chunk (entry offset, width | 1 << 16
    // if an entry names another block's row, rows, first shared-memory slot),
    // ck_blk the chunk range of every block, entries (each row's other-block
    // parents first)
    // sliced (entry u of lane l of a chunk at offset + 32 u + l), one orow/dinv
    // per chunk lane (-1 / 0 for lanes without a row)
    int32_t ck_gen = -1, ck_nb = 0, ck_width = 0;
    size_t ck_slots = 0;          // most rows of one block (shared-memory slots)
    int64_t ck_bytes = 0;
    int64_t cross_edges = 0, edges = 0;   // of the current partition
    int32_t *ck_info = nullptr, *ck_blk = nullptr, *ck_col = nullptr, *ck_orow = nullptr;
    double *ck_val = nullptr, *ck_dinv = nullptr;
    float *ck_s32 = nullptr, *ck_dinv32 = nullptr;
    void *ck_bd = nullptr;        // workspace: b_i / A_ii per chunk lane (8 bytes a lane, FP32 uses half)
};

}  // namespace sptrsv

struct sptrsv_plan {
    sptrsv::HostSchedule h;
    int32_t values = 0;
    int32_t device = -1;
    bool reversed = false;        // UPPER / LOWER_TRANSPOSED: analysed as L' with ids i' = n-1-i
    int32_t triangle = SPTRSV_TRI_LOWER;
    int32_t num_sms = 0;
    int64_t nnz_off = 0;
    int32_t max_row_off = 0;      // most off-diagonal entries in one row
    int64_t device_bytes = 0;
    double analyze_ms = 0.0;
    double lnorm = 0.0;           // ||L||inf in FP64 (backward-error test of the refinement)
    int32_t sticky_status = 0;    // device error seen by an asynchronous solve
    sptrsv::DeviceBuffers d;
    // autotuner memo: best launch shape per (dtype, precision, nrhs class); the slot of the
    // call being served is selected by sptrsv_solve before it picks a configuration
    struct TunedCfg {
        bool valid = false;
        int32_t sync = 0, lanes = 0, threads = 0, blocks_per_sm = 0, rhs_tile = 0, eager_sum = 0, partition = 0;
        double ms = 0.0;
    };
    TunedCfg tuned[16];
    int32_t tuned_slot = -1;
};
using TunedCfg = sptrsv_plan::TunedCfg;

namespace sptrsv {
// analyze.cpp
int validate_csr(const sptrsv_csr *A);
// Block-local partition (used by SPTRSV_SYNC_LOCAL).  Rows are taken in
// (wavefront, id) order; row v's off-diagonal parents are col[rp[row_of[v]] ..
// rp[row_of[v] + 1]) (original ids).  Outputs: blk[v] in [0, nb), lidx[v] = v's
// position in its block's (wavefront, id) list, load[b] = rows of block b.
// Returns false if the rows do not fit nb blocks of row_cap rows.
bool local_partition(int32_t n, int32_t nb, int32_t row_cap, const std::vector<int32_t> &level, int32_t nlevels,
                     const int32_t *rp, const int32_t *col, const int32_t *row_of, std::vector<int32_t> &blk,
                     std::vector<int32_t> &lidx, std::vector<int32_t> &load);
// Contiguous ranges of row ids: block b takes rows floor(b n / nb) ..
// floor((b+1) n / nb) - 1, each block's list in (wavefront, id) order.  Same
// outputs and failure as local_partition.
bool range_partition(int32_t n, int32_t nb, int32_t row_cap, const std::vector<int32_t> &level, int32_t nlevels,
                     std::vector<int32_t> &blk, std::vector<int32_t> &lidx, std::vector<int32_t> &load);
// Structured-grid partition: when the off-diagonal offsets of the factor are
// dominated by nested strides 1 | s1 | s2 (a 3D grid numbered in natural order:
// x-lines of s1 rows, planes of s2 rows), rows are grouped into pencils along
// the fastest stride and the (line, plane) index space is cut into TA x TB <= nb
// rectangular tiles, one per block.  Every dependency then goes to the same
// tile or one with a larger line or plane index, so the blocks' dependency
// graph is acyclic and a dependency path crosses at most TA + TB - 2 tiles.
// Lists in (wavefront, id) order.  Returns false when no such strides exist
// (or a tile exceeds row_cap); the caller falls back to local_partition.
bool grid_partition(int32_t n, int32_t nb, int32_t row_cap, const std::vector<int32_t> &level, int32_t nlevels,
                    const int32_t *rp, const int32_t *col, const int32_t *row_of, std::vector<int32_t> &blk,
                    std::vector<int32_t> &lidx, std::vector<int32_t> &load);
// A schedule read from a saved plan instead of computed (analysed numbering).
struct GivenSchedule {
    int32_t mode = SPTRSV_SCHED_LEVELS, k = 1, S = 0, sched_blocks = 1, coarse_vertices = 0;
    const int32_t *sigma = nullptr, *pi = nullptr;
    int32_t loc_nb = 0;                                  // saved block-local partition, if any
    const int32_t *loc_blk = nullptr, *loc_lidx = nullptr;
};
int build_schedule(const sptrsv_csr *A, const sptrsv_analyze_opts &o, HostSchedule &h,
                   const GivenSchedule *given = nullptr);
// sptrsv_analyze's body; `given` replaces the scheduler by a validated saved schedule.
int analyze_impl(const sptrsv_csr *csr, sptrsv_analyze_opts o, const GivenSchedule *given, sptrsv_plan **out);
// The lower factor a plan analyses: `csr` itself (LOWER) or L' numbered backwards
// (UPPER, LOWER_TRANSPOSED) built in rp/col/val; validated.  *use points to it.
int lower_factor(const sptrsv_csr *csr, int32_t triangle, std::vector<int32_t> &rp, std::vector<int32_t> &col,
                 std::vector<double> &val, sptrsv_csr &lowered, const sptrsv_csr **use);
// Smallest safe shared-memory x ring of a one-block walk (0: none), as build_schedule sets it.
int32_t ring_rows_of(const sptrsv_csr *A, const HostSchedule &h);
// analyze_gpu.cu: the wavefront schedule, its Sec. 5 order and the device layout
// computed on `device` from the analysed lower CSR (validated); fills p->h and p->d.
// reversed: A is L' with ids i' = n-1-i (UPPER, LOWER_TRANSPOSED); the device
// column ids and permutation are written in the caller's numbering.
int analyze_levels_device(sptrsv_plan *p, const sptrsv_csr *A, int device, int32_t values, bool reversed);
// analyze_gpu.cu: the block-local layout's values gathered on the device from the
// device-order arrays (entry q <- src[q], row t <- rsrc[t]); allocates l_val/l_dinv
// and/or l_s32/l_dinv32 as the plan holds FP64 and/or FP32 values.
int local_values_device(sptrsv_plan *p, const std::vector<int32_t> &src, const std::vector<int32_t> &rsrc,
                        int64_t *bytes);
// Wavefronts of a validated lower factor; returns their number.
int32_t factor_levels(const sptrsv_csr *A, std::vector<int32_t> &level);
// A saved block-local partition is usable: blocks in range, every block's list a
// permutation of 0..load-1 in (wavefront, id) order.
bool partition_valid(int32_t n, int32_t nb, const int32_t *blk, const int32_t *lidx, const std::vector<int32_t> &level);
// growlocal.cpp
int32_t growlocal_schedule(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k,
                           double alpha0, double growth, double L, double accept,
                           int32_t *sigma, int32_t *pi);
// GrowLocal with explicit vertex weights (a coarsened DAG).
int32_t growlocal_weighted(int32_t n, const int32_t *rowptr, const int32_t *col, const int64_t *weight, int32_t k,
                           double alpha0, double growth, double L, double accept, int32_t *sigma, int32_t *pi);
// funnel.cpp: Funnel + GrowLocal (Sec. 4): triangle transitive reduction, in-funnel
// coarsening with parts of weight <= max_weight, GrowLocal on the coarsened DAG,
// each row taking its part's superstep and core.  *parts = coarsened vertices;
// part_of (optional) receives every row's part, parts numbered by root id.
// threads: host threads of the triangle reduction (0: one per hardware thread).
int32_t funnel_growlocal(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k, double alpha0,
                         double growth, double L, double accept, double max_weight, int32_t threads, int32_t *sigma,
                         int32_t *pi, int32_t *parts, std::vector<int32_t> *part_of = nullptr);
// Block-parallel GrowLocal (Sec. 3.1): rows cut into `blocks` diagonal blocks of
// floor(b n / blocks) .. floor((b+1) n / blocks) - 1, each block's sub-DAG
// scheduled on one of `threads` host threads (0: one per hardware thread, at
// most one per block), block schedules concatenated in block order.  blocks <= 1
// is growlocal_schedule.  Returns the total number of supersteps.
int32_t growlocal_blocks(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t k,
                         double alpha0, double growth, double L, double accept,
                         int32_t blocks, int32_t threads, int32_t *sigma, int32_t *pi);
// device.cu
int upload_plan(sptrsv_plan *p, const sptrsv_csr *A);
void free_device(sptrsv_plan *p);
int device_sm_count(int device, int32_t *out);
}  // namespace sptrsv
