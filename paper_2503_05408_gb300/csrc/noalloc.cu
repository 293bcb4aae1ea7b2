// Allocation-free forward substitution on a caller-owned device CSR factor.
//
// Some callers cannot let a library call cudaMalloc: code whose every device
// byte is drawn from its own pool or budget, and latency-critical loops where
// an allocation may synchronise the device.  sptrsv_solve_csr_noalloc serves
// them: the caller passes the factor, b and x (all device memory it owns), and
// the only scratch the kernel needs - one ready flag per row and a few control
// words - lives in the file-scope array below, which every GPU that loads this
// library holds until the process exits.
//
// The kernel is a variant of the per-row ready-flag executor: rows are taken
// in natural order (topological for a lower-triangular factor), one warp per
// row, and each row waits on its parents' flags.  A flag holds the epoch of
// the call that set it, so the flags are never cleared between calls; the
// control words are cleared by a memset at the start of every call.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "plan.hpp"

namespace sptrsv {
namespace {

constexpr int kCtlWords = 64;                              // 256 bytes of control words
constexpr int32_t kMaxRows = SPTRSV_NOALLOC_MAX_ROWS;

// [0] status word, [1 .. kCtlWords) spare, [kCtlWords ...] one ready flag per row.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kCtlWords + kMaxRows];

struct DeviceSlot {
    bool ready = false;
    uint32_t *scratch = nullptr;   // device address of g_noalloc_scratch on this device
    uint32_t epoch = 0;
    int sms = 0;
    int blocks_per_sm = 0;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;

__device__ __forceinline__ void put_status(uint32_t *ctl, int32_t code) {
    atomicCAS(reinterpret_cast<int *>(ctl), 0, code);
}

__global__ void __launch_bounds__(256, 1)
k_flags_csr_noalloc(int32_t n, int64_t nnz, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                    const double *__restrict__ val, const double *__restrict__ b, double *x, uint32_t *scratch,
                    uint32_t epoch, long long timeout_ns) {
    uint32_t *ctl = scratch;
    uint32_t *flags = scratch + kCtlWords;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < n; r += nw) {
        const int32_t beg = rowptr[r], end = rowptr[r + 1];
        // the factor is not validated on the host: check what would break memory safety
        if (beg < 0 || end <= beg || int64_t(end) > nnz || col[end - 1] != r) {
            if (lane == 0) put_status(ctl, SPTRSV_ERR_ARG);
            break;
        }
        bool ok = true;
        double acc = 0.0;
        for (int q = beg + lane; q < end - 1; q += 32) {
            const int32_t c = col[q];
            if (c < 0 || c >= r) {                     // not strictly lower: would wait forever
                put_status(ctl, SPTRSV_ERR_NOT_LOWER);
                ok = false;
                break;
            }
            const uint32_t *f = flags + c;
            if (ld_acquire(f) != epoch) {
                const long long t0 = gtimer();
                unsigned spins = 0;
                while (ld_acquire(f) != epoch) {
                    if ((++spins & 63u) == 1) {
                        if (*reinterpret_cast<volatile int32_t *>(ctl) != 0) { ok = false; break; }
                        if (gtimer() - t0 > timeout_ns) {
                            put_status(ctl, SPTRSV_ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
                if (!ok) break;
            }
            acc += val[q] * x[c];
        }
        if (!__all_sync(0xffffffffu, ok)) break;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            x[r] = (b[r] - acc) / val[end - 1];
            st_release(flags + r, epoch);
        }
        __syncwarp();
    }
}

// Per-device set-up, run once with that device current: resolve the device
// address of the scratch array (its name in host code is only a stand-in).
int setup_device(int dev, DeviceSlot &slot) {
    void *addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) {
        (void)cudaGetLastError();
        return fail(SPTRSV_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") +
                                         cudaGetErrorString(e));
    }
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_flags_csr_noalloc, 256, 0);
    if (e != cudaSuccess || sms <= 0 || per_sm <= 0)
        return fail(SPTRSV_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    slot.scratch = static_cast<uint32_t *>(addr);
    slot.sms = sms;
    slot.blocks_per_sm = per_sm < 2 ? per_sm : 2;
    slot.ready = true;
    return SPTRSV_OK;
}

}  // namespace
}  // namespace sptrsv

using namespace sptrsv;

extern "C" int sptrsv_solve_csr_noalloc(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                                        const double *val, const double *b, double *x,
                                        sptrsv_stream stream) {
    clear_error();
    if (n < 0 || nnz < 0) return fail(SPTRSV_ERR_ARG, "negative size");
    if (n > kMaxRows)
        return fail(SPTRSV_ERR_ARG, "sptrsv_solve_csr_noalloc handles at most " + std::to_string(kMaxRows) +
                                        " rows (its scratch array is fixed); got n = " + std::to_string(n) +
                                        " - use sptrsv_analyze + sptrsv_solve instead");
    if (n == 0) return SPTRSV_OK;
    if (!rowptr || !col || !val || !b || !x) return fail(SPTRSV_ERR_ARG, "NULL device pointer");
    if (nnz < n || nnz > INT32_MAX) return fail(SPTRSV_ERR_ARG, "nnz must be in [n, 2^31)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(SPTRSV_ERR_ARG, "sptrsv_solve_csr_noalloc: device index " + std::to_string(dev) +
                                        " exceeds the " + std::to_string(kMaxDevices) + " devices it tracks");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *scratch;
    uint32_t epoch;
    int grid;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        DeviceSlot &slot = g_slots[dev];
        if (!slot.ready) {
            int st = setup_device(dev, slot);
            if (st) return st;
        }
        if (++slot.epoch == 0) {               // flags wrapped: clear them once
            e = cudaMemsetAsync(slot.scratch + kCtlWords, 0, size_t(kMaxRows) * sizeof(uint32_t), s);
            if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, cudaGetErrorString(e));
            slot.epoch = 1;
        }
        scratch = slot.scratch;
        epoch = slot.epoch;
        grid = slot.sms * slot.blocks_per_sm;
    }
    e = cudaMemsetAsync(scratch, 0, kCtlWords * sizeof(uint32_t), s);     // status and counters
    if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, cudaGetErrorString(e));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;                          // co-residency or error
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const long long timeout_ns = 2000000000LL;
    e = cudaLaunchKernelEx(&cfg, k_flags_csr_noalloc, n, nnz, rowptr, col, val, b, x, scratch, epoch, timeout_ns);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(SPTRSV_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    int32_t status = 0;
    e = cudaMemcpyAsync(&status, scratch, sizeof(status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SPTRSV_ERR_CUDA, cudaGetErrorString(e));
    if (status) return fail(status, std::string("device reported ") + sptrsv_status_string(status));
    return SPTRSV_OK;
}
