// Continuous-batching serving loop over resident factors.
//
// Clients submit solve requests (factor id, b/x in device memory or in host
// memory, number of right-hand sides).  A dispatcher thread admits requests in arrival order as soon as
// their device workspace fits the remaining HBM budget, packs every admitted
// request into one launch of the batched executor on a free stream slot, and
// keeps going while earlier launches still run: requests that arrive while
// others are on the GPU are admitted as slots and memory free up, and their
// work overlaps on the device.  Completion is observed through per-slot events;
// latency is completion time minus submission time.
//
// A second mode, SPTRSV_SERVE_SERIAL_F64, serves the same stream the plain way
// - one request per sptrsv_solve launch in FP64, one stream, arrival order -
// so both are measured by identical bookkeeping.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "plan.hpp"

namespace sptrsv {
namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int32_t fid = 0, nrhs = 0;
    const double *b = nullptr;
    double *x = nullptr;
    int64_t ld = 0;
    // host requests: b and x live in host memory; they are staged through device
    // buffers carved from the arena next to the workspace (n x nrhs each, ld = n)
    bool host = false;
    const double *b_host = nullptr;
    double *x_host = nullptr;
    int64_t ldb_host = 0, ldx_host = 0;
    size_t io_off = 0;             // offset of the staged b (then x) inside the request's arena block
    double t_arrive = 0.0, t_done = 0.0;
    int32_t state = 0;              // 0 pending, 1 in flight, 2 done
    size_t ws_off = 0, ws_bytes = 0;
    sptrsv_report rep{};
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    BatchItem *h_items = nullptr, *d_items = nullptr;
    ItemResult *h_res = nullptr, *d_res = nullptr;
    unsigned int *d_cursor = nullptr;
    std::vector<uint64_t> reqs;
    bool busy = false;
};

// First-fit allocator over the workspace arena (offsets), coalescing on free.
struct Arena {
    char *base = nullptr;
    size_t size = 0, in_use = 0, peak = 0;
    std::map<size_t, size_t> free_list;
    void init(char *b, size_t s) {
        base = b;
        size = s;
        free_list.clear();
        if (s) free_list[0] = s;
    }
    bool alloc(size_t bytes, size_t &off) {
        if (bytes == 0) {
            off = 0;
            return true;
        }
        for (auto it = free_list.begin(); it != free_list.end(); ++it)
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_list.erase(it);
                if (rest) free_list[off + bytes] = rest;
                in_use += bytes;
                peak = std::max(peak, in_use);
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        if (bytes == 0) return;
        in_use -= bytes;
        auto nx = free_list.lower_bound(off);
        size_t start = off, len = bytes;
        if (nx != free_list.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                start = pv->first;
                len += pv->second;
                free_list.erase(pv);
            }
        }
        nx = free_list.lower_bound(off);
        if (nx != free_list.end() && off + bytes == nx->first) {
            len += nx->second;
            free_list.erase(nx);
        }
        free_list[start] = len;
    }
};

constexpr size_t kServeRingBudget = 64 * 1024;
constexpr size_t kServeSmem = 96 * 1024;          // dynamic shared memory of every serving launch

// Upper bound of a request's workspace (refinement vectors + staged right-hand sides).
size_t workspace_bytes(const sptrsv_plan *p, int nrhs, bool refine) {
    const size_t v = (size_t(p->h.n) * size_t(nrhs) * sizeof(float) + 255) & ~size_t(255);
    const size_t bdev = (size_t(p->h.n) * size_t(nrhs) * (refine ? sizeof(float) : sizeof(double)) + 64 + 255) &
                        ~size_t(255);
    return (refine ? 2 * v : 0) + bdev;
}

// Device staging of a host request's b and x (n x nrhs doubles each).
size_t host_io_bytes(const sptrsv_plan *p, int nrhs) {
    return 2 * ((size_t(p->h.n) * size_t(nrhs) * sizeof(double) + 255) & ~size_t(255));
}

// Copies between a host request's buffers and its device staging (column-major).
cudaError_t stage_in(const Request &r, int32_t n, double *db, cudaStream_t s) {
    return cudaMemcpy2DAsync(db, size_t(n) * sizeof(double), r.b_host, size_t(r.ldb_host) * sizeof(double),
                             size_t(n) * sizeof(double), size_t(r.nrhs), cudaMemcpyHostToDevice, s);
}
cudaError_t stage_out(const Request &r, int32_t n, const double *dx, cudaStream_t s) {
    return cudaMemcpy2DAsync(r.x_host, size_t(r.ldx_host) * sizeof(double), dx, size_t(n) * sizeof(double),
                             size_t(n) * sizeof(double), size_t(r.nrhs), cudaMemcpyDeviceToHost, s);
}

}  // namespace
}  // namespace sptrsv

using namespace sptrsv;

struct sptrsv_server {
    int device = 0;
    size_t budget = 0;
    sptrsv_serve_opts opts{};
    bool refine = false;
    std::vector<sptrsv_plan *> factors;
    size_t factor_bytes = 0;
    void *arena_mem = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    std::vector<Slot> slots;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<int> worker_error{0};
    std::string worker_msg;
    // statistics
    std::vector<double> latencies;
    double t_first = -1.0, t_last = 0.0;
    int64_t submitted = 0, completed = 0, rejected = 0, launches = 0, items = 0;
    int threads = 256, per_sm = 1, sms = 1;
    size_t smem = 0;
    BatchCfg cfg{};
    int64_t inflight = 0;
};

namespace sptrsv {
namespace {

void finish_request(sptrsv_server *S, uint64_t id, const sptrsv_report &rep, double t) {
    Request &r = S->reqs[id];
    r.state = 2;
    r.t_done = t;
    r.rep = rep;
    r.rep.latency_s = t - r.t_arrive;
    S->arena.release(r.ws_off, r.ws_bytes);   // workspace and, for host requests, the staging
    S->latencies.push_back(t - r.t_arrive);
    S->t_last = std::max(S->t_last, t);
    ++S->completed;
    --S->inflight;
}

// Continuous mode: harvest finished slots, then fill free slots with admissible
// pending requests, one duration class per launch.
// Duration class of a request: its factor's critical path (wavefronts) in
// decades, 0: < 1000, 1: < 10000, 2: longer.
int duration_class(const sptrsv_server *S, uint64_t id) {
    const int32_t lv = S->factors[S->reqs.at(id).fid]->h.nlevels;
    return lv < 1000 ? 0 : lv < 10000 ? 1 : 2;
}

bool continuous_step(sptrsv_server *S) {
    bool did = false;
    for (Slot &sl : S->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        const double t = now_s();
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t i = 0; i < sl.reqs.size(); ++i) {
            sptrsv_report rep{};
            rep.status = q == cudaSuccess ? sl.h_res[i].status : SPTRSV_ERR_CUDA;
            rep.sweeps = sl.h_res[i].sweeps;
            rep.dnorm = sl.h_res[i].dnorm;
            rep.berr = sl.h_res[i].berr;
            rep.sync = SPTRSV_SYNC_CTA;
            rep.threads = S->threads;
            rep.lanes = kVariantLanes[sl.h_items[i].variant];
            finish_request(S, sl.reqs[i], rep, t);
        }
        sl.reqs.clear();
        sl.busy = false;
        did = true;
        S->cv.notify_all();
    }
    for (Slot &sl : S->slots) {
        if (sl.busy) continue;
        int cnt = 0;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            // A launch lasts as long as its longest item and holds its stream
            // until then, so a launch takes requests of one duration class only
            // (the class of the oldest pending request, then its peers in arrival
            // order): long dependency chains do not hold short requests back.
            const int cls = S->pending.empty() ? 0 : duration_class(S, S->pending.front());
            for (auto pit = S->pending.begin(); pit != S->pending.end() && cnt < S->opts.max_batch;) {
                const uint64_t id = *pit;
                if (duration_class(S, id) != cls) {
                    ++pit;
                    continue;
                }
                Request &r = S->reqs[id];
                const sptrsv_plan *p = S->factors[r.fid];
                BatchItem &it = sl.h_items[cnt];
                batch_fill_item(it, p, r.nrhs, S->refine, kServeRingBudget);
                if (batch_item_smem(it, S->refine) > S->smem) it.staged = 0;   // launch smem is fixed
                size_t off = 0;
                const size_t ws = (batch_item_workspace(it, S->refine) + 255) & ~size_t(255);
                const size_t need = ws + (r.host ? host_io_bytes(p, r.nrhs) : 0);
                if (!S->arena.alloc(need, off)) break;             // FIFO: wait for memory
                pit = S->pending.erase(pit);
                r.state = 1;
                r.ws_off = off;
                r.ws_bytes = need;
                if (r.host) {                                       // staged in the arena after the workspace
                    r.io_off = off + ws;
                    r.b = reinterpret_cast<double *>(S->arena.base + r.io_off);
                    r.x = reinterpret_cast<double *>(S->arena.base + r.io_off + host_io_bytes(p, r.nrhs) / 2);
                    r.ld = std::max<int64_t>(p->h.n, 1);
                }
                it.b = r.b;
                it.x = r.x;
                it.ldb = it.ldx = r.ld;
                if (ws) batch_bind_workspace(it, S->arena.base + off, S->refine);
                sl.reqs.push_back(id);
                ++cnt;
            }
        }
        if (cnt == 0) break;
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < cnt && e == cudaSuccess; ++i) {          // host requests: b in
            const Request &r = S->reqs[sl.reqs[i]];
            if (r.host) e = stage_in(r, S->factors[r.fid]->h.n, const_cast<double *>(r.b), sl.stream);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.d_items, sl.h_items, size_t(cnt) * sizeof(BatchItem), cudaMemcpyHostToDevice,
                                sl.stream);
        const int grid = std::max(1, std::min(cnt, S->sms * S->per_sm));
        int st = e == cudaSuccess ? batch_launch(sl.d_items, cnt, sl.d_res, sl.d_cursor, S->cfg, grid, S->threads,
                                                 S->smem, sl.stream)
                                  : SPTRSV_ERR_CUDA;
        if (!st) e = cudaMemcpyAsync(sl.h_res, sl.d_res, size_t(cnt) * sizeof(ItemResult), cudaMemcpyDeviceToHost,
                                     sl.stream);
        for (int i = 0; i < cnt && !st && e == cudaSuccess; ++i) {   // host requests: x out, inside the request
            const Request &r = S->reqs[sl.reqs[i]];
            if (r.host) e = stage_out(r, S->factors[r.fid]->h.n, r.x, sl.stream);
        }
        if (!st && e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        if (st || e != cudaSuccess) {
            S->worker_error = SPTRSV_ERR_CUDA;
            S->worker_msg = std::string("serving launch failed: ") + cudaGetErrorString(e);
            for (int i = 0; i < cnt; ++i) sl.h_res[i].status = SPTRSV_ERR_CUDA;
        }
        sl.busy = true;
        ++S->launches;
        S->items += cnt;
        did = true;
    }
    return did;
}

// Plain FP64 per-request baseline: one request per launch, one stream, arrival order.
bool serial_step(sptrsv_server *S) {
    uint64_t id;
    Request r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->pending.empty()) return false;
        id = S->pending.front();
        S->pending.pop_front();
        S->reqs[id].state = 1;
        r = S->reqs[id];
    }
    Slot &sl = S->slots[0];
    sptrsv_plan *p = S->factors[r.fid];
    sptrsv_solve_opts o;
    sptrsv_solve_opts_default(&o);
    o.precision = SPTRSV_PREC_F64;
    sptrsv_report rep{};
    int st = SPTRSV_OK;
    if (r.host) {          // one request at a time: its staging always fits the arena
        size_t off = 0;
        const size_t io = host_io_bytes(p, r.nrhs);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (!S->arena.alloc(io, off)) st = SPTRSV_ERR_BUDGET;
            else S->reqs[id].ws_off = off, S->reqs[id].ws_bytes = io;
        }
        r.b = reinterpret_cast<double *>(S->arena.base + off);
        r.x = reinterpret_cast<double *>(S->arena.base + off + io / 2);
        r.ld = std::max<int64_t>(p->h.n, 1);
        if (!st && stage_in(r, p->h.n, const_cast<double *>(r.b), sl.stream) != cudaSuccess) st = SPTRSV_ERR_CUDA;
    }
    if (!st)
        st = sptrsv_solve(p, r.b, r.x, r.nrhs, r.ld, SPTRSV_F64, &o, reinterpret_cast<sptrsv_stream>(sl.stream), &rep);
    if (!st && r.host) {
        cudaError_t e = stage_out(r, p->h.n, r.x, sl.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sl.stream);
        if (e != cudaSuccess) st = SPTRSV_ERR_CUDA;
    }
    if (st) rep.status = st;
    const double t = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    finish_request(S, id, rep, t);
    S->cv.notify_all();
    return true;
}

void worker_main(sptrsv_server *S) {
    cudaSetDevice(S->device);
    while (!S->stop.load()) {
        const bool did = S->opts.mode == SPTRSV_SERVE_SERIAL_F64 ? serial_step(S) : continuous_step(S);
        if (!did) {
            std::unique_lock<std::mutex> lk(S->mu);
            const bool idle = S->pending.empty() && S->inflight == 0;
            S->cv.wait_for(lk, std::chrono::microseconds(idle ? 500 : 20));
        }
    }
}

int ensure_arena(sptrsv_server *S) {
    if (S->arena_mem) return SPTRSV_OK;
    if (S->factor_bytes >= S->budget) return fail(SPTRSV_ERR_BUDGET, "resident factors fill the HBM budget");
    size_t size = S->budget - S->factor_bytes;
    cudaError_t e = cudaMalloc(&S->arena_mem, size);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(SPTRSV_ERR_OOM, std::string("workspace arena: ") + cudaGetErrorString(e));
    }
    S->arena.init(static_cast<char *>(S->arena_mem), size);
    return SPTRSV_OK;
}

}  // namespace
}  // namespace sptrsv

extern "C" {

void sptrsv_serve_opts_default(sptrsv_serve_opts *o) {
    if (!o) return;
    o->mode = SPTRSV_SERVE_CONTINUOUS;
    o->streams = 8;
    o->max_batch = 256;
    o->precision = SPTRSV_PREC_F32_REFINE;
    o->max_iters = 6;
    o->refine_tol = 1e-13;
    o->threads = 256;
    o->device = 0;
}

int sptrsv_serve_create(size_t hbm_budget, const sptrsv_serve_opts *opts, sptrsv_server **out) {
    clear_error();
    if (!out) return fail(SPTRSV_ERR_ARG, "out is NULL");
    *out = nullptr;
    sptrsv_serve_opts o;
    sptrsv_serve_opts_default(&o);
    if (opts) o = *opts;
    if (o.mode != SPTRSV_SERVE_CONTINUOUS && o.mode != SPTRSV_SERVE_SERIAL_F64) return fail(SPTRSV_ERR_ARG, "mode");
    if (o.streams < 1 || o.streams > 64 || o.max_batch < 1 || o.max_batch > 4096)
        return fail(SPTRSV_ERR_ARG, "streams in [1, 64], max_batch in [1, 4096]");
    if (o.threads < 32 || o.threads > 512 || o.threads % 32) return fail(SPTRSV_ERR_ARG, "threads");
    if (o.precision != SPTRSV_PREC_F64 && o.precision != SPTRSV_PREC_F32_REFINE) return fail(SPTRSV_ERR_ARG, "precision");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || o.device < 0 || o.device >= count) {
        (void)cudaGetLastError();
        return fail(SPTRSV_ERR_CUDA, "no such CUDA device");
    }
    sptrsv_server *S = new sptrsv_server();
    S->device = o.device;
    S->budget = hbm_budget;
    S->opts = o;
    S->refine = o.mode == SPTRSV_SERVE_CONTINUOUS && o.precision == SPTRSV_PREC_F32_REFINE;
    S->threads = o.threads;
    S->cfg = BatchCfg{S->refine ? 1 : 0, o.max_iters, o.refine_tol};
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    int st = SPTRSV_OK;
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    S->smem = kServeSmem;
    st = batch_occupancy(S->threads, S->smem, &S->per_sm);
    const int nslots = o.mode == SPTRSV_SERVE_SERIAL_F64 ? 1 : o.streams;
    S->slots.resize(nslots);
    for (Slot &sl : S->slots) {
        if (st) break;
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_items, size_t(o.max_batch) * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_items, size_t(o.max_batch) * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_res, size_t(o.max_batch) * sizeof(ItemResult));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_res, size_t(o.max_batch) * sizeof(ItemResult));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_cursor, sizeof(unsigned int));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            st = fail(SPTRSV_ERR_CUDA, std::string("serving slot: ") + cudaGetErrorString(e));
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st) {
        sptrsv_serve_destroy(S);
        return st;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return SPTRSV_OK;
}

int sptrsv_serve_register(sptrsv_server *S, sptrsv_plan *plan, int32_t *factor_id) {
    clear_error();
    if (!S || !plan || !factor_id) return fail(SPTRSV_ERR_ARG, "NULL argument");
    if (plan->device != S->device) return fail(SPTRSV_ERR_ARG, "plan lives on another device");
    if (S->refine && !(plan->values & SPTRSV_VALUES_F32)) return fail(SPTRSV_ERR_ARG, "plan has no FP32 values");
    if (!S->refine && !(plan->values & SPTRSV_VALUES_F64)) return fail(SPTRSV_ERR_ARG, "plan has no FP64 values");
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->arena_mem) return fail(SPTRSV_ERR_ARG, "register every factor before the first submit");
    if (S->factor_bytes + size_t(plan->device_bytes) > S->budget)
        return fail(SPTRSV_ERR_BUDGET, "factor does not fit in the HBM budget");
    S->factor_bytes += size_t(plan->device_bytes);
    S->factors.push_back(plan);
    *factor_id = int32_t(S->factors.size()) - 1;
    return SPTRSV_OK;
}

}  // extern "C"

namespace sptrsv {
namespace {
int submit_request(sptrsv_server *S, Request r, uint64_t *req_id) {
    if (S->worker_error) return fail(S->worker_error, S->worker_msg);
    std::unique_lock<std::mutex> lk(S->mu);
    if (r.fid < 0 || r.fid >= int32_t(S->factors.size())) return fail(SPTRSV_ERR_ARG, "unknown factor id");
    const sptrsv_plan *p = S->factors[r.fid];
    const int64_t n1 = std::max<int64_t>(p->h.n, 1);
    if (r.host ? (r.ldb_host < n1 || r.ldx_host < n1) : r.ld < n1) return fail(SPTRSV_ERR_ARG, "ld < n");
    if (!S->arena_mem && (S->opts.mode == SPTRSV_SERVE_CONTINUOUS || r.host)) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(S->device);
        const int st = ensure_arena(S);
        if (prev >= 0) cudaSetDevice(prev);
        if (st) return st;
    }
    size_t need = S->opts.mode == SPTRSV_SERVE_CONTINUOUS ? workspace_bytes(p, r.nrhs, S->refine) + 256 : 0;
    if (r.host) need += host_io_bytes(p, r.nrhs);
    if (need > S->arena.size) {
        ++S->rejected;
        return fail(SPTRSV_ERR_BUDGET, "request workspace exceeds the HBM budget left by the resident factors");
    }
    r.t_arrive = now_s();
    if (S->t_first < 0) S->t_first = r.t_arrive;
    const uint64_t id = S->next_id++;
    S->reqs[id] = r;
    S->pending.push_back(id);
    ++S->submitted;
    ++S->inflight;
    *req_id = id;
    S->cv.notify_all();
    return SPTRSV_OK;
}
}  // namespace
}  // namespace sptrsv

extern "C" {

int sptrsv_serve_submit(sptrsv_server *S, int32_t factor_id, const double *b, double *x, int32_t nrhs,
                        int64_t ld, uint64_t *req_id) {
    clear_error();
    if (!S || !req_id || !b || !x || nrhs < 1) return fail(SPTRSV_ERR_ARG, "bad argument");
    Request r;
    r.fid = factor_id;
    r.nrhs = nrhs;
    r.b = b;
    r.x = x;
    r.ld = ld;
    return submit_request(S, r, req_id);
}

int sptrsv_serve_submit_host(sptrsv_server *S, int32_t factor_id, const double *b_host, int64_t ldb, double *x_host,
                             int64_t ldx, int32_t nrhs, uint64_t *req_id) {
    clear_error();
    if (!S || !req_id || !b_host || !x_host || nrhs < 1) return fail(SPTRSV_ERR_ARG, "bad argument");
    Request r;
    r.fid = factor_id;
    r.nrhs = nrhs;
    r.host = true;
    r.b_host = b_host;
    r.x_host = x_host;
    r.ldb_host = ldb;
    r.ldx_host = ldx;
    return submit_request(S, r, req_id);
}

int sptrsv_serve_poll(sptrsv_server *S, uint64_t req_id, sptrsv_report *out) {
    if (!S) return fail(SPTRSV_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return fail(SPTRSV_ERR_ARG, "unknown request id");
    if (it->second.state != 2) return SPTRSV_ERR_PENDING;
    const sptrsv_report rep = it->second.rep;
    if (out) *out = rep;
    S->reqs.erase(it);
    if (rep.status) return fail(rep.status, std::string("request failed: ") + sptrsv_status_string(rep.status));
    return SPTRSV_OK;
}

int sptrsv_serve_wait(sptrsv_server *S, uint64_t req_id, double timeout_s, sptrsv_report *out) {
    if (!S) return fail(SPTRSV_ERR_ARG, "server is NULL");
    {
        std::unique_lock<std::mutex> lk(S->mu);
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
        while (true) {
            auto it = S->reqs.find(req_id);
            if (it == S->reqs.end()) return fail(SPTRSV_ERR_ARG, "unknown request id");
            if (it->second.state == 2) break;
            if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout) return SPTRSV_ERR_PENDING;
        }
    }
    return sptrsv_serve_poll(S, req_id, out);
}

int sptrsv_serve_drain(sptrsv_server *S, double timeout_s) {
    if (!S) return fail(SPTRSV_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->inflight > 0)
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout) return fail(SPTRSV_ERR_PENDING, "drain timed out");
    return SPTRSV_OK;
}

int sptrsv_serve_stats(sptrsv_server *S, sptrsv_serve_statistics *out) {
    if (!S || !out) return fail(SPTRSV_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->launches = S->launches;
    out->mean_batch = S->launches ? double(S->items) / double(S->launches) : (S->completed ? 1.0 : 0.0);
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
        if (l.empty()) return 0.0;
        const size_t i = std::min(l.size() - 1, size_t(q * double(l.size() - 1) + 0.5));
        return l[i] * 1e3;
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.empty() ? 0.0 : l.back() * 1e3;
    out->mean_ms = 0.0;
    for (double v : l) out->mean_ms += v * 1e3;
    if (!l.empty()) out->mean_ms /= double(l.size());
    const double span = S->t_last - S->t_first;
    out->solves_per_s = (span > 0 && S->completed) ? double(S->completed) / span : 0.0;
    out->peak_workspace_bytes = int64_t(S->arena.peak);
    out->arena_bytes = int64_t(S->arena.size);
    out->factor_bytes = int64_t(S->factor_bytes);
    return SPTRSV_OK;
}

void sptrsv_serve_destroy(sptrsv_server *S) {
    if (!S) return;
    S->stop = true;
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_items) cudaFreeHost(sl.h_items);
        if (sl.d_items) cudaFree(sl.d_items);
        if (sl.h_res) cudaFreeHost(sl.h_res);
        if (sl.d_res) cudaFree(sl.d_res);
        if (sl.d_cursor) cudaFree(sl.d_cursor);
    }
    if (S->arena_mem) cudaFree(S->arena_mem);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
