// Saved plans: the factor, its superstep schedule and the block-local
// partition in one file, so a later process rebuilds the plan without running
// the scheduler (GrowLocal, Sec. 3) or the partition again.  The schedule
// depends only on the pattern, so the analysis is paid once per factor (the
// amortisation threshold of Table 7.6 counts it against every solve).
//
// Layout (little-endian; both supported hosts are):
//   char     magic[8]   "SPTRSVPL"
//   uint32   version    1
//   uint32   order      0x01020304 as written by the saving host
//   int32    n, triangle
//   int64    nnz
//   int32    mode, k, supersteps, sched_blocks, loc_nb, coarse_vertices
//   int32    rowptr[n + 1], col[nnz]; double val[nnz]   the caller's factor
//   int32    sigma[n], pi[n]                           analysed numbering
//   int32    loc_blk[n], loc_lidx[n]                   only if loc_nb > 0
//   uint64   checksum of everything after the header
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "plan.hpp"

namespace sptrsv {
namespace {

constexpr char kMagic[8] = {'S', 'P', 'T', 'R', 'S', 'V', 'P', 'L'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kOrder = 0x01020304u;

struct Header {
    char magic[8];
    uint32_t version, order;
    int32_t n, triangle;
    int64_t nnz;
    int32_t mode, k, S, sched_blocks, loc_nb, coarse;
};
static_assert(sizeof(Header) == 56, "saved plan header layout");

// Checksum over 8-byte words: h = (h ^ w) * odd constant, then a final mix
// (splitmix64's finaliser); catches truncation and flipped bytes.
struct Sum {
    uint64_t h = 0x9e3779b97f4a7c15ull;
    void add(const void *p, size_t bytes) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        size_t i = 0;
        for (; i + 8 <= bytes; i += 8) {
            uint64_t w;
            std::memcpy(&w, c + i, 8);
            h = (h ^ w) * 0x100000001b3ull;
        }
        uint64_t w = 0;
        std::memcpy(&w, c + i, bytes - i);
        h = (h ^ w ^ (uint64_t(bytes) << 56)) * 0x100000001b3ull;
    }
    uint64_t value() const {
        uint64_t z = h;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
};

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) std::fclose(f);
    }
};

}  // namespace

int load_body(FILE *f, const Header &hd, const sptrsv_analyze_opts *opts, sptrsv_plan **out);

}  // namespace sptrsv

using namespace sptrsv;

extern "C" {

int sptrsv_plan_save(const sptrsv_plan *p, const sptrsv_csr *csr, const char *path) {
    clear_error();
    if (!p || !csr || !path) return fail(SPTRSV_ERR_ARG, "NULL argument");
    const HostSchedule &h = p->h;
    if (csr->n != h.n || csr->nnz != h.nnz) return fail(SPTRSV_ERR_ARG, "factor size differs from the plan's");
    // the factor must have the plan's pattern: same wavefronts, schedule valid on it
    std::vector<int32_t> rp, col, level;
    std::vector<double> val;
    sptrsv_csr lowered;
    const sptrsv_csr *A = nullptr;
    int st = lower_factor(csr, p->triangle, rp, col, val, lowered, &A);
    if (st) return st;
    if (factor_levels(A, level) != h.nlevels || level != h.level)
        return fail(SPTRSV_ERR_ARG, "factor pattern differs from the plan's (wavefronts differ)");
    for (int32_t v = 0; v < h.n; ++v)
        for (int32_t q = A->rowptr[v]; q < A->rowptr[v + 1] - 1; ++q) {
            const int32_t u = A->col[q];
            if (h.sigma[u] > h.sigma[v] || (h.sigma[u] == h.sigma[v] && h.pi[u] != h.pi[v]))
                return fail(SPTRSV_ERR_ARG, "factor pattern differs from the plan's (schedule invalid on it)");
        }
    const bool part = h.loc_nb > 0 && h.loc_blk.size() == size_t(h.n);
    Header hd{};
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = kVersion;
    hd.order = kOrder;
    hd.n = h.n;
    hd.triangle = p->triangle;
    hd.nnz = h.nnz;
    hd.mode = h.mode;
    hd.k = h.k;
    hd.S = h.S;
    hd.sched_blocks = h.sched_blocks;
    hd.loc_nb = part ? h.loc_nb : 0;
    hd.coarse = h.coarse_vertices;
    const std::string tmp = std::string(path) + ".tmp";
    File out;
    out.f = std::fopen(tmp.c_str(), "wb");
    if (!out.f) return fail(SPTRSV_ERR_IO, "cannot create " + tmp);
    Sum sum;
    bool ok = std::fwrite(&hd, sizeof(hd), 1, out.f) == 1;
    auto put = [&](const void *a, size_t bytes) {
        if (!ok || bytes == 0) return;
        sum.add(a, bytes);
        ok = std::fwrite(a, 1, bytes, out.f) == bytes;
    };
    const size_t n = size_t(h.n), nnz = size_t(h.nnz);
    put(csr->rowptr, (n + 1) * sizeof(int32_t));
    put(csr->col, nnz * sizeof(int32_t));
    put(csr->val, nnz * sizeof(double));
    put(h.sigma.data(), n * sizeof(int32_t));
    put(h.pi.data(), n * sizeof(int32_t));
    if (part) {
        put(h.loc_blk.data(), n * sizeof(int32_t));
        put(h.loc_lidx.data(), n * sizeof(int32_t));
    }
    const uint64_t c = sum.value();
    ok = ok && std::fwrite(&c, sizeof(c), 1, out.f) == 1;
    ok = (std::fclose(out.f) == 0) && ok;
    out.f = nullptr;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(SPTRSV_ERR_IO, std::string("cannot write ") + path);
    }
    return SPTRSV_OK;
}

int sptrsv_plan_load(const char *path, const sptrsv_analyze_opts *opts, sptrsv_plan **out) {
    clear_error();
    if (!path || !out) return fail(SPTRSV_ERR_ARG, "NULL argument");
    *out = nullptr;
    File in;
    in.f = std::fopen(path, "rb");
    if (!in.f) return fail(SPTRSV_ERR_IO, std::string("cannot open ") + path);
    Header hd{};
    if (std::fread(&hd, sizeof(hd), 1, in.f) != 1) return fail(SPTRSV_ERR_IO, "truncated plan file");
    if (std::memcmp(hd.magic, kMagic, 8) != 0) return fail(SPTRSV_ERR_ARG, "not a saved plan");
    if (hd.version != kVersion) return fail(SPTRSV_ERR_ARG, "saved plan of another format version");
    if (hd.order != kOrder) return fail(SPTRSV_ERR_ARG, "saved plan of another byte order");
    if (hd.n < 0 || hd.nnz < hd.n || hd.nnz > (int64_t(1) << 31) - 1 || hd.loc_nb < 0 || hd.k < 1 ||
        hd.k > (1 << 20) || hd.S < 0 || hd.S > hd.n || hd.coarse < 0 || hd.coarse > hd.n ||
        (hd.mode != SPTRSV_SCHED_LEVELS && hd.mode != SPTRSV_SCHED_GROWLOCAL))
        return fail(SPTRSV_ERR_ARG, "saved plan: bad header");
    const size_t n = size_t(hd.n), nnz = size_t(hd.nnz);
    {   // the size the header promises, before allocating anything
        const uint64_t want = sizeof(Header) + (n + 1) * 4 + nnz * 12 + n * 8 + (hd.loc_nb > 0 ? n * 8 : 0) + 8;
        if (std::fseek(in.f, 0, SEEK_END) != 0) return fail(SPTRSV_ERR_IO, "cannot seek in plan file");
        const long have = std::ftell(in.f);
        if (have < 0 || uint64_t(have) != want) return fail(SPTRSV_ERR_IO, "plan file has the wrong size");
        if (std::fseek(in.f, long(sizeof(Header)), SEEK_SET) != 0)
            return fail(SPTRSV_ERR_IO, "cannot seek in plan file");
    }
    try {
        return load_body(in.f, hd, opts, out);
    } catch (const std::bad_alloc &) {
        return fail(SPTRSV_ERR_OOM, "host allocation failed while loading a plan");
    }
}

}  // extern "C"

namespace sptrsv {

int load_body(FILE *f, const Header &hd, const sptrsv_analyze_opts *opts, sptrsv_plan **out) {
    const size_t n = size_t(hd.n), nnz = size_t(hd.nnz);
    std::vector<int32_t> rowptr(n + 1), col(nnz), sigma(n), pi(n), blk, lidx;
    std::vector<double> val(nnz);
    Sum sum;
    bool ok = true;
    auto get = [&](void *a, size_t bytes) {
        if (!ok || bytes == 0) return;
        ok = std::fread(a, 1, bytes, f) == bytes;
        if (ok) sum.add(a, bytes);
    };
    get(rowptr.data(), (n + 1) * sizeof(int32_t));
    get(col.data(), nnz * sizeof(int32_t));
    get(val.data(), nnz * sizeof(double));
    get(sigma.data(), n * sizeof(int32_t));
    get(pi.data(), n * sizeof(int32_t));
    if (hd.loc_nb > 0) {
        blk.resize(n);
        lidx.resize(n);
        get(blk.data(), n * sizeof(int32_t));
        get(lidx.data(), n * sizeof(int32_t));
    }
    uint64_t c = 0;
    ok = ok && std::fread(&c, sizeof(c), 1, f) == 1;
    if (!ok) return fail(SPTRSV_ERR_IO, "truncated plan file");
    if (c != sum.value()) return fail(SPTRSV_ERR_ARG, "saved plan: checksum mismatch");
    sptrsv_analyze_opts o;
    sptrsv_analyze_opts_default(&o);
    if (opts) {
        o.device = opts->device;
        o.values = opts->values;
    }
    o.triangle = hd.triangle;
    sptrsv_csr A{hd.n, hd.nnz, rowptr.data(), col.data(), val.data()};
    GivenSchedule g;
    g.mode = hd.mode;
    g.k = hd.k;
    g.S = hd.S;
    g.sched_blocks = hd.sched_blocks;
    g.coarse_vertices = hd.coarse;
    g.sigma = sigma.data();
    g.pi = pi.data();
    g.loc_nb = hd.loc_nb;
    g.loc_blk = blk.data();
    g.loc_lidx = lidx.data();
    return analyze_impl(&A, o, &g, out);
}

}  // namespace sptrsv
