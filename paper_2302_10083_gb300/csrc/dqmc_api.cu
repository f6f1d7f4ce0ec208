// dqmc_api.cu -- the C ABI of libdqmc.so (declared in include/dqmc.h and
// include/dqmc_plan.h): argument checks, the pass plan, the workspace layout,
// and the host entry points with their per-device buffer cache.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "dqmc.h"
#include "dqmc_plan.h"
#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"

namespace dqmc {

static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t bitmap_words(int n) { return (pow3(n) + 31) / 32; }
uint64_t bitmap_alloc_bytes(int n) { return align_up((pow3(n) + 7) / 8, 16); }

// ------------------------------------------------------------------- plans
//
// n <= 12: one tile holds the whole function in shared memory (one pass of
// the tile_pass kernel in dqmc_sweep.cu).
//
// n >= 13 (H = n - 5 >= 8 high digits): streaming passes of 2187-row tiles
// (dqmc_pass.cu).  The high digits are split into a first group G0 = 0..6 and
// groups G1 < G2 < ... of at most 6 digits; a tile holds one group's digits
// plus 7 - K inner digits (the lowest high digits) for contiguous runs.
//   first       truth table -> Merge chunk digits and G0 (digits >= 7 still 0/1)
//   merge       Merge G1 .. G(last-1), sparse rows in and out
//   merge-last  Merge the last group, then Reduce it (and chunk digits
//               {0, 1, 2} when there is no middle group)
//   reduce      Reduce the middle groups above G1, top down; the first of
//               them also Reduces chunk digits {0, 1, 2}
//   out         Reduce G1 (each cell against its '*' neighbours in G1 read
//               from the neighbour tiles in the state, as the previous pass
//               left it), G0 and chunk digits {3, 4} (all five when no reduce
//               pass took {0, 1, 2}), write the dense bitmap, the count and
//               the list.
// Every digit is merged once before any Reduce and reduced exactly once.
// G1 needs no pass of its own: a tile of the out pass holds G0, and the rows
// of its G1 neighbours are whole tiles of the same shape (3^7 contiguous
// rows), 3^j tiles away for G1 digit 7 + j; the 3^(7+K1) rows that share the
// higher digits (51 MB at K1 = 6) stay in L2 while their tiles are swept.

static FixedDigits fixed_of(const std::vector<int> &digits, const std::vector<bool> &merged)
{
    FixedDigits f;
    for (int d : digits) {
        f.w3[f.n] = pow3(d);
        f.w2[f.n] = 1ull << d;
        f.r[f.n] = merged[d] ? 3 : 2;
        f.j[f.n] = (uint8_t)d;
        ++f.n;
    }
    return f;
}

static uint64_t radix_product(const FixedDigits &f)
{
    uint64_t t = 1;
    for (int i = 0; i < f.n; ++i) t *= f.r[i];
    return t;
}

// One pass = one phase over tiles of group digits a..a+K-1 and inner digits
// 0..B-1; every other high digit is fixed per tile (radix 2 while it is not
// merged yet, else 3), in ascending digit order, so tile index order is rho
// order.
static SuperPassDesc make_pass(int load, int a, int K, int B, int H, const std::vector<bool> &merged)
{
    SuperPassDesc sp;
    sp.nph = 1;
    PhaseDesc &ph = sp.ph[0];
    ph.load = load;
    ph.a = a;
    ph.K = K;
    ph.B = B;
    ph.tiles = 1;
    std::vector<int> outer;
    for (int d = 0; d < H; ++d)
        if (!(d < B) && !(d >= a && d < a + K)) outer.push_back(d);
    sp.sb = fixed_of(outer, merged);
    sp.n_sb = radix_product(sp.sb);
    sp.window = (uint32_t)std::min<uint64_t>(sp.n_sb, 0xffffffffu);
    sp.groups = 1;
    sp.step_size = (uint32_t)sp.n_sb;
    sp.n_steps = 1;
    return sp;
}

Plan make_plan(int n)
{
    Plan p;
    p.n = n;
    p.C = n < kChunkDigits ? n : kChunkDigits;
    p.H = n - p.C;
    const int H = p.H;
    if (H <= kMaxSmemGroup) {
        Pass ps;
        ps.kind = kPassFirst;
        ps.K = H;
        ps.tiles = 1;
        ps.fuse_reduce = ps.chunk_reduce = ps.write_out = true;
        p.passes.push_back(ps);
        p.state_rows = 0;
        return p;
    }
    p.state_rows = pow3(H);
    std::vector<int> starts, sizes;
    const int rest = H - kTileDigits;
    const int ng = (rest + kMaxStreamGroup - 1) / kMaxStreamGroup;
    int at = kTileDigits;
    for (int i = 0; i < ng; ++i) {
        const int k = rest / ng + (i < rest % ng ? 1 : 0);
        starts.push_back(at);
        sizes.push_back(k);
        at += k;
    }
    std::vector<bool> merged(H, false);
    int slot = 0;
    auto push = [&](SuperPassDesc sp) {
        sp.slot = slot++;
        p.sps.push_back(sp);
    };
    {   // first: G0 from the truth table
        SuperPassDesc sp = make_pass(kLoadTT, 0, kTileDigits, 0, H, merged);
        sp.ph[0].merge = 1;
        push(sp);
        for (int d = 0; d < kTileDigits; ++d) merged[d] = true;
    }
    for (int i = 0; i < ng; ++i) {   // merge G1 .. ; the last one also Reduces
        const int a = starts[i], K = sizes[i], B = kTileDigits - K;
        SuperPassDesc sp = make_pass(kLoadSparse, a, K, B, H, merged);
        sp.ph[0].merge = 1;
        if (i == ng - 1) {
            sp.ph[0].reduce = 1;
            // with a middle Reduce pass to come, that pass and the bitmap pass
            // take the chunk digits instead (at n = 24, chunk digits {0, 1}
            // cost this pass 3.8 ms and the middle Reduce 3.0 ms)
            sp.ph[0].chunk_mask = (ng >= 2) ? 0 : 0x07;
        }
        push(sp);
        for (int d = a; d < a + K; ++d) merged[d] = true;
    }
    for (int i = ng - 2; i >= 1; --i) {   // reduce the middle groups above G1, top down
        const int a = starts[i], K = sizes[i], B = kTileDigits - K;
        SuperPassDesc sp = make_pass(kLoadFull, a, K, B, H, merged);
        sp.ph[0].reduce = 1;
        sp.ph[0].chunk_mask = (i == ng - 2) ? 0x07 : 0;
        push(sp);
    }
    {   // out: G1 from the neighbour tiles, G0, the bitmap, the count and the list
        SuperPassDesc sp = make_pass(kLoadFull, 0, kTileDigits, 0, H, merged);
        sp.ph[0].reduce = 1;
        sp.ph[0].out = 1;
        sp.ph[0].chunk_mask = (ng == 2) ? 0x1f : 0x18;   // ng == 2: no reduce pass took {0, 1, 2}
        if (ng >= 2) {
            sp.ph[0].nbr_a = starts[0];
            sp.ph[0].nbr_K = sizes[0];
        }
        push(sp);
    }
    p.n_done = 0;
    p.out_tiles = pow3(H) / kTileRows;
    return p;
}

CtrlLayout ctrl_layout(const Plan &p)
{
    CtrlLayout c;
    const uint64_t u32 = 1 + kCtrlTickets + p.n_done;
    c.status_u64 = (u32 * 4 + 7) / 8;
    c.bytes = align_up((c.status_u64 + p.out_tiles) * 8, 256);
    return c;
}

int plan_passes(const Plan &p) { return p.sps.empty() ? (int)p.passes.size() : (int)p.sps.size(); }

static std::string fixed_json(const FixedDigits &f)
{
    std::string s = "[";
    for (int i = 0; i < f.n; ++i) {
        s += (i ? "," : "");
        s += "[" + std::to_string((int)f.j[i]) + "," + std::to_string((int)f.r[i]) + "]";
    }
    return s + "]";
}

std::string describe_plan(const Plan &p)
{
    std::string s = "{\"n\":" + std::to_string(p.n) + ",\"C\":" + std::to_string(p.C) +
                    ",\"H\":" + std::to_string(p.H) + ",\"state_rows\":" + std::to_string(p.state_rows) +
                    ",\"out_tiles\":" + std::to_string(p.out_tiles) + ",\"passes\":[";
    if (p.sps.empty()) {
        const Pass &q = p.passes[0];
        char buf[256];
        snprintf(buf, sizeof buf,
                 "{\"kind\":\"whole\",\"n_sb\":1,\"window\":1,\"sb\":[],\"phases\":[{\"load\":\"tt\",\"K\":%d,"
                 "\"B\":0,\"a\":0,\"merge\":1,\"reduce\":1,\"chunk_mask\":%d,\"out\":1,\"nbr_a\":0,\"nbr_K\":0,"
                 "\"tiles\":1,\"fix\":[]}]}",
                 q.K, (1 << p.C) - 1);
        s += buf;
    }
    static const char *loads[] = {"tt", "sparse", "full"};
    for (size_t i = 0; i < p.sps.size(); ++i) {
        const SuperPassDesc &sp = p.sps[i];
        s += std::string(i ? "," : "") + "{\"kind\":\"super\",\"n_sb\":" + std::to_string(sp.n_sb) +
             ",\"window\":" + std::to_string(sp.window) + ",\"step_size\":" + std::to_string(sp.step_size) +
             ",\"n_steps\":" + std::to_string(sp.n_steps) + ",\"groups\":" + std::to_string(sp.groups) +
             ",\"sb\":" + fixed_json(sp.sb) + ",\"phases\":[";
        for (int k = 0; k < sp.nph; ++k) {
            const PhaseDesc &q = sp.ph[k];
            char buf[256];
            snprintf(buf, sizeof buf,
                     "%s{\"load\":\"%s\",\"K\":%d,\"B\":%d,\"a\":%d,\"merge\":%d,\"reduce\":%d,\"chunk_mask\":%d,"
                     "\"out\":%d,\"nbr_a\":%d,\"nbr_K\":%d,\"tiles\":%u,\"fix\":",
                     k ? "," : "", loads[q.load], q.K, q.B, q.a, q.merge, q.reduce, q.chunk_mask, q.out, q.nbr_a,
                     q.nbr_K, q.tiles);
            s += buf + fixed_json(q.fix) + "}";
        }
        s += "]}";
    }
    s += "]}";
    return s;
}

Workspace workspace_layout(int n)
{
    Workspace w;
    const Plan p = make_plan(n);
    uint64_t at = 0;
    w.state_off = at;
    w.state_bytes = p.state_rows * kChunkBytes;
    at = align_up(at + w.state_bytes, 256);
    w.count_off = at;
    at = align_up(at + 256, 256);
    w.ctrl_off = at;
    w.ctrl_bytes = p.sps.empty() ? 256 : ctrl_layout(p).bytes;
    at = align_up(at + w.ctrl_bytes, 256);
    w.n_blocks = (bitmap_words(n) + kListWordsPerBlock - 1) / kListWordsPerBlock;
    w.blk_counts_off = at;
    at = align_up(at + 4 * w.n_blocks, 256);
    w.blk_offs_off = at;
    at = align_up(at + 8 * w.n_blocks, 256);
    w.total = at;
    return w;
}

static int map_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return DQMC_OK;
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    if (e == cudaErrorMemoryAllocation) return DQMC_ENOMEM;
    return DQMC_ECUDA;
}

static bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

// ------------------------------------------------------------ host-API cache

struct DeviceCache {
    std::mutex mu;
    cudaStream_t stream = nullptr;
    void *buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // on, dc, bitmap, work, pairs
    uint64_t cap[5] = {0, 0, 0, 0, 0};
    unsigned long long *h_count = nullptr;  // pinned
    unsigned long long *d_count = nullptr;
};

static std::mutex g_cache_mu;
static DeviceCache *g_cache[64];

static DeviceCache *cache_for_current_device(int *status)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *status = map_cuda(e == cudaSuccess ? cudaErrorInvalidDevice : e);
        return nullptr;
    }
    std::lock_guard<std::mutex> g(g_cache_mu);
    if (!g_cache[dev]) {
        DeviceCache *c = new DeviceCache();
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_count, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_count, 256);
        if (e != cudaSuccess) {
            *status = map_cuda(e);
            delete c;
            return nullptr;
        }
        g_cache[dev] = c;
    }
    return g_cache[dev];
}

static int ensure(DeviceCache *c, int i, uint64_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (c->cap[i] >= bytes) return DQMC_OK;
    if (c->buf[i]) cudaFree(c->buf[i]);
    c->buf[i] = nullptr;
    c->cap[i] = 0;
    cudaError_t e = cudaMalloc(&c->buf[i], bytes);
    if (e != cudaSuccess) return map_cuda(e);
    c->cap[i] = bytes;
    return DQMC_OK;
}

}  // namespace dqmc

using namespace dqmc;

// ----------------------------------------------------------------- C ABI

extern "C" const char *dqmc_strerror(int status)
{
    switch (status) {
    case DQMC_OK: return "ok";
    case DQMC_EINVAL: return "invalid argument";
    case DQMC_ENOMEM: return "out of device memory";
    case DQMC_ETRUNC: return "list truncated to cap";
    case DQMC_ECUDA: return "CUDA runtime error";
    case DQMC_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

extern "C" int dqmc_version(void) { return 10000; }

extern "C" uint64_t dqmc_bitmap_bytes(uint32_t n)
{
    return n > DQMC_MAX_N ? 0 : (pow3((int)n) + 7) / 8;
}

extern "C" uint64_t dqmc_bitmap_alloc_bytes(uint32_t n)
{
    return n > DQMC_MAX_N ? 0 : bitmap_alloc_bytes((int)n);
}

extern "C" uint64_t dqmc_workspace_bytes(uint32_t n)
{
    return n > DQMC_MAX_N ? 0 : workspace_layout((int)n).total;
}

extern "C" int dqmc_plan_json(uint32_t n, char *buf, uint64_t cap)
{
    if (n > DQMC_MAX_N || (!buf && cap)) return DQMC_EINVAL;
    const std::string s = describe_plan(make_plan((int)n));
    if (cap) {
        const size_t k = s.size() < cap - 1 ? s.size() : (size_t)(cap - 1);
        memcpy(buf, s.data(), k);
        buf[k] = 0;
    }
    return (int)s.size();
}

extern "C" int dqmc_plan_passes(uint32_t n)
{
    if (n > DQMC_MAX_N) return DQMC_EINVAL;
    return plan_passes(make_plan((int)n));
}

// HBM bytes a super-pass must move by design: its first phase's reads (from
// the previous pass) and its last writes (rows of the state, or the bitmap);
// rows handed from one phase to the next stay in L2 and are not counted.
static uint64_t super_bytes(const Plan &p, int i, bool with_dc)
{
    const SuperPassDesc &sp = p.sps[i];
    const PhaseDesc &p0 = sp.ph[0];
    const uint64_t RE = pow3(p0.B), NB = 1ull << p0.K, RG = pow3(p0.K);
    const uint64_t tiles0 = (uint64_t)p0.tiles * sp.n_sb;
    uint64_t rd = 0, wr = 0;
    if (p0.load == kLoadTT) rd = tiles0 * NB * 4 * (with_dc ? 2 : 1);
    else if (p0.load == kLoadSparse) rd = tiles0 * NB * RE * kChunkBytes;
    else rd = tiles0 * RG * RE * kChunkBytes;
    const PhaseDesc &pl = sp.ph[sp.nph - 1];
    if (pl.out) {
        wr = (pow3(p.n) + 7) / 8;
    } else if (sp.nph == 1 && p0.load == kLoadSparse && !p0.reduce) {
        wr = tiles0 * (RG - NB) * RE * kChunkBytes;     // only the rows the Merge created
    } else {
        // every row of the pass's super-blocks
        uint64_t rows = sp.n_sb;
        const PhaseDesc &q = sp.ph[0];
        uint64_t inner = pow3(q.K) * pow3(q.B);
        for (int k = 0; k < q.fix.n; ++k) inner *= 3;   // all digits merged by the end
        rows *= inner;
        wr = rows * kChunkBytes;
    }
    return rd + wr;
}

extern "C" uint64_t dqmc_pass_bytes(uint32_t n, int pass, int with_dc)
{
    if (n > DQMC_MAX_N) return 0;
    const Plan p = make_plan((int)n);
    if (p.sps.empty()) return pass_bytes(p, pass, with_dc != 0);
    if (pass < 0 || pass >= (int)p.sps.size()) return 0;
    return super_bytes(p, pass, with_dc != 0);
}

extern "C" int dqmc_compact_dev(uint32_t n, const void *d_bitmap, uint32_t *d_pairs, uint64_t cap,
                                uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream);

static int check_dev_args(uint32_t n, const void *d_on, const void *d_dc, const void *d_work,
                          uint64_t work_bytes)
{
    if (n > DQMC_MAX_N || !d_on) return DQMC_EINVAL;
    const uintptr_t in_align = n >= 5 ? 4 : 1;
    if (!aligned(d_on, in_align) || (d_dc && !aligned(d_dc, in_align))) return DQMC_EINVAL;
    if (work_bytes < workspace_layout((int)n).total) return DQMC_EINVAL;
    if (!d_work || !aligned(d_work, 256)) return DQMC_EINVAL;
    return DQMC_OK;
}

static int sweep_dev(uint32_t n, int first, int last, const void *d_on, const void *d_dc, void *d_bitmap,
                     uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream,
                     uint32_t *d_pairs = nullptr, uint64_t cap = 0, uint32_t flags = 0)
{
    if (flags & ~(uint32_t)DQMC_COMPLEMENT) return DQMC_EINVAL;
    const uint32_t inv = (flags & DQMC_COMPLEMENT) ? ~0u : 0u;
    int st = check_dev_args(n, d_on, d_dc, d_work, work_bytes);
    if (st) return st;
    if (!d_bitmap || !aligned(d_bitmap, 16)) return DQMC_EINVAL;
    if (d_count && !aligned(d_count, 8)) return DQMC_EINVAL;
    const Plan plan = make_plan((int)n);
    const int np = plan_passes(plan);
    if (last < 0) last = np;
    if (first < 0 || first >= last || last > np) return DQMC_EINVAL;
    const Workspace w = workspace_layout((int)n);
    char *base = static_cast<char *>(d_work);
    // The bitmap may be written over the state (d_bitmap == d_work, n >= 13);
    // any other overlap of the bitmap with the workspace is refused.
    const char *bm = static_cast<const char *>(d_bitmap);
    const bool inplace = !plan.sps.empty() && bm == base + w.state_off;
    if (!inplace && bm < base + work_bytes && base < bm + bitmap_alloc_bytes((int)n)) return DQMC_EINVAL;
    unsigned long long *cnt = d_count ? reinterpret_cast<unsigned long long *>(d_count)
                                      : reinterpret_cast<unsigned long long *>(base + w.count_off);
    if (plan.sps.empty())
        return map_cuda(launch_sweep(plan, d_on, d_dc, base + w.state_off, static_cast<uint32_t *>(d_bitmap),
                                     cnt, static_cast<cudaStream_t>(stream), first, last, nullptr, inv));
    return map_cuda(launch_super(plan, d_on, d_dc, base + w.state_off, static_cast<uint32_t *>(d_bitmap), cnt,
                                 d_pairs, cap, base + w.ctrl_off, static_cast<cudaStream_t>(stream), first, last,
                                 nullptr, inv, inplace));
}

extern "C" int dqmc_primes_dev(uint32_t n, const void *d_on, const void *d_dc, void *d_bitmap,
                               uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream)
{
    return sweep_dev(n, 0, -1, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream);
}

extern "C" int dqmc_sweep_pass_dev(uint32_t n, int pass, const void *d_on, const void *d_dc, void *d_bitmap,
                                   uint32_t *d_pairs, uint64_t cap, uint64_t *d_count, void *d_work,
                                   uint64_t work_bytes, void *stream)
{
    if (pass < 0 || n > DQMC_MAX_N || (cap && !d_pairs) || (d_pairs && !aligned(d_pairs, 8))) return DQMC_EINVAL;
    if (d_pairs && !d_count) return DQMC_EINVAL;
    const Plan plan = make_plan((int)n);
    if (!plan.sps.empty())
        return sweep_dev(n, pass, pass + 1, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream,
                         cap ? d_pairs : nullptr, cap);
    int st = sweep_dev(n, pass, pass + 1, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream);
    if (st || !d_pairs || pass != plan_passes(plan) - 1) return st;
    return dqmc_compact_dev(n, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes, stream);
}

extern "C" int dqmc_sweep_passes_dev(uint32_t n, int first, int last, const void *d_on, const void *d_dc,
                                     void *d_bitmap, uint32_t *d_pairs, uint64_t cap, uint64_t *d_count, void *d_work,
                                     uint64_t work_bytes, void *stream)
{
    if (first < 0 || last <= first || n > DQMC_MAX_N || (cap && !d_pairs) || (d_pairs && !aligned(d_pairs, 8)))
        return DQMC_EINVAL;
    if (d_pairs && !d_count) return DQMC_EINVAL;
    const Plan plan = make_plan((int)n);
    if (last > plan_passes(plan)) return DQMC_EINVAL;
    if (plan.sps.empty()) {
        for (int i = first; i < last; ++i) {
            const int st = dqmc_sweep_pass_dev(n, i, d_on, d_dc, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes,
                                               stream);
            if (st) return st;
        }
        return DQMC_OK;
    }
    return sweep_dev(n, first, last, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream,
                     cap ? d_pairs : nullptr, cap);
}

extern "C" int dqmc_selftest_timeout(uint32_t n, void *d_work, uint64_t work_bytes, uint64_t wait_ns, void *stream)
{
    if (n > DQMC_MAX_N || !d_work || !aligned(d_work, 256) || wait_ns > 1000000000ull) return DQMC_EINVAL;
    const Plan plan = make_plan((int)n);
    const Workspace w = workspace_layout((int)n);
    if (plan.sps.empty() || work_bytes < w.total) return DQMC_EINVAL;
    return map_cuda(launch_selftest_wait(static_cast<char *>(d_work) + w.ctrl_off, w.ctrl_bytes, wait_ns,
                                         static_cast<cudaStream_t>(stream)));
}

extern "C" int dqmc_compact_dev(uint32_t n, const void *d_bitmap, uint32_t *d_pairs, uint64_t cap,
                                uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream)
{
    if (n > DQMC_MAX_N || !d_bitmap || !d_count || (cap && !d_pairs)) return DQMC_EINVAL;
    if (!aligned(d_bitmap, 16) || !aligned(d_count, 8) || (d_pairs && !aligned(d_pairs, 8)))
        return DQMC_EINVAL;
    const Workspace w = workspace_layout((int)n);
    if (!d_work || !aligned(d_work, 256) || work_bytes < w.total) return DQMC_EINVAL;
    char *base = static_cast<char *>(d_work);
    return map_cuda(launch_compact((int)n, static_cast<const uint32_t *>(d_bitmap), d_pairs, cap,
                                   reinterpret_cast<unsigned long long *>(d_count),
                                   reinterpret_cast<uint32_t *>(base + w.blk_counts_off),
                                   reinterpret_cast<unsigned long long *>(base + w.blk_offs_off),
                                   static_cast<cudaStream_t>(stream)));
}

extern "C" int dqmc_primes_dev_ex(uint32_t n, const void *d_on, const void *d_dc, uint32_t flags, void *d_bitmap,
                                  uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream)
{
    return sweep_dev(n, 0, -1, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream, nullptr, 0, flags);
}

extern "C" int dqmc_list_dev_ex(uint32_t n, const void *d_on, const void *d_dc, uint32_t flags, void *d_bitmap,
                                uint32_t *d_pairs, uint64_t cap, uint64_t *d_count, void *d_work,
                                uint64_t work_bytes, void *stream)
{
    if (!d_count || (cap && !d_pairs) || (d_pairs && !aligned(d_pairs, 8))) return DQMC_EINVAL;
    if (n <= DQMC_MAX_N && !make_plan((int)n).sps.empty())  // the bitmap pass also writes the list
        return sweep_dev(n, 0, -1, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream,
                         cap ? d_pairs : nullptr, cap, flags);
    int st = dqmc_primes_dev_ex(n, d_on, d_dc, flags, d_bitmap, d_count, d_work, work_bytes, stream);
    if (st) return st;
    return dqmc_compact_dev(n, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes, stream);
}

extern "C" int dqmc_list_dev(uint32_t n, const void *d_on, const void *d_dc, void *d_bitmap,
                             uint32_t *d_pairs, uint64_t cap, uint64_t *d_count, void *d_work,
                             uint64_t work_bytes, void *stream)
{
    return dqmc_list_dev_ex(n, d_on, d_dc, 0, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes, stream);
}

extern "C" int dqmc_dev_status(uint32_t n, const void *d_work, uint64_t work_bytes, void *stream)
{
    if (n > DQMC_MAX_N || !d_work || work_bytes < workspace_layout((int)n).total) return DQMC_EINVAL;
    const Workspace w = workspace_layout((int)n);
    uint32_t err = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (make_plan((int)n).sps.empty()) return map_cuda(e);  // the one-tile pass has no device waits
    if (e == cudaSuccess)
        e = cudaMemcpy(&err, static_cast<const char *>(d_work) + w.ctrl_off, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return map_cuda(e);
    return err == 0 ? DQMC_OK : (err == kErrTimeout ? DQMC_ETIMEOUT : DQMC_ECUDA);
}

// Host entry points: copy in, run, copy out, wait.
static int host_run(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint8_t *out_bitmap,
                    uint32_t *out_pairs, uint64_t cap, uint64_t *out_count, bool want_list, uint32_t flags = 0)
{
    if (n > DQMC_MAX_N || !on_bits || (flags & ~(uint32_t)DQMC_COMPLEMENT)) return DQMC_EINVAL;
    if (want_list && cap && !out_pairs) return DQMC_EINVAL;
    int st = DQMC_OK;
    DeviceCache *c = cache_for_current_device(&st);
    if (!c) return st;
    std::lock_guard<std::mutex> g(c->mu);
    const uint64_t tt = ((1ull << n) + 7) / 8;
    const uint64_t tt_alloc = align_up(tt, 16);
    const Workspace w = workspace_layout((int)n);
    // n = DQMC_MAX_N: the bitmap is written over the state (one array of
    // 111.6 GB instead of 217.5 GB); smaller n keep a bitmap buffer of their own.
    const bool inplace = n >= (uint32_t)DQMC_MAX_N && !make_plan((int)n).sps.empty();
    if ((st = ensure(c, 0, tt_alloc))) return st;
    if (dc_bits && (st = ensure(c, 1, tt_alloc))) return st;
    if (inplace) {
        if (c->buf[2]) cudaFree(c->buf[2]);   // a bitmap buffer left by a smaller n
        c->buf[2] = nullptr;
        c->cap[2] = 0;
    } else if ((st = ensure(c, 2, bitmap_alloc_bytes((int)n)))) {
        return st;
    }
    if ((st = ensure(c, 3, w.total))) return st;
    void *d_bitmap = inplace ? static_cast<char *>(c->buf[3]) + w.state_off : c->buf[2];
    // A list buffer in pinned host memory that the device can address (8-byte
    // aligned) is written by the kernels directly (over NVLink-C2C on a
    // Grace-based node), so the list needs no copy after the sweep; any other
    // buffer gets the list through a device buffer and one copy.
    uint32_t *d_pairs = nullptr;
    bool direct = false;
    if (want_list && cap) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, out_pairs) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer && (uintptr_t)pa.devicePointer % 8 == 0) {
            d_pairs = static_cast<uint32_t *>(pa.devicePointer);
            direct = true;
        } else {
            cudaGetLastError();   // pageable memory: not an error
            if ((st = ensure(c, 4, 8 * cap))) return st;
            d_pairs = static_cast<uint32_t *>(c->buf[4]);
        }
    }
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemcpyAsync(c->buf[0], on_bits, tt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && dc_bits) e = cudaMemcpyAsync(c->buf[1], dc_bits, tt, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return map_cuda(e);
    uint64_t *dcount = reinterpret_cast<uint64_t *>(c->d_count);
    if (want_list)
        st = dqmc_list_dev_ex(n, c->buf[0], dc_bits ? c->buf[1] : nullptr, flags, d_bitmap, d_pairs, cap, dcount,
                              c->buf[3], c->cap[3], s);
    else
        st = dqmc_primes_dev_ex(n, c->buf[0], dc_bits ? c->buf[1] : nullptr, flags, d_bitmap, dcount, c->buf[3],
                                c->cap[3], s);
    if (st) return st;
    e = cudaMemcpyAsync(c->h_count, c->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out_bitmap)
        e = cudaMemcpyAsync(out_bitmap, d_bitmap, dqmc_bitmap_bytes(n), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda(e);
    if ((st = dqmc_dev_status(n, c->buf[3], c->cap[3], s))) return st;
    const uint64_t count = *c->h_count;
    if (out_count) *out_count = count;
    if (want_list && cap && !direct) {
        const uint64_t k = count < cap ? count : cap;
        if (k) {
            e = cudaMemcpy(out_pairs, c->buf[4], 8 * k, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return map_cuda(e);
        }
    }
    if (want_list && count > cap) return DQMC_ETRUNC;
    return DQMC_OK;
}

extern "C" int dqmc_primes(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
                           uint8_t *out_prime_bitmap)
{
    return host_run(n, on_bits, dc_bits, out_prime_bitmap, nullptr, 0, nullptr, false);
}

extern "C" int dqmc_count(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint64_t *out_count)
{
    if (!out_count) return DQMC_EINVAL;
    return host_run(n, on_bits, dc_bits, nullptr, nullptr, 0, out_count, false);
}

extern "C" int dqmc_list(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint32_t *out_pairs,
                         uint64_t cap, uint64_t *out_count)
{
    return host_run(n, on_bits, dc_bits, nullptr, out_pairs, cap, out_count, true);
}

extern "C" int dqmc_primes_ex(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint32_t flags,
                              uint8_t *out_prime_bitmap, uint64_t *out_count)
{
    return host_run(n, on_bits, dc_bits, out_prime_bitmap, nullptr, 0, out_count, false, flags);
}

extern "C" int dqmc_list_ex(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint32_t flags,
                            uint32_t *out_pairs, uint64_t cap, uint64_t *out_count)
{
    return host_run(n, on_bits, dc_bits, nullptr, out_pairs, cap, out_count, true, flags);
}

extern "C" void dqmc_release(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    DeviceCache *c = nullptr;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        c = g_cache[dev];
    }
    if (!c) return;
    // Only the buffers go: a host call on another thread may hold this entry
    // and be waiting for its lock, so the entry itself (its stream and count
    // words, a few bytes) stays for the life of the process.
    std::lock_guard<std::mutex> g2(c->mu);
    for (int i = 0; i < 5; ++i) {
        if (c->buf[i]) cudaFree(c->buf[i]);
        c->buf[i] = nullptr;
        c->cap[i] = 0;
    }
}
