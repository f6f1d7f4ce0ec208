// dqmc_api.cu -- the C ABI of libdqmc.so (declared in include/dqmc.h and
// include/dqmc_plan.h): argument checks, the pass plan, the workspace layout,
// and the host entry points with their per-device buffer cache.
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

// Pass plan for n variables.
//   n <= 12: one tile holds the whole function in shared memory (one pass).
//   n >= 13: the high digits are split into a first group of 7 (contiguous
//   rows) and groups of at most 6 (each row carried with its inner neighbour
//   digit for 96-byte runs).  Merge goes group by group from the low digits;
//   the last Merge pass also Reduces its digits and the chunk digits; the other
//   groups are then Reduced from the top down, the first group last, and that
//   pass writes the bitmap.
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
        ps.B = 0;
        ps.a = 0;
        ps.tiles = 1;
        ps.fuse_reduce = ps.chunk_reduce = ps.write_out = true;
        p.passes.push_back(ps);
        p.state_rows = 0;
        return p;
    }
    p.state_rows = pow3(H);
    std::vector<int> starts, sizes;
    starts.push_back(0);
    sizes.push_back(kMaxSmemGroup);
    const int rest = H - kMaxSmemGroup;
    const int ng = (rest + kMaxStreamGroup - 1) / kMaxStreamGroup;
    int at = kMaxSmemGroup;
    for (int i = 0; i < ng; ++i) {
        const int k = rest / ng + (i < rest % ng ? 1 : 0);
        starts.push_back(at);
        sizes.push_back(k);
        at += k;
    }
    const int G = (int)sizes.size();
    {   // first group: truth table -> rows with digits >= 7 binary
        Pass ps;
        ps.kind = kPassFirst;
        ps.K = sizes[0];
        ps.top_binary = true;
        ps.w_top = pow3(sizes[0]);
        ps.tiles = 1ull << (H - sizes[0]);
        p.passes.push_back(ps);
    }
    for (int i = 1; i < G; ++i) {
        const bool last = (i == G - 1);
        Pass ps;
        ps.kind = kPassMerge;
        ps.K = sizes[i];
        ps.B = 1;
        ps.a = starts[i];
        ps.n_mid = pow3(starts[i] - 1);
        ps.w_g = pow3(starts[i]);
        ps.w_top = pow3(starts[i] + sizes[i]);
        ps.top_binary = !last;
        const int top = H - starts[i] - sizes[i];
        ps.tiles = ps.n_mid * (last ? 1ull : (1ull << top));
        ps.fuse_reduce = ps.chunk_reduce = last;
        p.passes.push_back(ps);
    }
    for (int i = G - 2; i >= 1; --i) {
        Pass ps;
        ps.kind = kPassReduce;
        ps.K = sizes[i];
        ps.B = 1;
        ps.a = starts[i];
        ps.n_mid = pow3(starts[i] - 1);
        ps.w_g = pow3(starts[i]);
        ps.w_top = pow3(starts[i] + sizes[i]);
        ps.tiles = ps.n_mid * pow3(H - starts[i] - sizes[i]);
        p.passes.push_back(ps);
    }
    {
        Pass ps;
        ps.kind = kPassReduce;
        ps.K = sizes[0];
        ps.B = 0;
        ps.a = 0;
        ps.w_top = pow3(sizes[0]);
        ps.tiles = pow3(H - sizes[0]);
        ps.write_out = true;
        p.passes.push_back(ps);
    }
    return p;
}

std::string describe_plan(const Plan &p)
{
    std::string s = "{\"n\":" + std::to_string(p.n) + ",\"C\":" + std::to_string(p.C) +
                    ",\"H\":" + std::to_string(p.H) + ",\"state_rows\":" + std::to_string(p.state_rows) +
                    ",\"passes\":[";
    for (size_t i = 0; i < p.passes.size(); ++i) {
        const Pass &q = p.passes[i];
        static const char *kinds[] = {"first", "merge", "reduce"};
        char buf[512];
        snprintf(buf, sizeof buf,
                 "%s{\"kind\":\"%s\",\"K\":%d,\"B\":%d,\"a\":%d,\"top_binary\":%d,\"fuse_reduce\":%d,"
                 "\"chunk_reduce\":%d,\"write_out\":%d,\"tiles\":%llu,\"n_mid\":%llu,\"w_g\":%llu,\"w_top\":%llu}",
                 i ? "," : "", kinds[q.kind], q.K, q.B, q.a, (int)q.top_binary, (int)q.fuse_reduce,
                 (int)q.chunk_reduce, (int)q.write_out, (unsigned long long)q.tiles,
                 (unsigned long long)q.n_mid, (unsigned long long)q.w_g, (unsigned long long)q.w_top);
        s += buf;
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
    return (int)make_plan((int)n).passes.size();
}

extern "C" uint64_t dqmc_pass_bytes(uint32_t n, int pass, int with_dc)
{
    if (n > DQMC_MAX_N) return 0;
    return pass_bytes(make_plan((int)n), pass, with_dc != 0);
}

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
                     uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream)
{
    int st = check_dev_args(n, d_on, d_dc, d_work, work_bytes);
    if (st) return st;
    if (!d_bitmap || !aligned(d_bitmap, 16)) return DQMC_EINVAL;
    if (d_count && !aligned(d_count, 8)) return DQMC_EINVAL;
    const Plan plan = make_plan((int)n);
    if (last < 0) last = (int)plan.passes.size();
    if (first < 0 || first >= last || last > (int)plan.passes.size()) return DQMC_EINVAL;
    const Workspace w = workspace_layout((int)n);
    char *base = static_cast<char *>(d_work);
    unsigned long long *cnt = d_count ? reinterpret_cast<unsigned long long *>(d_count)
                                      : reinterpret_cast<unsigned long long *>(base + w.count_off);
    return map_cuda(launch_sweep(plan, d_on, d_dc, base + w.state_off, static_cast<uint32_t *>(d_bitmap),
                                 cnt, static_cast<cudaStream_t>(stream), first, last));
}

extern "C" int dqmc_primes_dev(uint32_t n, const void *d_on, const void *d_dc, void *d_bitmap,
                               uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream)
{
    return sweep_dev(n, 0, -1, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream);
}

extern "C" int dqmc_sweep_pass_dev(uint32_t n, int pass, const void *d_on, const void *d_dc, void *d_bitmap,
                                   uint64_t *d_count, void *d_work, uint64_t work_bytes, void *stream)
{
    if (pass < 0) return DQMC_EINVAL;
    return sweep_dev(n, pass, pass + 1, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream);
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

extern "C" int dqmc_list_dev(uint32_t n, const void *d_on, const void *d_dc, void *d_bitmap,
                             uint32_t *d_pairs, uint64_t cap, uint64_t *d_count, void *d_work,
                             uint64_t work_bytes, void *stream)
{
    if (!d_count) return DQMC_EINVAL;
    int st = dqmc_primes_dev(n, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream);
    if (st) return st;
    return dqmc_compact_dev(n, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes, stream);
}

// Host entry points: copy in, run, copy out, wait.
static int host_run(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint8_t *out_bitmap,
                    uint32_t *out_pairs, uint64_t cap, uint64_t *out_count, bool want_list)
{
    if (n > DQMC_MAX_N || !on_bits) return DQMC_EINVAL;
    if (want_list && cap && !out_pairs) return DQMC_EINVAL;
    int st = DQMC_OK;
    DeviceCache *c = cache_for_current_device(&st);
    if (!c) return st;
    std::lock_guard<std::mutex> g(c->mu);
    const uint64_t tt = ((1ull << n) + 7) / 8;
    const uint64_t tt_alloc = align_up(tt, 16);
    const Workspace w = workspace_layout((int)n);
    if ((st = ensure(c, 0, tt_alloc))) return st;
    if (dc_bits && (st = ensure(c, 1, tt_alloc))) return st;
    if ((st = ensure(c, 2, bitmap_alloc_bytes((int)n)))) return st;
    if ((st = ensure(c, 3, w.total))) return st;
    if (want_list && cap && (st = ensure(c, 4, 8 * cap))) return st;
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemcpyAsync(c->buf[0], on_bits, tt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && dc_bits) e = cudaMemcpyAsync(c->buf[1], dc_bits, tt, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return map_cuda(e);
    uint64_t *dcount = reinterpret_cast<uint64_t *>(c->d_count);
    if (want_list)
        st = dqmc_list_dev(n, c->buf[0], dc_bits ? c->buf[1] : nullptr, c->buf[2],
                           static_cast<uint32_t *>(cap ? c->buf[4] : nullptr), cap, dcount, c->buf[3],
                           c->cap[3], s);
    else
        st = dqmc_primes_dev(n, c->buf[0], dc_bits ? c->buf[1] : nullptr, c->buf[2], dcount, c->buf[3],
                             c->cap[3], s);
    if (st) return st;
    e = cudaMemcpyAsync(c->h_count, c->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out_bitmap)
        e = cudaMemcpyAsync(out_bitmap, c->buf[2], dqmc_bitmap_bytes(n), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda(e);
    const uint64_t count = *c->h_count;
    if (out_count) *out_count = count;
    if (want_list && cap) {
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

extern "C" void dqmc_release(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> g(g_cache_mu);
    DeviceCache *c = g_cache[dev];
    if (!c) return;
    {
        std::lock_guard<std::mutex> g2(c->mu);
        for (int i = 0; i < 5; ++i)
            if (c->buf[i]) cudaFree(c->buf[i]);
        if (c->d_count) cudaFree(c->d_count);
        if (c->h_count) cudaFreeHost(c->h_count);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
    g_cache[dev] = nullptr;
}
