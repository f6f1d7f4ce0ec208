// dqmc_batch.cu -- the batch driver: many independent functions, grouped by
// n, swept by one launch per (n, pass) and captured into one CUDA graph.
//
// Every function is swept as dqmc_primes sweeps one function (DenseQMC,
// arXiv 2302.10083, Algorithm 3, Section 4.1).  n <= 12: the one-tile kernel,
// one CTA per function, the whole state in shared memory.  n = 13, 14: the
// streaming pass kernels in batch mode, block b on tile b % tiles of function
// list[b / tiles], each function with its own state in the workspace.
#include <cstring>
#include <mutex>
#include <vector>

#include "dqmc.h"
#include "dqmc_batch.h"
#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"

namespace dqmc {

namespace {

constexpr int kClasses = DQMC_BATCH_MAX_N + 1;

uint64_t align_up_b(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

int map_err(cudaError_t e)
{
    if (e == cudaSuccess) return DQMC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DQMC_ENOMEM : DQMC_ECUDA;
}

// Where each part of the workspace starts (bytes from its base).
struct BatchLayout {
    uint64_t fn_off = 0;            // uint32 function ids, grouped by n (largest n first)
    uint64_t tt_off = 0, dc_off = 0, bm_off = 0;   // uint64 per function id
    uint64_t ctrl_off[kClasses] = {};
    uint64_t state_off[kClasses] = {};
    uint64_t total = 0;
};

BatchLayout batch_layout(uint32_t nfun, const uint32_t count[kClasses])
{
    BatchLayout L;
    uint64_t at = 0;
    L.fn_off = at;
    at = align_up_b(at + 4ull * nfun, 256);
    L.tt_off = at;
    at = align_up_b(at + 8ull * nfun, 256);
    L.dc_off = at;
    at = align_up_b(at + 8ull * nfun, 256);
    L.bm_off = at;
    at = align_up_b(at + 8ull * nfun, 256);
    for (int c = 0; c < kClasses; ++c) {
        if (!count[c]) continue;
        const Plan p = make_plan(c);
        if (p.sps.empty()) continue;
        L.ctrl_off[c] = at;
        at = align_up_b(at + ctrl_layout(p).bytes, 256);
        L.state_off[c] = at;
        at = align_up_b(at + (uint64_t)count[c] * p.state_rows * kChunkBytes, 256);
    }
    L.total = at;
    return L;
}

struct BatchCache {
    std::mutex mu;
    void *work = nullptr;
    uint64_t work_cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    // what the graph was captured for
    std::vector<uint32_t> n;
    std::vector<uint64_t> tt, dc, bm;
    bool has_dc = false;
    const void *arena = nullptr;
    void *counts = nullptr, *bitmaps = nullptr;
};

std::mutex g_batch_mu;
BatchCache *g_batch[64];

BatchCache *batch_cache(int *st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *st = e == cudaSuccess ? DQMC_EINVAL : map_err(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> g(g_batch_mu);
    if (!g_batch[dev]) {
        BatchCache *c = new BatchCache();
        e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            *st = map_err(e);
            delete c;
            return nullptr;
        }
        g_batch[dev] = c;
    }
    return g_batch[dev];
}

bool same_batch(const BatchCache &c, uint32_t nfun, const uint32_t *n, const uint64_t *tt, const uint64_t *dc,
                const uint64_t *bm, const void *arena, void *counts, void *bitmaps)
{
    if (!c.exec || c.n.size() != nfun || c.arena != arena || c.counts != counts || c.bitmaps != bitmaps) return false;
    if (c.has_dc != (dc != nullptr)) return false;
    if (memcmp(c.n.data(), n, 4ull * nfun) || memcmp(c.tt.data(), tt, 8ull * nfun) ||
        memcmp(c.bm.data(), bm, 8ull * nfun))
        return false;
    return !dc || !memcmp(c.dc.data(), dc, 8ull * nfun);
}

}  // namespace

}  // namespace dqmc

using namespace dqmc;

extern "C" uint64_t dqmc_batch_workspace_bytes(uint32_t nfun, const uint32_t *n)
{
    if (nfun && !n) return 0;
    uint32_t count[kClasses] = {};
    for (uint32_t f = 0; f < nfun; ++f) {
        if (n[f] > DQMC_BATCH_MAX_N) return 0;
        ++count[n[f]];
    }
    return batch_layout(nfun, count).total;
}

extern "C" int dqmc_batch_run(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                              const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps,
                              const uint64_t *bm_off, void *stream)
{
    if (nfun == 0) return DQMC_OK;
    if (nfun > (1u << 24) || !n || !tt_off || !bm_off || !d_tt_arena || !d_out_count || !d_out_bitmaps)
        return DQMC_EINVAL;
    if ((uintptr_t)d_tt_arena % 4 || (uintptr_t)d_out_count % 8 || (uintptr_t)d_out_bitmaps % 16)
        return DQMC_EINVAL;
    uint32_t count[kClasses] = {};
    for (uint32_t f = 0; f < nfun; ++f) {
        if (n[f] > DQMC_BATCH_MAX_N) return DQMC_EINVAL;
        const uint64_t a = n[f] >= 5 ? 4 : 1;
        if (tt_off[f] % a || bm_off[f] % 16) return DQMC_EINVAL;
        if (dc_off && dc_off[f] != ~0ull && dc_off[f] % a) return DQMC_EINVAL;
        ++count[n[f]];
    }
    int st = DQMC_OK;
    BatchCache *c = batch_cache(&st);
    if (!c) return st;
    std::lock_guard<std::mutex> g(c->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (same_batch(*c, nfun, n, tt_off, dc_off, bm_off, d_tt_arena, d_out_count, d_out_bitmaps))
        return map_err(cudaGraphLaunch(c->exec, s));

    // ---- new batch: workspace, function tables, then capture the graph
    const BatchLayout L = batch_layout(nfun, count);
    cudaError_t e = cudaSuccess;
    if (c->work_cap < L.total) {
        if (c->exec) cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
        if (c->work) {
            e = cudaStreamSynchronize(s);   // earlier launches may still use the old workspace
            if (e == cudaSuccess) e = cudaFree(c->work);
            c->work = nullptr;
            c->work_cap = 0;
            if (e != cudaSuccess) return map_err(e);
        }
        e = cudaMalloc(&c->work, L.total);
        if (e != cudaSuccess) return map_err(e);
        c->work_cap = L.total;
    }
    char *work = static_cast<char *>(c->work);
    // function ids grouped by n, largest n first (the big classes start first)
    std::vector<uint32_t> ids;
    ids.reserve(nfun);
    uint32_t class_at[kClasses] = {};
    for (int cl = kClasses - 1; cl >= 0; --cl) {
        class_at[cl] = (uint32_t)ids.size();
        for (uint32_t f = 0; f < nfun; ++f)
            if ((int)n[f] == cl) ids.push_back(f);
    }
    std::vector<uint64_t> dcv(nfun, ~0ull);
    if (dc_off) memcpy(dcv.data(), dc_off, 8ull * nfun);
    // the tables go in with ordinary copies (stream-ordered: the graph below
    // runs after them)
    e = cudaMemcpyAsync(work + L.fn_off, ids.data(), 4ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(work + L.tt_off, tt_off, 8ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(work + L.dc_off, dcv.data(), 8ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(work + L.bm_off, bm_off, 8ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors die at return
    if (e != cudaSuccess) return map_err(e);

    if (c->exec) cudaGraphExecDestroy(c->exec);
    c->exec = nullptr;
    cudaStream_t cs = c->cap_stream;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return map_err(e);
    cudaError_t le = cudaMemsetAsync(d_out_count, 0, 8ull * nfun, cs);
    for (int cl = kClasses - 1; cl >= 0 && le == cudaSuccess; --cl) {
        if (!count[cl]) continue;
        BatchArgs b;
        b.fn = reinterpret_cast<const uint32_t *>(work + L.fn_off) + class_at[cl];
        b.nfun = count[cl];
        b.tt_off = reinterpret_cast<const uint64_t *>(work + L.tt_off);
        b.dc_off = reinterpret_cast<const uint64_t *>(work + L.dc_off);
        b.bm_off = reinterpret_cast<const uint64_t *>(work + L.bm_off);
        b.arena = static_cast<const uint8_t *>(d_tt_arena);
        b.bitmaps = static_cast<uint8_t *>(d_out_bitmaps);
        b.count = reinterpret_cast<unsigned long long *>(d_out_count);
        const Plan p = make_plan(cl);
        if (p.sps.empty())
            le = launch_sweep(p, nullptr, nullptr, nullptr, nullptr, nullptr, cs, 0, -1, &b);
        else
            le = launch_super(p, nullptr, nullptr, work + L.state_off[cl], nullptr, nullptr, nullptr, 0,
                              work + L.ctrl_off[cl], cs, 0, plan_passes(p), &b);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return map_err(le != cudaSuccess ? le : e);
    }
    e = cudaGraphInstantiate(&c->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->exec = nullptr;
        return map_err(e);
    }
    c->n.assign(n, n + nfun);
    c->tt.assign(tt_off, tt_off + nfun);
    c->bm.assign(bm_off, bm_off + nfun);
    c->has_dc = dc_off != nullptr;
    if (dc_off) c->dc.assign(dc_off, dc_off + nfun);
    else c->dc.clear();
    c->arena = d_tt_arena;
    c->counts = d_out_count;
    c->bitmaps = d_out_bitmaps;
    return map_err(cudaGraphLaunch(c->exec, s));
}

extern "C" int dqmc_batch_release(void)
{
    int st = DQMC_OK;
    BatchCache *c = batch_cache(&st);
    if (!c) return st;
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = cudaDeviceSynchronize();
    if (c->exec) cudaGraphExecDestroy(c->exec);
    c->exec = nullptr;
    if (c->work) {
        cudaError_t e2 = cudaFree(c->work);
        if (e == cudaSuccess) e = e2;
    }
    c->work = nullptr;
    c->work_cap = 0;
    c->n.clear();
    return map_err(e);
}
