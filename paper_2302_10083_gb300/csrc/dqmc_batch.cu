// dqmc_batch.cu -- the batch driver: many independent functions, grouped by
// n, one launch per n (per pass on the streaming path), captured into one
// CUDA graph with one branch per n, and the autotuner that picks each n's
// launch.
//
// Every function is swept as dqmc_primes sweeps one function (DenseQMC,
// arXiv 2302.10083, Algorithm 3, Section 4.1).  Two paths per n:
//   * shared memory (5 <= n <= 14, dqmc_fn.cu): a function's whole state in
//     shared memory (a cluster of three CTAs for n = 14), fpc functions per
//     CTA, tg threads each, D high digits per step;
//   * tiles: n <= 12 the one-tile kernel of dqmc_sweep.cu, one CTA per
//     function; n = 13, 14 the streaming pass kernels in batch mode, each
//     function with its own state in the workspace.
// The autotuner times every launchable choice on the caller's batch and
// keeps the fastest per n.
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

// The launch of one n: path, then the shared-memory kernel's shape.
struct ClassConfig {
    uint32_t path = DQMC_BATCH_PATH_TILES;
    FnConfig fn;
};

// Shared-memory shape of one n that needs no scratch (the server's): threads
// per function, functions per CTA, digits per step, CTAs per function
// (measured best on a GB300 for 5958 functions of that n; n = 14 on a
// cluster of nine).
ClassConfig smem_config(int n)
{
    ClassConfig c;
    if (n < kFnMinN || n > kFnMaxN) return c;
    static const int tg[kClasses] = {0, 0, 0, 0, 0, 32, 32, 32, 32, 32, 32, 128, 256, 1024, 256};
    static const int fpc[kClasses] = {0, 0, 0, 0, 0, 6, 8, 8, 8, 6, 8, 2, 1, 1, 1};
    static const int dig[kClasses] = {0, 0, 0, 0, 0, 2, 2, 2, 3, 2, 3, 3, 3, 3, 3};
    c.path = DQMC_BATCH_PATH_SMEM;
    c.fn.tg = tg[n];
    c.fn.fpc = fpc[n];
    c.fn.digits = dig[n];
    c.fn.ctas = n == 14 ? 9 : 1;
    return c;
}

// Built-in table (the autotuner's choices on the 65,536-function batch on a
// GB300): shared memory for 5 <= n <= 14, n = 14 on one CTA per SM doing the
// thirds of the top digit in turn (3.6 ms against 4.2 ms for the streaming
// kernels and 5.5 ms for nine-CTA clusters), the tile kernel below n = 5.
ClassConfig default_config(int n)
{
    if (n < kFnMinN) return ClassConfig{};
    ClassConfig c = smem_config(n);
    if (n == 14) {
        c.fn.tg = 1024;
        c.fn.ctas = 1;
    }
    return c;
}

std::mutex g_cfg_mu;
ClassConfig g_cfg[kClasses];
bool g_cfg_init = false;
uint64_t g_cfg_gen = 1;     // bumped by every change; a graph records the one it was captured with

void config_snapshot(ClassConfig out[kClasses], uint64_t *gen)
{
    std::lock_guard<std::mutex> g(g_cfg_mu);
    if (!g_cfg_init) {
        for (int c = 0; c < kClasses; ++c) g_cfg[c] = default_config(c);
        g_cfg_init = true;
    }
    for (int c = 0; c < kClasses; ++c) out[c] = g_cfg[c];
    if (gen) *gen = g_cfg_gen;
}

bool config_ok(int n, const ClassConfig &c)
{
    if (n < 0 || n >= kClasses) return false;
    if (c.path == DQMC_BATCH_PATH_TILES) return true;
    return c.path == DQMC_BATCH_PATH_SMEM && fn_config_ok(n, c.fn);
}

// The streaming path keeps a device state per function (n >= 13 only).
bool needs_state(int n, const ClassConfig &c) { return c.path == DQMC_BATCH_PATH_TILES && n >= 13; }

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
    uint64_t scratch_off = 0;       // n = 14 in one CTA: a third per CTA slot
    uint32_t scratch_ctas = 0;
    uint64_t ctr_off = 0;           // one-launch mode: a queue counter per n
    uint64_t total = 0;
};

// CTA slots of the one-CTA n = 14 kernel: one per SM (210 KB of shared memory each).
uint32_t thirds_slots()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return 160;   // no device to ask (workspace sizing on a host without one)
    }
    return (uint32_t)sms;
}

BatchLayout batch_layout(uint32_t nfun, const uint32_t count[kClasses], const ClassConfig cfg[kClasses])
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
        if (!count[c] || !needs_state(c, cfg[c])) continue;
        const Plan p = make_plan(c);
        if (p.sps.empty()) continue;
        L.ctrl_off[c] = at;
        at = align_up_b(at + ctrl_layout(p).bytes, 256);
        L.state_off[c] = at;
        at = align_up_b(at + (uint64_t)count[c] * p.state_rows * kChunkBytes, 256);
    }
    if (count[14]) {   // reserved whenever n = 14 is present, so that the autotuner can try it
        L.scratch_ctas = thirds_slots();
        L.scratch_off = at;
        at = align_up_b(at + (uint64_t)L.scratch_ctas * kFnThirdBytes, 256);
    }
    L.ctr_off = at;
    at = align_up_b(at + 4ull * kClasses, 256);
    L.total = at;
    return L;
}

struct BatchCache {
    std::mutex mu;
    void *work = nullptr;
    uint64_t work_cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t branch[kClasses] = {};
    cudaEvent_t fork = nullptr, join[kClasses] = {};
    cudaEvent_t t0 = nullptr, t1 = nullptr;     // autotuner timing
    cudaGraphExec_t exec = nullptr;
    uint64_t cfg_gen = 0;
    bool one = false;           // captured as one persistent launch
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
        for (int k = 0; k < kClasses && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&c->branch[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreate(&c->t0);
        if (e == cudaSuccess) e = cudaEventCreate(&c->t1);
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
                const uint64_t *bm, const void *arena, void *counts, void *bitmaps, uint64_t gen, bool one)
{
    if (!c.exec || c.cfg_gen != gen || c.one != one || c.n.size() != nfun || c.arena != arena || c.counts != counts ||
        c.bitmaps != bitmaps)
        return false;
    if (c.has_dc != (dc != nullptr)) return false;
    if (memcmp(c.n.data(), n, 4ull * nfun) || memcmp(c.tt.data(), tt, 8ull * nfun) ||
        memcmp(c.bm.data(), bm, 8ull * nfun))
        return false;
    return !dc || !memcmp(c.dc.data(), dc, 8ull * nfun);
}

// Check a batch's arrays; count[] gets the functions per n.
int check_batch(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps, const uint64_t *bm_off,
                uint32_t count[kClasses])
{
    if (nfun > (1u << 24) || !n || !tt_off || !bm_off || !d_tt_arena || !d_out_count || !d_out_bitmaps)
        return DQMC_EINVAL;
    if ((uintptr_t)d_tt_arena % 4 || (uintptr_t)d_out_count % 8 || (uintptr_t)d_out_bitmaps % 16)
        return DQMC_EINVAL;
    for (int c = 0; c < kClasses; ++c) count[c] = 0;
    for (uint32_t f = 0; f < nfun; ++f) {
        if (n[f] > DQMC_BATCH_MAX_N) return DQMC_EINVAL;
        const uint64_t a = n[f] >= 5 ? 4 : 1;
        if (tt_off[f] % a || bm_off[f] % 16) return DQMC_EINVAL;
        if (dc_off && dc_off[f] != ~0ull && dc_off[f] % a) return DQMC_EINVAL;
        ++count[n[f]];
    }
    return DQMC_OK;
}

// Make the workspace at least L.total bytes and copy the function tables in
// (ids grouped by n, largest n first; class_at[n] = first index of n).
int upload_tables(BatchCache &c, const BatchLayout &L, uint32_t nfun, const uint32_t *n, const uint64_t *tt_off,
                  const uint64_t *dc_off, const uint64_t *bm_off, uint32_t class_at[kClasses], cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (c.work_cap < L.total) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        c.exec = nullptr;
        if (c.work) {
            e = cudaStreamSynchronize(s);   // earlier launches may still use the old workspace
            if (e == cudaSuccess) e = cudaFree(c.work);
            c.work = nullptr;
            c.work_cap = 0;
            if (e != cudaSuccess) return map_err(e);
        }
        e = cudaMalloc(&c.work, L.total);
        if (e != cudaSuccess) return map_err(e);
        c.work_cap = L.total;
    }
    char *work = static_cast<char *>(c.work);
    std::vector<uint32_t> ids;
    ids.reserve(nfun);
    for (int cl = kClasses - 1; cl >= 0; --cl) {
        class_at[cl] = (uint32_t)ids.size();
        for (uint32_t f = 0; f < nfun; ++f)
            if ((int)n[f] == cl) ids.push_back(f);
    }
    std::vector<uint64_t> dcv(nfun, ~0ull);
    if (dc_off) memcpy(dcv.data(), dc_off, 8ull * nfun);
    // ordinary stream-ordered copies: the launches below run after them
    e = cudaMemcpyAsync(work + L.fn_off, ids.data(), 4ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(work + L.tt_off, tt_off, 8ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(work + L.dc_off, dcv.data(), 8ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(work + L.bm_off, bm_off, 8ull * nfun, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors die at return
    return map_err(e);
}

// Enqueue the sweep of every function of one n.
cudaError_t launch_class(BatchCache &c, const BatchLayout &L, int cl, const ClassConfig &cc, uint32_t first,
                         uint32_t count, const void *d_tt_arena, void *d_out_count, void *d_out_bitmaps,
                         cudaStream_t s)
{
    char *work = static_cast<char *>(c.work);
    BatchArgs b;
    b.fn = reinterpret_cast<const uint32_t *>(work + L.fn_off) + first;
    b.nfun = count;
    b.tt_off = reinterpret_cast<const uint64_t *>(work + L.tt_off);
    b.dc_off = reinterpret_cast<const uint64_t *>(work + L.dc_off);
    b.bm_off = reinterpret_cast<const uint64_t *>(work + L.bm_off);
    b.arena = static_cast<const uint8_t *>(d_tt_arena);
    b.bitmaps = static_cast<uint8_t *>(d_out_bitmaps);
    b.count = reinterpret_cast<unsigned long long *>(d_out_count);
    if (L.scratch_ctas) {
        b.scratch = work + L.scratch_off;
        b.scratch_ctas = L.scratch_ctas;
    }
    if (cc.path == DQMC_BATCH_PATH_SMEM) return launch_fn_batch(cl, b, cc.fn, s);
    const Plan p = make_plan(cl);
    if (p.sps.empty()) return launch_sweep(p, nullptr, nullptr, nullptr, nullptr, nullptr, s, 0, -1, &b);
    return launch_super(p, nullptr, nullptr, work + L.state_off[cl], nullptr, nullptr, nullptr, 0,
                        work + L.ctrl_off[cl], s, 0, plan_passes(p), &b);
}

// The one-launch shape of each n present, largest n first (launch_fn_queue):
// the n's shared-memory shape from the launch table when it is one CTA per
// function, else the built-in one; as many groups as the CTA's threads,
// its shared memory and the named barriers allow, and groups of more than
// one warp widened to use all the threads (n = 12: 3 groups of 320).
QueueSetup queue_setup(const BatchLayout &L, const uint32_t count[kClasses], const uint32_t class_at[kClasses],
                       const ClassConfig cfg[kClasses], void *work)
{
    QueueSetup q;
    for (int cl = kClasses - 1; cl >= 0; --cl) {
        if (!count[cl]) continue;
        QueueClass k;
        k.n = (uint32_t)cl;
        k.first = class_at[cl];
        k.count = count[cl];
        if (cl < kFnMinN) {
            k.tg = 32;
            k.groups = kQueueThreads / 32;
        } else {
            const ClassConfig cc = (cfg[cl].path == DQMC_BATCH_PATH_SMEM && cfg[cl].fn.ctas == 1) ? cfg[cl]
                                                                                                     : default_config(cl);
            k.digits = (uint32_t)cc.fn.digits;
            if (cl == 14) {
                k.tg = kQueueThreads;
                k.groups = 1;
            } else {
                k.tg = (uint32_t)(cc.fn.tg == 64 ? 128 : cc.fn.tg);
                uint32_t g = kQueueThreads / k.tg;
                const uint64_t by_smem = kFnMaxSmem / queue_fn_smem(cl);
                if (g > by_smem) g = (uint32_t)by_smem;
                if (k.tg > 32 && g > 15) g = 15;
                k.groups = g;
                // when shared memory caps the groups, spread the CTA's threads over them
                if (k.tg > 32 && g * k.tg < (uint32_t)kQueueThreads) k.tg = kQueueThreads / g / 32 * 32;
            }
        }
        const uint64_t sm = (uint64_t)k.groups * queue_fn_smem(cl);
        if (sm > q.smem) q.smem = sm;
        q.cls[q.nclass++] = k;
    }
    q.ctr = reinterpret_cast<uint32_t *>(static_cast<char *>(work) + L.ctr_off);
    q.ctas = thirds_slots();
    if (count[14] && L.scratch_ctas < q.ctas) q.ctas = L.scratch_ctas;
    return q;
}

}  // namespace

cudaError_t launch_batch_in_smem(int n, const BatchArgs &b, cudaStream_t s)
{
    if (n < 0 || n > kFnMaxN) return cudaErrorInvalidValue;
    if (n < kFnMinN) return launch_sweep(make_plan(n), nullptr, nullptr, nullptr, nullptr, nullptr, s, 0, -1, &b);
    ClassConfig cfg[kClasses];
    config_snapshot(cfg, nullptr);
    // the server has no scratch for the one-CTA n = 14 kernel: clusters there
    const bool usable = cfg[n].path == DQMC_BATCH_PATH_SMEM && !(n == 14 && cfg[n].fn.ctas == 1);
    const ClassConfig cc = usable ? cfg[n] : smem_config(n);
    return launch_fn_batch(n, b, cc.fn, s);
}

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
    ClassConfig cfg[kClasses];
    config_snapshot(cfg, nullptr);
    return batch_layout(nfun, count, cfg).total;
}

// dqmc_batch_run and dqmc_batch_run_one_launch: the graph is captured once
// per batch (and mode) and launched again for the same batch.
static int batch_run(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                     const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps, const uint64_t *bm_off,
                     void *stream, bool one)
{
    if (nfun == 0) return DQMC_OK;
    uint32_t count[kClasses];
    int st = check_batch(nfun, n, tt_off, d_tt_arena, dc_off, d_out_count, d_out_bitmaps, bm_off, count);
    if (st != DQMC_OK) return st;
    BatchCache *c = batch_cache(&st);
    if (!c) return st;
    std::lock_guard<std::mutex> g(c->mu);
    ClassConfig cfg[kClasses];
    uint64_t gen = 0;
    config_snapshot(cfg, &gen);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (same_batch(*c, nfun, n, tt_off, dc_off, bm_off, d_tt_arena, d_out_count, d_out_bitmaps, gen, one))
        return map_err(cudaGraphLaunch(c->exec, s));

    // ---- new batch: workspace, function tables, then capture the graph:
    // zero the counts, then one branch per n (largest n first), joined at the
    // end; or, in one-launch mode, zero the queue counters and launch the
    // queue kernel once
    const BatchLayout L = batch_layout(nfun, count, cfg);
    uint32_t class_at[kClasses];
    st = upload_tables(*c, L, nfun, n, tt_off, dc_off, bm_off, class_at, s);
    if (st != DQMC_OK) return st;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    c->exec = nullptr;
    cudaStream_t cs = c->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return map_err(e);
    cudaError_t le = cudaMemsetAsync(d_out_count, 0, 8ull * nfun, cs);
    if (one) {
        const QueueSetup q = queue_setup(L, count, class_at, cfg, c->work);
        BatchArgs b;
        char *work = static_cast<char *>(c->work);
        b.fn = reinterpret_cast<const uint32_t *>(work + L.fn_off);
        b.nfun = nfun;
        b.tt_off = reinterpret_cast<const uint64_t *>(work + L.tt_off);
        b.dc_off = reinterpret_cast<const uint64_t *>(work + L.dc_off);
        b.bm_off = reinterpret_cast<const uint64_t *>(work + L.bm_off);
        b.arena = static_cast<const uint8_t *>(d_tt_arena);
        b.bitmaps = static_cast<uint8_t *>(d_out_bitmaps);
        b.count = reinterpret_cast<unsigned long long *>(d_out_count);
        if (L.scratch_ctas) {
            b.scratch = work + L.scratch_off;
            b.scratch_ctas = L.scratch_ctas;
        }
        if (le == cudaSuccess) le = cudaMemsetAsync(q.ctr, 0, 4ull * kClasses, cs);
        if (le == cudaSuccess) le = launch_fn_queue(b, q, cs);
    } else {
        if (le == cudaSuccess) le = cudaEventRecord(c->fork, cs);
        bool joined[kClasses] = {};
        for (int cl = kClasses - 1; cl >= 0 && le == cudaSuccess; --cl) {
            if (!count[cl]) continue;
            cudaStream_t bs = c->branch[cl];
            le = cudaStreamWaitEvent(bs, c->fork, 0);
            if (le == cudaSuccess)
                le = launch_class(*c, L, cl, cfg[cl], class_at[cl], count[cl], d_tt_arena, d_out_count, d_out_bitmaps, bs);
            if (le == cudaSuccess) le = cudaEventRecord(c->join[cl], bs);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(cs, c->join[cl], 0);
            joined[cl] = le == cudaSuccess;
        }
        // every branch that was forked must be joined before the capture ends
        for (int cl = 0; cl < kClasses && le != cudaSuccess; ++cl)
            if (count[cl] && !joined[cl]) {
                cudaEventRecord(c->join[cl], c->branch[cl]);
                cudaStreamWaitEvent(cs, c->join[cl], 0);
            }
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
    c->cfg_gen = gen;
    c->one = one;
    return map_err(cudaGraphLaunch(c->exec, s));
}

extern "C" int dqmc_batch_run(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                              const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps,
                              const uint64_t *bm_off, void *stream)
{
    return batch_run(nfun, n, tt_off, d_tt_arena, dc_off, d_out_count, d_out_bitmaps, bm_off, stream, false);
}

extern "C" int dqmc_batch_run_one_launch(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off,
                                         const void *d_tt_arena, const uint64_t *dc_off, uint64_t *d_out_count,
                                         void *d_out_bitmaps, const uint64_t *bm_off, void *stream)
{
    return batch_run(nfun, n, tt_off, d_tt_arena, dc_off, d_out_count, d_out_bitmaps, bm_off, stream, true);
}

extern "C" int dqmc_batch_get_config(uint32_t n, dqmc_batch_config *out)
{
    if (n > DQMC_BATCH_MAX_N || !out) return DQMC_EINVAL;
    ClassConfig cfg[kClasses];
    config_snapshot(cfg, nullptr);
    out->path = cfg[n].path;
    out->threads_per_fn = (uint32_t)cfg[n].fn.tg;
    out->fns_per_cta = (uint32_t)cfg[n].fn.fpc;
    out->digits_per_step = (uint32_t)cfg[n].fn.digits;
    out->ctas_per_fn = (uint32_t)cfg[n].fn.ctas;
    return DQMC_OK;
}

static ClassConfig from_public(const dqmc_batch_config &c)
{
    ClassConfig cc;
    cc.path = c.path;
    cc.fn.tg = (int)c.threads_per_fn;
    cc.fn.fpc = (int)c.fns_per_cta;
    cc.fn.digits = (int)c.digits_per_step;
    cc.fn.ctas = (int)c.ctas_per_fn;
    if (cc.path == DQMC_BATCH_PATH_TILES) cc.fn = FnConfig{};
    return cc;
}

extern "C" int dqmc_batch_set_config(uint32_t n, const dqmc_batch_config *cfg)
{
    if (n > DQMC_BATCH_MAX_N || !cfg) return DQMC_EINVAL;
    if (cfg->threads_per_fn > 4096 || cfg->fns_per_cta > 64 || cfg->digits_per_step > 8 || cfg->ctas_per_fn > 64)
        return DQMC_EINVAL;
    const ClassConfig cc = from_public(*cfg);
    if (!config_ok((int)n, cc)) return DQMC_EINVAL;
    ClassConfig cur[kClasses];
    config_snapshot(cur, nullptr);   // makes sure the defaults are in place
    std::lock_guard<std::mutex> g(g_cfg_mu);
    g_cfg[n] = cc;
    ++g_cfg_gen;
    return DQMC_OK;
}

extern "C" int dqmc_batch_autotune(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                                   const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps,
                                   const uint64_t *bm_off, uint32_t reps, void *stream, float *out_ms)
{
    if (out_ms)
        for (int c = 0; c < kClasses; ++c) out_ms[c] = -1.0f;
    if (nfun == 0) return DQMC_OK;
    if (reps == 0 || reps > 1000) return DQMC_EINVAL;
    uint32_t count[kClasses];
    int st = check_batch(nfun, n, tt_off, d_tt_arena, dc_off, d_out_count, d_out_bitmaps, bm_off, count);
    if (st != DQMC_OK) return st;
    BatchCache *c = batch_cache(&st);
    if (!c) return st;
    std::lock_guard<std::mutex> g(c->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the workspace of the streaming path for every n, so that every choice can run
    ClassConfig tiles[kClasses];
    const BatchLayout L = batch_layout(nfun, count, tiles);
    uint32_t class_at[kClasses];
    st = upload_tables(*c, L, nfun, n, tt_off, dc_off, bm_off, class_at, s);
    if (st != DQMC_OK) return st;
    // the graph (if any) was captured for another workspace layout
    if (c->exec) cudaGraphExecDestroy(c->exec);
    c->exec = nullptr;

    ClassConfig best[kClasses];
    config_snapshot(best, nullptr);
    for (int cl = 0; cl < kClasses; ++cl) {
        if (!count[cl]) continue;
        std::vector<ClassConfig> cand;
        cand.push_back(ClassConfig{});     // the tile / streaming path
        if (cl >= kFnMinN)
            for (int ctas : {1, 3, 9})
                for (int d : {2, 3})
                    for (int tg : {32, 64, 128, 256, 512, 1024})
                        for (int fpc : {1, 2, 3, 4, 6, 8}) {
                            ClassConfig cc;
                            cc.path = DQMC_BATCH_PATH_SMEM;
                            cc.fn.tg = tg;
                            cc.fn.fpc = fpc;
                            cc.fn.digits = d;
                            cc.fn.ctas = ctas;
                            // no more functions per CTA than the class has
                            if (fpc > 1 && (uint32_t)fpc > count[cl]) continue;
                            if (fn_config_ok(cl, cc.fn)) cand.push_back(cc);
                        }
        float best_ms = -1.0f;
        for (const ClassConfig &cc : cand) {
            cudaError_t e = cudaSuccess;
            for (uint32_t r = 0; r <= reps && e == cudaSuccess; ++r) {
                if (r == 1) e = cudaEventRecord(c->t0, s);
                if (e == cudaSuccess) e = cudaMemsetAsync(d_out_count, 0, 8ull * nfun, s);
                if (e == cudaSuccess)
                    e = launch_class(*c, L, cl, cc, class_at[cl], count[cl], d_tt_arena, d_out_count, d_out_bitmaps, s);
            }
            if (e == cudaSuccess) e = cudaEventRecord(c->t1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(c->t1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->t0, c->t1);
            if (e != cudaSuccess) {
                // a choice that does not launch on this device (e.g. no room for a
                // cluster) is skipped; an error that sticks to the context is not
                cudaGetLastError();
                const cudaError_t sticky = cudaStreamSynchronize(s);
                if (sticky != cudaSuccess) return map_err(sticky);
                continue;
            }
            ms /= (float)reps;
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                best[cl] = cc;
            }
        }
        if (out_ms) out_ms[cl] = best_ms;
    }
    {
        std::lock_guard<std::mutex> gc(g_cfg_mu);
        for (int cl = 0; cl < kClasses; ++cl)
            if (count[cl]) g_cfg[cl] = best[cl];
        ++g_cfg_gen;
    }
    return DQMC_OK;
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
