// dqmc_server.cu -- the serving loop: a job queue admitted by device-memory
// footprint, small jobs batched on arrival, large jobs on their own streams,
// completion signalled by host callbacks.
//
// Each job is swept as dqmc_primes sweeps one function (DenseQMC, arXiv
// 2302.10083, Algorithm 3, Section 4.1).  Jobs with n <= 14 go to batched
// launches (whole functions in shared memory, the launch shapes of the batch
// driver's table); larger jobs run the streaming pass kernels on a stream of
// their own.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dqmc.h"
#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"
#include "dqmc_server.h"

namespace dqmc {
namespace {

constexpr uint64_t kNone = ~0ull;
constexpr uint64_t kGrain = 256;
constexpr int kSmallMaxN = kFnMaxN;      // 14: the whole state in shared memory (3 CTAs for 14)
constexpr size_t kMaxBatch = 4096;                        // small jobs per batched launch

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

uint64_t up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

int map_err(cudaError_t e)
{
    if (e == cudaSuccess) return DQMC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DQMC_ENOMEM : DQMC_ECUDA;
}

// First-fit allocator over the byte range [0, size) in 256-byte grains.
class RangeAlloc {
public:
    void reset(uint64_t size)
    {
        free_.clear();
        size_ = size;
        used_ = peak_ = 0;
        if (size) free_[0] = size;
    }
    uint64_t alloc(uint64_t bytes)
    {
        bytes = up(bytes ? bytes : 1, kGrain);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const uint64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return off;
        }
        return kNone;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        if (off == kNone) return;
        bytes = up(bytes ? bytes : 1, kGrain);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && off + bytes == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }
    uint64_t size() const { return size_; }

private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t size_ = 0, used_ = 0, peak_ = 0;
};

struct Job {
    uint32_t n = 0, flags = 0;
    int state = DQMC_JOB_QUEUED;
    std::vector<uint8_t> on, dc;   // host copies until uploaded
    uint64_t t_submit = 0, t_done = 0, count = 0;
    uint64_t keep_off = kNone, keep_bytes = 0;   // bitmap slot (+ count word for large jobs)
};

uint64_t tt_bytes(uint32_t n) { return ((1ull << n) + 7) / 8; }

}  // namespace
}  // namespace dqmc

using namespace dqmc;

struct dqmc_server;

namespace dqmc {
namespace {

// One launch unit: a large job, or a batch of small jobs.  Everything the
// launch needs is moved in here while the server lock is held; the launch
// itself (host copies into pinned memory, CUDA calls) runs without the lock.
struct Group {
    dqmc_server *srv = nullptr;
    std::vector<uint64_t> jobs;                // ids (batch: by n, largest first)
    std::vector<uint32_t> ns;
    std::vector<std::vector<uint8_t>> on, dc;  // the jobs' truth tables
    std::vector<uint64_t> keep;                // bitmap slots (device arena offsets)
    uint64_t tmp_off = kNone, tmp_bytes = 0;   // device: tables, truth tables, state
    uint64_t pin_off = kNone, pin_bytes = 0;   // pinned: staging and counts out
    uint64_t counts_pin = 0;                   // offset of the counts in the pinned block
    int stream = -1;                           // large-job stream, -1 for the batch stream
    bool batch = false;
    // batch block layout (same offsets in the device and the pinned block)
    uint64_t fn_at = 0, tt_at = 0, dc_at = 0, bm_at = 0, cnt_at = 0;
    std::vector<uint64_t> tt_pos, dc_pos;
};

void CUDART_CB on_done(void *arg);

}  // namespace
}  // namespace dqmc

struct dqmc_server {
    int dev = 0, mode = DQMC_SERVER_CONCURRENT;
    uint8_t *d_base = nullptr;
    uint8_t *h_base = nullptr;
    RangeAlloc dalloc, halloc;
    std::vector<cudaStream_t> streams;
    std::vector<char> stream_busy;
    cudaStream_t batch_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<uint64_t, Job> jobs;
    std::deque<uint64_t> queue;
    uint64_t next_id = 0;
    bool stop = false, dirty = false;
    int running_groups = 0;
    uint64_t running_jobs = 0;
    int sticky = DQMC_OK;
    std::thread sched;
    uint64_t st_submitted = 0, st_done = 0, st_batches = 0, st_batched_jobs = 0, st_peak_running = 0;

    void run();
    std::vector<Group *> admit();
    Group *prepare_single(uint64_t id, int si);
    Group *prepare_batch(const std::vector<uint64_t> &arrived);
    void exec(Group *g);
    void fail(Group *g, cudaError_t e);
    void finish(Group *g);
};

namespace dqmc {
namespace {

void CUDART_CB on_done(void *arg)
{
    Group *g = static_cast<Group *>(arg);
    g->srv->finish(g);
}

// Device bytes of a job's kept part (bitmap slot, then an 8-byte count for a
// job that runs alone) and of its temporary part (truth tables, workspace).
uint64_t keep_bytes_of(uint32_t n) { return up(bitmap_alloc_bytes((int)n), kGrain) + kGrain; }
uint64_t tmp_bytes_of(uint32_t n, bool dc)
{
    const uint64_t tt = up(tt_bytes(n), kGrain);
    return tt * (dc ? 2 : 1) + (n > (uint32_t)kSmallMaxN ? workspace_layout((int)n).total : 0);
}

}  // namespace
}  // namespace dqmc

void dqmc_server::finish(Group *g)
{
    std::lock_guard<std::mutex> lk(mu);
    const uint64_t t = now_ns();
    const uint64_t *counts = reinterpret_cast<const uint64_t *>(h_base + g->pin_off + g->counts_pin);
    for (size_t i = 0; i < g->jobs.size(); ++i) {
        Job &j = jobs[g->jobs[i]];
        j.count = counts[i];
        j.state = DQMC_JOB_DONE;
        j.t_done = t;
        if (j.flags & DQMC_JOB_DISCARD_BITMAP) {
            dalloc.release(j.keep_off, j.keep_bytes);
            j.keep_off = kNone;
        }
    }
    dalloc.release(g->tmp_off, g->tmp_bytes);
    halloc.release(g->pin_off, g->pin_bytes);
    if (g->stream >= 0) stream_busy[g->stream] = 0;
    --running_groups;
    running_jobs -= g->jobs.size();
    st_done += g->jobs.size();
    dirty = true;
    delete g;
    cv.notify_all();
}

// Reserve device and pinned memory for a job on its own stream; nullptr if
// it does not fit now.  Called with the lock held.
Group *dqmc_server::prepare_single(uint64_t id, int si)
{
    Job &j = jobs[id];
    const bool has_dc = !j.dc.empty();
    const uint64_t tta = up(tt_bytes(j.n), kGrain);
    const uint64_t keep_bytes = keep_bytes_of(j.n), tmp = tmp_bytes_of(j.n, has_dc);
    const uint64_t pin_bytes = tta * (has_dc ? 2 : 1) + kGrain;
    const uint64_t keep = dalloc.alloc(keep_bytes);
    const uint64_t tmp_off = keep == kNone ? kNone : dalloc.alloc(tmp);
    const uint64_t pin_off = tmp_off == kNone ? kNone : halloc.alloc(pin_bytes);
    if (pin_off == kNone) {
        dalloc.release(tmp_off, tmp);
        dalloc.release(keep, keep_bytes);
        return nullptr;
    }
    Group *g = new Group();
    g->srv = this;
    g->jobs.push_back(id);
    g->ns.push_back(j.n);
    g->on.push_back(std::move(j.on));
    g->dc.push_back(std::move(j.dc));
    g->keep.push_back(keep);
    g->tmp_off = tmp_off;
    g->tmp_bytes = tmp;
    g->pin_off = pin_off;
    g->pin_bytes = pin_bytes;
    g->counts_pin = tta * (has_dc ? 2 : 1);
    g->stream = si;
    j.keep_off = keep;
    j.keep_bytes = keep_bytes;
    j.state = DQMC_JOB_RUNNING;
    if (si >= 0) stream_busy[si] = 1;
    ++running_groups;
    running_jobs += 1;
    st_peak_running = std::max<uint64_t>(st_peak_running, running_jobs);
    return g;
}

// Reserve memory for small jobs waiting together; nullptr if they do not fit
// now.  Called with the lock held.
Group *dqmc_server::prepare_batch(const std::vector<uint64_t> &arrived)
{
    const uint32_t k = (uint32_t)arrived.size();
    std::vector<uint64_t> ids(arrived);   // grouped by n, largest first
    std::stable_sort(ids.begin(), ids.end(), [&](uint64_t a, uint64_t b) { return jobs[a].n > jobs[b].n; });
    Group *g = new Group();
    g->srv = this;
    g->batch = true;
    g->fn_at = 0;
    g->tt_at = up(4ull * k, 16);
    g->dc_at = g->tt_at + 8ull * k;
    g->bm_at = g->dc_at + 8ull * k;
    g->cnt_at = g->bm_at + 8ull * k;
    uint64_t at = up(g->cnt_at + 8ull * k, kGrain);
    g->tt_pos.resize(k);
    g->dc_pos.assign(k, kNone);
    for (uint32_t i = 0; i < k; ++i) {
        const Job &j = jobs[ids[i]];
        g->tt_pos[i] = at;
        at += up(tt_bytes(j.n), 16);
        if (!j.dc.empty()) {
            g->dc_pos[i] = at;
            at += up(tt_bytes(j.n), 16);
        }
    }
    const uint64_t block = up(at, kGrain);
    // bitmap slots first (they outlive the batch), then the block
    std::vector<uint64_t> keep(k, kNone);
    bool ok = true;
    for (uint32_t i = 0; i < k && ok; ++i) {
        keep[i] = dalloc.alloc(keep_bytes_of(jobs[ids[i]].n));
        ok = keep[i] != kNone;
    }
    const uint64_t tmp = ok ? dalloc.alloc(block) : kNone;
    const uint64_t pin = tmp != kNone ? halloc.alloc(block) : kNone;
    if (pin == kNone) {
        dalloc.release(tmp, block);
        for (uint32_t i = 0; i < k; ++i) dalloc.release(keep[i], keep_bytes_of(jobs[ids[i]].n));
        delete g;
        return nullptr;
    }
    g->tmp_off = tmp;
    g->tmp_bytes = block;
    g->pin_off = pin;
    g->pin_bytes = block;
    g->counts_pin = g->cnt_at;
    g->jobs = ids;
    g->keep = keep;
    for (uint32_t i = 0; i < k; ++i) {
        Job &j = jobs[ids[i]];
        g->ns.push_back(j.n);
        g->on.push_back(std::move(j.on));
        g->dc.push_back(std::move(j.dc));
        j.keep_off = keep[i];
        j.keep_bytes = keep_bytes_of(j.n);
        j.state = DQMC_JOB_RUNNING;
    }
    ++running_groups;
    running_jobs += k;
    st_peak_running = std::max<uint64_t>(st_peak_running, running_jobs);
    ++st_batches;
    st_batched_jobs += k;
    return g;
}

// A launch could not be enqueued: its jobs end with the error, and the
// server keeps it (sticky).  Work already enqueued may still use the
// group's memory, so that memory stays reserved.
void dqmc_server::fail(Group *g, cudaError_t e)
{
    std::lock_guard<std::mutex> lk(mu);
    sticky = map_err(e);
    for (uint64_t id : g->jobs) {
        jobs[id].state = DQMC_JOB_DONE;
        jobs[id].t_done = now_ns();
    }
    --running_groups;
    running_jobs -= g->jobs.size();
    dirty = true;
    delete g;
    cv.notify_all();
}

// Enqueue a prepared group (no lock held): truth tables into pinned memory,
// one H2D copy, the sweep, counts out, then a host callback that completes
// the jobs.  The callback is the last use of g here.
void dqmc_server::exec(Group *g)
{
    uint8_t *hp = h_base + g->pin_off;
    uint8_t *dp = d_base + g->tmp_off;
    cudaStream_t s = g->stream >= 0 ? streams[g->stream] : batch_stream;
    cudaError_t e = cudaSuccess;
    if (!g->batch) {
        const uint32_t n = g->ns[0];
        const bool has_dc = !g->dc[0].empty();
        const uint64_t tt = tt_bytes(n), tta = up(tt, kGrain);
        memcpy(hp, g->on[0].data(), tt);
        if (has_dc) memcpy(hp + tta, g->dc[0].data(), tt);
        uint8_t *d_bitmap = d_base + g->keep[0];
        unsigned long long *d_count =
            reinterpret_cast<unsigned long long *>(d_bitmap + up(bitmap_alloc_bytes((int)n), kGrain));
        uint8_t *d_work = dp + tta * (has_dc ? 2 : 1);
        e = cudaMemcpyAsync(dp, hp, tta * (has_dc ? 2 : 1), cudaMemcpyHostToDevice, s);
        const Plan p = make_plan((int)n);
        if (e == cudaSuccess) {
            if (p.sps.empty()) {
                e = launch_sweep(p, dp, has_dc ? dp + tta : nullptr, nullptr, reinterpret_cast<uint32_t *>(d_bitmap),
                                 d_count, s);
            } else {
                const Workspace w = workspace_layout((int)n);
                e = launch_super(p, dp, has_dc ? dp + tta : nullptr, d_work + w.state_off,
                                 reinterpret_cast<uint32_t *>(d_bitmap), d_count, nullptr, 0, d_work + w.ctrl_off, s,
                                 0, plan_passes(p));
            }
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hp + g->counts_pin, d_count, 8, cudaMemcpyDeviceToHost, s);
    } else {
        const uint32_t k = (uint32_t)g->jobs.size();
        uint32_t *fn = reinterpret_cast<uint32_t *>(hp + g->fn_at);
        uint64_t *tto = reinterpret_cast<uint64_t *>(hp + g->tt_at);
        uint64_t *dco = reinterpret_cast<uint64_t *>(hp + g->dc_at);
        uint64_t *bmo = reinterpret_cast<uint64_t *>(hp + g->bm_at);
        memset(hp + g->cnt_at, 0, 8ull * k);
        for (uint32_t i = 0; i < k; ++i) {
            fn[i] = i;
            tto[i] = g->tmp_off + g->tt_pos[i];   // offsets from the device arena base
            dco[i] = g->dc_pos[i] == kNone ? kNone : g->tmp_off + g->dc_pos[i];
            bmo[i] = g->keep[i];
            memcpy(hp + g->tt_pos[i], g->on[i].data(), tt_bytes(g->ns[i]));
            if (g->dc_pos[i] != kNone) memcpy(hp + g->dc_pos[i], g->dc[i].data(), tt_bytes(g->ns[i]));
        }
        e = cudaMemcpyAsync(dp, hp, g->tmp_bytes, cudaMemcpyHostToDevice, s);
        for (uint32_t i = 0; i < k && e == cudaSuccess;) {
            const uint32_t n = g->ns[i];
            uint32_t m = i;
            while (m < k && g->ns[m] == n) ++m;
            BatchArgs b;
            b.fn = reinterpret_cast<const uint32_t *>(dp + g->fn_at) + i;
            b.nfun = m - i;
            b.tt_off = reinterpret_cast<const uint64_t *>(dp + g->tt_at);
            b.dc_off = reinterpret_cast<const uint64_t *>(dp + g->dc_at);
            b.bm_off = reinterpret_cast<const uint64_t *>(dp + g->bm_at);
            b.arena = d_base;
            b.bitmaps = d_base;
            b.count = reinterpret_cast<unsigned long long *>(dp + g->cnt_at);
            e = launch_batch_in_smem((int)n, b, s);
            i = m;
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hp + g->cnt_at, dp + g->cnt_at, 8ull * k, cudaMemcpyDeviceToHost, s);
    }
    g->on.clear();
    g->dc.clear();
    if (e == cudaSuccess) e = cudaLaunchHostFunc(s, on_done, g);
    if (e != cudaSuccess) fail(g, e);
}

// Choose what to start now, in arrival order, and reserve its memory (lock
// held, host work only).  Small jobs go into one batch; a large job that does
// not fit (or finds no free stream) stops later large jobs from passing it,
// so large jobs keep their order.
std::vector<Group *> dqmc_server::admit()
{
    std::vector<Group *> out;
    if (sticky) return out;
    if (mode == DQMC_SERVER_SERIAL) {
        // one job at a time, on the same kernels as the concurrent mode: a
        // small job is a batch of one (its footprint has no workspace)
        if (running_groups || queue.empty()) return out;
        const uint64_t id = queue.front();
        Group *g = (int)jobs[id].n <= kSmallMaxN ? prepare_batch(std::vector<uint64_t>{id}) : prepare_single(id, 0);
        if (g) {
            queue.pop_front();
            out.push_back(g);
        }
        return out;
    }
    std::vector<uint64_t> small;
    bool large_blocked = false;
    for (auto it = queue.begin(); it != queue.end();) {
        Job &j = jobs[*it];
        if ((int)j.n <= kSmallMaxN) {
            if (small.size() < kMaxBatch) {
                small.push_back(*it);
                it = queue.erase(it);
            } else {
                ++it;
            }
            continue;
        }
        if (large_blocked) {
            ++it;
            continue;
        }
        int si = -1;
        for (size_t q = 0; q < streams.size(); ++q)
            if (!stream_busy[q]) {
                si = (int)q;
                break;
            }
        Group *g = si < 0 ? nullptr : prepare_single(*it, si);
        if (!g) {
            large_blocked = true;
            ++it;
            continue;
        }
        out.push_back(g);
        it = queue.erase(it);
    }
    while (!small.empty()) {
        if (Group *g = prepare_batch(small)) {
            out.push_back(g);
            break;
        }
        // did not fit: put the newer half back at the front, try the older half
        const size_t keep = small.size() / 2;
        for (size_t i = small.size(); i > keep; --i) queue.push_front(small[i - 1]);
        small.resize(keep);
    }
    return out;
}

// The scheduler thread: under the lock it only decides and reserves; the
// CUDA calls happen after the lock is released, so a completion callback
// (which takes the lock) never waits on a thread that waits on the driver.
void dqmc_server::run()
{
    cudaSetDevice(dev);
    for (;;) {
        std::vector<Group *> todo;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return dirty || stop; });
            dirty = false;
            if (sticky && !queue.empty()) {
                // a launch failed: nothing more is started, the queued jobs
                // end with the error (their waiters see it)
                const uint64_t t = now_ns();
                for (uint64_t id : queue) {
                    jobs[id].state = DQMC_JOB_DONE;
                    jobs[id].t_done = t;
                }
                queue.clear();
                cv.notify_all();
            }
            if (stop && queue.empty() && running_groups == 0) break;
            todo = admit();
        }
        for (Group *g : todo) exec(g);
    }
}

// ----------------------------------------------------------------- C ABI

extern "C" uint64_t dqmc_server_job_bytes(uint32_t n, int with_dc)
{
    if (n > DQMC_MAX_N) return 0;
    return keep_bytes_of(n) + tmp_bytes_of(n, with_dc != 0);
}

extern "C" int dqmc_server_create(uint64_t hbm_bytes, uint32_t streams, int mode, dqmc_server **out)
{
    if (!out || hbm_bytes < (1u << 20) || streams == 0 || streams > 32) return DQMC_EINVAL;
    if (mode != DQMC_SERVER_CONCURRENT && mode != DQMC_SERVER_SERIAL) return DQMC_EINVAL;
    *out = nullptr;
    dqmc_server *s = new dqmc_server();
    s->mode = mode;
    cudaError_t e = cudaGetDevice(&s->dev);
    // pinned staging: the truth tables of the jobs being uploaded, tables, counts
    const uint64_t pinned = std::min<uint64_t>(hbm_bytes / 8, 1ull << 30);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_base, hbm_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_base, pinned);
    for (uint32_t i = 0; e == cudaSuccess && i < (mode == DQMC_SERVER_SERIAL ? 1u : streams); ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->batch_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        const int st = map_err(e);
        for (cudaStream_t q : s->streams) cudaStreamDestroy(q);
        if (s->batch_stream) cudaStreamDestroy(s->batch_stream);
        if (s->d_base) cudaFree(s->d_base);
        if (s->h_base) cudaFreeHost(s->h_base);
        delete s;
        return st;
    }
    s->stream_busy.assign(s->streams.size(), 0);
    s->dalloc.reset(hbm_bytes);
    s->halloc.reset(pinned);
    s->sched = std::thread([s] { s->run(); });
    *out = s;
    return DQMC_OK;
}

extern "C" int dqmc_server_destroy(dqmc_server *s)
{
    if (!s) return DQMC_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    s->sched.join();
    cudaError_t e = cudaSuccess;
    for (cudaStream_t q : s->streams) {
        cudaError_t e2 = cudaStreamSynchronize(q);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(q);
    }
    cudaError_t e2 = cudaStreamSynchronize(s->batch_stream);
    if (e == cudaSuccess) e = e2;
    cudaStreamDestroy(s->batch_stream);
    cudaFree(s->d_base);
    cudaFreeHost(s->h_base);
    const int st = s->sticky;
    delete s;
    return e != cudaSuccess ? map_err(e) : st;
}

extern "C" int dqmc_server_submit(dqmc_server *s, uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
                                  uint32_t flags, uint64_t *job)
{
    if (!s || !on_bits || !job || n > DQMC_MAX_N || (flags & ~DQMC_JOB_DISCARD_BITMAP)) return DQMC_EINVAL;
    const uint64_t tt = tt_bytes(n);
    if (dqmc_server_job_bytes(n, dc_bits != nullptr) > s->dalloc.size()) return DQMC_EINVAL;
    Job j;
    j.n = n;
    j.flags = flags;
    j.on.assign(on_bits, on_bits + tt);
    if (dc_bits) j.dc.assign(dc_bits, dc_bits + tt);
    j.t_submit = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->sticky) return s->sticky;
    const uint64_t id = s->next_id++;
    s->jobs.emplace(id, std::move(j));
    s->queue.push_back(id);
    ++s->st_submitted;
    s->dirty = true;
    s->cv.notify_all();
    *job = id;
    return DQMC_OK;
}

extern "C" int dqmc_server_query(dqmc_server *s, uint64_t job, int *state, uint64_t *count, const void **d_bitmap,
                                 uint64_t *t_submit_ns, uint64_t *t_done_ns)
{
    if (!s) return DQMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return DQMC_EINVAL;
    const Job &j = it->second;
    if (state) *state = j.state;
    if (count) *count = j.state == DQMC_JOB_DONE ? j.count : 0;
    if (d_bitmap)
        *d_bitmap = (j.state == DQMC_JOB_DONE && j.keep_off != kNone) ? s->d_base + j.keep_off : nullptr;
    if (t_submit_ns) *t_submit_ns = j.t_submit;
    if (t_done_ns) *t_done_ns = j.t_done;
    return s->sticky;
}

extern "C" int dqmc_server_copy_bitmap(dqmc_server *s, uint64_t job, uint8_t *out, uint64_t cap)
{
    if (!s || !out) return DQMC_EINVAL;
    const uint8_t *src = nullptr;
    uint64_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job);
        if (it == s->jobs.end() || it->second.state != DQMC_JOB_DONE || it->second.keep_off == kNone)
            return DQMC_EINVAL;
        bytes = (pow3((int)it->second.n) + 7) / 8;
        src = s->d_base + it->second.keep_off;
    }
    if (cap < bytes) return DQMC_EINVAL;
    return map_err(cudaMemcpy(out, src, bytes, cudaMemcpyDeviceToHost));
}

extern "C" int dqmc_server_wait(dqmc_server *s, uint64_t job, uint32_t timeout_ms)
{
    if (!s) return DQMC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return DQMC_EINVAL;
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto jt = s->jobs.find(job);
        return jt == s->jobs.end() || jt->second.state == DQMC_JOB_DONE || s->sticky != DQMC_OK;
    });
    if (s->sticky) return s->sticky;
    return ok ? DQMC_OK : DQMC_ETIMEOUT;
}

extern "C" int dqmc_server_free_job(dqmc_server *s, uint64_t job)
{
    if (!s) return DQMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end() || it->second.state != DQMC_JOB_DONE) return DQMC_EINVAL;
    s->dalloc.release(it->second.keep_off, it->second.keep_bytes);
    s->jobs.erase(it);
    s->dirty = true;
    s->cv.notify_all();
    return DQMC_OK;
}

extern "C" int dqmc_server_stats(dqmc_server *s, uint64_t out[8])
{
    if (!s || !out) return DQMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = s->st_submitted;
    out[1] = s->st_done;
    out[2] = s->st_batches;
    out[3] = s->st_batched_jobs;
    out[4] = s->dalloc.used();
    out[5] = s->dalloc.peak();
    out[6] = s->st_peak_running;
    out[7] = s->dalloc.size();
    return DQMC_OK;
}

extern "C" int dqmc_server_replay(dqmc_server *s, uint32_t njobs, const double *t_arrive_s, const uint32_t *n,
                                  const uint8_t *const *on_bits, const uint8_t *const *dc_bits, uint64_t *count_out,
                                  double *latency_s_out, double *span_s)
{
    if (!s || (njobs && (!t_arrive_s || !n || !on_bits))) return DQMC_EINVAL;
    std::vector<uint64_t> ids(njobs), due(njobs);
    const uint64_t t0 = now_ns();
    int st = DQMC_OK;
    for (uint32_t j = 0; j < njobs && st == DQMC_OK; ++j) {
        due[j] = t0 + (uint64_t)(t_arrive_s[j] * 1e9);
        for (;;) {
            const uint64_t t = now_ns();
            if (t >= due[j]) break;
            if (due[j] - t > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(due[j] - t - 100000));
        }
        st = dqmc_server_submit(s, n[j], on_bits[j], dc_bits ? dc_bits[j] : nullptr, DQMC_JOB_DISCARD_BITMAP,
                                &ids[j]);
    }
    if (st != DQMC_OK) return st;
    uint64_t last = 0;
    for (uint32_t j = 0; j < njobs; ++j) {
        while ((st = dqmc_server_wait(s, ids[j], 60000)) == DQMC_ETIMEOUT) {
        }
        if (st != DQMC_OK) return st;
        uint64_t cnt = 0, td = 0;
        int state = 0;
        dqmc_server_query(s, ids[j], &state, &cnt, nullptr, nullptr, &td);
        if (count_out) count_out[j] = cnt;
        if (latency_s_out) latency_s_out[j] = (double)(td - std::min(td, due[j])) * 1e-9;
        last = std::max(last, td);
        dqmc_server_free_job(s, ids[j]);
    }
    if (span_s) *span_s = njobs ? (double)(last - due[0]) * 1e-9 : 0.0;
    return DQMC_OK;
}
