// dqmc_cover.cu -- the second step of the Quine-McCluskey method (arXiv
// 2302.10083, Section 1: choose a subset of the prime implicants that covers
// the function, a SetCover instance, NP-hard, so a heuristic): essential
// primes, then greedy.
//
//   essential  a prime that is the only one covering some ON minterm;
//   greedy     then, while some ON minterm is uncovered, the prime that
//              covers the most uncovered ON minterms (ties: the lowest index
//              in the given list).
// Don't-care minterms need no cover.  The state is one bit per minterm
// ("still to cover"); a prime (mask, value) with w wildcards covers the 2^w
// minterms value | deposit(k, ~mask), k < 2^w, which one warp per prime
// enumerates (lanes split k).  The greedy part runs one level of the maximum
// count per round (level_kernel), which takes exactly the primes the
// one-at-a-time rule takes, in the same order.
#include <cstdint>
#include <cstring>
#include <vector>

#include "dqmc.h"

namespace dqmc {
namespace cover {

constexpr int kThreads = 256;

// k-th minterm of the cube (mask, value): value with the bits of k deposited
// in the free (wildcard) positions, lowest first
__device__ __forceinline__ uint32_t cube_minterm(uint32_t free_bits, uint32_t value, uint32_t k)
{
    uint32_t t = value;
    while (free_bits) {
        const uint32_t low = free_bits & (0u - free_bits);
        if (k & 1u) t |= low;
        k >>= 1;
        free_bits &= free_bits - 1;
    }
    return t;
}

__device__ __forceinline__ bool get_bit(const uint32_t *bits, uint32_t t) { return (bits[t >> 5] >> (t & 31)) & 1u; }

// per ON minterm: how many primes cover it, and the first one counted
__global__ void incidence_kernel(const uint2 *pairs, uint64_t np, uint32_t full, const uint32_t *todo,
                                 uint32_t *cnt, uint32_t *who)
{
    const uint64_t p = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= np) return;
    const uint2 mv = pairs[p];
    const uint32_t free_bits = ~mv.x & full;
    const uint64_t nk = 1ull << __popc(free_bits);
    for (uint64_t k = lane; k < nk; k += 32) {
        const uint32_t t = cube_minterm(free_bits, mv.y, (uint32_t)k);
        if (!get_bit(todo, t)) continue;
        if (atomicAdd(cnt + t, 1u) == 0u) who[t] = (uint32_t)p;
    }
}

__global__ void essential_kernel(const uint32_t *cnt, const uint32_t *who, const uint32_t *todo, uint64_t m,
                                 uint8_t *sel)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m && get_bit(todo, (uint32_t)t) && cnt[t] == 1u) sel[who[t]] = 1;
}

// the minterms of every selected prime are covered
__global__ void cover_kernel(const uint2 *pairs, uint64_t np, uint32_t full, const uint8_t *sel, uint32_t *todo)
{
    const uint64_t p = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= np || !sel[p]) return;
    const uint2 mv = pairs[p];
    const uint32_t free_bits = ~mv.x & full;
    const uint64_t nk = 1ull << __popc(free_bits);
    for (uint64_t k = lane; k < nk; k += 32) {
        const uint32_t t = cube_minterm(free_bits, mv.y, (uint32_t)k);
        atomicAnd(todo + (t >> 5), ~(1u << (t & 31)));
    }
}

// uncovered ON minterms of prime p (all lanes of the warp get the sum)
__device__ __forceinline__ uint32_t warp_count(const uint2 *pairs, uint64_t p, uint32_t full, const uint32_t *todo,
                                               int lane)
{
    const uint2 mv = pairs[p];
    const uint32_t free_bits = ~mv.x & full;
    const uint64_t nk = 1ull << __popc(free_bits);
    uint32_t c = 0;
    for (uint64_t k = lane; k < nk; k += 32) c += get_bit(todo, cube_minterm(free_bits, mv.y, (uint32_t)k));
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    return c;
}

// every unselected prime's count of uncovered ON minterms, and their maximum
__global__ void count_kernel(const uint2 *pairs, uint64_t np, uint32_t full, const uint8_t *sel,
                             const uint32_t *todo, uint32_t *cnt, unsigned int *best)
{
    const uint64_t p = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= np) return;
    const uint32_t c = sel[p] ? 0u : warp_count(pairs, p, full, todo, lane);
    if (lane == 0) {
        cnt[p] = c;
        if (c) atomicMax(best, c);
    }
}

// One greedy level, by one warp, primes in index order: a prime whose count
// was the maximum is taken if it still is (then its minterms are covered).
// Every other prime's count is below the maximum and can only fall, so the
// lowest-index prime still at the maximum is exactly the prime that taking
// one prime at a time (most uncovered minterms, lowest index) would take next.
__global__ void level_kernel(const uint2 *pairs, uint64_t np, uint32_t full, uint8_t *sel, uint32_t *todo,
                             const uint32_t *cnt, uint32_t best)
{
    const int lane = threadIdx.x;
    for (uint64_t p0 = 0; p0 < np; p0 += 32) {
        const uint64_t mine = p0 + lane;
        const bool cand = mine < np && !sel[mine] && cnt[mine] == best;
        uint32_t m = __ballot_sync(0xffffffffu, cand);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const uint64_t p = p0 + l;
            if (warp_count(pairs, p, full, todo, lane) != best) continue;
            if (lane == 0) sel[p] = 1;
            const uint2 mv = pairs[p];
            const uint32_t free_bits = ~mv.x & full;
            const uint64_t nk = 1ull << __popc(free_bits);
            for (uint64_t k = lane; k < nk; k += 32) {
                const uint32_t t = cube_minterm(free_bits, mv.y, (uint32_t)k);
                atomicAnd(todo + (t >> 5), ~(1u << (t & 31)));
            }
            __syncwarp();
        }
    }
}

static int map_err(cudaError_t e)
{
    if (e == cudaSuccess) return DQMC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DQMC_ENOMEM : DQMC_ECUDA;
}

struct Bufs {
    std::vector<void *> ptrs;
    cudaError_t alloc(void **p, uint64_t bytes)
    {
        *p = nullptr;
        const cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Bufs()
    {
        for (void *q : ptrs) cudaFree(q);
    }
};

static int run(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, const uint32_t *pairs, uint64_t np,
               uint32_t *out_sel, uint64_t *out_nsel)
{
    const uint64_t m = 1ull << n, words = (m + 31) / 32;
    const uint32_t full = (uint32_t)(m - 1);   // the n variable bits
    // still to cover: the ON minterms (a minterm in DC too is a don't-care)
    std::vector<uint32_t> todo(words, 0u), dcw;
    std::memcpy(todo.data(), on_bits, (m + 7) / 8);
    if (dc_bits) {
        dcw.assign(words, 0u);
        std::memcpy(dcw.data(), dc_bits, (m + 7) / 8);
        for (uint64_t w = 0; w < words; ++w) todo[w] &= ~dcw[w];
    }
    if (m < 32) todo[0] &= (1u << m) - 1u;
    Bufs B;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return map_err(e);
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    uint32_t *d_todo = nullptr, *d_cnt = nullptr, *d_who = nullptr;
    uint2 *d_pairs = nullptr;
    uint8_t *d_sel = nullptr;
    if ((e = B.alloc((void **)&d_todo, words * 4)) != cudaSuccess) return map_err(e);
    if ((e = B.alloc((void **)&d_cnt, m * 4)) != cudaSuccess) return map_err(e);
    if ((e = B.alloc((void **)&d_who, m * 4)) != cudaSuccess) return map_err(e);
    if ((e = B.alloc((void **)&d_pairs, np * 8)) != cudaSuccess) return map_err(e);
    if ((e = B.alloc((void **)&d_sel, np)) != cudaSuccess) return map_err(e);
    e = cudaMemcpyAsync(d_todo, todo.data(), words * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && np) e = cudaMemcpyAsync(d_pairs, pairs, np * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, m * 4, s);
    if (e == cudaSuccess && np) e = cudaMemsetAsync(d_sel, 0, np, s);
    if (e != cudaSuccess) return map_err(e);
    const unsigned gp = (unsigned)((np * 32 + kThreads - 1) / kThreads);   // a warp per prime
    const unsigned gm = (unsigned)((m + kThreads - 1) / kThreads);
    if (np) {
        incidence_kernel<<<gp, kThreads, 0, s>>>(d_pairs, np, full, d_todo, d_cnt, d_who);
        essential_kernel<<<gm, kThreads, 0, s>>>(d_cnt, d_who, d_todo, m, d_sel);
        cover_kernel<<<gp, kThreads, 0, s>>>(d_pairs, np, full, d_sel, d_todo);
    }
    // greedy, one level of the maximum count per round (rounds <= the largest count)
    uint32_t *d_c = nullptr;
    unsigned int *d_b = nullptr;
    if ((e = B.alloc((void **)&d_c, np * 4)) != cudaSuccess) return map_err(e);
    if ((e = B.alloc((void **)&d_b, 4)) != cudaSuccess) return map_err(e);
    for (uint64_t round = 0; round < np; ++round) {   // each round takes at least one prime
        if ((e = cudaMemsetAsync(d_b, 0, 4, s)) != cudaSuccess) return map_err(e);
        count_kernel<<<gp, kThreads, 0, s>>>(d_pairs, np, full, d_sel, d_todo, d_c, d_b);
        unsigned int best = 0;
        if ((e = cudaMemcpyAsync(&best, d_b, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return map_err(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_err(e);
        if (best == 0) break;   // nothing left to cover
        level_kernel<<<1, 32, 0, s>>>(d_pairs, np, full, d_sel, d_todo, d_c, best);
    }
    std::vector<uint8_t> sel(np);
    if (np && (e = cudaMemcpyAsync(sel.data(), d_sel, np, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return map_err(e);
    if ((e = cudaMemcpyAsync(todo.data(), d_todo, words * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return map_err(e);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess) return map_err(e);
    for (uint64_t w = 0; w < words; ++w)
        if (todo[w]) return DQMC_EINVAL;   // the primes given do not cover the ON-set
    uint64_t k = 0;
    for (uint64_t p = 0; p < np; ++p)
        if (sel[p]) out_sel[k++] = (uint32_t)p;
    *out_nsel = k;
    return DQMC_OK;
}

}  // namespace cover
}  // namespace dqmc

extern "C" int dqmc_cover(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, const uint32_t *pairs,
                          uint64_t count, uint32_t *out_sel, uint64_t *out_nsel)
{
    if (n > DQMC_COVER_MAX_N || !on_bits || !out_nsel || (count && (!pairs || !out_sel)) || count > 0xffffffffull)
        return DQMC_EINVAL;
    return dqmc::cover::run(n, on_bits, dc_bits, pairs, count, out_sel, out_nsel);
}
