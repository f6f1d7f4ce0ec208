// dqmc_sparse.cu -- SparseQMC on the GPU: the classic level-by-level
// Quine-McCluskey (arXiv 2302.10083, Algorithm 1) with the paper's optimised
// data layout for sparse functions (Section 5, "SparseQMC").
//
// A cube is a 2n-bit code, two bits per variable x_i (bits 2(i-1), 2i-1):
// 00 = '0', 01 = '1', 10 = '*' (Section 5, bit-based representation).  Level
// w is the set L_w of implicants with w wildcards, kept twice: as a list
// (sequential) and as a hash set with linear probing (membership; bit 63 of
// a slot is the control flag "redundant").  Level w from level w - 1:
//   generate  for each s in L_{w-1} and each position i with s_i = '0' and no
//             wildcard before position i, if t = s with t_i = '1' is in
//             L_{w-1}, then s with '*' at i joins L_w.  Every u in L_w is
//             made exactly once this way: from its first wildcard position
//             (the paper's rule against repeated generation);
//   insert    the list of L_w into its hash set;
//   mark      for each u in L_w and each wildcard position j of u, the two
//             cubes u with '0' and with '1' at j are flagged redundant in
//             L_{w-1} (the extra pass the rule makes necessary);
//   collect   the unflagged cubes of L_{w-1} are prime.
// The primes are then sorted by rho (a radix sort) and written as (mask,
// value) pairs in ascending rho, the order of dqmc_list.
#include <cstdio>
#include <cstring>
#include <vector>

#include "dqmc.h"

namespace dqmc {
namespace sparse {

constexpr uint64_t kEmpty = ~0ull;             // an empty hash slot
constexpr uint64_t kRedundant = 1ull << 63;    // control flag of a slot
constexpr int kThreads = 256;

// Fibonacci hashing of a code into a table of 2^lg slots
__device__ __forceinline__ uint64_t slot_of(uint64_t code, int lg)
{
    return (code * 0x9E3779B97F4A7C15ull) >> (64 - lg);
}

__device__ __forceinline__ void ht_insert(uint64_t *tab, int lg, uint64_t code)
{
    const uint64_t mask = (1ull << lg) - 1;
    for (uint64_t s = slot_of(code, lg), probes = 0; probes <= mask; s = (s + 1) & mask, ++probes) {
        const unsigned long long prev =
            atomicCAS(reinterpret_cast<unsigned long long *>(tab + s), (unsigned long long)kEmpty, code);
        if (prev == kEmpty || (prev & ~kRedundant) == code) return;
    }
}

// Slot holding code, or -1
__device__ __forceinline__ int64_t ht_find(const uint64_t *tab, int lg, uint64_t code)
{
    const uint64_t mask = (1ull << lg) - 1;
    for (uint64_t s = slot_of(code, lg), probes = 0; probes <= mask; s = (s + 1) & mask, ++probes) {
        const uint64_t v = __ldcg(reinterpret_cast<const unsigned long long *>(tab + s));
        if (v == kEmpty) return -1;
        if ((v & ~kRedundant) == code) return (int64_t)s;
    }
    return -1;
}

// Append x to a list of capacity cap (warp-aggregated); past cap only counted
__device__ __forceinline__ void list_append(uint64_t *list, unsigned long long *len, uint64_t cap, uint64_t x)
{
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(len, (unsigned long long)__popc(act));
    base = __shfl_sync(act, base, leader);
    const unsigned long long at = base + __popc(act & ((1u << lane) - 1u));
    if (at < cap) list[at] = x;
}

// Spread the n bits of minterm t into a code: bit i of t -> bit 2i
__device__ __forceinline__ uint64_t spread2(uint32_t t)
{
    uint64_t x = t;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

// L_0: the minterms of the support (ON or DC; with inv, (not ON) or DC), one
// thread per truth-table word of 32 minterms (m < 32: one partial word).
__global__ void seed_kernel(const uint32_t *on, const uint32_t *dc, uint32_t inv, uint64_t words, uint32_t m_bits,
                            uint64_t *list, unsigned long long *len, uint64_t cap)
{
    const uint64_t wi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (wi >= words) return;
    uint32_t x = on[wi] ^ inv;
    if (dc) x |= dc[wi];
    if (m_bits < 32) x &= (1u << m_bits) - 1u;
    while (x) {
        const int b = __ffs(x) - 1;
        x &= x - 1;
        list_append(list, len, cap, spread2((uint32_t)(wi * 32 + b)));
    }
}

__global__ void insert_kernel(const uint64_t *list, uint64_t len, uint64_t *tab, int lg)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) ht_insert(tab, lg, list[i]);
}

__global__ void fill_kernel(uint64_t *p, uint64_t len, uint64_t v)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) p[i] = v;
}

// generate: L_w from L_{w-1} (list prev, hash set tab)
__global__ void generate_kernel(const uint64_t *prev, uint64_t len, const uint64_t *tab, int lg, int n,
                                uint64_t *next, unsigned long long *next_len, uint64_t cap)
{
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    const uint64_t s = prev[k];
    for (int i = 0; i < n; ++i) {
        const uint64_t sym = (s >> (2 * i)) & 3u;
        if (sym == 2) break;          // no merge at or after the first wildcard
        if (sym != 0) continue;
        const uint64_t t = s | (1ull << (2 * i));
        if (ht_find(tab, lg, t) >= 0) list_append(next, next_len, cap, s | (2ull << (2 * i)));
    }
}

// mark: every merge pair of every u in L_w is redundant in L_{w-1}
__global__ void mark_kernel(const uint64_t *cur, uint64_t len, uint64_t *tab, int lg, int n)
{
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    const uint64_t u = cur[k];
    for (int j = 0; j < n; ++j) {
        if (((u >> (2 * j)) & 3u) != 2) continue;
        const uint64_t s0 = u & ~(3ull << (2 * j));
        for (int v = 0; v < 2; ++v) {
            const int64_t sl = ht_find(tab, lg, s0 | ((uint64_t)v << (2 * j)));
            if (sl >= 0 && !(tab[sl] & kRedundant))
                atomicOr(reinterpret_cast<unsigned long long *>(tab + sl), (unsigned long long)kRedundant);
        }
    }
}

// rho and the packed (mask, value) of a code
__device__ __forceinline__ void code_rho_pair(uint64_t c, int n, uint64_t &rho, uint64_t &mv)
{
    uint64_t r = 0, w = 1;
    uint32_t m = 0, val = 0;
    for (int i = 0; i < n; ++i) {
        const uint32_t sym = (uint32_t)((c >> (2 * i)) & 3u);
        r += w * sym;   // '0' -> 0, '1' -> 1, '*' -> 2: the symbols' rho values
        w *= 3;
        if (sym != 2) m |= 1u << i;
        if (sym == 1) val |= 1u << i;
    }
    rho = r;
    mv = ((uint64_t)val << 32) | m;
}

// collect: the unflagged cubes of a level's hash set are prime
__global__ void collect_kernel(const uint64_t *tab, uint64_t slots, int n, uint64_t *keys, uint64_t *vals,
                               unsigned long long *len, uint64_t cap)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slots) return;
    const uint64_t v = tab[i];
    if (v == kEmpty || (v & kRedundant)) return;
    uint64_t rho, mv;
    code_rho_pair(v, n, rho, mv);
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(len, (unsigned long long)__popc(act));
    base = __shfl_sync(act, base, leader);
    const unsigned long long at = base + __popc(act & ((1u << lane) - 1u));
    if (at < cap) {
        keys[at] = rho;
        vals[at] = mv;
    }
}

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort of (key, value) pairs by 8-bit digits.  A block owns
// a tile of kSortTile consecutive pairs; its 8 warps own 512 each, taken in
// rounds of 32.  Per digit pass: each block's digit histogram (digit-major,
// block-minor in global memory), one exclusive scan of it, then the scatter:
// a pair's place is its digit's scanned base for the block, plus the counts
// of that digit in the block's earlier warps, earlier rounds of its warp, and
// earlier lanes of its round (__match_any_sync), so equal digits keep their
// order.
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerWarp = 512;
constexpr int kSortTile = kSortWarps * kSortPerWarp;   // 4096

__global__ void hist_kernel(const uint64_t *keys, uint64_t len, int shift, uint32_t *hist, uint32_t nblocks)
{
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        const uint64_t k = t0 + i;
        if (k < len) atomicAdd(&h[(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(uint64_t)d * nblocks + blockIdx.x] = h[d];
}

// exclusive scan of cnt in place, by one block of 1024 threads
__global__ void scan_kernel(uint32_t *cnt, uint64_t n)
{
    __shared__ uint32_t part[1024];
    const uint64_t per = (n + 1023) / 1024;
    const uint64_t b0 = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint64_t i = b0; i < b0 + per && i < n; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t y = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum;
    for (uint64_t i = b0; i < b0 + per && i < n; ++i) {
        const uint32_t c = cnt[i];
        cnt[i] = run;
        run += c;
    }
}

__global__ void scatter_kernel(const uint64_t *keys, const uint64_t *vals, uint64_t len, int shift,
                               const uint32_t *base, uint32_t nblocks, uint64_t *okeys, uint64_t *ovals)
{
    __shared__ uint32_t wcnt[kSortWarps][256];   // per warp: its pairs of each digit, then their offsets
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * kSortTile + (uint64_t)w * kSortPerWarp;
    for (int r = 0; r < kSortPerWarp; r += 32) {
        const uint64_t k = t0 + r + lane;
        const bool in = k < len;
        const uint32_t d = in ? (uint32_t)((keys[k] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (in && lane == __ffs(peers) - 1) wcnt[w][d] += __popc(peers);
    }
    __syncthreads();
    // offsets: the digit's base for this block, then the earlier warps' counts
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        uint32_t run = base[(uint64_t)d * nblocks + blockIdx.x];
        for (int ww = 0; ww < kSortWarps; ++ww) {
            const uint32_t c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < kSortPerWarp; r += 32) {
        const uint64_t k = t0 + r + lane;
        const bool in = k < len;
        const uint64_t key = in ? keys[k] : 0ull;
        const uint32_t d = in ? (uint32_t)((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (in) {
            const uint32_t at = wcnt[w][d] + __popc(peers & ((1u << lane) - 1u));
            okeys[at] = key;
            ovals[at] = vals[k];
        }
        __syncwarp();
        if (in && lane == __ffs(peers) - 1) wcnt[w][d] += __popc(peers);
        __syncwarp();
    }
}

__global__ void pairs_kernel(const uint64_t *vals, uint64_t len, uint2 *out)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = make_uint2((uint32_t)vals[i], (uint32_t)(vals[i] >> 32));
}

// Device buffers of one call, freed together.
struct Bufs {
    std::vector<void *> ptrs;
    cudaError_t alloc(void **p, uint64_t bytes)
    {
        *p = nullptr;
        const cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(void *p)
    {
        for (auto &q : ptrs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
    ~Bufs()
    {
        for (void *q : ptrs)
            if (q) cudaFree(q);
    }
};

static unsigned blocks_for(uint64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

static uint64_t pow3u(uint32_t n)
{
    uint64_t p = 1;
    for (uint32_t i = 0; i < n; ++i) p *= 3u;
    return p;
}

static int lg_slots(uint64_t len)
{
    int lg = 4;
    while ((1ull << lg) < 2 * len) ++lg;   // load factor at most 1/2
    return lg;
}

static int map_err(cudaError_t e)
{
    if (e == cudaSuccess) return DQMC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DQMC_ENOMEM : DQMC_ECUDA;
}

static uint64_t read_counter(unsigned long long *d, cudaStream_t s, cudaError_t &e)
{
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return h;
}

static int run(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint32_t flags, uint32_t *out_pairs,
               uint64_t cap, uint64_t *out_count)
{
    const uint64_t m = 1ull << n;
    const uint64_t words = (m + 31) / 32;
    const uint32_t m_bits = m < 32 ? (uint32_t)m : 32u;
    const uint32_t inv = (flags & DQMC_COMPLEMENT) ? ~0u : 0u;
    // the support's size, for L_0
    std::vector<uint32_t> hon(words, 0u), hdc;
    std::memcpy(hon.data(), on_bits, (m + 7) / 8);
    if (dc_bits) {
        hdc.assign(words, 0u);
        std::memcpy(hdc.data(), dc_bits, (m + 7) / 8);
    }
    uint64_t len = 0;
    for (uint64_t w = 0; w < words; ++w) {
        uint32_t x = hon[w] ^ inv;
        if (dc_bits) x |= hdc[w];
        if (m_bits < 32) x &= (1u << m_bits) - 1u;
        len += (uint64_t)__builtin_popcount(x);
    }
    Bufs B;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return map_err(e);
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    uint32_t *d_on = nullptr, *d_dc = nullptr;
    unsigned long long *d_cnt = nullptr;   // [0] list length, [1] primes
    uint64_t *cur = nullptr;
    if ((e = B.alloc((void **)&d_on, words * 4)) != cudaSuccess) return map_err(e);
    if ((e = cudaMemcpyAsync(d_on, hon.data(), words * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return map_err(e);
    if (dc_bits) {
        if ((e = B.alloc((void **)&d_dc, words * 4)) != cudaSuccess) return map_err(e);
        if ((e = cudaMemcpyAsync(d_dc, hdc.data(), words * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return map_err(e);
    }
    if ((e = B.alloc((void **)&d_cnt, 16)) != cudaSuccess) return map_err(e);
    if ((e = B.alloc((void **)&cur, len * 8)) != cudaSuccess) return map_err(e);
    if ((e = cudaMemsetAsync(d_cnt, 0, 16, s)) != cudaSuccess) return map_err(e);
    if (words) seed_kernel<<<blocks_for(words), kThreads, 0, s>>>(d_on, d_dc, inv, words, m_bits, cur, d_cnt, len);
    // the primes found so far, as (rho, packed mask / value)
    uint64_t pcap = len > 1024 ? len : 1024, np = 0;
    uint64_t *keys = nullptr, *vals = nullptr;
    if ((e = B.alloc((void **)&keys, pcap * 8)) != cudaSuccess) return map_err(e);
    if ((e = B.alloc((void **)&vals, pcap * 8)) != cudaSuccess) return map_err(e);
    for (int w = 1; w <= (int)n + 1 && len > 0; ++w) {
        // the hash set of L_{w-1}
        const int lg = lg_slots(len);
        uint64_t *tab = nullptr;
        if ((e = B.alloc((void **)&tab, (1ull << lg) * 8)) != cudaSuccess) return map_err(e);
        fill_kernel<<<blocks_for(1ull << lg), kThreads, 0, s>>>(tab, 1ull << lg, kEmpty);
        insert_kernel<<<blocks_for(len), kThreads, 0, s>>>(cur, len, tab, lg);
        // L_w (grown and generated again when its first guess is short)
        uint64_t ncap = len, nlen = 0;
        uint64_t *next = nullptr;
        if (w <= (int)n) {
            for (;;) {
                if ((e = B.alloc((void **)&next, ncap * 8)) != cudaSuccess) return map_err(e);
                if ((e = cudaMemsetAsync(d_cnt, 0, 8, s)) != cudaSuccess) return map_err(e);
                generate_kernel<<<blocks_for(len), kThreads, 0, s>>>(cur, len, tab, lg, (int)n, next, d_cnt, ncap);
                nlen = read_counter(d_cnt, s, e);
                if (e != cudaSuccess) return map_err(e);
                if (nlen <= ncap) break;
                B.release(next);
                ncap = nlen;
            }
            if (nlen) mark_kernel<<<blocks_for(nlen), kThreads, 0, s>>>(next, nlen, tab, lg, (int)n);
        }
        // the primes of L_{w-1}
        for (;;) {
            if ((e = cudaMemcpyAsync(d_cnt + 1, &np, 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) return map_err(e);
            collect_kernel<<<blocks_for(1ull << lg), kThreads, 0, s>>>(tab, 1ull << lg, (int)n, keys, vals,
                                                                        d_cnt + 1, pcap);
            const uint64_t got = read_counter(d_cnt + 1, s, e);
            if (e != cudaSuccess) return map_err(e);
            if (got <= pcap) {
                np = got;
                break;
            }
            // grow the prime arrays, keeping the primes of earlier levels
            uint64_t *k2 = nullptr, *v2 = nullptr;
            const uint64_t cap2 = got + got / 2;
            if ((e = B.alloc((void **)&k2, cap2 * 8)) != cudaSuccess) return map_err(e);
            if ((e = B.alloc((void **)&v2, cap2 * 8)) != cudaSuccess) return map_err(e);
            if (np && (e = cudaMemcpyAsync(k2, keys, np * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                return map_err(e);
            if (np && (e = cudaMemcpyAsync(v2, vals, np * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                return map_err(e);
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_err(e);
            B.release(keys);
            B.release(vals);
            keys = k2;
            vals = v2;
            pcap = cap2;
        }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_err(e);
        B.release(tab);
        B.release(cur);
        cur = next;
        len = nlen;
    }
    // ascending rho: LSD radix sort, 8 bits a pass, over the bits rho can have
    if (np > 1) {
        int bits = 1;
        while (bits < 64 && (1ull << bits) < pow3u(n)) ++bits;
        const uint32_t nblocks = (uint32_t)((np + kSortTile - 1) / kSortTile);
        uint64_t *k2 = nullptr, *v2 = nullptr;
        uint32_t *hist = nullptr;
        if ((e = B.alloc((void **)&k2, np * 8)) != cudaSuccess) return map_err(e);
        if ((e = B.alloc((void **)&v2, np * 8)) != cudaSuccess) return map_err(e);
        if ((e = B.alloc((void **)&hist, (uint64_t)nblocks * 256 * 4)) != cudaSuccess) return map_err(e);
        for (int shift = 0; shift < bits; shift += 8) {
            hist_kernel<<<nblocks, kSortThreads, 0, s>>>(keys, np, shift, hist, nblocks);
            scan_kernel<<<1, 1024, 0, s>>>(hist, (uint64_t)nblocks * 256);
            scatter_kernel<<<nblocks, kSortThreads, 0, s>>>(keys, vals, np, shift, hist, nblocks, k2, v2);
            uint64_t *t = keys;
            keys = k2;
            k2 = t;
            t = vals;
            vals = v2;
            v2 = t;
        }
    }
    const uint64_t kout = np < cap ? np : cap;
    if (kout) {
        uint2 *d_pairs = nullptr;
        if ((e = B.alloc((void **)&d_pairs, kout * 8)) != cudaSuccess) return map_err(e);
        pairs_kernel<<<blocks_for(kout), kThreads, 0, s>>>(vals, kout, d_pairs);
        if ((e = cudaMemcpyAsync(out_pairs, d_pairs, kout * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return map_err(e);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return map_err(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_err(e);
    if (out_count) *out_count = np;
    return np > cap ? DQMC_ETRUNC : DQMC_OK;
}

}  // namespace sparse
}  // namespace dqmc

extern "C" int dqmc_sparse_list(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits, uint32_t flags,
                                uint32_t *out_pairs, uint64_t cap, uint64_t *out_count)
{
    if (n > DQMC_SPARSE_MAX_N || !on_bits || (cap && !out_pairs) || (flags & ~(uint32_t)DQMC_COMPLEMENT))
        return DQMC_EINVAL;
    return dqmc::sparse::run(n, on_bits, dc_bits, flags, out_pairs, cap, out_count);
}
