// dqmc_list.cu -- stream compaction of the prime bitmap into (mask, value)
// pairs in ascending rho (the output extraction step of Algorithm 4,
// arXiv 2302.10083 Section 4.2: every set bit of the final state is a prime).
//
// Three launches: per-block popcounts of the dense bitmap, one exclusive scan
// of the block counts (which also yields the total), then each block scans its
// words again and writes the pairs of its set bits at its global offset.  The
// base-3 digits of rho are decoded five at a time through a 243-entry table.
#include "dqmc_internal.h"

namespace dqmc {

constexpr int kListThreads = 256;
constexpr int kWordsPerThread = kListWordsPerBlock / kListThreads;  // 16

__global__ void __launch_bounds__(kListThreads)
list_count_kernel(const uint32_t *__restrict__ bm, uint64_t n_words, uint32_t *__restrict__ blk_counts)
{
    const uint64_t w0 = (uint64_t)blockIdx.x * kListWordsPerBlock;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < kWordsPerThread; ++j) {
        const uint64_t w = w0 + (uint64_t)j * kListThreads + threadIdx.x;
        if (w < n_words) c += __popc(__ldg(bm + w));
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __shared__ uint32_t red[kListThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kListThreads / 32; ++i) t += red[i];
        blk_counts[blockIdx.x] = t;
    }
}

// Single-CTA exclusive scan of the block counts; writes the total to *total.
__global__ void __launch_bounds__(1024)
list_scan_kernel(const uint32_t *__restrict__ blk_counts, uint64_t n_blocks,
                 unsigned long long *__restrict__ blk_offs, unsigned long long *__restrict__ total)
{
    const int T = blockDim.x;
    const uint64_t per = (n_blocks + T - 1) / T;
    const uint64_t b0 = per * threadIdx.x;
    const uint64_t b1 = (b0 + per < n_blocks) ? b0 + per : n_blocks;
    unsigned long long s = 0;
    for (uint64_t b = b0; b < b1; ++b) s += blk_counts[b];
    // block-wide exclusive scan of s
    __shared__ unsigned long long warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long t = (lane < (T >> 5)) ? warp_tot[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long run = (x - s) + (wid > 0 ? warp_tot[wid - 1] : 0ull);
    for (uint64_t b = b0; b < b1; ++b) {
        blk_offs[b] = run;
        run += blk_counts[b];
    }
    if (threadIdx.x == T - 1) *total = run;
}

__global__ void __launch_bounds__(kListThreads)
list_emit_kernel(const uint32_t *__restrict__ bm, uint64_t n_words, int n,
                 const unsigned long long *__restrict__ blk_offs,
                 uint32_t *__restrict__ pairs, uint64_t cap)
{
    // t5m[r] / t5v[r]: mask and value bits of the five base-3 digits of r < 243.
    __shared__ uint8_t t5m[243], t5v[243];
    __shared__ unsigned long long warp_tot[kListThreads / 32];
    for (int r = threadIdx.x; r < 243; r += blockDim.x) {
        int q = r, m = 0, v = 0;
        for (int i = 0; i < 5; ++i) {
            const int d = q % 3;
            q /= 3;
            if (d != 2) m |= 1 << i;
            if (d == 1) v |= 1 << i;
        }
        t5m[r] = (uint8_t)m;
        t5v[r] = (uint8_t)v;
    }
    // thread t owns words [w0 + 16t, w0 + 16t + 16): contiguous, so a
    // block-wide exclusive scan of the per-thread counts gives ascending order.
    const uint64_t wbase = (uint64_t)blockIdx.x * kListWordsPerBlock + (uint64_t)threadIdx.x * kWordsPerThread;
    uint32_t wv[kWordsPerThread];
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < kWordsPerThread; ++j) {
        const uint64_t w = wbase + j;
        wv[j] = (w < n_words) ? __ldg(bm + w) : 0u;
        c += __popc(wv[j]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = c;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    unsigned long long before = 0;
    for (int i = 0; i < wid; ++i) before += warp_tot[i];
    unsigned long long k = blk_offs[blockIdx.x] + before + (x - c);
    const uint32_t nmask = (n >= 32) ? 0xffffffffu : ((1u << n) - 1u);
#pragma unroll
    for (int j = 0; j < kWordsPerThread; ++j) {
        uint32_t bits = wv[j];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            if (k < cap) {
                const uint64_t rho = (wbase + j) * 32u + (uint64_t)b;
                const uint64_t q0 = rho / 243u;
                uint32_t r = (uint32_t)(rho - q0 * 243u);
                uint32_t q = (uint32_t)q0;  // < 3^20 for n <= 25
                uint32_t m = t5m[r], v = t5v[r];
#pragma unroll
                for (int g = 1; g < 5; ++g) {
                    const uint32_t qq = q / 243u;
                    r = q - qq * 243u;
                    q = qq;
                    m |= (uint32_t)t5m[r] << (5 * g);
                    v |= (uint32_t)t5v[r] << (5 * g);
                }
                pairs[2 * k] = m & nmask;
                pairs[2 * k + 1] = v & nmask;
            }
            ++k;
        }
    }
}

cudaError_t launch_compact(int n, const uint32_t *d_bitmap, uint32_t *d_pairs, uint64_t cap,
                           unsigned long long *d_count, uint32_t *d_blk_counts,
                           unsigned long long *d_blk_offs, cudaStream_t stream)
{
    const uint64_t n_words = bitmap_words(n);
    const uint64_t n_blocks = (n_words + kListWordsPerBlock - 1) / kListWordsPerBlock;
    if (n_blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    list_count_kernel<<<(unsigned)n_blocks, kListThreads, 0, stream>>>(d_bitmap, n_words, d_blk_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    list_scan_kernel<<<1, 1024, 0, stream>>>(d_blk_counts, n_blocks, d_blk_offs, d_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cap == 0 || d_pairs == nullptr) return cudaSuccess;
    list_emit_kernel<<<(unsigned)n_blocks, kListThreads, 0, stream>>>(d_bitmap, n_words, n, d_blk_offs,
                                                                      d_pairs, cap);
    return cudaGetLastError();
}

}  // namespace dqmc
