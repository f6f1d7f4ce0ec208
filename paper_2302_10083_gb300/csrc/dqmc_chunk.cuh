// dqmc_chunk.cuh -- the 256-bit chunk: five ternary digits held in eight
// 32-bit registers, and the Merge / Reduce steps of those digits done with
// funnel shifts and masks.
//
// Layout of the device state (DenseQMC, arXiv 2302.10083, Section 4.2 gives the
// two-layer idea; this is a GB300 variant of it): cube rho = r * 3^C + q with
// q < 3^C the index of the C = min(n, 5) lowest digits and r the index of the
// n - C high digits.  Row r is one 32-byte chunk (a DRAM sector), bit q of the
// chunk is cube (r, q); bits 3^C..255 are always zero.  243 of 256 bits are
// used at C = 5 (5% padding).
#pragma once

#include <cstdint>
#include <type_traits>

namespace dqmc {

constexpr int kChunkDigits = 5;
constexpr int kChunkWords = 8;
constexpr int kChunkBytes = 32;

__host__ __device__ constexpr uint64_t pow3(int k)
{
    uint64_t p = 1;
    for (int i = 0; i < k; ++i) p *= 3u;
    return p;
}

__host__ __device__ constexpr int digit_of(int q, int i)
{
    for (int j = 0; j < i; ++j) q /= 3;
    return q % 3;
}

// m[C][i][v][w]: bit b of word w is set iff q = 32w + b < 3^C and digit i of q
// equals v.  Digit value 2 is the wildcard '*'.
struct MaskTable {
    uint32_t m[kChunkDigits + 1][kChunkDigits][3][kChunkWords];
};

__host__ __device__ constexpr MaskTable make_mask_table()
{
    MaskTable t{};
    for (int C = 0; C <= kChunkDigits; ++C)
        for (int i = 0; i < kChunkDigits; ++i)
            for (int v = 0; v < 3; ++v)
                for (int w = 0; w < kChunkWords; ++w) {
                    uint32_t x = 0;
                    if (i < C)
                        for (int b = 0; b < 32; ++b) {
                            const int q = 32 * w + b;
                            if (q < (int)pow3(C) && digit_of(q, i) == v) x |= 1u << b;
                        }
                    t.m[C][i][v][w] = x;
                }
    return t;
}

// Position of minterm t (its C low bits) inside the chunk: sum bit_i(t) 3^i.
__host__ __device__ constexpr int spread_pos(int t)
{
    int q = 0, w = 1;
    for (int i = 0; i < kChunkDigits; ++i) {
        if ((t >> i) & 1) q += w;
        w *= 3;
    }
    return q;
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// Word w of (v << S) as a 256-bit value.
template <int S>
__device__ __forceinline__ uint32_t shl_word(const uint32_t (&v)[kChunkWords], int w)
{
    constexpr int ws = S >> 5, bs = S & 31;
    const int src = w - ws;
    const uint32_t hi = (src >= 0) ? v[src] : 0u;
    if constexpr (bs == 0) return hi;
    const uint32_t lo = (src - 1 >= 0) ? v[src - 1] : 0u;
    return __funnelshift_l(lo, hi, bs);
}

// Word w of (v >> S) as a 256-bit value.
template <int S>
__device__ __forceinline__ uint32_t shr_word(const uint32_t (&v)[kChunkWords], int w)
{
    constexpr int ws = S >> 5, bs = S & 31;
    const int src = w + ws;
    const uint32_t lo = (src < kChunkWords) ? v[src] : 0u;
    if constexpr (bs == 0) return lo;
    const uint32_t hi = (src + 1 < kChunkWords) ? v[src + 1] : 0u;
    return __funnelshift_r(lo, hi, bs);
}

}  // namespace dqmc
