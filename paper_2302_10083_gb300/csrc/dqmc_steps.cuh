// dqmc_steps.cuh -- Merge and Reduce of several high digits at once on rows
// held in shared memory (DenseQMC, arXiv 2302.10083, Algorithm 3, Section
// 4.1), shared by the whole-function kernel (dqmc_fn.cu) and the last Merge
// pass of the streaming sweep (dqmc_pass.cu).
//
// Rows are 32 bytes (one chunk of 243 cells, dqmc_chunk.cuh) at byte 32 r of
// the array, no swizzle.  A step takes D digits J .. J+D-1 of the row index
// (weights 3^J ..): a thread loads the 3^D rows of one block (one 8-byte
// slice of each) into registers, does the D digits there and writes the
// block back.  Within a step the blocks are disjoint, so working in place
// reads the state the step started from.  A warp reads 8 rows at an odd
// stride (3^j apart, or consecutive), which spreads them over the four
// 128-byte bank phases (two wavefronts per 256 bytes), and one base address
// plus compile-time offsets reach a block's rows.
#pragma once

#include <cstdint>

#include "dqmc_chunk.cuh"

namespace dqmc {

// sum of 3^i over the set bits i of x (x < 2^K)
template <int K>
__device__ __forceinline__ int spread3k(int x)
{
    int r = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) r += ((x >> i) & 1) * (int)pow3(i);
    return r;
}

// Compile-time digit helpers over block indices t < 3^D.
__host__ __device__ constexpr int twos_of(int t, int D)
{
    int c = 0;
    for (int i = 0; i < D; ++i, t /= 3) c += (t % 3) == 2;
    return c;
}
__host__ __device__ constexpr bool binary_above(int t, int d, int D)
{
    for (int i = 0; i < D; ++i, t /= 3)
        if (i > d && (t % 3) == 2) return false;
    return true;
}

struct SubSync {
    int id, nthreads;
    bool whole;
    __device__ __forceinline__ void operator()() const
    {
        if (whole) __syncthreads();
        else asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
    }
};

// Merge of digits J .. J+DD-1 (of the HL digits a CTA holds): blocks of
// 3^DD rows whose lower digits take any value and whose higher digits are 0/1.
template <int HL, int J, int DD>
__device__ __forceinline__ void merge_step(uint4 *S, int lt, int tg)
{
    constexpr int P = (int)pow3(J);
    constexpr int T = (int)pow3(DD);
    constexpr int items = P * (1 << (HL - J - DD)) * 4;
    for (int it = lt; it < items; it += tg) {
        const int q = it & 3, r = it >> 2;
        const int lo = r % P, hb = r / P;
        const int base = lo + (int)pow3(J + DD) * spread3k<HL - J - DD>(hb);
        uint2 *bp = reinterpret_cast<uint2 *>(S) + 4 * base + q;   // slice q of row base
        uint2 x[T];
        static_for<0, T>([&](auto Ti) {
            constexpr int t = decltype(Ti)::value;
            if constexpr (twos_of(t, DD) == 0) x[t] = bp[4 * t * P];
        });
        static_for<0, DD>([&](auto Di) {
            constexpr int d = decltype(Di)::value;
            constexpr int w = (int)pow3(d);
            static_for<0, T>([&](auto Ti) {
                constexpr int t = decltype(Ti)::value;
                if constexpr ((t / w) % 3 == 2 && binary_above(t, d, DD)) {
                    x[t].x = x[t - 2 * w].x & x[t - w].x;
                    x[t].y = x[t - 2 * w].y & x[t - w].y;
                }
            });
        });
        static_for<0, T>([&](auto Ti) {
            constexpr int t = decltype(Ti)::value;
            if constexpr (twos_of(t, DD) > 0) bp[4 * t * P] = x[t];
        });
    }
}

// Reduce of digits J .. J+DD-1 over all rows: each cell loses its bit if one
// of its '*' neighbours in these digits is set, all read from the block as
// the step found it (rows are updated in order of their number of '*'
// digits, so a row is overwritten only after every row that reads it).
template <int HL, int J, int DD>
__device__ __forceinline__ void reduce_step(uint4 *S, int lt, int tg)
{
    constexpr int P = (int)pow3(J);
    constexpr int T = (int)pow3(DD);
    constexpr int items = (int)pow3(HL - DD) * 4;
    for (int it = lt; it < items; it += tg) {
        const int q = it & 3, r = it >> 2;
        const int lo = r % P, hi = r / P;
        const int base = lo + hi * (int)pow3(J + DD);
        uint2 *bp = reinterpret_cast<uint2 *>(S) + 4 * base + q;   // slice q of row base
        uint2 x[T];
        static_for<0, T>([&](auto Ti) {
            constexpr int t = decltype(Ti)::value;
            x[t] = bp[4 * t * P];
        });
        {
            // Only a set cell of a row with a '*' in these digits clears
            // anything: with none set, the block stays as it is.
            uint32_t src = 0;
            static_for<0, T>([&](auto Ti) {
                constexpr int t = decltype(Ti)::value;
                if constexpr (twos_of(t, DD) > 0) src |= x[t].x | x[t].y;
            });
            if (src == 0) continue;
        }
        static_for<0, DD>([&](auto Ki) {
            constexpr int k = decltype(Ki)::value;   // number of '*' digits of the rows updated now
            static_for<0, T>([&](auto Ti) {
                constexpr int t = decltype(Ti)::value;
                if constexpr (twos_of(t, DD) == k) {
                    uint32_t ax = 0, ay = 0;
                    static_for<0, DD>([&](auto Di) {
                        constexpr int d = decltype(Di)::value;
                        constexpr int w = (int)pow3(d);
                        constexpr int td = (t / w) % 3;
                        if constexpr (td != 2) {
                            ax |= x[t + (2 - td) * w].x;
                            ay |= x[t + (2 - td) * w].y;
                        }
                    });
                    x[t].x &= ~ax;
                    x[t].y &= ~ay;
                }
            });
        });
        static_for<0, T>([&](auto Ti) {
            constexpr int t = decltype(Ti)::value;
            if constexpr (twos_of(t, DD) < DD) bp[4 * t * P] = x[t];
        });
    }
}

template <int HL, int J, int D, typename Sync>
__device__ __forceinline__ void merge_all(uint4 *S, int lt, int tg, const Sync &sync)
{
    if constexpr (J < HL) {
        constexpr int DD = (HL - J < D) ? HL - J : D;
        merge_step<HL, J, DD>(S, lt, tg);
        sync();
        merge_all<HL, J + DD, D, Sync>(S, lt, tg, sync);
    }
}

template <int HL, int J, int D, typename Sync>
__device__ __forceinline__ void reduce_all(uint4 *S, int lt, int tg, const Sync &sync)
{
    if constexpr (J < HL) {
        constexpr int DD = (HL - J < D) ? HL - J : D;
        reduce_step<HL, J, DD>(S, lt, tg);
        sync();
        reduce_all<HL, J + DD, D, Sync>(S, lt, tg, sync);
    }
}


}  // namespace dqmc
