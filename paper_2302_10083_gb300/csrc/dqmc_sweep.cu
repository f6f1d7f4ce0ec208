// dqmc_sweep.cu -- the dense ternary sweep on the device.
//
// What is computed (DenseQMC, arXiv 2302.10083, Algorithm 3 in Section 4.1):
//   MergeAll: for every digit i and every triple (s, t, u) of cubes that differ
//     only in digit i (values 0, 1, *): S(u) |= S(s) & S(t)   (Merge).
//   ReduceAll: for every digit i and every such triple:
//     S(s) &= ~S(u), S(t) &= ~S(u)                            (Reduce).
// The result is the set of prime implicants of the support ON u DC.
//
// How it is scheduled on GB300 (this differs from the paper's CPU layout):
//   * State layout: row r (index of the n-5 high digits) x chunk q (index of the
//     5 low digits, 243 bits in a 32-byte sector).  The chunk digits are merged
//     and reduced in registers with funnel shifts and constant masks
//     (dqmc_chunk.cuh), the high digits row-wise on whole 32-bit words.
//   * Merge order is free and cubes with a '*' in a digit that is not merged yet
//     are zero, so the low digits go first: the first pass reads the truth table
//     and only ever writes rows whose unmerged digits are 0/1; each later Merge
//     pass reads only rows whose group digits are 0/1.  Only the last Merge pass
//     writes the whole state.
//   * Reduce is fused into the last Merge pass (for its digits and the chunk
//     digits) and the remaining digits are reduced group by group; the last
//     group writes the dense bitmap and counts its bits.  Doing Reduce in
//     groups, each group reading the state left by the previous ones, gives
//     the same set as the paper's digit-by-digit in-place loop: a cube with an
//     implicant one-digit extension loses its bit in the first group that holds
//     such a digit, because that extension is still set when the group reads
//     it (its own clearing would need an extension of the cube in an earlier
//     group), and primes are never cleared.
#include <cstdio>

#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"

namespace dqmc {

static __constant__ MaskTable kMasks = make_mask_table();

struct PassArgs {
    const uint32_t *on;
    const uint32_t *dc;
    uint32_t inv;               // ~0u: sweep the complement (support = (not ON) or DC)
    uint4 *state;               // 2 x uint4 per row
    uint32_t *out;              // dense bitmap words
    unsigned long long *count;
    uint64_t n_mid, w_g, w_top;
    uint64_t total_rows;        // 3^H
    uint64_t out_words;         // ceil(3^n / 32)
    uint64_t out_alloc_words;   // bitmap allocation in words (16-byte multiple)
    int top_binary, fuse_reduce, chunk_reduce, write_out;
    // Batch mode (bfn non-null, one tile per function): block b works on
    // function bfn[b]; on / dc / out / count come from the batch tables.
    const uint32_t *bfn;
    const uint64_t *btt_off, *bdc_off, *bbm_off;   // byte offsets; bdc_off ~0: no don't-cares
    const uint8_t *barena;
    uint8_t *bbitmaps;
    unsigned long long *bcount;
};

__device__ __forceinline__ uint64_t spread3(uint64_t x)
{
    uint64_t r = 0, w = 1;
    while (x) {
        if (x & 1) r += w;
        x >>= 1;
        w *= 3u;
    }
    return r;
}

// Shared-memory slot (in uint4 units) of quad h of tile row r.  The quad
// order flips every four rows so that eight consecutive rows read by a
// quarter-warp hit eight different 16-byte bank groups.
__device__ __forceinline__ int slot(int r, int h) { return 2 * r + (h ^ ((r >> 2) & 1)); }

__device__ __forceinline__ void load_row(const uint4 *s, int r, uint32_t (&v)[kChunkWords])
{
    const uint4 q0 = s[slot(r, 0)];
    const uint4 q1 = s[slot(r, 1)];
    v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
    v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
}

__device__ __forceinline__ void or_row(const uint4 *s, int r, uint32_t (&acc)[kChunkWords])
{
    const uint4 q0 = s[slot(r, 0)];
    const uint4 q1 = s[slot(r, 1)];
    acc[0] |= q0.x; acc[1] |= q0.y; acc[2] |= q0.z; acc[3] |= q0.w;
    acc[4] |= q1.x; acc[5] |= q1.y; acc[6] |= q1.z; acc[7] |= q1.w;
}

__device__ __forceinline__ void store_row(uint4 *s, int r, const uint32_t (&v)[kChunkWords])
{
    s[slot(r, 0)] = make_uint4(v[0], v[1], v[2], v[3]);
    s[slot(r, 1)] = make_uint4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// 2^C truth-table bits -> chunk, then Merge over the C chunk digits (Merge of
// Section 4.1: the '*' cell becomes the AND of its 0-cell and 1-cell; before
// digit i is merged every '*' cell of digit i is zero, so OR and assignment
// agree).
template <int C>
__device__ __forceinline__ void chunk_from_minterms(uint32_t x, uint32_t (&v)[kChunkWords])
{
#pragma unroll
    for (int w = 0; w < kChunkWords; ++w) v[w] = 0;
#pragma unroll
    for (int t = 0; t < (1 << C); ++t) {
        const int q = spread_pos(t);
        v[q >> 5] |= ((x >> t) & 1u) << (q & 31);
    }
    static_for<0, C>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int d = (int)pow3(i);
        uint32_t nv[kChunkWords];
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w)
            nv[w] = v[w] | (shl_word<d>(v, w) & shl_word<2 * d>(v, w) & kMasks.m[C][i][2][w]);
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) v[w] = nv[w];
    });
}

// Reduce over the C chunk digits, all read from v: acc collects, for every
// cell with digit i in {0, 1}, its '*' neighbour in digit i.
template <int C>
__device__ __forceinline__ void chunk_reduce_acc(const uint32_t (&v)[kChunkWords],
                                                 uint32_t (&acc)[kChunkWords])
{
    static_for<0, C>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int d = (int)pow3(i);
        uint32_t y[kChunkWords];
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) y[w] = v[w] & kMasks.m[C][i][2][w];
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) acc[w] |= shr_word<d>(y, w) | shr_word<2 * d>(y, w);
    });
}

// 32 bits of the tile's padded result stream starting at tile bit p (p may be
// negative down to -31; bits outside [0, R*C3) read as zero).
template <int C>
__device__ __forceinline__ uint32_t extract32(const uint32_t *st, int p, int R)
{
    constexpr int C3 = (int)pow3(C);
    // p < 0 only for the first word of a misaligned tile: its low -p bits
    // belong to the previous tile, so read from bit 0 and shift up.
    const int up = (p < 0) ? -p : 0;
    p = (p < 0) ? 0 : p;
    const int m = p / C3;
    if (m >= R) return 0u;
    const int off = p - m * C3;
    const int w = off >> 5, s = off & 31;
    auto word = [&](int row, int ww) -> uint32_t {
        const int sl = slot(row, ww >> 2);
        return st[4 * sl + (ww & 3)];
    };
    const uint32_t lo = word(m, w);
    const uint32_t hi = (w + 1 < kChunkWords) ? word(m, w + 1) : 0u;
    uint32_t x = __funnelshift_r(lo, hi, s);
    const int rem = C3 - off;
    if (rem < 32 && m + 1 < R) x |= word(m + 1, 0) << rem;
    return x << up;
}

constexpr int kThreads = 256;

// One tile: 3^K group rows x 3^B inner rows, for one assignment of the other
// high digits.  KIND selects where the rows come from (truth table, sparse
// Merge input, full state); the flags select what happens after the Merge.
template <int C, int K, int B, int KIND>
__global__ void __launch_bounds__(kThreads) tile_pass(const PassArgs p)
{
    constexpr int RG = (int)pow3(K);
    constexpr int RE = (int)pow3(B);
    constexpr int R = RG * RE;
    constexpr int NB = 1 << K;
    extern __shared__ uint4 smem[];
    __shared__ uint16_t sp3[NB];

    const uint32_t *p_on = p.on, *p_dc = p.dc;
    uint32_t *p_out = p.out;
    unsigned long long *p_count = p.count;
    uint64_t tile = blockIdx.x;
    if (p.bfn) {
        const uint32_t id = p.bfn[blockIdx.x];
        tile = 0;
        p_on = reinterpret_cast<const uint32_t *>(p.barena + p.btt_off[id]);
        const uint64_t dco = p.bdc_off[id];
        p_dc = dco == ~0ull ? nullptr : reinterpret_cast<const uint32_t *>(p.barena + dco);
        p_out = reinterpret_cast<uint32_t *>(p.bbitmaps + p.bbm_off[id]);
        p_count = p.bcount + id;
    }
    const uint64_t mid = tile % p.n_mid;
    const uint64_t topi = tile / p.n_mid;
    const uint64_t top_t = p.top_binary ? spread3(topi) : topi;
    const uint64_t base = mid * RE + top_t * p.w_top;  // row of (g = 0, e = 0)

    for (int i = threadIdx.x; i < NB; i += blockDim.x) sp3[i] = (uint16_t)spread3((uint64_t)i);
    __syncthreads();

    if constexpr (KIND == kPassFirst) {
        // a = 0, B = 0: the 2^K binary group rows come from truth-table words
        // topi * 2^K .. topi * 2^K + 2^K - 1 (each word = the 32 minterms of a chunk).
        for (int gb = threadIdx.x; gb < NB; gb += blockDim.x) {
            uint32_t x;
            if constexpr (C == kChunkDigits) {
                const uint64_t wi = topi * NB + gb;
                x = __ldg(p_on + wi) ^ p.inv;
                if (p_dc) x |= __ldg(p_dc + wi);
            } else {
                const uint8_t *on8 = reinterpret_cast<const uint8_t *>(p_on);
                const uint8_t *dc8 = reinterpret_cast<const uint8_t *>(p_dc);
                // 2^C <= 16 minterms: one byte, two for C = 4
                x = on8[0];
                if constexpr (C == 4) x |= (uint32_t)on8[1] << 8;
                x ^= p.inv;   // bits past 2^C are masked below
                if (dc8) {
                    x |= dc8[0];
                    if constexpr (C == 4) x |= (uint32_t)dc8[1] << 8;
                }
                x &= (1u << (1 << C)) - 1u;
            }
            uint32_t v[kChunkWords];
            chunk_from_minterms<C>(x, v);
            store_row(smem, sp3[gb], v);
        }
    } else if constexpr (KIND == kPassMerge) {
        // rows with every group digit in {0, 1}
        for (int pc = threadIdx.x; pc < NB * RE * 2; pc += blockDim.x) {
            const int h = pc & 1, ri = pc >> 1;
            const int gb = ri / RE, e = ri - gb * RE;
            const int g = sp3[gb];
            const uint64_t row = base + e + (uint64_t)g * p.w_g;
            cp_async16(&smem[slot(g * RE + e, h)], &p.state[2 * row + h]);
        }
        cp_async_wait_all();
    } else {
        for (int pc = threadIdx.x; pc < R * 2; pc += blockDim.x) {
            const int h = pc & 1, ri = pc >> 1;
            const int g = ri / RE, e = ri - g * RE;
            const uint64_t row = base + e + (uint64_t)g * p.w_g;
            cp_async16(&smem[slot(ri, h)], &p.state[2 * row + h]);
        }
        cp_async_wait_all();
    }
    __syncthreads();

    if constexpr (KIND == kPassFirst || KIND == kPassMerge) {
        // Merge the group digits one after another (digit j: rows with digit j
        // = 0, lower group digits any value, higher group digits 0/1).
        static_for<0, K>([&](auto J) {
            constexpr int j = decltype(J)::value;
            constexpr int dj = (int)pow3(j);
            constexpr int items = dj * (1 << (K - 1 - j)) * RE * 2;
            for (int it = threadIdx.x; it < items; it += blockDim.x) {
                const int h = it & 1;
                int r = it >> 1;
                const int e = r % RE;
                r /= RE;
                const int lo = r % dj;
                const int hb = r / dj;
                const int g = lo + 3 * dj * (int)sp3[hb];
                const int r0 = g * RE + e;
                const uint4 s0 = smem[slot(r0, h)];
                const uint4 s1 = smem[slot(r0 + dj * RE, h)];
                smem[slot(r0 + 2 * dj * RE, h)] =
                    make_uint4(s0.x & s1.x, s0.y & s1.y, s0.z & s1.z, s0.w & s1.w);
            }
            __syncthreads();
        });
        if (!p.fuse_reduce) {
            for (int pc = threadIdx.x; pc < R * 2; pc += blockDim.x) {
                const int h = pc & 1, ri = pc >> 1;
                const int g = ri / RE, e = ri - g * RE;
                const uint64_t row = base + e + (uint64_t)g * p.w_g;
                p.state[2 * row + h] = smem[slot(ri, h)];
            }
            return;
        }
    }

    // Reduce the group digits (and the chunk digits if asked), every row read
    // from the tile as it is now.
    uint4 *staging = smem + 2 * R;
    unsigned long long bits = 0;
    for (int ri = threadIdx.x; ri < R; ri += blockDim.x) {
        const int g = ri / RE, e = ri - g * RE;
        uint32_t v[kChunkWords], acc[kChunkWords];
        load_row(smem, ri, v);
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) acc[w] = 0;
        int gg = g;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int dgt = gg % 3;
            gg /= 3;
            if (dgt != 2) or_row(smem, ri + (2 - dgt) * (int)pow3(j) * RE, acc);
        }
        if (p.chunk_reduce) chunk_reduce_acc<C>(v, acc);
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) v[w] &= ~acc[w];
        if (p.write_out) {
            store_row(staging, ri, v);
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) bits += __popc(v[w]);
        } else {
            const uint64_t row = base + e + (uint64_t)g * p.w_g;
            p.state[2 * row] = make_uint4(v[0], v[1], v[2], v[3]);
            p.state[2 * row + 1] = make_uint4(v[4], v[5], v[6], v[7]);
        }
    }
    if (!p.write_out) return;

    // Count: one atomic per warp.
    for (int o = 16; o > 0; o >>= 1) bits += __shfl_down_sync(0xffffffffu, bits, o);
    if ((threadIdx.x & 31) == 0 && bits) atomicAdd(p_count, bits);
    __syncthreads();

    // Dense bitmap: the tile is rows base .. base + R - 1 (B = 0, a = 0), i.e.
    // bits base*3^C .. (base+R)*3^C - 1 of the output.  The first and last
    // words may be shared with the neighbouring tiles and are written with
    // masked atomics; all other words belong to this tile alone.
    constexpr uint64_t C3 = pow3(C);
    const uint64_t bit0 = base * C3;
    const int o = (int)(bit0 & 31);
    const uint64_t W0 = bit0 >> 5;
    const uint64_t L = (uint64_t)R * C3;
    const int nw = (int)((o + L + 31) >> 5);
    const bool last_tile = (base + R == p.total_rows);
    const int tail = (int)((o + L) & 31);
    const uint32_t *st = reinterpret_cast<const uint32_t *>(staging);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
        const uint32_t val = extract32<C>(st, 32 * i - o, R);
        const bool shared_prev = (i == 0 && o != 0);
        const bool shared_next = (i == nw - 1 && !last_tile && tail != 0);
        uint32_t *dst = p_out + W0 + i;
        if (!shared_prev && !shared_next) {
            *dst = val;
        } else {
            uint32_t m = 0xffffffffu;
            if (shared_prev) m &= 0xffffffffu << o;
            if (shared_next) m &= (1u << tail) - 1u;
            atomicAnd(dst, val | ~m);
            atomicOr(dst, val & m);
        }
    }
    if (last_tile)
        for (uint64_t w = p.out_words + threadIdx.x; w < p.out_alloc_words; w += blockDim.x)
            p_out[w] = 0u;
}

// ------------------------------------------------------------------ dispatch

template <int C, int K, int B, int KIND>
static cudaError_t launch_one(const Pass &ps, const PassArgs &a, cudaStream_t stream)
{
    constexpr int R = (int)(pow3(K) * pow3(B));
    const size_t smem = (size_t)R * kChunkBytes * (a.write_out ? 2 : 1);
    auto kern = tile_pass<C, K, B, KIND>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ps.tiles == 0) return cudaSuccess;
    if (ps.tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)ps.tiles, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int KIND, int B>
static cudaError_t dispatch_k(int C, const Pass &ps, const PassArgs &a, cudaStream_t s)
{
    if (C < kChunkDigits) {
        if constexpr (KIND == kPassFirst && B == 0) {
            switch (C) {
            case 0: return launch_one<0, 0, 0, KIND>(ps, a, s);
            case 1: return launch_one<1, 0, 0, KIND>(ps, a, s);
            case 2: return launch_one<2, 0, 0, KIND>(ps, a, s);
            case 3: return launch_one<3, 0, 0, KIND>(ps, a, s);
            case 4: return launch_one<4, 0, 0, KIND>(ps, a, s);
            }
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (B == 0) {
        switch (ps.K) {
        case 0: if constexpr (KIND == kPassFirst) return launch_one<5, 0, 0, KIND>(ps, a, s); else break;
        case 1: return launch_one<5, 1, 0, KIND>(ps, a, s);
        case 2: return launch_one<5, 2, 0, KIND>(ps, a, s);
        case 3: return launch_one<5, 3, 0, KIND>(ps, a, s);
        case 4: return launch_one<5, 4, 0, KIND>(ps, a, s);
        case 5: return launch_one<5, 5, 0, KIND>(ps, a, s);
        case 6: return launch_one<5, 6, 0, KIND>(ps, a, s);
        case 7: return launch_one<5, 7, 0, KIND>(ps, a, s);
        }
    } else if constexpr (KIND != kPassFirst) {
        switch (ps.K) {
        case 1: return launch_one<5, 1, B, KIND>(ps, a, s);
        case 2: return launch_one<5, 2, B, KIND>(ps, a, s);
        case 3: return launch_one<5, 3, B, KIND>(ps, a, s);
        case 4: return launch_one<5, 4, B, KIND>(ps, a, s);
        case 5: return launch_one<5, 5, B, KIND>(ps, a, s);
        case 6: return launch_one<5, 6, B, KIND>(ps, a, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep(const Plan &plan, const void *d_on, const void *d_dc, void *d_state,
                         uint32_t *d_bitmap, unsigned long long *d_count, cudaStream_t stream, int first,
                         int last, const BatchArgs *batch, uint32_t tt_invert)
{
    if (last < 0) last = (int)plan.passes.size();
    if (first < 0 || last > (int)plan.passes.size() || first > last) return cudaErrorInvalidValue;
    if (batch && batch->nfun == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (first == 0 && !batch) {
        e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return e;
    }
    PassArgs a{};
    a.on = static_cast<const uint32_t *>(d_on);
    a.dc = static_cast<const uint32_t *>(d_dc);
    a.inv = tt_invert;
    a.state = static_cast<uint4 *>(d_state);
    a.out = d_bitmap;
    a.count = d_count;
    a.total_rows = pow3(plan.H);
    a.out_words = bitmap_words(plan.n);
    a.out_alloc_words = bitmap_alloc_bytes(plan.n) / 4;
    if (batch) {
        a.bfn = batch->fn;
        a.btt_off = batch->tt_off;
        a.bdc_off = batch->dc_off;
        a.bbm_off = batch->bm_off;
        a.barena = batch->arena;
        a.bbitmaps = batch->bitmaps;
        a.bcount = batch->count;
    }
    for (int pi = first; pi < last; ++pi) {
        Pass ps = plan.passes[pi];
        if (batch) ps.tiles = batch->nfun;   // one-tile plans: a CTA per function
        a.n_mid = ps.n_mid;
        a.w_g = ps.w_g;
        a.w_top = ps.w_top;
        a.top_binary = ps.top_binary;
        a.fuse_reduce = ps.fuse_reduce;
        a.chunk_reduce = ps.chunk_reduce;
        a.write_out = ps.write_out;
        // n <= 12 only: one tile, the whole function (n >= 13 runs dqmc_super.cu)
        e = (ps.kind == kPassFirst) ? dispatch_k<kPassFirst, 0>(plan.C, ps, a, stream) : cudaErrorInvalidValue;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

uint64_t pass_bytes(const Plan &plan, int i, bool with_dc)
{
    if (i < 0 || i >= (int)plan.passes.size()) return 0;
    const Pass &ps = plan.passes[i];
    const uint64_t RG = pow3(ps.K), RE = pow3(ps.B), NB = 1ull << ps.K;
    uint64_t rd = 0, wr = 0;
    if (ps.kind == kPassFirst) {
        const uint64_t tt = ((1ull << plan.n) + 7) / 8;
        rd = ps.write_out ? tt : ps.tiles * NB * 4;
        if (with_dc) rd *= 2;
    } else if (ps.kind == kPassMerge) {
        rd = ps.tiles * NB * RE * kChunkBytes;
    } else {
        rd = ps.tiles * RG * RE * kChunkBytes;
    }
    wr = ps.write_out ? (pow3(plan.n) + 7) / 8 : ps.tiles * RG * RE * kChunkBytes;
    return rd + wr;
}

}  // namespace dqmc
