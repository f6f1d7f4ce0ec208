// dqmc_pass.cu -- the sweep for n >= 13: streaming passes of 2187-row tiles.
//
// Algorithm 3 of DenseQMC (arXiv 2302.10083, Section 4.1) on the padded
// device state: row r (index of the n-5 high digits) is one 32-byte chunk
// holding the 243 cells of the five low digits (dqmc_chunk.cuh).  Each pass
// is one kernel; one CTA owns one tile of 3^7 = 2187 rows, in which the pass's
// group digits (a .. a+K-1) and 7-K inner digits (0 .. 6-K, contiguous rows)
// vary; every other high digit is fixed per tile.
//
// Per tile:
//   load   truth-table words (first pass), the rows whose group digits are
//          0/1 (Merge input), or all rows, into shared memory (cp.async);
//   Merge  the group digits one after another (Merge of Section 4.1: the
//          '*' row becomes the AND of its 0 row and 1 row; '*' rows of an
//          unmerged digit are zero, so assignment equals the paper's OR);
//   Reduce the group digits and the pass's chunk digits, every row read from
//          the tile as loaded (Reduce of Section 4.1: a cell loses its bit
//          when its '*' neighbour in a reduced digit is set).  Reducing digits
//          in groups, each group reading the state the previous groups left,
//          gives the paper's result: a cube with an implicant one-digit
//          extension is cleared in the first group that holds such a digit
//          (the extension is still set then: clearing it would need an
//          extension of the cube in an earlier group), and primes are never
//          cleared;
//   store  rows back to the state, or, in the last pass, the dense bitmap
//          (each warp funnel-shifts its 32 rows into place in shared memory),
//          the count, and the (mask, value) list placed by a decoupled
//          look-back over the tiles in rho order.
//
// Every global index is checked against its buffer before the access (ck):
// a bad one is recorded in the error word and the access skipped.
#include <cstdio>

#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"

namespace dqmc {

static __constant__ MaskTable kMasksP = make_mask_table();

// Lookup tables over the 7 digits of a tile and the 5 chunk digits.
struct PassTables {
    uint8_t has_star[kTileRows];   // the index has a '*' digit
    uint8_t m7[kTileRows];         // bit d: digit d is 0 or 1 (a literal)
    uint8_t v7[kTileRows];         // bit d: digit d is 1
    uint8_t t5m[243], t5v[243];    // the same for the 5 chunk digits
    uint16_t sp3[128];             // sum of 3^d over the set bits d of the index
};

__host__ __device__ constexpr PassTables make_pass_tables()
{
    PassTables t{};
    for (int i = 0; i < kTileRows; ++i) {
        int q = i, star = 0, m = 0, v = 0;
        for (int d = 0; d < 7; ++d) {
            const int dg = q % 3;
            q /= 3;
            if (dg == 2) star = 1;
            else m |= 1 << d;
            if (dg == 1) v |= 1 << d;
        }
        t.has_star[i] = (uint8_t)star;
        t.m7[i] = (uint8_t)m;
        t.v7[i] = (uint8_t)v;
    }
    for (int i = 0; i < 243; ++i) {
        int q = i, m = 0, v = 0;
        for (int d = 0; d < 5; ++d) {
            const int dg = q % 3;
            q /= 3;
            if (dg != 2) m |= 1 << d;
            if (dg == 1) v |= 1 << d;
        }
        t.t5m[i] = (uint8_t)m;
        t.t5v[i] = (uint8_t)v;
    }
    for (int i = 0; i < 128; ++i) {
        int r = 0, w = 1, x = i;
        while (x) {
            if (x & 1) r += w;
            x >>= 1;
            w *= 3;
        }
        t.sp3[i] = (uint16_t)r;
    }
    return t;
}

static __device__ const PassTables g_tab = make_pass_tables();

struct PassParams {
    const uint32_t *on;
    const uint32_t *dc;
    uint4 *state;
    uint32_t *out;
    unsigned long long *count;
    uint2 *pairs;               // null: no list
    uint64_t cap;
    uint32_t *ctrl;             // control block: [0] error word, [1..] ticket counters
    unsigned long long *status; // look-back slots, one per bitmap tile
    uint64_t state_rows, tt_words, out_tiles, total_rows;
    uint64_t out_words, out_alloc_words;
    uint64_t wait_ns;
    uint64_t w_g;               // 3^a
    uint32_t nmask;             // (1 << n) - 1
    int H, chunk_mask, slot;
    FixedDigits fix;            // digits fixed per tile, ascending
};

constexpr int kThreads = 256;
constexpr int kRounds = (kTileRows + kThreads - 1) / kThreads;  // 9
constexpr unsigned long long kFlagA = 1ull << 62, kFlagP = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
// The last warp of a tile stages the bits of kTileRows % 32 = 11 rows in those
// rows' 88 words; the staged words, rounded up to whole uint4, fit, and so
// do the 9 words the list reads from the start of the last row.
static_assert(kTileRows % 32 == 11, "tile tail");
static_assert(4 * ((31 + 243 * 11 + 127) / 128) <= 8 * 11, "tail staging fits its rows");
static_assert((31 + 243 * 10) / 32 + 9 <= 8 * 11, "tail list reads fit its rows");
static_assert((31 + 243 * 31) / 32 + 9 <= 8 * 32, "list reads fit a warp's rows");

enum PassMode : int { kModeMerge = 0, kModeMergeReduce = 1, kModeReduce = 2, kModeOut = 3 };

__device__ __forceinline__ void report(const PassParams &P, uint64_t idx)
{
    if (atomicCAS(P.ctrl, 0u, kErrBounds) == 0u)
        printf("dqmc: index %llu out of range (block %d)\n", (unsigned long long)idx, (int)blockIdx.x);
}

// true when cond holds; otherwise records the bad index and returns false
__device__ __forceinline__ bool ck(const PassParams &P, bool cond, uint64_t idx)
{
    if (cond) return true;
    report(P, idx);
    return false;
}

__device__ __forceinline__ int slotp(int r, int h) { return 2 * r + (h ^ ((r >> 2) & 1)); }

__device__ __forceinline__ void cp_async16p(void *smem_dst, const void *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_p()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64p(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void chunk_reduce_masked_p(const uint32_t (&v)[kChunkWords],
                                                      uint32_t (&acc)[kChunkWords], int mask)
{
    static_for<0, kChunkDigits>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int d = (int)pow3(i);
        if ((mask >> i) & 1) {
            uint32_t y[kChunkWords];
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) y[w] = v[w] & kMasksP.m[kChunkDigits][i][2][w];
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) acc[w] |= shr_word<d>(y, w) | shr_word<2 * d>(y, w);
        }
    });
}

__device__ __forceinline__ void chunk_from_word_p(uint32_t x, uint32_t (&v)[kChunkWords])
{
#pragma unroll
    for (int w = 0; w < kChunkWords; ++w) v[w] = 0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const int q = spread_pos(t);
        v[q >> 5] |= ((x >> t) & 1u) << (q & 31);
    }
    static_for<0, kChunkDigits>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int d = (int)pow3(i);
        uint32_t nv[kChunkWords];
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w)
            nv[w] = v[w] | (shl_word<d>(v, w) & shl_word<2 * d>(v, w) & kMasksP.m[kChunkDigits][i][2][w]);
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) v[w] = nv[w];
    });
}

// Decoupled look-back (warp 0): primes in the bitmap tiles before tile T.
// This tile's aggregate (or, for T = 0, its prefix) is already published.
__device__ unsigned long long lookback_p(const PassParams &P, uint64_t T, bool &ok)
{
    const int lane = threadIdx.x & 31;
    ok = true;
    if (T == 0) return 0;
    unsigned long long excl = 0;
    long long j = (long long)T - 1;
    const uint64_t t0 = globaltimer_p();
    for (;;) {
        const long long idx = j - lane;
        const unsigned long long s = (idx >= 0) ? ld_volatile_u64p(&P.status[idx]) : kFlagP;
        const unsigned flag = (unsigned)(s >> 62);
        if (__any_sync(0xffffffffu, flag == 0)) {
            bool stop = false;
            if (lane == 0) {
                if (*reinterpret_cast<volatile uint32_t *>(P.ctrl) != 0) stop = true;
                else if (globaltimer_p() - t0 > P.wait_ns) {
                    atomicCAS(P.ctrl, 0u, kErrTimeout);
                    stop = true;
                }
            }
            if (__shfl_sync(0xffffffffu, (int)stop, 0)) {
                ok = false;
                return 0;
            }
            __nanosleep(64);
            continue;
        }
        const unsigned pm = __ballot_sync(0xffffffffu, flag == 2);
        const int first = pm ? __ffs(pm) - 1 : 31;
        unsigned long long v = (lane <= first) ? (s & kValMask) : 0ull;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pm) break;
        j -= 32;
    }
    return excl;
}

struct PassShared {
    FixedDigits fix;
    uint64_t base, ttb, tile;
    unsigned long long excl;
    uint32_t warp_tot[kThreads / 32];
    uint32_t tile_mask, tile_val;
    int list_ok;
};

template <int K, int B, int LOAD, int MODE>
__global__ void __launch_bounds__(kThreads, 3)
pass_kernel(const __grid_constant__ PassParams P)
{
    constexpr int RE = (int)pow3(B);
    constexpr int RG = (int)pow3(K);
    constexpr int R = RG * RE;
    constexpr int NB = 1 << K;
    static_assert(R == kTileRows, "tiles are 2187 rows");
    extern __shared__ uint4 tile[];
    __shared__ PassShared S;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    // ---------------------------------------------------------------- tile
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&P.fix);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&S.fix);
        for (int i = tid; i < (int)(sizeof(FixedDigits) / 4); i += kThreads) dst[i] = src[i];
    }
    __syncthreads();
    if (tid == 0) {
        uint64_t t = blockIdx.x;
        if (MODE == kModeOut && P.pairs) t = atomicAdd(P.ctrl + 1 + P.slot, 1u);  // tiles start in rho order
        uint64_t base = 0, ttb = 0, x = t;
        for (int i = 0; i < S.fix.n; ++i) {
            uint64_t d;
            if (S.fix.r[i] == 2) {
                d = x & 1u;
                x >>= 1;
            } else {
                const uint64_t q = x / 3u;
                d = x - 3u * q;
                x = q;
            }
            base += d * S.fix.w3[i];
            ttb += d * S.fix.w2[i];
        }
        S.base = base;
        S.ttb = ttb;
        S.tile = t;
    }
    __syncthreads();
    const uint64_t base = S.base, ttb = S.ttb;
    const uint64_t w_g = P.w_g;
    uint4 *const state = P.state;
    const uint64_t state_rows = P.state_rows;

    // ---------------------------------------------------------------- load
    if constexpr (LOAD == kLoadTT) {
        for (int gb = tid; gb < NB; gb += kThreads) {
            if (!ck(P, ttb + gb < P.tt_words, ttb + gb)) continue;
            uint32_t x = __ldg(P.on + ttb + gb);
            if (P.dc) x |= __ldg(P.dc + ttb + gb);
            uint32_t v[kChunkWords];
            chunk_from_word_p(x, v);
            const int r = __ldg(&g_tab.sp3[gb]);
            tile[slotp(r, 0)] = make_uint4(v[0], v[1], v[2], v[3]);
            tile[slotp(r, 1)] = make_uint4(v[4], v[5], v[6], v[7]);
        }
    } else {
        constexpr int rows_in = (LOAD == kLoadSparse) ? NB * RE : R;
        for (int pc = tid; pc < rows_in * 2; pc += kThreads) {
            const int h = pc & 1, ri = pc >> 1;
            const int q = ri / RE, e = ri - q * RE;
            const int g = (LOAD == kLoadSparse) ? (int)__ldg(&g_tab.sp3[q]) : q;
            const uint64_t row = base + e + (uint64_t)g * w_g;
            if (!ck(P, row < state_rows, row)) continue;
            cp_async16p(&tile[slotp(g * RE + e, h)], &state[2 * row + h]);
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();

    // --------------------------------------------------------------- Merge
    if constexpr (MODE == kModeMerge || MODE == kModeMergeReduce) {
        static_for<0, K>([&](auto J) {
            constexpr int j = decltype(J)::value;
            constexpr int dj = (int)pow3(j);
            constexpr int items = dj * (1 << (K - 1 - j)) * RE * 2;
            for (int it = tid; it < items; it += kThreads) {
                const int h = it & 1;
                int r = it >> 1;
                const int e = r % RE;
                r /= RE;
                const int lo = r % dj;
                const int hb = r / dj;
                const int g = lo + 3 * dj * (int)__ldg(&g_tab.sp3[hb]);
                const int r0 = g * RE + e;
                const uint4 s0 = tile[slotp(r0, h)];
                const uint4 s1 = tile[slotp(r0 + dj * RE, h)];
                tile[slotp(r0 + 2 * dj * RE, h)] = make_uint4(s0.x & s1.x, s0.y & s1.y, s0.z & s1.z, s0.w & s1.w);
            }
            __syncthreads();
        });
    }

    if constexpr (MODE == kModeMerge) {
        // Write the rows the Merge created (rows whose group digits are all
        // 0/1 came from the state unchanged), or all rows when they came from
        // the truth table.
        for (int pc = tid; pc < R * 2; pc += kThreads) {
            const int h = pc & 1, ri = pc >> 1;
            const int g = ri / RE, e = ri - g * RE;
            if (LOAD != kLoadTT && !__ldg(&g_tab.has_star[g])) continue;
            const uint64_t row = base + e + (uint64_t)g * w_g;
            if (!ck(P, row < state_rows, row)) continue;
            state[2 * row + h] = tile[slotp(ri, h)];
        }
        return;
    } else {
        // ------------------------------------------------------- Reduce rows
        const int cmask = P.chunk_mask;
        uint32_t my_count = 0;
        // out: this tile's bits are bits bit0 .. bit0 + R*243 - 1 of the bitmap
        const uint64_t bit0 = base * 243u;
        const uint32_t o = (uint32_t)(bit0 & 31);
        const uint64_t W0 = bit0 >> 5;
        const bool last_tile = (base + R == P.total_rows);
        uint8_t *const cnt = reinterpret_cast<uint8_t *>(tile + 2 * R);  // primes per row (OUT)

#pragma unroll 1
        for (int rd = 0; rd < kRounds; ++rd) {
            const int ri = rd * kThreads + tid;
            uint32_t v[kChunkWords];
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) v[w] = 0;
            if (ri < R) {
                const uint4 q0 = tile[slotp(ri, 0)], q1 = tile[slotp(ri, 1)];
                v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
                v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
                uint32_t acc[kChunkWords];
#pragma unroll
                for (int w = 0; w < kChunkWords; ++w) acc[w] = 0;
                int gg = ri / RE;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int dg = gg % 3;
                    gg /= 3;
                    if (dg != 2) {
                        const int nb = ri + (2 - dg) * (int)pow3(j) * RE;
                        const uint4 a0 = tile[slotp(nb, 0)], a1 = tile[slotp(nb, 1)];
                        acc[0] |= a0.x; acc[1] |= a0.y; acc[2] |= a0.z; acc[3] |= a0.w;
                        acc[4] |= a1.x; acc[5] |= a1.y; acc[6] |= a1.z; acc[7] |= a1.w;
                    }
                }
                if (cmask) chunk_reduce_masked_p(v, acc, cmask);
#pragma unroll
                for (int w = 0; w < kChunkWords; ++w) v[w] &= ~acc[w];
            }
            if constexpr (MODE != kModeOut) {
                if (ri < R) {
                    const int g = ri / RE, e = ri - g * RE;
                    const uint64_t row = base + e + (uint64_t)g * w_g;
                    if (ck(P, row < state_rows, row)) {
                        state[2 * row] = make_uint4(v[0], v[1], v[2], v[3]);
                        state[2 * row + 1] = make_uint4(v[4], v[5], v[6], v[7]);
                    }
                }
            } else {
                // ------------------------------------- count and dense bits
                uint32_t c = 0;
#pragma unroll
                for (int w = 0; w < kChunkWords; ++w) c += __popc(v[w]);
                my_count += c;
                if (ri < R) cnt[ri] = (uint8_t)c;  // <= 243
                // A row is read only by rows of smaller index (its '*'
                // neighbours lie above it), so once this round's reads are
                // done its rows' slots are free: each warp stages the dense
                // bits of its 32 rows there and keeps them for the list.
                __syncthreads();
                const int q0 = rd * kThreads + wid * 32;
                const int nrows = min(32, R - q0);
                if (nrows > 0) {
                    uint32_t *const stg = reinterpret_cast<uint32_t *>(tile + 2 * q0);
                    // these rows are tile bits o + 243*q0 ..: words S0 .. of the
                    // bitmap, starting at bit o of word S0
                    const uint32_t hi_bit = o + 243u * (uint32_t)nrows;  // end of these rows' bits
                    const int nw4 = (int)((hi_bit + 127u) >> 7);          // uint4 words holding them
                    for (int i = lane; i < nw4; i += 32) reinterpret_cast<uint4 *>(stg)[i] = make_uint4(0u, 0u, 0u, 0u);
                    __syncwarp();
                    if (ri < R) {
                        const uint32_t lb = o + 243u * (uint32_t)lane;
                        const uint32_t k0 = lb >> 5, s = lb & 31;
                        const uint32_t cw = (s + 243u + 31u) >> 5;  // 8 or 9 words
                        uint32_t w9[9];
                        w9[0] = v[0] << s;
#pragma unroll
                        for (int j = 1; j < 8; ++j) w9[j] = __funnelshift_l(v[j - 1], v[j], s);
                        w9[8] = __funnelshift_l(v[7], 0u, s);
                        atomicOr(&stg[k0], w9[0]);
#pragma unroll
                        for (int j = 1; j < 8; ++j) {
                            if ((uint32_t)j < cw - 1) stg[k0 + j] = w9[j];
                            else if ((uint32_t)j == cw - 1) atomicOr(&stg[k0 + j], w9[j]);
                        }
                        if (cw == 9) atomicOr(&stg[k0 + 8], w9[8]);
                    }
                    __syncwarp();
                    const uint64_t S0 = W0 + (uint64_t)243 * (uint64_t)(q0 >> 5);
                    if (nrows == 32 && ck(P, S0 + 244 <= P.out_alloc_words, S0 + 244)) {
                        // 32 full rows: words 1 .. 242 hold only these rows' bits;
                        // word 0 holds them from bit o up, word 243 below bit o.
                        uint32_t *const dstw = P.out + S0;
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int j = 1 + lane + 32 * k;
                            if (j <= 242) dstw[j] = stg[j];
                        }
                        if (lane == 0) {
                            if (o == 0) {
                                dstw[0] = stg[0];
                            } else {
                                const uint32_t m = 0xffffffffu << o;
                                atomicAnd(dstw, stg[0] | ~m);
                                atomicOr(dstw, stg[0] & m);
                            }
                        } else if (lane == 1 && o != 0) {
                            const uint32_t m = (1u << o) - 1u;
                            atomicAnd(dstw + 243, stg[243] | ~m);
                            atomicOr(dstw + 243, stg[243] & m);
                        }
                    } else for (int j = lane; j < 244; j += 32) {
                        // bits of word j owned by these rows: [lo, hi)
                        const int lo = (j == 0) ? (int)o : 0;
                        int hi = (int)min(hi_bit - 32u * (uint32_t)j, 32u);
                        if ((uint32_t)(32 * j) >= hi_bit) hi = 0;
                        const uint64_t wi = S0 + (uint64_t)j;
                        if (last_tile && wi == P.out_words - 1 && hi > lo) hi = 32;  // bits past 3^n are 0
                        if (hi <= lo) continue;
                        if (!ck(P, wi < P.out_alloc_words, wi)) continue;
                        const uint32_t val = stg[j];
                        uint32_t *dst = P.out + wi;
                        if (lo == 0 && hi == 32) {
                            *dst = val;
                        } else {
                            const uint32_t m = (hi == 32 ? 0xffffffffu : ((1u << hi) - 1u)) & (0xffffffffu << lo);
                            atomicAnd(dst, val | ~m);
                            atomicOr(dst, val & m);
                        }
                    }
                }
            }
        }

        if constexpr (MODE == kModeOut) {
            if (last_tile)
                for (uint64_t w = P.out_words + tid; w < P.out_alloc_words; w += kThreads) P.out[w] = 0u;
            // tile count
            uint32_t x = my_count;
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) S.warp_tot[wid] = x;
            __syncthreads();
            uint32_t tile_total = 0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) tile_total += S.warp_tot[w];
            if (tid == 0 && tile_total) atomicAdd(P.count, (unsigned long long)tile_total);
            if (P.pairs) {
                const uint64_t T = S.tile;
                if (wid == 0) {
                    bool ok = true;
                    unsigned long long ex = 0;
                    if (ck(P, T < P.out_tiles, T)) {
                        if (lane == 0)
                            atomicExch(&P.status[T], (T == 0 ? kFlagP : kFlagA) | (unsigned long long)tile_total);
                        ex = lookback_p(P, T, ok);
                        if (lane == 0 && ok && T > 0) atomicExch(&P.status[T], kFlagP | (ex + tile_total));
                    } else {
                        ok = false;
                    }
                    if (lane == 0) {
                        S.excl = ex;
                        S.list_ok = ok;
                        // mask / value bits of the high digits >= 7 (fixed in this tile)
                        uint64_t xt = T;
                        uint32_t m = 0, vv = 0;
                        for (int d = kTileDigits; d < P.H; ++d) {
                            const uint64_t q = xt / 3u;
                            const uint32_t dg = (uint32_t)(xt - 3u * q);
                            xt = q;
                            if (dg != 2) m |= 1u << (5 + d);
                            if (dg == 1) vv |= 1u << (5 + d);
                        }
                        S.tile_mask = m;
                        S.tile_val = vv;
                    }
                }
                __syncthreads();
                if (S.list_ok) {
                    // rows 9t .. 9t+8 belong to thread t < 243: prefix over rows
                    constexpr int kPer = kTileRows / 243;  // 9
                    uint32_t mine = 0;
                    if (tid < 243)
                        for (int k = 0; k < kPer; ++k) mine += cnt[tid * kPer + k];
                    uint32_t incl = mine;
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += y;
                    }
                    __syncthreads();
                    if (lane == 31) S.warp_tot[wid] = incl;
                    __syncthreads();
                    uint32_t before = incl - mine;
                    for (int w = 0; w < wid; ++w) before += S.warp_tot[w];
                    unsigned long long k = S.excl + before;
                    const uint64_t cap = P.cap;
                    const uint32_t nmask = P.nmask;
                    if (tid < 243 && mine && k < cap) {
                        for (int kk = 0; kk < kPer; ++kk) {
                            const int ri = tid * kPer + kk;
                            if (!cnt[ri]) continue;
                            // this row's 243 bits, staged in its warp's slots
                            const uint32_t *const stg = reinterpret_cast<const uint32_t *>(tile + 2 * (ri & ~31));
                            const uint32_t lb = o + 243u * (uint32_t)(ri & 31);
                            const uint32_t s = lb & 31;
                            uint32_t words[9];
#pragma unroll
                            for (int j = 0; j < 9; ++j) words[j] = stg[(lb >> 5) + j];
                            const uint32_t rm = S.tile_mask | ((uint32_t)__ldg(&g_tab.m7[ri]) << 5);
                            const uint32_t rv = S.tile_val | ((uint32_t)__ldg(&g_tab.v7[ri]) << 5);
#pragma unroll
                            for (int w = 0; w < kChunkWords; ++w) {
                                uint32_t bits = __funnelshift_r(words[w], words[w + 1], s);
                                if (w == kChunkWords - 1) bits &= (1u << (243 - 224)) - 1u;
                                while (bits) {
                                    const int bb = __ffs(bits) - 1;
                                    bits &= bits - 1;
                                    const int q = 32 * w + bb;
                                    if (k < cap)
                                        P.pairs[k] = make_uint2((rm | __ldg(&g_tab.t5m[q])) & nmask,
                                                                (rv | __ldg(&g_tab.t5v[q])) & nmask);
                                    ++k;
                                }
                            }
                        }
                    }
                }
            }
        }
    }
}

// One thread waits on a counter that nothing increments: the bounded wait must
// give up after wait_ns and leave kErrTimeout in the error word.
__global__ void selftest_wait_kernel(const __grid_constant__ PassParams P)
{
    if (threadIdx.x != 0) return;
    const volatile uint32_t *ctr = P.ctrl + 1 + kCtrlTickets;
    const uint64_t t0 = globaltimer_p();
    for (;;) {
        if (*ctr >= 1u) return;
        if (globaltimer_p() - t0 > P.wait_ns) {
            atomicCAS(P.ctrl, 0u, kErrTimeout);
            return;
        }
        __nanosleep(256);
    }
}

cudaError_t launch_selftest_wait(void *d_ctrl, uint64_t ctrl_bytes, uint64_t wait_ns, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(d_ctrl, 0, ctrl_bytes, stream);
    if (e != cudaSuccess) return e;
    PassParams p{};
    p.ctrl = static_cast<uint32_t *>(d_ctrl);
    p.wait_ns = wait_ns;
    selftest_wait_kernel<<<1, 32, 0, stream>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ dispatch

template <int K, int B, int LOAD, int MODE>
static cudaError_t launch_pass_k(const PassParams &p, uint64_t tiles, cudaStream_t stream)
{
    size_t smem = (size_t)kTileRows * kChunkBytes;
    if (MODE == kModeOut) smem += (size_t)kTileRows;
    auto kern = pass_kernel<K, B, LOAD, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (tiles == 0) return cudaSuccess;
    if (tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)tiles, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

template <int LOAD, int MODE>
static cudaError_t dispatch_group(int K, const PassParams &p, uint64_t tiles, cudaStream_t s)
{
    switch (K) {
    case 1: return launch_pass_k<1, 6, LOAD, MODE>(p, tiles, s);
    case 2: return launch_pass_k<2, 5, LOAD, MODE>(p, tiles, s);
    case 3: return launch_pass_k<3, 4, LOAD, MODE>(p, tiles, s);
    case 4: return launch_pass_k<4, 3, LOAD, MODE>(p, tiles, s);
    case 5: return launch_pass_k<5, 2, LOAD, MODE>(p, tiles, s);
    case 6: return launch_pass_k<6, 1, LOAD, MODE>(p, tiles, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_super(const Plan &plan, const void *d_on, const void *d_dc, void *d_state, uint32_t *d_bitmap,
                         unsigned long long *d_count, uint32_t *d_pairs, uint64_t cap, void *d_ctrl,
                         cudaStream_t stream, int first, int last)
{
    const CtrlLayout cl = ctrl_layout(plan);
    cudaError_t e = cudaSuccess;
    if (first == 0) {
        e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_ctrl, 0, cl.bytes, stream);
        if (e != cudaSuccess) return e;
    }
    PassParams a{};
    a.on = static_cast<const uint32_t *>(d_on);
    a.dc = static_cast<const uint32_t *>(d_dc);
    a.state = static_cast<uint4 *>(d_state);
    a.out = d_bitmap;
    a.count = d_count;
    a.pairs = reinterpret_cast<uint2 *>(d_pairs);
    a.cap = d_pairs ? cap : 0;
    a.ctrl = static_cast<uint32_t *>(d_ctrl);
    a.status = reinterpret_cast<unsigned long long *>(d_ctrl) + cl.status_u64;
    a.state_rows = plan.state_rows;
    a.tt_words = ((1ull << plan.n) + 31) / 32;
    a.out_tiles = plan.out_tiles;
    a.total_rows = pow3(plan.H);
    a.out_words = bitmap_words(plan.n);
    a.out_alloc_words = bitmap_alloc_bytes(plan.n) / 4;
    a.wait_ns = 1000000000ull;
    a.nmask = (uint32_t)((1ull << plan.n) - 1);
    a.H = plan.H;
    for (int i = first; i < last; ++i) {
        const SuperPassDesc &sp = plan.sps[i];
        const PhaseDesc &ph = sp.ph[0];
        a.w_g = pow3(ph.a);
        a.chunk_mask = ph.chunk_mask;
        a.slot = sp.slot;
        a.fix = sp.sb;
        const uint64_t tiles = sp.n_sb;
        if (ph.load == kLoadTT)
            e = (ph.K == kTileDigits) ? launch_pass_k<kTileDigits, 0, kLoadTT, kModeMerge>(a, tiles, stream)
                                      : cudaErrorInvalidValue;
        else if (ph.out)
            e = (ph.K == kTileDigits) ? launch_pass_k<kTileDigits, 0, kLoadFull, kModeOut>(a, tiles, stream)
                                      : cudaErrorInvalidValue;
        else if (ph.merge && ph.reduce)
            e = dispatch_group<kLoadSparse, kModeMergeReduce>(ph.K, a, tiles, stream);
        else if (ph.merge)
            e = dispatch_group<kLoadSparse, kModeMerge>(ph.K, a, tiles, stream);
        else
            e = dispatch_group<kLoadFull, kModeReduce>(ph.K, a, tiles, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dqmc
