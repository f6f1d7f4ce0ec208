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
//   load   the first pass reads truth-table words (tt_pass_kernel); the
//          others copy the rows whose group digits are 0/1 (Merge input) or
//          every row into shared memory: cp.async of 16-byte pieces, or, in
//          the bitmap pass, whose tile is contiguous, TMA bulk copies issued
//          by one thread on an mbarrier whose wait is bounded;
//   Merge  the group digits (Merge of Section 4.1: the '*' row becomes the
//          AND of its 0 row and 1 row; '*' rows of an unmerged digit are zero
//          in the state, so assignment equals the paper's OR);
//   Reduce the group digits, then each row's chunk digits (Reduce of Section
//          4.1: a cell loses its bit when its '*' neighbour in a reduced digit
//          is set).  Reducing digits in groups, each group reading the state
//          the previous groups left, gives the paper's result: a cube with an
//          implicant one-digit extension is cleared in the first group that
//          holds such a digit (the extension is still set then: clearing it
//          would need an extension of the cube in an earlier group), and
//          primes are never cleared.  The bitmap pass also reduces the group
//          just above its tile (the neighbour group) against the '*'
//          neighbour tiles, read from the state as the last Merge pass left
//          it; a block or row with no set cell skips the work that could
//          only leave it as it is;
//   store  rows back to the state, or, in the last pass, the dense bitmap
//          (each warp funnel-shifts its 96 rows into their own, no longer
//          needed, slots of the tile; a region with no set cell writes zero
//          words), the count, and the (mask, value) list placed by a
//          decoupled look-back over the tiles in rho order.  The bitmap may be
//          written over the state itself (in-place mode): each tile then
//          waits for its look-back before it writes a bitmap word.
//
// Two kernels:
//   mr_pass_kernel   the last Merge pass and the Reduce passes: the tile
//                    row-major in shared memory, Merge and Reduce several
//                    digits at a time in register blocks (dqmc_steps.cuh);
//   unit_pass_kernel the Merge-only passes (a thread per unit: the three tile
//                    rows that differ only in tile digit 0, one digit per
//                    step) and the bitmap pass (row-major tile, Reduce in
//                    register blocks, then the per-region bitmap and list).
//
// Every global index is checked against its buffer before the access (ck):
// a bad one is recorded in the error word and the access skipped.
#include <cstdio>

#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"
#include "dqmc_steps.cuh"

namespace dqmc {

static __constant__ MaskTable kMasksP = make_mask_table();

constexpr int kUnits = kTileRows / 3;  // 729 units of three rows per tile
// Shared memory of a unit pass, in 16-byte slots: the tile (6 slots per unit;
// see uslot), then one unit of zeros that stands for the '*' neighbour a '*'
// digit does not have.
template <bool PAD>
constexpr int tile_slots() { return 6 * kUnits; }
template <bool PAD>
constexpr size_t unit_smem() { return (size_t)(tile_slots<PAD>() + 6) * 16; }

// Lookup tables over tile units and the 5 chunk digits.
struct PassTables {
    uint16_t code[kUnits];      // bit d (d < 6): unit digit d is 0/1; bit 8+d: it is 1
    uint16_t c5[243];           // chunk cell q: bits 0..4 literal digits, bits 8..12 digits = 1
    uint16_t sp3[128];          // sum of 3^d over the set bits d of the index
};

__host__ __device__ constexpr PassTables make_pass_tables()
{
    PassTables t{};
    for (int u = 0; u < kUnits; ++u) {
        int q = u, m = 0, v = 0;
        for (int d = 0; d < 6; ++d) {
            const int dg = q % 3;
            q /= 3;
            if (dg != 2) m |= 1 << d;
            if (dg == 1) v |= 1 << d;
        }
        t.code[u] = (uint16_t)(m | (v << 8));
    }
    for (int i = 0; i < 243; ++i) {
        int q = i, m = 0, v = 0;
        for (int d = 0; d < 5; ++d) {
            const int dg = q % 3;
            q /= 3;
            if (dg != 2) m |= 1 << d;
            if (dg == 1) v |= 1 << d;
        }
        t.c5[i] = (uint16_t)(m | (v << 8));
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
    uint32_t inv;               // ~0u: sweep the complement (support = (not ON) or DC)
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
    int H, slot;
    // bitmap pass: the first nbr_k fixed digits (high digits 7 .. 6+nbr_k) are
    // reduced against the '*' neighbour tiles read from the state (0: none)
    int nbr_k;
    // bitmap pass: the bitmap is written over the state (out == state).  A
    // tile's bitmap lies at or before its own rows (bit 243 r of the bitmap
    // for row r at byte 32 r of the state), so it only overwrites rows of
    // itself and of tiles before it; those tiles, and the tiles before them
    // that read their rows as '*' neighbours, have all read them once they
    // have published their counts.  So each tile waits for its look-back
    // before it writes a bitmap word.
    int inplace;
    FixedDigits fix;            // digits fixed per tile, ascending
    // Batch mode (bfn non-null): block b works on tile b % tiles_per_fn of
    // function bfn[b / tiles_per_fn]; its truth tables, bitmap and count come
    // from the batch tables, its state is state + (b / tiles_per_fn) *
    // bstate_stride, and on / dc / out / count above are unused.
    const uint32_t *bfn;
    const uint64_t *btt_off, *bdc_off, *bbm_off;   // byte offsets; bdc_off ~0: no don't-cares
    const uint8_t *barena;
    uint8_t *bbitmaps;
    unsigned long long *bcount;
    uint64_t bstate_stride;     // uint4 per function
    uint32_t tiles_per_fn;
};

// The function a block works on: its buffers and its tile index.
struct FnBufs {
    const uint32_t *on, *dc;
    uint4 *state;
    uint32_t *out;
    unsigned long long *count;
    uint64_t tile;
};

__device__ __forceinline__ FnBufs fn_bufs(const PassParams &P)
{
    FnBufs f{P.on, P.dc, P.state, P.out, P.count, blockIdx.x};
    if (P.bfn) {
        const uint32_t fi = blockIdx.x / P.tiles_per_fn;
        f.tile = blockIdx.x - (uint64_t)fi * P.tiles_per_fn;
        const uint32_t id = P.bfn[fi];
        f.on = reinterpret_cast<const uint32_t *>(P.barena + P.btt_off[id]);
        const uint64_t dco = P.bdc_off[id];
        f.dc = dco == ~0ull ? nullptr : reinterpret_cast<const uint32_t *>(P.barena + dco);
        f.state = P.state + (uint64_t)fi * P.bstate_stride;
        f.out = reinterpret_cast<uint32_t *>(P.bbitmaps + P.bbm_off[id]);
        f.count = P.bcount + id;
    }
    return f;
}

constexpr int kMaxNbr = 6;          // neighbour-group digits of the bitmap pass
constexpr int kThreads = 256;       // threads per CTA of the first pass
constexpr int kOutStepDigits = 3;   // bitmap pass: tile digits reduced per step
constexpr int kOutThreads = 384;    // threads per CTA of the bitmap pass and the Merge-only passes
constexpr int kMaxWarps = kOutThreads / 32;
constexpr unsigned long long kFlagA = 1ull << 62, kFlagP = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

// Bitmap staging (last pass): a region of 32 units spans 6 * 32 + 8 slots
// (800 words); their 32 * 729 bits, starting at bit o < 32, take at most 730
// words.  The last region has 729 - 22 * 32 = 25 units (6 * 25 + 6 slots).
static_assert(kUnits == 22 * 32 + 25, "tile units");
static_assert((31 + 32 * 729 + 31) / 32 <= 4 * (6 * 32), "full staging fits its region");
static_assert((31 + 25 * 729 + 31) / 32 <= 4 * (6 * 25), "tail staging fits its region");

// Modes of unit_pass_kernel (the last Merge pass and the Reduce passes run in
// mr_pass_kernel).
enum PassMode : int { kModeMerge = 0, kModeOut = 3 };

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

// Shared-memory slot (uint4) of 16-byte piece c (row c/2, half c%2) of unit u:
//   plain (PAD, the bitmap pass): row-major as in the state, row r at bytes
//     32r .. 32r+31, so bulk copies move whole runs of units and the Merge /
//     Reduce steps of dqmc_steps.cuh work on it;
//   swizzled (the Merge-only passes): every other group of four units has its
//     row halves swapped, so that the eight lanes of a quarter-warp reading the
//     same piece of consecutive units (or of units three apart, the Merge of
//     unit digit 0) hit eight different 16-byte bank groups.
template <bool PAD>
__device__ __forceinline__ int uslot(int u, int c)
{
    if constexpr (PAD) return 6 * u + c;
    else return 6 * u + (c ^ ((u >> 2) & 1));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async16p(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bulk copy (TMA, no tensor map) of bytes (a multiple of 16, both addresses
// 16-byte aligned) from global to shared memory, completing on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// L2 prefetch of `bytes` (a multiple of 16) at a 16-byte aligned address.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Bitmap pass: the tile this many tickets later is brought into L2 when a
// tile starts, so that its own bulk copies find it there (0: none).  About
// two tiles per SM ahead (measured at n = 24: 0 / 76 / 152 / 228 / 304 / 456
// / 912 tickets: 30.0 / 29.7 / 29.5 / 29.4 / 29.35 / 29.6 / 30.9 ms; further
// ahead the lines leave L2 before they are used).
constexpr uint64_t kPrefetchAhead = 304;

// The first pass's tile layout: row r, half h.
__device__ __forceinline__ int slotp(int r, int h) { return 2 * r + (h ^ ((r >> 2) & 1)); }

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

// Reduce of the chunk digits in CM (bit i = chunk digit i): acc gains every
// cell whose '*' neighbour in such a digit is set in v.
template <int CM>
__device__ __forceinline__ void chunk_reduce_p(const uint32_t (&v)[kChunkWords], uint32_t (&acc)[kChunkWords])
{
    static_for<0, kChunkDigits>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int d = (int)pow3(i);
        if constexpr ((CM >> i) & 1) {
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
    uint64_t base, ttb, tile;
    uint64_t bar;                         // mbarrier of the tile's bulk loads
    unsigned long long excl;
    uint32_t warp_tot[kMaxWarps];
    uint32_t rcnt[32];                    // primes per 32-unit region (bitmap pass)
    uint32_t tile_mask, tile_val;         // literal / value bits of the digits fixed per tile
    uint32_t nbr_off[kMaxNbr];            // bitmap pass: '*' neighbour tiles, uint4 offsets from the tile
    int n_nbr;
    int list_ok, overflow, next_region, load_fail;
    uint16_t c5[243];                     // copy of the chunk-cell table
    uint16_t code[kUnits];                // copy of the unit-digit table
};

// A decoded tile: its first state row, its first truth-table word, the
// literal / value bits of the digits fixed per tile (bit 5 + j for high digit
// j) and, for the bitmap pass, its '*' neighbour tiles in the neighbour group.
struct TileInfo {
    uint64_t base, ttb, tile;
    uint32_t mask, val;
    uint32_t nbr_off[kMaxNbr];      // uint4 offsets from the tile's first row
    int n_nbr;
};

// Tile id t -> TileInfo, from the fixed-digit table in the kernel parameters.
__device__ __forceinline__ void decode_tile(const PassParams &P, uint64_t t, TileInfo &T)
{
    const FixedDigits &f = P.fix;
    uint64_t base = 0, ttb = 0;
    uint32_t m = 0, vv = 0;
    uint32_t dlo = 0;   // 2 bits per digit: values of the first kMaxNbr fixed digits
    auto put = [&](int i, uint32_t d) {
        base += d * f.w3[i];
        ttb += d * f.w2[i];
        if (d != 2) m |= 1u << (kChunkDigits + f.j[i]);
        if (d == 1) vv |= 1u << (kChunkDigits + f.j[i]);
        if (i < kMaxNbr) dlo |= d << (2 * i);
    };
    if (t >> 32) {
        uint64_t x = t;
        for (int i = 0; i < f.n; ++i) {
            uint32_t d;
            if (f.r[i] == 2) {
                d = (uint32_t)(x & 1u);
                x >>= 1;
            } else {
                const uint64_t q = x / 3u;
                d = (uint32_t)(x - 3u * q);
                x = q;
            }
            put(i, d);
        }
    } else {
        uint32_t x = (uint32_t)t;   // the usual case: 32-bit division by 3
        for (int i = 0; i < f.n; ++i) {
            uint32_t d;
            if (f.r[i] == 2) {
                d = x & 1u;
                x >>= 1;
            } else {
                const uint32_t q = x / 3u;
                d = x - 3u * q;
                x = q;
            }
            put(i, d);
        }
    }
    T.base = base;
    T.ttb = ttb;
    T.tile = t;
    T.mask = m;
    T.val = vv;
    // The '*' neighbour of this tile in each neighbour-group digit that is
    // 0/1 here: the tile with that digit set to '*', (2 - d) 3^j rows on.
    int nn = 0;
    for (int i = 0; i < P.nbr_k && i < kMaxNbr; ++i) {
        const uint32_t d = (dlo >> (2 * i)) & 3u;
        if (d == 2) continue;
        const uint64_t off = (uint64_t)(2 - d) * f.w3[i];
        if (ck(P, base + off + kTileRows <= P.state_rows && 2 * off < (1ull << 32), base + off))
            T.nbr_off[nn++] = (uint32_t)(2 * off);
    }
    T.n_nbr = nn;
}

// Tile id -> PassShared (S.base, S.ttb, S.tile_mask / val, the neighbours).
// Thread 0 only; the caller's next barrier publishes S.  With kTicket and a
// list, tiles take ids in the order they start, so a tile's look-back waits
// only on tiles already running.
template <bool kTicket>
__device__ __forceinline__ void decode_tile0(const PassParams &P, PassShared &S, uint64_t tile)
{
    uint64_t t = tile;
    if (kTicket && (P.pairs || P.inplace)) t = atomicAdd(P.ctrl + 1 + P.slot, 1u);
    TileInfo T;
    decode_tile(P, t, T);
    S.base = T.base;
    S.ttb = T.ttb;
    S.tile = T.tile;
    S.tile_mask = T.mask;
    S.tile_val = T.val;
    for (int i = 0; i < T.n_nbr; ++i) S.nbr_off[i] = T.nbr_off[i];
    S.n_nbr = T.n_nbr;
}

// ------------------------------------------------------------ first pass
// Truth table -> rows with the chunk digits and tile digits 0..6 merged
// (digits >= 7 are still 0/1: their '*' rows are not written).
__global__ void __launch_bounds__(kThreads, 3) tt_pass_kernel(const __grid_constant__ PassParams P)
{
    constexpr int R = kTileRows;
    extern __shared__ uint4 tile[];
    __shared__ PassShared S;
    const int tid = threadIdx.x;
    const FnBufs F = fn_bufs(P);
    if (tid == 0) decode_tile0<false>(P, S, F.tile);
    __syncthreads();
    const uint64_t base = S.base, ttb = S.ttb;

    for (int gb = tid; gb < (1 << kTileDigits); gb += kThreads) {
        if (!ck(P, ttb + gb < P.tt_words, ttb + gb)) continue;
        uint32_t x = __ldg(F.on + ttb + gb) ^ P.inv;
        if (F.dc) x |= __ldg(F.dc + ttb + gb);
        uint32_t v[kChunkWords];
        chunk_from_word_p(x, v);
        const int r = __ldg(&g_tab.sp3[gb]);
        tile[slotp(r, 0)] = make_uint4(v[0], v[1], v[2], v[3]);
        tile[slotp(r, 1)] = make_uint4(v[4], v[5], v[6], v[7]);
    }
    __syncthreads();
    static_for<0, kTileDigits>([&](auto J) {
        constexpr int j = decltype(J)::value;
        constexpr int dj = (int)pow3(j);
        constexpr int items = dj * (1 << (kTileDigits - 1 - j)) * 2;
        for (int it = tid; it < items; it += kThreads) {
            const int h = it & 1;
            const int r = it >> 1;
            const int lo = r % dj;
            const int hb = r / dj;
            const int r0 = lo + 3 * dj * (int)__ldg(&g_tab.sp3[hb]);
            const uint4 s0 = tile[slotp(r0, h)];
            const uint4 s1 = tile[slotp(r0 + dj, h)];
            tile[slotp(r0 + 2 * dj, h)] = make_uint4(s0.x & s1.x, s0.y & s1.y, s0.z & s1.z, s0.w & s1.w);
        }
        __syncthreads();
    });
    for (int pc = tid; pc < R * 2; pc += kThreads) {
        const int h = pc & 1, ri = pc >> 1;
        const uint64_t row = base + ri;
        if (!ck(P, row < P.state_rows, row)) continue;
        F.state[2 * row + h] = tile[slotp(ri, h)];
    }
}

// List of one bitmap tile read back from the bitmap it has written (its
// warp regions had more pairs than their slots hold).  Rows 9t .. 9t+8 of the
// tile belong to thread t < 243.  Every thread of the block calls this.
__device__ __noinline__ void emit_from_bitmap(const PassParams &P, PassShared &S, const uint32_t *out, uint64_t base)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    auto row_bits = [&](int ri, uint32_t (&bw)[kChunkWords]) {
        const uint64_t b = (base + (uint64_t)ri) * 243u;
        const uint64_t wb = b >> 5;
        const uint32_t sh = (uint32_t)(b & 31);
        uint32_t wd[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) wd[j] = (wb + j < P.out_words) ? __ldcg(out + wb + j) : 0u;
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) bw[w] = __funnelshift_r(wd[w], wd[w + 1], sh);
        bw[kChunkWords - 1] &= (1u << (243 - 224)) - 1u;
    };
    uint32_t mine = 0;
    if (tid < 243)
        for (int r = 0; r < 9; ++r) {
            uint32_t bw[kChunkWords];
            row_bits(9 * tid + r, bw);
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) mine += __popc(bw[w]);
        }
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
        for (int r = 0; r < 9; ++r) {
            const int u = 3 * tid + r / 3, kr = r % 3;
            uint32_t bw[kChunkWords];
            row_bits(9 * tid + r, bw);
            const uint32_t code = __ldg(&g_tab.code[u]);
            const uint32_t m7 = (kr != 2 ? 1u : 0u) | ((code & 0x3fu) << 1);
            const uint32_t v7 = (kr == 1 ? 1u : 0u) | (((code >> 8) & 0x3fu) << 1);
            const uint32_t rm = S.tile_mask | (m7 << 5);
            const uint32_t rv = S.tile_val | (v7 << 5);
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) {
                uint32_t bits = bw[w];
                while (bits) {
                    const int bb = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const uint32_t c5 = S.c5[32 * w + bb];
                    if (k < cap) P.pairs[k] = make_uint2((rm | (c5 & 0x1fu)) & nmask, (rv | (c5 >> 8)) & nmask);
                    ++k;
                }
            }
        }
    }
}

// ------------------------------------------------------------ unit passes
//
// B >= 1: tile row e + 3^B g (inner e < 3^B, group index g < 3^K); unit
//         u = eh + RU g holds e = 3 eh .. 3 eh + 2 (RU = 3^(B-1)); its group
//         digits are unit digits B-1 .. 5.
// B == 0: the bitmap pass (a = 0): unit u holds tile rows 3u .. 3u+2, i.e.
//         state rows base + 3u + k; tile digit 0 and unit digits 0 .. 5 are
//         the group digits.
template <int MODE>
constexpr int unit_threads() { return (MODE == kModeOut || MODE == kModeMerge) ? kOutThreads : kThreads; }

template <int K, int B, int LOAD, int MODE, int CM>
__global__ void __launch_bounds__(unit_threads<MODE>(), 3) unit_pass_kernel(const __grid_constant__ PassParams P)
{
    constexpr int NT = unit_threads<MODE>();
    static_assert(MODE == kModeMerge || MODE == kModeOut, "Merge-only and bitmap passes (the others: mr_pass_kernel)");
    static_assert(K + B == kTileDigits, "tiles are 3^7 rows");
    static_assert(B >= 1 || (MODE == kModeOut && LOAD == kLoadFull), "B = 0 only in the bitmap pass");
    constexpr int RU = (B == 0) ? 1 : (int)pow3(B - 1);
    constexpr int D0 = (B == 0) ? 0 : B - 1;    // lowest group unit digit
    constexpr int NB = 1 << K;
    constexpr bool PAD = (B == 0);   // the bitmap pass: padded layout, bulk loads
    constexpr int kZeroSlot = tile_slots<PAD>();
    auto uslot = [](int u, int c) { return dqmc::uslot<PAD>(u, c); };
    extern __shared__ uint4 tile[];
    __shared__ PassShared S;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    const FnBufs F = fn_bufs(P);
    if (tid == 0) {
        decode_tile0<MODE == kModeOut>(P, S, F.tile);
        S.overflow = 0;
        if constexpr (B == 0) {
            // The bitmap pass's tile is one contiguous block of the state (and
            // of shared memory): thread 0 starts its copy (six TMA bulk copies)
            // at once, before the first barrier.
            S.load_fail = 0;
            mbar_init(&S.bar, 1);
            if (*reinterpret_cast<volatile uint32_t *>(P.ctrl) != 0u) {
                // An earlier tile gave up (or found a bad index): the sweep's
                // outputs are already invalid, so this tile issues no copies
                // and sweeps nothing.
                S.load_fail = 2;
            } else {
                constexpr uint32_t kPart = (uint32_t)(kTileRows * kChunkBytes / 6);
                static_assert(kTileRows * kChunkBytes % 6 == 0 && kPart % 16 == 0, "16-byte multiples");
                const uint64_t last = S.base + kTileRows - 1;
                if (ck(P, last < P.state_rows, last)) {
                    mbar_expect_tx(&S.bar, (uint32_t)kUnits * 96u);
                    const char *src = reinterpret_cast<const char *>(&F.state[2 * S.base]);
                    for (int q = 0; q < 6; ++q)
                        bulk_g2s(reinterpret_cast<char *>(tile) + q * kPart, src + q * kPart, kPart, &S.bar);
                    // the bitmap pass's tiles are contiguous in rho order: tile t
                    // starts at row t 3^7
                    const uint64_t t2 = S.tile + kPrefetchAhead;
                    if (kPrefetchAhead && !P.bfn && t2 < P.out_tiles && (t2 + 1) * kTileRows <= P.state_rows)
                        bulk_prefetch_l2(&F.state[2 * t2 * kTileRows], (uint32_t)(kTileRows * kChunkBytes));
                } else {
                    S.load_fail = 2;   // a tile past the state (reported): not loaded, not swept
                }
            }
        }
    }
    __syncthreads();
    if constexpr (B == 0) {
        if (S.load_fail == 2) {   // nothing in flight: leave at once
            if (tid == 0) mbar_inval(&S.bar);
            return;
        }
    }
    // the unit tables are copied while the tile's loads are in flight (below)
    auto fill_tables = [&]() {
        for (int i = tid; i < kUnits; i += NT) S.code[i] = g_tab.code[i];
        if constexpr (MODE == kModeOut)
            for (int i = tid; i < 243; i += NT) S.c5[i] = g_tab.c5[i];
    };
    const uint64_t base = S.base;
    const uint64_t w_g = P.w_g;
    uint4 *const state = F.state;
    uint32_t *const out = F.out;
    const uint64_t state_rows = P.state_rows;
    // first state row of unit u
    auto unit_row = [&](int u) -> uint64_t {
        if constexpr (B == 0) {
            return base + 3u * (uint64_t)u;
        } else {
            const int g = u / RU, eh = u - g * RU;
            return base + 3u * (uint64_t)eh + (uint64_t)g * w_g;
        }
    };

    // ---------------------------------------------------------------- load
    // The bitmap pass's tile is in flight (issued above) and completes on one
    // mbarrier whose wait is bounded.  Other tiles are 96-byte runs far apart:
    // cp.async of 16-byte pieces, consecutive lanes on consecutive pieces.
    if constexpr (B == 0) {
        if (tid < 6) tile[kZeroSlot + tid] = make_uint4(0u, 0u, 0u, 0u);
        fill_tables();
        const uint64_t t0 = globaltimer_p();
        while (!mbar_try_wait(&S.bar, 0)) {
            if (globaltimer_p() - t0 > P.wait_ns) {
                if (atomicCAS(P.ctrl, 0u, kErrTimeout) == 0u)
                    printf("dqmc: tile load did not complete (block %d)\n", (int)blockIdx.x);
                S.load_fail = 1;
                break;
            }
        }
        __syncthreads();
        if (S.load_fail) {
            // Give copies still in flight a bounded time to land, then leave.
            // Every later tile sees the error word before it issues copies of
            // its own and leaves without touching shared memory, so a copy
            // that lands after this CTA is gone can only reach shared memory
            // no tile of this sweep reads.
            if (tid == 0) {
                const uint64_t t1 = globaltimer_p();
                while (!mbar_try_wait(&S.bar, 0) && globaltimer_p() - t1 < P.wait_ns) {
                }
            }
            __syncthreads();
            return;
        }
        if (tid == 0) mbar_inval(&S.bar);   // every thread has seen the tile land
    } else {
        constexpr int units_in = (LOAD == kLoadSparse) ? NB * RU : kUnits;
        for (int p = tid; p < units_in * 6; p += NT) {
            const int q = p / 6, c = p - 6 * q;
            int u = q;
            if constexpr (LOAD == kLoadSparse) {
                const int gb = q / RU, eh = q - gb * RU;
                u = eh + RU * (int)__ldg(&g_tab.sp3[gb]);
            }
            const uint64_t row0 = unit_row(u);
            if (!ck(P, row0 + 2 < state_rows, row0 + 2)) continue;
            cp_async16p(&tile[uslot(u, c)], &state[2 * row0 + c]);
        }
        if (tid < 6) tile[kZeroSlot + tid] = make_uint4(0u, 0u, 0u, 0u);
        fill_tables();
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
    }

    // --------------------------------------------------------------- Merge
    if constexpr (MODE == kModeMerge) {
        static_for<0, K>([&](auto J) {
            constexpr int d = D0 + decltype(J)::value;
            constexpr int Dd = (int)pow3(d);
            // units whose digit d is '*' and whose later group digits are
            // still 0/1: RU * 3^j * 2^(K-1-j) <= 243 of them
            constexpr int j = decltype(J)::value;
            constexpr int Dj = (int)pow3(j);
            constexpr int items = RU * Dj * (1 << (K - 1 - j));
            static_assert(items <= NT, "one unit per thread");
            if (tid < items) {
                const int eh = tid % RU, rest = tid / RU;
                const int lo = rest % Dj, hb = rest / Dj;
                const int u = eh + RU * (lo + 2 * Dj + 3 * Dj * (int)__ldg(&g_tab.sp3[hb]));
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const uint4 s0 = tile[uslot(u - 2 * Dd, c)];
                    const uint4 s1 = tile[uslot(u - Dd, c)];
                    tile[uslot(u, c)] = make_uint4(s0.x & s1.x, s0.y & s1.y, s0.z & s1.z, s0.w & s1.w);
                }
            }
            __syncthreads();
        });
    }

    if constexpr (MODE == kModeMerge) {
        // Write the units the Merge created (a '*' in a group digit); the
        // others came from the state unchanged.
        constexpr uint32_t gmask = (0x3fu >> D0) << D0;
        for (int p = tid; p < kUnits * 6; p += NT) {
            const int u = p / 6, c = p - 6 * u;
            if (!(~(uint32_t)S.code[u] & gmask)) continue;
            const uint64_t row0 = unit_row(u);
            if (!ck(P, row0 + 2 < state_rows, row0 + 2)) continue;
            state[2 * row0 + c] = tile[uslot(u, c)];
        }
        return;
    } else {
        // ------------------------------------------------------- Reduce units
        uint32_t my_count = 0;
        // out: this tile's bits are bits bit0 .. bit0 + 2187*243 - 1 of the bitmap
        const uint64_t bit0 = base * 243u;
        const uint32_t o = (uint32_t)(bit0 & 31);
        const uint64_t W0 = bit0 >> 5;
        const bool last_tile = (base + kTileRows == P.total_rows);

        {
            // Reduce of tile digits 0..6 on whole rows (the tile is row-major),
            // three digits per step with one barrier each (dqmc_steps.cuh); then
            // each thread reduces the chunk digits of its rows (if this pass has
            // any) and counts them.
            // Tile digits 0..5 in two steps; digit 6 in the row loop below.
            static_assert(kTileDigits == 7 && kOutStepDigits == 3, "two steps of three digits, then digit 6");
            reduce_step<kTileDigits, 0, 3>(tile, tid, NT);
            __syncthreads();
            reduce_step<kTileDigits, 3, 3>(tile, tid, NT);
            __syncthreads();
            // Neighbour group (bitmap pass): a cell is also cleared when its
            // '*' neighbour in a neighbour-group digit is set in the state as
            // the previous pass left it.  The neighbour tiles are never
            // written by this pass, so every tile reads them unchanged; the
            // result is exact in any order with the tile's own Reduce steps
            // (a set cell is always an implicant, and a cell with an implicant
            // extension in such a digit finds it still set: clearing that
            // extension would take an implicant extension of the cell in an
            // earlier group).
            // A row with no set cell stays empty whatever its neighbours
            // hold, so it reads no neighbour row and skips the chunk digits
            // (the tile itself is always read and its bitmap always written).
            // Tile digit 6 is reduced here too: a row whose digit 6 is 0/1
            // reads its '*' row (729 or 1458 rows on) from the tile while the
            // thread that owns that row may be writing it back reduced, so a
            // bit is seen either as the two Reduce steps left it or final.
            // Either is exact: a cell whose only implicant extensions are in
            // digit 6 has its digit-6 extension prime, set in both; any other
            // extension is cleared through the neighbour group (read from the
            // state, unchanged in this pass) or the chunk digits (read from
            // the row as the steps left it, before this thread changes it).
            const int n_nbr = (MODE == kModeOut) ? S.n_nbr : 0;
            const uint4 *const tile_g = state + 2 * base;
            for (int r = tid; r < kTileRows; r += NT) {
                const uint4 q0 = tile[2 * r], q1 = tile[2 * r + 1];
                uint32_t v[kChunkWords] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                const bool any = ((q0.x | q0.y | q0.z | q0.w) | (q1.x | q1.y | q1.z | q1.w)) != 0u;
                if (any) {
                    uint32_t acc[kChunkWords] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
                    for (int k = 0; k < kMaxNbr; ++k) {
                        if (k < n_nbr) {
                            const uint4 *src = tile_g + S.nbr_off[k] + 2 * r;
                            const uint4 a0 = __ldcg(src), a1 = __ldcg(src + 1);
                            acc[0] |= a0.x; acc[1] |= a0.y; acc[2] |= a0.z; acc[3] |= a0.w;
                            acc[4] |= a1.x; acc[5] |= a1.y; acc[6] |= a1.z; acc[7] |= a1.w;
                        }
                    }
                    constexpr int R6 = (int)pow3(kTileDigits - 1);   // 729 rows per value of digit 6
                    if (r < 2 * R6) {
                        const int rs = r + (r < R6 ? 2 * R6 : R6);   // the row with digit 6 = '*'
                        const uint4 b0 = tile[2 * rs], b1 = tile[2 * rs + 1];
                        acc[0] |= b0.x; acc[1] |= b0.y; acc[2] |= b0.z; acc[3] |= b0.w;
                        acc[4] |= b1.x; acc[5] |= b1.y; acc[6] |= b1.z; acc[7] |= b1.w;
                    }
                    if constexpr (CM != 0) chunk_reduce_p<CM>(v, acc);
#pragma unroll
                    for (int w = 0; w < kChunkWords; ++w) v[w] &= ~acc[w];
                    tile[2 * r] = make_uint4(v[0], v[1], v[2], v[3]);     // only this thread writes row r here
                    tile[2 * r + 1] = make_uint4(v[4], v[5], v[6], v[7]);   // (others may read it: digit 6)
                }
#pragma unroll
                for (int w = 0; w < kChunkWords; ++w) my_count += __popc(v[w]);
            }
        }
        if constexpr (MODE == kModeOut) {
            // ------------------------------------------------ bitmap and list
            // The tile now holds the reduced rows, and the rounds counted
            // them: the tile's count is published first, so that warp 0's
            // look-back overlaps the other warps' regions.  Region r = units
            // 32r .. goes to one warp (taken in turn): count, dense bits into
            // the region's own slots, bitmap store, then the region's pairs
            // in those slots.
            uint32_t xs = my_count;
            for (int off = 16; off > 0; off >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, off);
            if (lane == 0) S.warp_tot[wid] = xs;
            if (tid == 0) S.next_region = 0;
            __syncthreads();
            uint32_t tile_total = 0;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) tile_total += S.warp_tot[w];
            if (tid == 0 && tile_total) atomicAdd(F.count, (unsigned long long)tile_total);
            if ((P.pairs || P.inplace) && wid == 0) {
                const uint64_t T = S.tile;
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
                }
            }
            if (P.inplace) __syncthreads();   // no bitmap word before the look-back
            constexpr int kRegions = (kUnits + 31) / 32;
            for (;;) {
                int r = 0;
                if (lane == 0) r = atomicAdd(&S.next_region, 1);
                r = __shfl_sync(0xffffffffu, r, 0);
                if (r >= kRegions) break;
                const int U0 = 32 * r;
                const int nun = min(32, kUnits - U0);
                const int u = U0 + lane;
                const bool valid = lane < nun;
                uint32_t x[3][kChunkWords];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (valid) {
                        const uint4 q0 = tile[uslot(u, 2 * k)], q1 = tile[uslot(u, 2 * k + 1)];
                        x[k][0] = q0.x; x[k][1] = q0.y; x[k][2] = q0.z; x[k][3] = q0.w;
                        x[k][4] = q1.x; x[k][5] = q1.y; x[k][6] = q1.z; x[k][7] = q1.w;
                    } else {
#pragma unroll
                        for (int w = 0; w < kChunkWords; ++w) x[k][w] = 0u;
                    }
                }
                uint32_t c3 = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int w = 0; w < kChunkWords; ++w) c3 += __popc(x[k][w]);
                // this unit's first pair among the region's (warp scan)
                uint32_t incl = c3;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += y;
                }
                const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
                if (lane == 0) S.rcnt[r] = wtot;
                __syncwarp();   // every lane holds its rows: the region's slots are free
                {
                    uint32_t *const stg = reinterpret_cast<uint32_t *>(tile + uslot(U0, 0));
                    // these units are tile bits 729*U0 ..: words S0 .. of the
                    // bitmap, starting at bit o of word S0.  Unit 'lane' starts
                    // at bit lb0 of stg; its rows follow each other.  A word
                    // shared by two rows of the unit is carried in a register,
                    // one shared with the next unit goes to the next lane.
                    const uint32_t lb0 = o + 729u * (uint32_t)lane;
                    const uint32_t s0 = lb0 & 31;
                    uint32_t *const uw = stg + (lb0 >> 5);
                    uint32_t carry = 0, first = 0;
                    // a region with no set cell writes zero words and stages nothing
                    const bool empty = (wtot == 0u);
                    if (valid && !empty) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const uint32_t sb = s0 + 243u * (uint32_t)k;  // row k's first bit, from uw
                            const uint32_t sh = sb & 31;
                            uint32_t *const rw = uw + (sb >> 5);
                            uint32_t w9[9];
                            w9[0] = (x[k][0] << sh) | carry;
#pragma unroll
                            for (int j = 1; j < 8; ++j) w9[j] = __funnelshift_l(x[k][j - 1], x[k][j], sh);
                            w9[8] = __funnelshift_l(x[k][7], 0u, sh);
                            // the row ends in word 8 (sh >= 13) or word 7
                            const bool nine = sh >= 13u;
                            if (k == 0) first = w9[0];
                            else rw[0] = w9[0];
#pragma unroll
                            for (int j = 1; j < 7; ++j) rw[j] = w9[j];
                            if (nine) rw[7] = w9[7];
                            carry = nine ? w9[8] : w9[7];
                        }
                    }
                    const uint32_t cin = __shfl_up_sync(0xffffffffu, carry, 1);
                    if (valid && !empty) {
                        uw[0] = first | (lane > 0 ? cin : 0u);
                        if (lane == nun - 1) uw[(s0 + 729u) >> 5] = carry;  // the region's last word
                    }
                    __syncwarp();
                    const uint32_t hi_bit = o + 729u * (uint32_t)nun;   // end of these units' bits
                    const uint64_t S0 = W0 + (uint64_t)729 * (uint64_t)(U0 >> 5);
                    if (nun == 32 && ck(P, S0 + 730 <= P.out_alloc_words, S0 + 730)) {
                        // 32 full units: words 1 .. 728 hold only their bits;
                        // word 0 holds them from bit o up, word 729 below bit o.
                        uint32_t *const dstw = out + S0;
                        if (empty) {
#pragma unroll 4
                            for (int j = 1 + lane; j <= 728; j += 32) dstw[j] = 0u;
                        } else {
#pragma unroll 4
                            for (int j = 1 + lane; j <= 728; j += 32) dstw[j] = stg[j];
                        }
                        if (lane == 0) {
                            const uint32_t v0 = empty ? 0u : stg[0];
                            if (o == 0) {
                                dstw[0] = v0;
                            } else {
                                const uint32_t m = 0xffffffffu << o;
                                atomicAnd(dstw, v0 | ~m);
                                atomicOr(dstw, v0 & m);
                            }
                        } else if (lane == 1 && o != 0) {
                            const uint32_t m = (1u << o) - 1u;
                            const uint32_t v1 = empty ? 0u : stg[729];
                            atomicAnd(dstw + 729, v1 | ~m);
                            atomicOr(dstw + 729, v1 & m);
                        }
                    } else {
                        const int nw = (int)((hi_bit + 31u) >> 5);
                        for (int j = lane; j < nw; j += 32) {
                            // bits of word j owned by these units: [lo, hi)
                            const int lo = (j == 0) ? (int)o : 0;
                            const int hi = (int)min(hi_bit - 32u * (uint32_t)j, 32u);
                            const uint64_t wi = S0 + (uint64_t)j;
                            const int hi2 = (last_tile && wi == P.out_words - 1) ? 32 : hi;  // bits past 3^n are 0
                            if (hi2 <= lo) continue;
                            if (!ck(P, wi < P.out_alloc_words, wi)) continue;
                            const uint32_t val = empty ? 0u : stg[j];
                            uint32_t *dst = out + wi;
                            if (lo == 0 && hi2 == 32) {
                                *dst = val;
                            } else {
                                const uint32_t m = (hi2 == 32 ? 0xffffffffu : ((1u << hi2) - 1u)) & (0xffffffffu << lo);
                                atomicAnd(dst, val | ~m);
                                atomicOr(dst, val & m);
                            }
                        }
                    }
                    __syncwarp();
                    // (mask, value) pairs of these units, in rho order, in the
                    // slots just freed; copied to the list after the look-back
                    if (P.pairs) {
                        if (wtot <= 12u * (uint32_t)nun) {   // a unit's 96 bytes hold 12 pairs
                            if (valid && c3) {
                                uint2 *pr = reinterpret_cast<uint2 *>(stg) + (incl - c3);
                                const uint32_t code = S.code[u];
                                const uint32_t nmask = P.nmask;
                                // cube bits: tile digits 1..6 are the unit digits
                                const uint32_t um = S.tile_mask | ((code & 0x3fu) << (kChunkDigits + 1));
                                const uint32_t uv = S.tile_val | (((code >> 8) & 0x3fu) << (kChunkDigits + 1));
                                // lanes walk their own row words; a word's
                                // bits come out in rho order
#pragma unroll
                                for (int k = 0; k < 3; ++k) {
                                    // tile digit 0 = k
                                    const uint32_t rm = um | (k != 2 ? 1u << kChunkDigits : 0u);
                                    const uint32_t rv = uv | (k == 1 ? 1u << kChunkDigits : 0u);
#pragma unroll
                                    for (int w = 0; w < kChunkWords; ++w) {
                                        uint32_t bits = x[k][w];
                                        while (bits) {
                                            const int bb = __ffs(bits) - 1;
                                            bits &= bits - 1;
                                            const uint32_t c5 = S.c5[32 * w + bb];
                                            *pr++ = make_uint2((rm | (c5 & 0x1fu)) & nmask, (rv | (c5 >> 8)) & nmask);
                                        }
                                    }
                                }
                            }
                        } else if (lane == 0) {
                            S.overflow = 1;
                        }
                    }
                }
            }
        }

        if constexpr (MODE == kModeOut) {
            if (last_tile)
                for (uint64_t w = P.out_words + tid; w < P.out_alloc_words; w += NT) out[w] = 0u;
            if (P.pairs) {
                __syncthreads();   // every region's pairs are in place, the look-back is done
                const uint64_t cap = P.cap;
                if (S.list_ok && !S.overflow) {
                    // each region's pairs to the list, region r = units 32r ..
                    constexpr int kRegions = (kUnits + 31) / 32;
                    static_assert(kRegions <= 32, "one lane per region");
                    const uint32_t rc = (lane < kRegions) ? S.rcnt[lane] : 0u;
                    uint32_t ri = rc;
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, ri, off);
                        if (lane >= off) ri += y;
                    }
                    for (int r = wid; r < kRegions; r += NT / 32) {
                        const uint32_t nr = __shfl_sync(0xffffffffu, rc, r);
                        const uint32_t off = __shfl_sync(0xffffffffu, ri, r) - nr;
                        const uint2 *src = reinterpret_cast<const uint2 *>(tile + uslot(32 * r, 0));
                        const unsigned long long k0 = S.excl + off;
                        for (uint32_t i = lane; i < nr; i += 32)
                            if (k0 + i < cap) P.pairs[k0 + i] = src[i];
                    }
                } else if (S.list_ok) {
                    // a region had more pairs than its slots hold: list this
                    // tile from the bitmap it has written (rows 9t .. 9t+8
                    // belong to thread t < 243)
                    emit_from_bitmap(P, S, out, base);
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

// --------------------------------------- last Merge pass and Reduce passes
// Whole rows: a tile's 3^7 rows (inner digits 0..B-1, then group digits B..6
// = high digits a..a+K-1) in shared memory, row-major with no swizzle
// (dqmc_steps.cuh).  MERGE (the last Merge pass): the rows whose group digits
// are 0/1 come in and the group digits are merged kMrDigits at a time; else
// every row comes in.  Then the group digits are reduced kMrDigits at a time
// (one barrier per step), each row's chunk digits in registers, and the rows
// go out from their threads when a group digit's rows are less than 1 MB
// apart, else back in place and out with consecutive lanes on consecutive
// 16-byte pieces (STAGE).  kMrDigits per step, mr_threads per CTA.
// Threads per CTA and digits per step (measured at n = 24: the last Merge
// pass 14.70 ms with 384 threads and 2 digits, 14.81 with 384 and 3; the
// middle Reduce pass 14.78 ms with 256 and 2, 17.26 with 384 and 3).
template <bool MERGE> constexpr int mr_threads() { return MERGE ? 384 : 256; }
constexpr int kMrDigits = 2;

template <int K, int B, int CM, bool STAGE, bool MERGE>
__global__ void __launch_bounds__(mr_threads<MERGE>(), 3) mr_pass_kernel(const __grid_constant__ PassParams P)
{
    constexpr int HL = K + B;           // tile digits
    constexpr int NT = mr_threads<MERGE>();
    constexpr int R = kTileRows;
    constexpr int RE = (int)pow3(B);   // inner rows per group-digit value
    constexpr int NB = 1 << K;
    static_assert(HL == kTileDigits && B >= 1, "tiles are 3^7 rows with at least one inner digit");
    extern __shared__ uint4 tile[];
    __shared__ PassShared S;
    const int tid = threadIdx.x;
    const FnBufs F = fn_bufs(P);
    if (tid == 0) decode_tile0<false>(P, S, F.tile);
    __syncthreads();
    const uint64_t base = S.base, w_g = P.w_g, state_rows = P.state_rows;
    uint4 *const state = F.state;
    // tile row e + RE*g (e: inner digits, g: group digits) is state row base + e + g*w_g
    auto state_row = [&](int ri) -> uint64_t {
        const int g = ri / RE, e = ri - g * RE;
        return base + (uint64_t)e + (uint64_t)g * w_g;
    };

    if constexpr (MERGE) {
        // the rows whose group digits are all 0/1
        for (int p = tid; p < NB * RE * 2; p += NT) {
            const int h = p & 1, q = p >> 1;
            const int gb = q / RE, e = q - gb * RE;
            const int g = (int)__ldg(&g_tab.sp3[gb]);
            const uint64_t row = base + (uint64_t)e + (uint64_t)g * w_g;
            if (!ck(P, row < state_rows, row)) continue;
            cp_async16p(&tile[2 * (e + RE * g) + h], &state[2 * row + h]);
        }
    } else {
        for (int p = tid; p < 2 * R; p += NT) {
            const uint64_t row = state_row(p >> 1);
            if (!ck(P, row < state_rows, row)) continue;
            cp_async16p(&tile[p], &state[2 * row + (p & 1)]);
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    const SubSync sync{1, NT, true};
    __syncthreads();

    if constexpr (MERGE) merge_all<HL, B, kMrDigits>(tile, tid, NT, sync);
    reduce_all<HL, B, kMrDigits>(tile, tid, NT, sync);

    // chunk digits, then out
    for (int ri = tid; ri < R; ri += NT) {
        const uint4 q0 = tile[2 * ri], q1 = tile[2 * ri + 1];
        uint32_t v[kChunkWords] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        uint32_t acc[kChunkWords] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        chunk_reduce_p<CM>(v, acc);
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) v[w] &= ~acc[w];
        if constexpr (STAGE) {
            // only this thread reads or writes row ri in this loop
            tile[2 * ri] = make_uint4(v[0], v[1], v[2], v[3]);
            tile[2 * ri + 1] = make_uint4(v[4], v[5], v[6], v[7]);
        } else {
            const uint64_t row = state_row(ri);
            if (!ck(P, row < state_rows, row)) continue;
            state[2 * row] = make_uint4(v[0], v[1], v[2], v[3]);
            state[2 * row + 1] = make_uint4(v[4], v[5], v[6], v[7]);
        }
    }
    if constexpr (STAGE) {
        __syncthreads();
        for (int p = tid; p < 2 * R; p += NT) {
            const uint64_t row = state_row(p >> 1);
            if (!ck(P, row < state_rows, row)) continue;
            state[2 * row + (p & 1)] = tile[p];
        }
    }
}

template <typename Kern>
static cudaError_t launch_tiles(Kern kern, size_t smem, const PassParams &p, uint64_t tiles, cudaStream_t stream,
                               int threads = kThreads)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (tiles == 0) return cudaSuccess;
    if (tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)tiles, threads, smem, stream>>>(p);
    return cudaGetLastError();
}

// A group digit's rows lie 3^a rows apart in the state.  When that is 1 MB or
// more, a warp storing one row per thread would touch many pages, so the row
// passes put their rows back in shared memory and store the tile with
// consecutive lanes on consecutive 16-byte pieces (STAGE) instead.
constexpr uint64_t kStageStrideBytes = 1ull << 20;

template <int K, int B, int LOAD, int MODE, int CM>
static cudaError_t launch_unit(const PassParams &p, uint64_t tiles, cudaStream_t stream)
{
    return launch_tiles(unit_pass_kernel<K, B, LOAD, MODE, CM>, unit_smem<B == 0>(), p, tiles, stream,
                        unit_threads<MODE>());
}

template <int K, int CM, bool MERGE>
static cudaError_t launch_mr(const PassParams &p, uint64_t tiles, cudaStream_t stream)
{
    constexpr int B = kTileDigits - K;
    const size_t smem = (size_t)kTileRows * kChunkBytes;
    constexpr int NT = mr_threads<MERGE>();
    if (p.w_g * kChunkBytes >= kStageStrideBytes)
        return launch_tiles(mr_pass_kernel<K, B, CM, true, MERGE>, smem, p, tiles, stream, NT);
    return launch_tiles(mr_pass_kernel<K, B, CM, false, MERGE>, smem, p, tiles, stream, NT);
}

template <int CM, bool MERGE>
static cudaError_t dispatch_mr(int K, const PassParams &p, uint64_t tiles, cudaStream_t s)
{
    switch (K) {
    case 1: return launch_mr<1, CM, MERGE>(p, tiles, s);
    case 2: return launch_mr<2, CM, MERGE>(p, tiles, s);
    case 3: return launch_mr<3, CM, MERGE>(p, tiles, s);
    case 4: return launch_mr<4, CM, MERGE>(p, tiles, s);
    case 5: return launch_mr<5, CM, MERGE>(p, tiles, s);
    case 6: return launch_mr<6, CM, MERGE>(p, tiles, s);
    }
    return cudaErrorInvalidValue;
}

template <int LOAD, int MODE, int CM>
static cudaError_t dispatch_group(int K, const PassParams &p, uint64_t tiles, cudaStream_t s)
{
    switch (K) {
    case 1: return launch_unit<1, 6, LOAD, MODE, CM>(p, tiles, s);
    case 2: return launch_unit<2, 5, LOAD, MODE, CM>(p, tiles, s);
    case 3: return launch_unit<3, 4, LOAD, MODE, CM>(p, tiles, s);
    case 4: return launch_unit<4, 3, LOAD, MODE, CM>(p, tiles, s);
    case 5: return launch_unit<5, 2, LOAD, MODE, CM>(p, tiles, s);
    case 6: return launch_unit<6, 1, LOAD, MODE, CM>(p, tiles, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_super(const Plan &plan, const void *d_on, const void *d_dc, void *d_state, uint32_t *d_bitmap,
                         unsigned long long *d_count, uint32_t *d_pairs, uint64_t cap, void *d_ctrl,
                         cudaStream_t stream, int first, int last, const BatchArgs *batch, uint32_t tt_invert,
                         bool inplace)
{
    const CtrlLayout cl = ctrl_layout(plan);
    cudaError_t e = cudaSuccess;
    if (batch) {
        if (batch->nfun == 0) return cudaSuccess;
        d_pairs = nullptr;
        cap = 0;
    }
    if (first == 0) {
        if (!batch) e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_ctrl, 0, cl.bytes, stream);
        if (e != cudaSuccess) return e;
    }
    PassParams a{};
    a.on = static_cast<const uint32_t *>(d_on);
    a.dc = static_cast<const uint32_t *>(d_dc);
    a.inv = tt_invert;
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
    a.inplace = (inplace && !batch) ? 1 : 0;
    a.H = plan.H;
    if (batch) {
        a.bfn = batch->fn;
        a.btt_off = batch->tt_off;
        a.bdc_off = batch->dc_off;
        a.bbm_off = batch->bm_off;
        a.barena = batch->arena;
        a.bbitmaps = batch->bitmaps;
        a.bcount = batch->count;
        a.bstate_stride = 2 * plan.state_rows;
    }
    for (int i = first; i < last; ++i) {
        const SuperPassDesc &sp = plan.sps[i];
        const PhaseDesc &ph = sp.ph[0];
        a.w_g = pow3(ph.a);
        a.slot = sp.slot;
        a.fix = sp.sb;
        a.nbr_k = ph.out ? ph.nbr_K : 0;   // the neighbour group is the first nbr_K fixed digits (7 ..)
        a.tiles_per_fn = (uint32_t)sp.n_sb;
        const uint64_t tiles = sp.n_sb * (batch ? batch->nfun : 1u);
        if (ph.load == kLoadTT)
            e = (ph.K == kTileDigits && ph.a == 0)
                    ? launch_tiles(tt_pass_kernel, (size_t)kTileRows * kChunkBytes, a, tiles, stream)
                    : cudaErrorInvalidValue;
        else if (ph.out && (ph.K != kTileDigits || ph.a != 0 || ph.nbr_K > kMaxNbr ||
                            (ph.nbr_K && ph.nbr_a != kTileDigits)))
            e = cudaErrorInvalidValue;
        else if (ph.out && ph.chunk_mask == 0x18)
            e = launch_unit<kTileDigits, 0, kLoadFull, kModeOut, 0x18>(a, tiles, stream);
        else if (ph.out && ph.chunk_mask == 0x1f)
            e = launch_unit<kTileDigits, 0, kLoadFull, kModeOut, 0x1f>(a, tiles, stream);
        else if (ph.out)
            e = cudaErrorInvalidValue;
        else if (ph.merge && ph.reduce && ph.chunk_mask == 0)
            e = dispatch_mr<0, true>(ph.K, a, tiles, stream);
        else if (ph.merge && ph.reduce && ph.chunk_mask == 0x07)
            e = dispatch_mr<0x07, true>(ph.K, a, tiles, stream);
        else if (ph.merge && !ph.reduce && ph.chunk_mask == 0)
            e = dispatch_group<kLoadSparse, kModeMerge, 0>(ph.K, a, tiles, stream);
        else if (!ph.merge && ph.reduce && ph.chunk_mask == 0x07)
            e = dispatch_mr<0x07, false>(ph.K, a, tiles, stream);
        else if (!ph.merge && ph.reduce && ph.chunk_mask == 0)
            e = dispatch_mr<0, false>(ph.K, a, tiles, stream);
        else
            e = cudaErrorInvalidValue;  // not a pass the plan makes
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dqmc
