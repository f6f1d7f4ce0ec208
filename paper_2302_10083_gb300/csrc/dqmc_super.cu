// dqmc_super.cu -- the sweep for n >= 13: persistent "super-pass" kernels.
//
// Algorithm 3 of DenseQMC (arXiv 2302.10083, Section 4.1) on the padded
// device state (row = 5 chunk digits in one 32-byte sector, see
// dqmc_chunk.cuh).  One launch runs one super-pass: CTAs take tickets from a
// global counter; a ticket names (phase, super-block, tile).  A tile is at
// most 729 rows: group digits a..a+K-1 and inner digits 0..B-1 vary inside it,
// the other digits are fixed.  Phase p of a super-block starts after every
// tile of phase p-1 of that block has signalled, so a block's rows stay in L2
// between phases and only its first read and last write reach HBM.  Tickets
// are issued in a software pipeline (phase 0 of block group g, phase 1 of
// group g-1, ...), so a tile only ever waits for tiles with smaller tickets,
// which running CTAs already hold: no deadlock, whatever the grid size.
//
// Per tile:
//   load   truth-table words (first pass), the rows whose group digits are
//          0/1 (Merge input), or all rows, into shared memory (cp.async);
//   Merge  the group digits one after another (Merge of Section 4.1:
//          '*'-row = 0-row AND 1-row);
//   Reduce the group digits (and chosen chunk digits) all from the tile as it
//          is after the Merge: a row loses the bits whose '*'-neighbour in any
//          reduced digit is set.  Grouping digits this way gives the same
//          final set as the paper's digit-by-digit in-place loop: a cube with
//          an implicant one-digit extension is cleared in the first phase that
//          holds such a digit (the extension is still set then, or an earlier
//          phase would hold a digit of that kind), and primes are never cleared;
//   store  rows back to the state, or, in the bitmap phase, the dense bitmap
//          (funnel-shifted rows combined in shared memory), the count, and
//          the (mask, value) list placed by a decoupled look-back over the
//          bitmap tiles in rho order.
#include <cstdio>
#include <cstdlib>

#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"

namespace dqmc {

static __constant__ MaskTable kMasksSP = make_mask_table();

struct Pow3Table {
    uint64_t p[27];
    uint64_t magic[7];   // ceil(2^32 / 3^k): x / 3^k = (x * magic) >> 32 for x < 2^16
};
__host__ __device__ constexpr Pow3Table make_pow3_table()
{
    Pow3Table t{};
    uint64_t v = 1;
    for (int i = 0; i < 27; ++i) {
        t.p[i] = v;
        v *= 3u;
    }
    for (int k = 0; k < 7; ++k) t.magic[k] = ((1ull << 32) + t.p[k] - 1) / t.p[k];
    return t;
}
static __constant__ Pow3Table kP3 = make_pow3_table();

__device__ __forceinline__ uint32_t div_pow3(uint32_t x, int k)
{
    return (uint32_t)(((uint64_t)x * kP3.magic[k]) >> 32);
}

struct SweepArgs {
    const uint32_t *on;
    const uint32_t *dc;
    uint4 *state;
    uint32_t *out;
    unsigned long long *count;
    uint2 *pairs;               // null: no list
    uint64_t cap;
    uint32_t *ctrl;             // control block (uint32 view)
    unsigned long long *status; // look-back slots
    uint64_t total_rows;        // 3^H
    uint64_t out_words, out_alloc_words;
    uint64_t wait_ns;           // bound of every device wait
    uint32_t nmask;             // (1 << n) - 1
    int H;
    // buffer sizes for the bounds checks
    uint64_t state_rows, tt_words, out_tiles, ctrl_words;
    int l2_discard;             // drop dead state lines from L2 in the bitmap phase
    unsigned long long *timing; // per-phase cycle sums of the tile segments (null: off)
};

// Bounds checks: every global and shared index is compared with its buffer
// before the access; a bad one is reported (printf, error word kErrBounds) and
// the access is skipped, so an index error cannot fault the GPU.
enum CheckWhat : int { kChkTT = 1, kChkTile, kChkState, kChkDiscard, kChkCtrl, kChkStatus, kChkStage, kChkOut,
                       kChkTable };
template <bool kCheck>
__device__ __forceinline__ bool ck(const SweepArgs &A, bool cond, int what, uint64_t idx, uint64_t lim)
{
    if constexpr (!kCheck) {
        return true;
    } else {
        if (cond) return true;
        atomicCAS(A.ctrl, 0u, kErrBounds);
        if (atomicAdd(A.ctrl + kCtrlTickets, 1u) < 16u)   // spare ticket slot counts reports
            printf("dqmc checked: what=%d idx=%llu lim=%llu block=%d thread=%d\n", what,
                   (unsigned long long)idx, (unsigned long long)lim, (int)blockIdx.x, (int)threadIdx.x);
        return false;
    }
}

constexpr int kSThreads = 256;
constexpr int kTimeSegs = 8;  // ticket+wait, load, merge, reduce, store/out, signal, tiles, (spare)
constexpr int kRounds = (kTileRowsMax + kSThreads - 1) / kSThreads;  // 3
constexpr unsigned long long kFlagA = 1ull << 62, kFlagP = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ int slot_s(int r, int h) { return 2 * r + (h ^ ((r >> 2) & 1)); }

__device__ __forceinline__ void cp_async16s(void *smem_dst, const void *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void discard_l2(const void *p)
{
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Mixed-radix decode of x over a list of fixed digits (first entry least significant).
__device__ __forceinline__ void decode_fixed(const FixedDigits &f, uint64_t x, uint64_t &row, uint64_t &tt)
{
    for (int i = 0; i < f.n; ++i) {
        uint64_t d;
        if (f.r[i] == 2) {
            d = x & 1u;
            x >>= 1;
        } else {
            const uint64_t q = x / 3u;
            d = x - 3u * q;
            x = q;
        }
        row += d * f.w3[i];
        tt += d * f.w2[i];
    }
}

__device__ __forceinline__ uint64_t total_tickets(const SuperPassDesc &sp)
{
    uint64_t t = 0;
    for (int p = 0; p < sp.nph; ++p) t += (uint64_t)sp.ph[p].tiles * sp.n_sb;
    return t;
}

// Tickets issued before pipeline step k: phase p runs block group k - p at step k.
__device__ __forceinline__ uint64_t step_offset(const SuperPassDesc &sp, uint64_t k)
{
    uint64_t off = 0;
    for (int p = 0; p < sp.nph; ++p) {
        if (k <= (uint64_t)p) continue;
        uint64_t nsb = (k - p) * sp.window;
        if (nsb > sp.n_sb) nsb = sp.n_sb;
        off += nsb * sp.ph[p].tiles;
    }
    return off;
}

__device__ __forceinline__ void decode_ticket(const SuperPassDesc &sp, uint64_t ticket, int &phase, uint64_t &sb,
                                              uint32_t &tile)
{
    const uint64_t groups = (sp.n_sb + sp.window - 1) / sp.window;
    uint64_t lo = 0, hi = groups + sp.nph - 1;  // step_offset(hi) = total > ticket
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) / 2;
        if (step_offset(sp, mid) <= ticket) lo = mid;
        else hi = mid;
    }
    uint64_t rem = ticket - step_offset(sp, lo);
    for (int p = 0; p < sp.nph; ++p) {
        if (lo < (uint64_t)p) break;
        const uint64_t g = lo - p;
        if (g >= groups) continue;
        uint64_t nsb = sp.n_sb - g * sp.window;
        if (nsb > sp.window) nsb = sp.window;
        const uint64_t cnt = nsb * sp.ph[p].tiles;
        if (rem < cnt) {
            phase = p;
            sb = g * sp.window + rem / sp.ph[p].tiles;
            tile = (uint32_t)(rem % sp.ph[p].tiles);
            return;
        }
        rem -= cnt;
    }
    phase = 0;  // unreachable for ticket < total
    sb = 0;
    tile = 0;
}

// Reduce over the chunk digits selected by mask (all read from v).
__device__ __forceinline__ void chunk_reduce_masked(const uint32_t (&v)[kChunkWords], uint32_t (&acc)[kChunkWords],
                                                    int mask)
{
    static_for<0, kChunkDigits>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int d = (int)pow3(i);
        if ((mask >> i) & 1) {
            uint32_t y[kChunkWords];
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) y[w] = v[w] & kMasksSP.m[kChunkDigits][i][2][w];
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) acc[w] |= shr_word<d>(y, w) | shr_word<2 * d>(y, w);
        }
    });
}

__device__ __forceinline__ void chunk_from_word(uint32_t x, uint32_t (&v)[kChunkWords])
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
            nv[w] = v[w] | (shl_word<d>(v, w) & shl_word<2 * d>(v, w) & kMasksSP.m[kChunkDigits][i][2][w]);
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) v[w] = nv[w];
    });
}

__device__ __forceinline__ bool wait_counter(const SweepArgs &A, const uint32_t *ctr, uint32_t need)
{
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (ld_acquire(ctr) >= need) return true;
        if (*reinterpret_cast<volatile uint32_t *>(A.ctrl) != 0) return false;
        if (globaltimer() - t0 > A.wait_ns) {
            atomicCAS(A.ctrl, 0u, kErrTimeout);
            return false;
        }
        __nanosleep(128);
    }
}

// Decoupled look-back over the bitmap tiles (warp 0).  Returns the number of
// primes in tiles 0..T-1; publishes this tile's inclusive prefix.
template <bool kCheck>
__device__ __forceinline__ unsigned long long lookback(const SweepArgs &A, uint64_t T, unsigned long long count,
                                                       bool &ok)
{
    if (!ck<kCheck>(A, T < A.out_tiles, kChkStatus, T, A.out_tiles)) {
        ok = false;
        return 0;
    }
    const int lane = threadIdx.x & 31;
    ok = true;
    // (this tile's aggregate, or for T = 0 its prefix, is already published)
    if (T == 0) return 0;
    unsigned long long excl = 0;
    long long j = (long long)T - 1;
    const uint64_t t0 = globaltimer();
    for (;;) {
        const long long idx = j - lane;
        const unsigned long long s = (idx >= 0) ? ld_volatile_u64(&A.status[idx]) : kFlagP;
        const unsigned flag = (unsigned)(s >> 62);
        if (__any_sync(0xffffffffu, flag == 0)) {
            bool stop = false;
            if (lane == 0) {
                if (*reinterpret_cast<volatile uint32_t *>(A.ctrl) != 0) stop = true;
                else if (globaltimer() - t0 > A.wait_ns) {
                    atomicCAS(A.ctrl, 0u, kErrTimeout);
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
    if (lane == 0) atomicExch(&A.status[T], kFlagP | (excl + count));
    return excl;
}

struct TileShared {
    uint16_t sp3[64];               // spread3 of 6-bit numbers
    uint8_t has_star[kTileRowsMax]; // group index has a '*' digit
    uint8_t m6[kTileRowsMax], v6[kTileRowsMax];  // mask / value bits of the 6 low high digits
    uint8_t t5m[243], t5v[243];     // mask / value bits of the 5 chunk digits
    uint32_t warp_tot[kRounds][kSThreads / 32];  // per round: inclusive warp totals of row counts
    // the current tile, decoded by thread 0
    uint64_t base, ttb, sb;
    unsigned long long excl;        // primes in the bitmap tiles before this one
    uint32_t tile_mask, tile_val;   // mask / value bits of the digits above the bitmap tile
    int p, abort, stop, list_ok;
    unsigned long long tsum[kMaxPhases][8];  // timing sums (thread 0)
};

// Mixed-radix decode of x over a list of fixed digits (first entry least
// significant), 32-bit digit arithmetic.
__device__ __forceinline__ void decode_fixed32(const FixedDigits &f, uint32_t x, uint64_t &row, uint64_t &tt)
{
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
        row += (uint64_t)d * f.w3[i];
        tt += (uint64_t)d * f.w2[i];
    }
}

// Ticket -> (phase, super-block, tile); false for an empty ticket.
__device__ __forceinline__ bool decode_ticket_step(const SuperPassDesc &sp, uint32_t ticket, int &phase, uint32_t &sb,
                                                   uint32_t &tile)
{
    const uint32_t step = ticket / sp.step_size;
    uint32_t r = ticket - step * sp.step_size;
    int p = sp.nph - 1;
    while (p > 0 && r < sp.ph_off[p]) --p;
    r -= sp.ph_off[p];
    if (step < (uint32_t)p) return false;
    const uint32_t g = step - p;
    if (g >= sp.groups) return false;
    const uint32_t tiles = sp.ph[p].tiles;
    const uint32_t sbl = r / tiles;
    const uint64_t sb64 = (uint64_t)g * sp.window + sbl;
    if (sb64 >= sp.n_sb) return false;
    phase = p;
    sb = (uint32_t)sb64;
    tile = r - sbl * tiles;
    return true;
}

// The kernel bounds-checks every global and shared index (ck): an index
// outside its buffer is reported and the access skipped, so the kernel cannot
// fault on one.
template <bool kCheck>
__global__ void __launch_bounds__(kSThreads, 3)
super_pass_kernel(const __grid_constant__ SuperPassDesc sp_param, const __grid_constant__ SweepArgs A)
{
    constexpr uint32_t kSlots = 2 * kTileRowsMax;
    extern __shared__ uint4 tile[];
    __shared__ TileShared S;
    // The pass descriptor is read with run-time indexes (phase, digit): one
    // copy per CTA in shared memory, indexed there, not in parameter space.
    __shared__ SuperPassDesc s_sp;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    {
        static_assert(sizeof(SuperPassDesc) % 4 == 0, "word copy");
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&sp_param);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&s_sp);
        for (int i = tid; i < (int)(sizeof(SuperPassDesc) / 4); i += kSThreads) dst[i] = src[i];
    }
    for (int i = tid; i < 64; i += kSThreads) {
        uint32_t r = 0, w = 1, x = i;
        while (x) {
            if (x & 1) r += w;
            x >>= 1;
            w *= 3;
        }
        S.sp3[i] = (uint16_t)r;
    }
    for (int i = tid; i < kTileRowsMax; i += kSThreads) {
        int q = i, star = 0, m = 0, v = 0;
        for (int d = 0; d < 6; ++d) {
            const int dg = q % 3;
            q /= 3;
            if (dg == 2) star = 1;
            else m |= 1 << d;
            if (dg == 1) v |= 1 << d;
        }
        S.has_star[i] = (uint8_t)star;
        S.m6[i] = (uint8_t)m;
        S.v6[i] = (uint8_t)v;
    }
    for (int i = tid; i < 243; i += kSThreads) {
        int q = i, m = 0, v = 0;
        for (int d = 0; d < 5; ++d) {
            const int dg = q % 3;
            q /= 3;
            if (dg != 2) m |= 1 << d;
            if (dg == 1) v |= 1 << d;
        }
        S.t5m[i] = (uint8_t)m;
        S.t5v[i] = (uint8_t)v;
    }
    __syncthreads();
    const SuperPassDesc &sp = s_sp;

    const int nph = sp.nph;
    const uint64_t total = (uint64_t)sp.n_steps * sp.step_size;
    uint32_t *const tickets = A.ctrl + 1;
    uint32_t *const done = A.ctrl + sp.done_off;
    const bool slot_ok = ck<kCheck>(A, sp.slot < kCtrlTickets - 1, kChkCtrl, sp.slot, kCtrlTickets - 1);
    const int slot = sp.slot;
    // Thread 0 holds the next ticket: it is taken while the current tile runs.
    uint32_t next = 0xffffffffu;
    if (tid == 0 && slot_ok) next = atomicAdd(tickets + slot, 1u);
    // Optional timing (thread 0): cycles per tile segment, summed per phase.
    const bool timing = (A.timing != nullptr);
    unsigned long long(&tsum)[kMaxPhases][kTimeSegs] = S.tsum;
    if (tid == 0)
        for (int q = 0; q < kMaxPhases; ++q)
            for (int g = 0; g < kTimeSegs; ++g) tsum[q][g] = 0;
    unsigned long long tcur = timing ? clock64() : 0ull;
    int tph = 0;
#define DQMC_TSEG(seg)                                                       \
    do {                                                                     \
        if (timing && tid == 0) {                                            \
            const unsigned long long now_ = clock64();                       \
            tsum[tph][(seg)] += now_ - tcur;                                 \
            tcur = now_;                                                     \
        }                                                                    \
    } while (0)

    for (;;) {
        if (tid == 0) {
            int stop = 0, valid = 0, abort = 0;
            for (;;) {
                const uint32_t ticket = next;
                if ((uint64_t)ticket >= total) {
                    stop = 1;
                    break;
                }
                next = atomicAdd(tickets + slot, 1u);
                int p;
                uint32_t sb, t;
                if (!decode_ticket_step(sp, ticket, p, sb, t)) continue;  // empty ticket
                uint64_t base = 0, ttb = 0;
                decode_fixed32(sp.sb, sb, base, ttb);
                decode_fixed32(sp.ph[p].fix, t, base, ttb);
                S.p = p;
                S.sb = sb;
                S.base = base;
                S.ttb = ttb;
                if (p > 0) {
                    const uint64_t di = sp.done_off + (uint64_t)sb * nph + (p - 1);
                    abort = !ck<kCheck>(A, di < A.ctrl_words, kChkCtrl, di, A.ctrl_words) ||
                            !wait_counter(A, done + (uint64_t)sb * nph + (p - 1), sp.ph[p - 1].tiles);
                    __threadfence();
                }
                valid = 1;
                break;
            }
            S.stop = stop;
            S.abort = abort;
        }
        __syncthreads();
        if (S.stop) break;
        const int p = S.p;
        tph = p;
        DQMC_TSEG(0);  // ticket, decode, dependency wait
        const uint64_t sb = S.sb;
        const uint64_t base = S.base, ttb = S.ttb;
        const bool signal = (p < nph - 1);   // later phases of this block wait for this tile
        if (S.abort) {
            __syncthreads();
            if (tid == 0 && signal) atomicAdd(done + sb * nph + p, 1u);
            continue;
        }
        // this tile's phase, in registers
        const int K = sp.ph[p].K, B = sp.ph[p].B;
        const int load = sp.ph[p].load, merge = sp.ph[p].merge, reduce = sp.ph[p].reduce;
        const int chunk_mask = sp.ph[p].chunk_mask, out = sp.ph[p].out;
        const uint32_t RE = (uint32_t)kP3.p[B];
        const uint32_t R = (uint32_t)kP3.p[K] * RE;
        const uint32_t NB = 1u << K;
        const uint64_t w_g = kP3.p[sp.ph[p].a];
        uint4 *const state = A.state;
        const uint64_t state_rows = A.state_rows;

        // ---------------------------------------------------------------- load
        if (load == kLoadTT) {
            const uint32_t *on = A.on, *dc = A.dc;
            for (uint32_t gb = tid; gb < NB; gb += kSThreads) {
                if (!ck<kCheck>(A, ttb + gb < A.tt_words, kChkTT, ttb + gb, A.tt_words)) continue;
                if (!ck<kCheck>(A, gb < 64, kChkTable, gb, 64)) continue;
                uint32_t x = __ldg(on + ttb + gb);
                if (dc) x |= __ldg(dc + ttb + gb);
                uint32_t v[kChunkWords];
                chunk_from_word(x, v);
                const int r = S.sp3[gb];
                if (!ck<kCheck>(A, (uint32_t)slot_s(r, 1) < kSlots && (uint32_t)slot_s(r, 0) < kSlots, kChkTile, r,
                                kTileRowsMax))
                    continue;
                tile[slot_s(r, 0)] = make_uint4(v[0], v[1], v[2], v[3]);
                tile[slot_s(r, 1)] = make_uint4(v[4], v[5], v[6], v[7]);
            }
        } else {
            const bool sparse = (load == kLoadSparse);
            const uint32_t npc = (sparse ? NB * RE : R) * 2;
            for (uint32_t pc = tid; pc < npc; pc += kSThreads) {
                const int h = pc & 1;
                const uint32_t ri = pc >> 1;
                const uint32_t q = div_pow3(ri, B);
                const uint32_t e = ri - q * RE;
                if (!ck<kCheck>(A, !sparse || q < 64, kChkTable, q, 64)) continue;
                const uint32_t g = sparse ? S.sp3[q] : q;
                const uint32_t srow = g * RE + e;
                const uint64_t row = base + e + (uint64_t)g * w_g;
                if (!ck<kCheck>(A, (uint32_t)slot_s(srow, h) < kSlots, kChkTile, srow, kTileRowsMax)) continue;
                if (!ck<kCheck>(A, row < state_rows, kChkState, row, state_rows)) continue;
                cp_async16s(&tile[slot_s(srow, h)], &state[2 * row + h]);
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        }
        __syncthreads();
        DQMC_TSEG(1);  // load
        if (out && A.l2_discard) {
            // The bitmap phase is the last reader of these rows: drop their
            // lines from L2 without writing them back (off unless
            // DQMC_L2_DISCARD=1).
            const uint64_t b0 = base * kChunkBytes, b1 = (base + R) * kChunkBytes;
            const uint64_t l0 = (b0 + 127) / 128, l1 = b1 / 128;
            const char *st = reinterpret_cast<const char *>(state);
            for (uint64_t l = l0 + tid; l < l1; l += kSThreads)
                if (ck<kCheck>(A, (l + 1) * 128 <= state_rows * kChunkBytes, kChkDiscard, l, state_rows / 4))
                    discard_l2(st + l * 128);
        }

        // --------------------------------------------------------------- Merge
        if (merge) {
            uint32_t dj = 1;
            for (int j = 0; j < K; ++j) {
                const uint32_t items = dj * (1u << (K - 1 - j)) * RE * 2;
                for (uint32_t it = tid; it < items; it += kSThreads) {
                    const int h = it & 1;
                    const uint32_t r = it >> 1;
                    const uint32_t q = div_pow3(r, B);
                    const uint32_t e = r - q * RE;
                    const uint32_t hb = div_pow3(q, j);
                    const uint32_t lo = q - hb * dj;
                    if (!ck<kCheck>(A, hb < 64, kChkTable, hb, 64)) continue;
                    const uint32_t g = lo + 3 * dj * S.sp3[hb];
                    const int r0 = g * RE + e;
                    if (!ck<kCheck>(A, (uint32_t)(r0 + 2 * dj * RE) < R, kChkTile, r0 + 2 * dj * RE, R)) continue;
                    const uint4 s0 = tile[slot_s(r0, h)];
                    const uint4 s1 = tile[slot_s(r0 + dj * RE, h)];
                    tile[slot_s(r0 + 2 * dj * RE, h)] = make_uint4(s0.x & s1.x, s0.y & s1.y, s0.z & s1.z, s0.w & s1.w);
                }
                dj *= 3;
                __syncthreads();
            }
        }

        DQMC_TSEG(2);  // Merge
        if (!reduce && !chunk_mask && !out) {
            // Merge only: write the rows the Merge created (rows whose group
            // digits are all 0/1 were read from the state unchanged), or all
            // rows when they came from the truth table.
            const bool all = (load == kLoadTT);
            for (uint32_t pc = tid; pc < R * 2; pc += kSThreads) {
                const int h = pc & 1;
                const uint32_t ri = pc >> 1;
                const uint32_t g = div_pow3(ri, B);
                if (!ck<kCheck>(A, g < (uint32_t)kTileRowsMax, kChkTable, g, kTileRowsMax)) continue;
                if (!all && !S.has_star[g]) continue;
                const uint32_t e = ri - g * RE;
                const uint64_t row = base + e + (uint64_t)g * w_g;
                if (!ck<kCheck>(A, row < state_rows, kChkState, row, state_rows)) continue;
                state[2 * row + h] = tile[slot_s(ri, h)];
            }
        } else {
            // ---------------------------------------------------------- Reduce
            uint32_t res[kRounds][kChunkWords];
#pragma unroll
            for (int rd = 0; rd < kRounds; ++rd) {
                const uint32_t ri = rd * kSThreads + tid;
                if (ri < R) {
                    const uint32_t g = div_pow3(ri, B);
                    uint32_t v[kChunkWords], acc[kChunkWords];
                    const uint4 q0 = tile[slot_s(ri, 0)], q1 = tile[slot_s(ri, 1)];
                    v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
                    v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
#pragma unroll
                    for (int w = 0; w < kChunkWords; ++w) acc[w] = 0;
                    if (reduce) {
                        uint32_t gg = g, wgt = RE;
                        for (int j = 0; j < K; ++j) {
                            const uint32_t q = gg / 3u;
                            const uint32_t dg = gg - 3u * q;
                            gg = q;
                            if (dg != 2 && ck<kCheck>(A, ri + (2 - dg) * wgt < R, kChkTile, ri + (2 - dg) * wgt, R)) {
                                const int nb = ri + (2 - dg) * wgt;
                                const uint4 a0 = tile[slot_s(nb, 0)], a1 = tile[slot_s(nb, 1)];
                                acc[0] |= a0.x; acc[1] |= a0.y; acc[2] |= a0.z; acc[3] |= a0.w;
                                acc[4] |= a1.x; acc[5] |= a1.y; acc[6] |= a1.z; acc[7] |= a1.w;
                            }
                            wgt *= 3;
                        }
                    }
                    if (chunk_mask) chunk_reduce_masked(v, acc, chunk_mask);
#pragma unroll
                    for (int w = 0; w < kChunkWords; ++w) res[rd][w] = v[w] & ~acc[w];
                } else {
#pragma unroll
                    for (int w = 0; w < kChunkWords; ++w) res[rd][w] = 0;
                }
            }

            DQMC_TSEG(3);  // Reduce (this thread)
            if (!out) {
                __syncthreads();  // every read of the tile is done before rows are overwritten in place
#pragma unroll
                for (int rd = 0; rd < kRounds; ++rd) {
                    const uint32_t ri = rd * kSThreads + tid;
                    if (ri < R) {
                        const uint32_t g = div_pow3(ri, B);
                        const uint32_t e = ri - g * RE;
                        const uint64_t row = base + e + (uint64_t)g * w_g;
                        if (!ck<kCheck>(A, row < state_rows, kChkState, row, state_rows)) continue;
                        state[2 * row] = make_uint4(res[rd][0], res[rd][1], res[rd][2], res[rd][3]);
                        state[2 * row + 1] = make_uint4(res[rd][4], res[rd][5], res[rd][6], res[rd][7]);
                    }
                }
            } else {
                // ------------------------------------ bitmap, count and list
                // (B = 0, a = 0: rows base .. base + R - 1, contiguous.)
                // Rows in rho order are (round, thread): per round, an
                // inclusive warp scan of the row counts and the warp totals.
                // excl[rd]: bits in this warp's rows before this thread's row
                // of round rd (< 7776: 13 bits), row count in the top bits.
                uint32_t cx[kRounds];
#pragma unroll
                for (int rd = 0; rd < kRounds; ++rd) {
                    uint32_t c = 0;
#pragma unroll
                    for (int w = 0; w < kChunkWords; ++w) c += __popc(res[rd][w]);
                    uint32_t x = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= o) x += y;
                    }
                    cx[rd] = (c << 16) | (x - c);
                    if (lane == 31) S.warp_tot[rd][wid] = x;
                }
                __syncthreads();  // tile reads done; warp totals visible
                uint32_t tile_total = 0;
#pragma unroll
                for (int rd = 0; rd < kRounds; ++rd)
#pragma unroll
                    for (int w = 0; w < kSThreads / 32; ++w) tile_total += S.warp_tot[rd][w];
                uint2 *const pairs = A.pairs;
                const uint64_t T = base / kTileRowsMax;
                if (tid == 0) {
                    if (tile_total) atomicAdd(A.count, (unsigned long long)tile_total);
                    // publish this tile's aggregate now; the prefix comes after the bitmap
                    if (pairs && ck<kCheck>(A, T < A.out_tiles, kChkStatus, T, A.out_tiles))
                        atomicExch(&A.status[T], (T == 0 ? kFlagP : kFlagA) | (unsigned long long)tile_total);
                }

                // Dense bitmap: rows base .. base+R-1 are bits base*243 ..
                // (base+R)*243-1 (words W0 .. W0+nw-1).  Each row is funnel-
                // shifted to its bit offset in a shared-memory copy of those
                // words (stored sh = W0 mod 4 words in, so that 16-byte
                // groups of the copy are 16-byte groups of the bitmap); words
                // shared by two rows are OR-ed in with shared atomics.
                uint32_t *stg = reinterpret_cast<uint32_t *>(tile);
                const uint64_t bit0 = base * 243u;
                const uint32_t o = (uint32_t)(bit0 & 31);
                const uint64_t W0 = bit0 >> 5;
                const uint32_t sh = (uint32_t)(W0 & 3);
                const uint32_t L = R * 243u;
                const uint32_t nw = (o + L + 31) >> 5;
                const uint32_t nq = (nw + sh + 3) >> 2;
                ck<kCheck>(A, nq <= kSlots, kChkStage, nq, kSlots);
                for (uint32_t i = tid; i < nq && i < kSlots; i += kSThreads) tile[i] = make_uint4(0u, 0u, 0u, 0u);
                __syncthreads();
#pragma unroll
                for (int rd = 0; rd < kRounds; ++rd) {
                    const uint32_t ri = rd * kSThreads + tid;
                    if (ri < R) {
                        const uint32_t lb = o + 243u * ri;
                        const uint32_t k0 = (lb >> 5) + sh, s = lb & 31;
                        const uint32_t c = (s + 243u + 31u) >> 5;  // 8 or 9 words
                        if (!ck<kCheck>(A, k0 + c <= kSlots * 4, kChkStage, k0 + c, kSlots * 4)) continue;
                        uint32_t w8[9];
                        w8[0] = res[rd][0] << s;
#pragma unroll
                        for (int j = 1; j < 8; ++j) w8[j] = __funnelshift_l(res[rd][j - 1], res[rd][j], s);
                        w8[8] = __funnelshift_l(res[rd][7], 0u, s);
                        atomicOr(&stg[k0], w8[0]);
#pragma unroll
                        for (int j = 1; j < 8; ++j) {
                            if ((uint32_t)j < c - 1) stg[k0 + j] = w8[j];
                            else if ((uint32_t)j == c - 1) atomicOr(&stg[k0 + j], w8[j]);
                        }
                        if (c == 9) atomicOr(&stg[k0 + 8], w8[8]);
                    }
                }
                __syncthreads();
                uint32_t *const outw = A.out;
                const uint64_t alloc_words = A.out_alloc_words;
                const bool last_tile = (base + R == A.total_rows);
                const uint32_t tail = (o + L) & 31;
                for (uint32_t cq = tid; cq < nq && cq < kSlots; cq += kSThreads) {
                    // bitmap words i = 4*cq + x - sh, x = 0..3
                    const long long i0 = (long long)(4 * cq) - (long long)sh;
                    if (i0 >= 1 && i0 + 3 <= (long long)nw - 2) {
                        const uint64_t wi = W0 + (uint64_t)i0;
                        if (!ck<kCheck>(A, wi + 4 <= alloc_words, kChkOut, wi, alloc_words)) continue;
                        *reinterpret_cast<uint4 *>(outw + wi) = tile[cq];
                        continue;
                    }
                    for (int x = 0; x < 4; ++x) {
                        const long long i = i0 + x;
                        if (i < 0 || i >= (long long)nw) continue;
                        const uint32_t val = stg[4 * cq + x];
                        const bool shared_prev = (i == 0 && o != 0);
                        const bool shared_next = (i == (long long)nw - 1 && !last_tile && tail != 0);
                        const uint64_t wi = W0 + (uint64_t)i;
                        if (!ck<kCheck>(A, wi < alloc_words, kChkOut, wi, alloc_words)) continue;
                        uint32_t *dst = outw + wi;
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
                }
                if (last_tile)
                    for (uint64_t w = A.out_words + tid; w < alloc_words; w += kSThreads) outw[w] = 0u;

                if (pairs) {
                    // The predecessors have had the bitmap's time to publish.
                    if (wid == 0) {
                        bool ok = true;
                        unsigned long long ex = 0;
                        if (T > 0) ex = lookback<kCheck>(A, T, tile_total, ok);
                        if (lane == 0) {
                            S.excl = ex;
                            S.list_ok = ok;
                            // mask / value bits of the digits above the tile (high digits >= 6)
                            uint64_t x = T;
                            uint32_t m = 0, v = 0;
                            for (int d = 6; d < A.H; ++d) {
                                const uint64_t q = x / 3u;
                                const uint32_t dg = (uint32_t)(x - 3u * q);
                                x = q;
                                if (dg != 2) m |= 1u << (5 + d);
                                if (dg == 1) v |= 1u << (5 + d);
                            }
                            S.tile_mask = m;
                            S.tile_val = v;
                        }
                    }
                    __syncthreads();
                    if (S.list_ok) {
                        const unsigned long long ex = S.excl;
                        const uint64_t cap = A.cap;
                        const uint32_t nmask = A.nmask;
                        uint32_t round_base = 0;
#pragma unroll
                        for (int rd = 0; rd < kRounds; ++rd) {
                            const uint32_t ri = rd * kSThreads + tid;
                            uint32_t rt = 0, bw = 0;
#pragma unroll
                            for (int w = 0; w < kSThreads / 32; ++w) {
                                const uint32_t v = S.warp_tot[rd][w];
                                rt += v;
                                if (w < wid) bw += v;
                            }
                            unsigned long long k = ex + round_base + bw + (cx[rd] & 0xffffu);
                            round_base += rt;
                            if ((cx[rd] >> 16) && k < cap &&
                                ck<kCheck>(A, ri < (uint32_t)kTileRowsMax, kChkTable, ri, kTileRowsMax)) {
                                const uint32_t rm = S.tile_mask | ((uint32_t)S.m6[ri] << 5);
                                const uint32_t rv = S.tile_val | ((uint32_t)S.v6[ri] << 5);
#pragma unroll
                                for (int w = 0; w < kChunkWords; ++w) {
                                    uint32_t bits = res[rd][w];
                                    while (bits) {
                                        const int b = __ffs(bits) - 1;
                                        bits &= bits - 1;
                                        const int q = 32 * w + b;  // < 243: padding bits stay 0
                                        if (k < cap && q < 243)
                                            pairs[k] = make_uint2((rm | S.t5m[q]) & nmask, (rv | S.t5v[q]) & nmask);
                                        ++k;
                                    }
                                }
                            }
                        }
                    }
                }
            }
        }

        DQMC_TSEG(4);  // store / bitmap / list
        // ------------------------------------------------------------- signal
        if (signal) {
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const uint64_t di = sp.done_off + sb * nph + p;
                if (ck<kCheck>(A, di < A.ctrl_words, kChkCtrl, di, A.ctrl_words)) atomicAdd(done + sb * nph + p, 1u);
            }
        }
        __syncthreads();  // the shared tile and S are reused by the next ticket
        DQMC_TSEG(5);  // signal, end barrier
        if (timing && tid == 0) tsum[tph][6] += 1;  // tiles
    }
#undef DQMC_TSEG
    if (timing && tid == 0)
        for (int q = 0; q < kMaxPhases; ++q)
            for (int g = 0; g < kTimeSegs; ++g)
                if (tsum[q][g]) atomicAdd(A.timing + q * kTimeSegs + g, tsum[q][g]);
}

// One thread waits on a phase counter that nothing increments: the bounded
// wait must give up after wait_ns and leave kErrTimeout in the error word.
__global__ void selftest_wait_kernel(const __grid_constant__ SweepArgs A)
{
    if (threadIdx.x == 0) wait_counter(A, A.ctrl + 1 + kCtrlTickets, 1u);
}

cudaError_t launch_selftest_wait(void *d_ctrl, uint64_t ctrl_bytes, uint64_t wait_ns, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(d_ctrl, 0, ctrl_bytes, stream);
    if (e != cudaSuccess) return e;
    SweepArgs a{};
    a.ctrl = static_cast<uint32_t *>(d_ctrl);
    a.wait_ns = wait_ns;
    selftest_wait_kernel<<<1, 32, 0, stream>>>(a);
    return cudaGetLastError();
}

static int occupancy_blocks(size_t smem)
{
    static int cached_dev = -1, cached_sms = 0, cached_blocks = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        cudaDeviceGetAttribute(&cached_sms, cudaDevAttrMultiProcessorCount, dev);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, super_pass_kernel<true>, kSThreads, smem);
        cached_blocks = b > 0 ? b : 1;
        cached_dev = dev;
    }
    return cached_sms * cached_blocks;
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
    const size_t smem = (size_t)kTileRowsMax * kChunkBytes;

    static const bool discard = [] {
        const char *v = getenv("DQMC_L2_DISCARD");
        return v && v[0] == '1';
    }();
    auto kern = super_pass_kernel<true>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SweepArgs a{};
    a.on = static_cast<const uint32_t *>(d_on);
    a.dc = static_cast<const uint32_t *>(d_dc);
    a.state = static_cast<uint4 *>(d_state);
    a.out = d_bitmap;
    a.count = d_count;
    a.pairs = reinterpret_cast<uint2 *>(d_pairs);
    a.cap = d_pairs ? cap : 0;
    a.ctrl = static_cast<uint32_t *>(d_ctrl);
    a.status = reinterpret_cast<unsigned long long *>(d_ctrl) + cl.status_u64;
    a.total_rows = pow3(plan.H);
    a.out_words = bitmap_words(plan.n);
    a.out_alloc_words = bitmap_alloc_bytes(plan.n) / 4;
    a.wait_ns = 1000000000ull;
    a.nmask = (uint32_t)((1ull << plan.n) - 1);
    a.H = plan.H;
    a.state_rows = plan.state_rows;
    a.tt_words = ((1ull << plan.n) + 31) / 32;
    a.out_tiles = plan.out_tiles;
    a.ctrl_words = cl.bytes / 4;
    a.l2_discard = discard ? 1 : 0;
    static const bool timing_on = [] {
        const char *v = getenv("DQMC_TIMING");
        return v && v[0] == '1';
    }();
    a.timing = timing_on ? reinterpret_cast<unsigned long long *>(static_cast<char *>(d_ctrl) + cl.timing_off)
                         : nullptr;
    const int resident = occupancy_blocks(smem);
    unsigned long long *const timing0 = a.timing;
    for (int i = first; i < last; ++i) {
        const SuperPassDesc &sp = plan.sps[i];
        a.timing = timing0 ? timing0 + (size_t)i * kTimingWordsPerPass : nullptr;
        uint64_t tickets = 0;
        for (int p = 0; p < sp.nph; ++p) tickets += (uint64_t)sp.ph[p].tiles * sp.n_sb;
        const uint64_t grid = tickets < (uint64_t)resident ? tickets : (uint64_t)resident;
        kern<<<(unsigned)grid, kSThreads, smem, stream>>>(sp, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dqmc
