// dqmc_fn.cu -- whole functions in shared memory, for batches of small and
// medium functions (5 <= n <= 14).
//
// What is computed is the sweep of DenseQMC (arXiv 2302.10083, Algorithm 3 in
// Section 4.1): MergeAll, S(u) |= S(s) & S(t) for every triple (s, t, u) that
// differs only in one digit (values 0, 1, *), then ReduceAll,
// S(s) &= ~S(u), S(t) &= ~S(u), and the dense bitmap and count of what is left
// (the prime implicants; output as in Algorithm 4, Section 4.2).
//
// How it is scheduled:
//   * One function's state (3^(n-5) rows of one 32-byte chunk, the layout of
//     dqmc_chunk.cuh) stays in shared memory from the truth table to the
//     bitmap: device memory sees the truth table once and the bitmap once.
//   * A CTA holds fpc functions, each worked on by tg threads with a named
//     barrier of its own.  Or a cluster of CL = 3 or 9 CTAs holds one function
//     (n = 13, 14; n = 14 takes 598 KB): the top one or two high digits are
//     the cluster digits, and CTA k holds the cubes whose cluster digits are
//     the base-3 digits of k.  Merge of a cluster digit needs no exchange: the
//     part with a '*' cluster digit is the Merge of the AND of the truth-table
//     parts of its 0 and 1 values (a cube with a '*' there covers one minterm
//     of each).  Reduce of a cluster digit reads the '*' CTA over distributed
//     shared memory, one digit after the other.
//   * The high digits are merged and reduced D at a time: a thread loads the
//     3^D rows of one block (one 8-byte slice of each), does the D digits in
//     registers and writes the block back.  Within one step the blocks are
//     disjoint, so working in place reads the state the step started from.
//     Merge goes from the lowest digit up, so a block only reads rows whose
//     higher digits are 0/1 (the others are still empty); Reduce may take the
//     digits in any order (the grouped form of ReduceAll, see dqmc_sweep.cu).
//   * The chunk digits are reduced per row in registers with funnel shifts;
//     each warp packs its 32 rows (243 words) in place and stores them to the
//     bitmap at once (coalesced; a cluster's CTAs, whose streams start inside
//     a word, go through a second phase with masked atomics at the seams).
#include <cooperative_groups.h>

#include "dqmc_chunk.cuh"
#include "dqmc_internal.h"
#include "dqmc_steps.cuh"

namespace cg = cooperative_groups;

namespace dqmc {

static __constant__ MaskTable kFnMasks = make_mask_table();

struct FnArgs {
    const uint32_t *fn;             // function ids of this launch (one n)
    uint32_t nfun;
    uint32_t tg;                    // threads per function (multiple of 32)
    uint32_t fpc;                   // functions per CTA (1 for a cluster)
    const uint64_t *tt_off, *dc_off, *bm_off;
    const uint8_t *arena;
    uint8_t *bitmaps;
    unsigned long long *count;
    uint64_t out_words, out_alloc_words;   // ceil(3^n / 32), bitmap slot in words
    uint4 *scratch;                 // n = 14 in one CTA: 3^8 rows per CTA of the grid
};

// Shared-memory layout of a function's rows: row r at bytes 32r .. 32r+31,
// no swizzle.  A Merge / Reduce step has lanes 4k..4k+3 on the four 8-byte
// slices of one row and eight rows per warp at an odd stride (3^j apart, or
// consecutive), which spreads them over all four 128-byte bank phases: two
// wavefronts per warp access, the least 256 bytes take.  Rows of a block are
// then a fixed number of bytes apart, so one base address and compile-time
// offsets reach all of them.
__device__ __forceinline__ int fslot(int r, int h) { return 2 * r + h; }

__device__ __forceinline__ void ld_row(const uint4 *S, int r, uint32_t (&v)[kChunkWords])
{
    const uint4 a = S[fslot(r, 0)], b = S[fslot(r, 1)];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void st_row(uint4 *S, int r, const uint32_t (&v)[kChunkWords])
{
    S[fslot(r, 0)] = make_uint4(v[0], v[1], v[2], v[3]);
    S[fslot(r, 1)] = make_uint4(v[4], v[5], v[6], v[7]);
}

// The 32 minterms of a chunk -> its 243 cells, Merged over the five chunk
// digits (before digit i is merged its '*' cells are zero, so OR equals
// assignment).
__device__ __forceinline__ void chunk_merge_from_tt(uint32_t x, uint32_t (&v)[kChunkWords])
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
            nv[w] = v[w] | (shl_word<d>(v, w) & shl_word<2 * d>(v, w) & kFnMasks.m[kChunkDigits][i][2][w]);
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) v[w] = nv[w];
    });
}

// Reduce of the five chunk digits of one row, all read from v.
__device__ __forceinline__ void chunk_reduce_row(uint32_t (&v)[kChunkWords])
{
    uint32_t acc[kChunkWords];
#pragma unroll
    for (int w = 0; w < kChunkWords; ++w) acc[w] = 0;
    static_for<0, kChunkDigits>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int d = (int)pow3(i);
        uint32_t y[kChunkWords];
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) y[w] = v[w] & kFnMasks.m[kChunkDigits][i][2][w];
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) acc[w] |= shr_word<d>(y, w) | shr_word<2 * d>(y, w);
    });
#pragma unroll
    for (int w = 0; w < kChunkWords; ++w) v[w] &= ~acc[w];
}

// Binary rows of one part of a function from its truth table (word g holds
// the 32 minterms of binary row g), chunk digits merged on the way.  The part
// holds the cubes whose top CD high digits (above the HL it holds) are the
// base-3 digits of `part`; word gb + 2^HL b0 + 2^(HL+1) b1 holds binary row gb
// with those digits (b0, b1), and a '*' digit ANDs both values.
template <int HL, int CD>
__device__ __forceinline__ void load_rows(uint4 *S, const uint32_t *on, const uint32_t *dc, int part, int lt, int tg)
{
    constexpr int NB = 1 << HL;
    const int cd0 = CD >= 1 ? part % 3 : 0, cd1 = CD >= 2 ? part / 3 : 0;
    for (int gb = lt; gb < NB; gb += tg) {
        uint32_t x = 0xffffffffu;
#pragma unroll
        for (int b1 = 0; b1 < (CD >= 2 ? 2 : 1); ++b1) {
            if (CD >= 2 && cd1 != 2 && b1 != cd1) continue;
#pragma unroll
            for (int b0 = 0; b0 < (CD >= 1 ? 2 : 1); ++b0) {
                if (CD >= 1 && cd0 != 2 && b0 != cd0) continue;
                const int wi = gb + (b0 << HL) + (b1 << (HL + 1));
                x &= __ldg(on + wi) | (dc ? __ldg(dc + wi) : 0u);
            }
        }
        uint32_t v[kChunkWords];
        chunk_merge_from_tt(x, v);
        st_row(S, spread3k<HL>(gb), v);
    }
}

// Chunk digits, count, and the rows packed into the dense stream in place: a
// warp takes regions of 32 rows (1 KB of shared memory; 32 rows of 243 cells
// are exactly 243 words), reduces each row's chunk digits in registers and
// writes the region's packed words to its start.  Lane l's row starts at bit
// 243 l of the region; the word it shares with the next row is completed by
// the next lane.  With DIRECT (a stream that starts at bit 0 of `out`) each
// region also goes to `out` at once.  Returns this thread's count of set cells.
template <int R, bool DIRECT>
__device__ __forceinline__ unsigned long long chunk_pack(uint4 *S, uint32_t *out, int lt, int tg)
{
    constexpr int C3 = (int)pow3(kChunkDigits);
    constexpr int NREG = (R + 31) / 32;
    constexpr int NP = (int)(((uint64_t)R * C3 + 31) / 32);   // packed words
    const int lane = (int)threadIdx.x & 31, nwarp = tg >> 5;
    uint32_t *Sw = reinterpret_cast<uint32_t *>(S);
    unsigned long long bits = 0;
    const int sh = (C3 * lane) & 31, w0 = (C3 * lane) >> 5;
    const bool k8 = sh + C3 > 256;                     // the row's last word is word 8 (else 7)
    const bool shares = ((sh + C3) & 31) != 0;         // the next row starts inside it
    for (int g = lt >> 5; g < NREG; g += nwarp) {
        const int r = 32 * g + lane;
        uint32_t v[kChunkWords];
        if (r < R) {
            ld_row(S, r, v);
            chunk_reduce_row(v);
        } else {
#pragma unroll
            for (int w = 0; w < kChunkWords; ++w) v[w] = 0;
        }
#pragma unroll
        for (int w = 0; w < kChunkWords; ++w) bits += __popc(v[w]);
        uint32_t o[kChunkWords + 1];
        o[0] = __funnelshift_l(0u, v[0], sh);
#pragma unroll
        for (int k = 1; k < kChunkWords; ++k) o[k] = __funnelshift_l(v[k - 1], v[k], sh);
        o[kChunkWords] = __funnelshift_l(v[kChunkWords - 1], 0u, sh);
        const uint32_t tailw = k8 ? o[8] : o[7];
        const uint32_t from_prev = __shfl_up_sync(0xffffffffu, tailw, 1);
        if (lane > 0 && sh != 0) o[0] |= from_prev;
        __syncwarp();   // every row of the region is in registers before it is overwritten
        if (r < R) {
            const bool own_last = !shares || lane == 31 || r + 1 >= R;
            uint32_t *dst = Sw + 256 * g + w0;
#pragma unroll
            for (int k = 0; k < 7; ++k) dst[k] = o[k];
            if (k8 || own_last) dst[7] = o[7];
            if (k8 && own_last) dst[8] = o[8];
        }
        __syncwarp();
        if constexpr (DIRECT) {
            const int nwords = (g == NREG - 1) ? NP - C3 * g : C3;
            const uint32_t *src = Sw + 256 * g;
            uint32_t *dst = out + C3 * g;
            for (int k = lane; k < nwords; k += 32) dst[k] = src[k];
        }
    }
    return bits;
}

// Part `part` of `parts` (rows part*R .. part*R + R-1 of the function) from
// its packed regions to the bitmap: its stream starts at bit part*R*243, and
// the words it shares with the neighbouring parts are written with masked
// atomics.  The last part also zeroes the slot past the stream.
template <int R>
__device__ __forceinline__ void stream_out(const uint4 *S, uint32_t *out, int part, int parts, uint64_t out_words,
                                           uint64_t alloc_words, int lt, int tg)
{
    constexpr int C3 = (int)pow3(kChunkDigits);
    constexpr int NP = (int)(((uint64_t)R * C3 + 31) / 32);
    const uint32_t *Sw = reinterpret_cast<const uint32_t *>(S);
    auto packed = [&](int j) -> uint32_t {   // packed word j is at word 256 (j / 243) + j % 243
        if (j < 0 || j >= NP) return 0u;
        const int g = j / C3;
        return Sw[256 * g + (j - g * C3)];
    };
    const uint64_t bit0 = (uint64_t)part * R * C3;
    const int o = (int)(bit0 & 31);
    const uint64_t W0 = bit0 >> 5;
    constexpr uint64_t L = (uint64_t)R * C3;
    const int nw = (int)((o + L + 31) >> 5);
    const bool last = part == parts - 1;
    const int tail = (int)((o + L) & 31);
    for (int i = lt; i < nw; i += tg) {
        const uint32_t val = o ? __funnelshift_l(packed(i - 1), packed(i), o) : packed(i);
        const bool shared_prev = (i == 0 && o != 0);
        const bool shared_next = (i == nw - 1 && !last && tail != 0);
        uint32_t *dst = out + W0 + i;
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
    if (last)
        for (uint64_t w = out_words + lt; w < alloc_words; w += tg) out[w] = 0u;
}

__device__ __forceinline__ void add_count(unsigned long long *count, unsigned long long bits)
{
    for (int off = 16; off > 0; off >>= 1) bits += __shfl_down_sync(0xffffffffu, bits, off);
    if ((threadIdx.x & 31) == 0 && bits) atomicAdd(count, bits);
}

template <int H, int CL, int D>
__global__ void __launch_bounds__(1024, 1) fn_kernel(const FnArgs a)
{
    static_assert(CL == 1 || CL == 3 || CL == 9, "clusters of 1, 3 or 9 CTAs");
    constexpr int CD = (CL == 9) ? 2 : (CL == 3) ? 1 : 0;   // cluster digits
    constexpr int HL = H - CD;                              // high digits one CTA holds
    constexpr int R = (int)pow3(HL);
    extern __shared__ uint4 fsmem[];

    const int tg = (int)a.tg;
    const int sub = (int)threadIdx.x / tg, lt = (int)threadIdx.x - sub * tg;
    int rank = 0;
    if constexpr (CL > 1) rank = (int)cg::this_cluster().block_rank();
    const uint64_t fi = (uint64_t)(blockIdx.x / CL) * a.fpc + sub;
    if (fi >= a.nfun) return;   // a whole sub-group (or a whole cluster) leaves together
    const SubSync sync{sub + 1, tg, a.fpc == 1};
    uint4 *S = fsmem + (size_t)sub * 2 * R;

    const uint32_t id = a.fn[fi];
    const uint32_t *on = reinterpret_cast<const uint32_t *>(a.arena + a.tt_off[id]);
    const uint64_t dco = a.dc_off[id];
    const uint32_t *dc = dco == ~0ull ? nullptr : reinterpret_cast<const uint32_t *>(a.arena + dco);
    uint32_t *out = reinterpret_cast<uint32_t *>(a.bitmaps + a.bm_off[id]);

    load_rows<HL, CD>(S, on, dc, rank, lt, tg);
    sync();
    merge_all<HL, 0, D>(S, lt, tg, sync);

    if constexpr (CL > 1) {
        // Reduce of the cluster digits, one after the other: for digit c, the
        // CTAs whose digit c is 0 or 1 clear what the CTA with a '*' there
        // (merged, and not modified in this step) has set.
        cg::cluster_group cl = cg::this_cluster();
        static_for<0, CD>([&](auto Ci) {
            constexpr int c = decltype(Ci)::value;
            constexpr int wc = (int)pow3(c);
            cl.sync();
            const int dgt = (rank / wc) % 3;
            if (dgt != 2) {
                const uint4 *T = cl.map_shared_rank(fsmem, rank + (2 - dgt) * wc);
                // eight remote loads in flight per thread
                constexpr int U = 8;
                for (int i0 = lt; i0 < 2 * R; i0 += U * tg) {
                    uint4 z[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int i = i0 + u * tg;
                        z[u] = i < 2 * R ? T[i] : make_uint4(0u, 0u, 0u, 0u);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int i = i0 + u * tg;
                        if (i < 2 * R) {
                            uint4 v = S[i];
                            v.x &= ~z[u].x; v.y &= ~z[u].y; v.z &= ~z[u].z; v.w &= ~z[u].w;
                            S[i] = v;
                        }
                    }
                }
            }
        });
        cl.sync();   // no CTA changes its rows (or leaves) while another still reads them
    }
    reduce_all<HL, 0, D>(S, lt, tg, sync);

    if constexpr (CL == 1) {
        // a single CTA's stream starts at bit 0 of the bitmap: each region
        // goes out as soon as it is packed (coalesced 4-byte stores)
        add_count(a.count + id, chunk_pack<R, true>(S, out, lt, tg));
        constexpr uint64_t NP = ((uint64_t)R * pow3(kChunkDigits) + 31) / 32;
        for (uint64_t w = NP + lt; w < a.out_alloc_words; w += tg) out[w] = 0u;   // at most three words
    } else {
        add_count(a.count + id, chunk_pack<R, false>(S, out, lt, tg));
        sync();
        stream_out<R>(S, out, rank, CL, a.out_words, a.out_alloc_words, lt, tg);
    }
}

// n = 14 by one thread group: the three thirds of the top high digit one after
// the other.  The '*' third is merged first and parked in T (a scratch slot
// of the group's own in device memory, 210 KB, read back from L2); thirds 0
// and 1 are merged, cleared by it (Reduce of the top digit), reduced and
// written out; then the '*' third comes back, is reduced and written out.
template <int D, typename Sync>
__device__ __forceinline__ void fn_thirds_one(const uint32_t *on, const uint32_t *dc, uint32_t *out,
                                              unsigned long long *count, uint64_t out_words, uint64_t alloc_words,
                                              uint4 *S, uint4 *T, int lt, int tg, const Sync &sync)
{
    constexpr int HL = 8, R = (int)pow3(HL);
    unsigned long long bits = 0;
    load_rows<HL, 1>(S, on, dc, 2, lt, tg);
    sync();
    merge_all<HL, 0, D>(S, lt, tg, sync);
    for (int i = lt; i < 2 * R; i += tg) T[i] = S[i];
    sync();   // the scratch copy is complete (and visible to the group) before S is reused
    for (int part = 0; part < 2; ++part) {
        load_rows<HL, 1>(S, on, dc, part, lt, tg);
        sync();
        merge_all<HL, 0, D>(S, lt, tg, sync);
        for (int i = lt; i < 2 * R; i += tg) {
            const uint4 z = T[i];
            uint4 v = S[i];
            v.x &= ~z.x; v.y &= ~z.y; v.z &= ~z.z; v.w &= ~z.w;
            S[i] = v;
        }
        sync();
        reduce_all<HL, 0, D>(S, lt, tg, sync);
        if (part == 0) {
            bits += chunk_pack<R, true>(S, out, lt, tg);   // third 0 starts at bit 0
        } else {
            bits += chunk_pack<R, false>(S, out, lt, tg);
            sync();
            stream_out<R>(S, out, part, 3, out_words, alloc_words, lt, tg);
        }
        sync();
    }
    for (int i = lt; i < 2 * R; i += tg) S[i] = T[i];
    sync();
    reduce_all<HL, 0, D>(S, lt, tg, sync);
    bits += chunk_pack<R, false>(S, out, lt, tg);
    sync();
    stream_out<R>(S, out, 2, 3, out_words, alloc_words, lt, tg);
    add_count(count, bits);
    sync();   // S and T are free for the next function
}

// n = 14 in one CTA (persistent: CTA b takes functions b, b + grid, ...),
// with the CTA's scratch slot.
template <int D>
__global__ void __launch_bounds__(1024, 1) fn_thirds_kernel(const FnArgs a)
{
    constexpr int R = (int)pow3(8);
    extern __shared__ uint4 fsmem[];
    const int tg = (int)blockDim.x, lt = (int)threadIdx.x;
    const SubSync sync{1, tg, true};
    uint4 *T = a.scratch + (size_t)blockIdx.x * 2 * R;
    for (uint64_t fi = blockIdx.x; fi < a.nfun; fi += gridDim.x) {
        const uint32_t id = a.fn[fi];
        const uint32_t *on = reinterpret_cast<const uint32_t *>(a.arena + a.tt_off[id]);
        const uint64_t dco = a.dc_off[id];
        const uint32_t *dc = dco == ~0ull ? nullptr : reinterpret_cast<const uint32_t *>(a.arena + dco);
        uint32_t *out = reinterpret_cast<uint32_t *>(a.bitmaps + a.bm_off[id]);
        fn_thirds_one<D>(on, dc, out, a.count + id, a.out_words, a.out_alloc_words, fsmem, T, lt, tg, sync);
    }
}

template <int H, int CL, int D>
static cudaError_t launch_fn_t(const FnArgs &a, uint32_t ctas, size_t smem, cudaStream_t s)
{
    auto kern = fn_kernel<H, CL, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && CL > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas * CL);
    cfg.blockDim = dim3(a.tg * a.fpc);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (CL > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int D>
static cudaError_t launch_fn_d(int n, int cl, const FnArgs &a, uint32_t ctas, size_t smem, cudaStream_t s)
{
    if (cl == 3) {
        if (n == 13) return launch_fn_t<8, 3, D>(a, ctas, smem, s);
        if (n == 14) return launch_fn_t<9, 3, D>(a, ctas, smem, s);
        return cudaErrorInvalidValue;
    }
    if (cl == 9) return n == 14 ? launch_fn_t<9, 9, D>(a, ctas, smem, s) : cudaErrorInvalidValue;
    if (cl != 1) return cudaErrorInvalidValue;
    switch (n) {
    case 5: return launch_fn_t<0, 1, D>(a, ctas, smem, s);
    case 6: return launch_fn_t<1, 1, D>(a, ctas, smem, s);
    case 7: return launch_fn_t<2, 1, D>(a, ctas, smem, s);
    case 8: return launch_fn_t<3, 1, D>(a, ctas, smem, s);
    case 9: return launch_fn_t<4, 1, D>(a, ctas, smem, s);
    case 10: return launch_fn_t<5, 1, D>(a, ctas, smem, s);
    case 11: return launch_fn_t<6, 1, D>(a, ctas, smem, s);
    case 12: return launch_fn_t<7, 1, D>(a, ctas, smem, s);
    case 13: return launch_fn_t<8, 1, D>(a, ctas, smem, s);
    }
    return cudaErrorInvalidValue;
}

template <int D>
static cudaError_t launch_thirds(const FnArgs &a, uint32_t ctas, size_t smem, cudaStream_t s)
{
    auto kern = fn_thirds_kernel<D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ctas, a.tg, smem, s>>>(a);
    return cudaGetLastError();
}

uint64_t fn_smem_bytes(int n, int fpc, int ctas)
{
    if (n < kFnMinN || n > kFnMaxN) return 0;
    // one CTA for n = 14 holds one third at a time
    const int cd = ctas == 9 ? 2 : (ctas == 3 || n == 14) ? 1 : 0;
    return (uint64_t)fpc * pow3(n - kChunkDigits - cd) * kChunkBytes;
}

bool fn_config_ok(int n, const FnConfig &c)
{
    if (n < kFnMinN || n > kFnMaxN) return false;
    if (c.digits != 2 && c.digits != 3) return false;
    if (c.tg < 32 || c.tg % 32 || c.fpc < 1 || c.fpc > 15) return false;
    if (c.tg * c.fpc > 1024) return false;
    // clusters: 3 CTAs for n = 13 and 14, 9 for n = 14, one function each;
    // one CTA for n = 14 runs the thirds in turn
    if (c.ctas == 3 && n != 13 && n != 14) return false;
    if (c.ctas == 9 && n != 14) return false;
    if (c.ctas != 1 && c.ctas != 3 && c.ctas != 9) return false;
    if (c.ctas > 1 && c.fpc != 1) return false;
    return fn_smem_bytes(n, c.fpc, c.ctas) <= kFnMaxSmem;
}

// ------------------------------------------------- the batch in one launch
// (launch_fn_queue, dqmc_internal.h.)  Thread groups synchronise with a
// named barrier of their own (barrier 1 + group), or __syncwarp for a group
// of one warp.
struct GroupSync {
    int id, nthreads;
    __device__ __forceinline__ void operator()() const
    {
        if (nthreads == 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
    }
};

struct QueueArgs {
    const uint32_t *fn;
    const uint64_t *tt_off, *dc_off, *bm_off;
    const uint8_t *arena;
    uint8_t *bitmaps;
    unsigned long long *count;
    uint32_t *ctr;
    uint4 *scratch;                 // n = 14: 3^8 rows per CTA of the grid
    uint32_t nclass;
    QueueClass cls[kFnMaxN + 1];
};

// shared memory of one function of n in the queue kernel: its rows (one third
// of them at n = 14), none below n = 5
__host__ __device__ constexpr uint64_t queue_fn_smem_d(int n)
{
    return n < kFnMinN ? 0 : pow3((n == 14 ? 13 : n) - kChunkDigits) * kChunkBytes;
}

// bitmap slot of an n-variable function in 32-bit words: ceil(3^n / 8) bytes
// rounded up to 16
__host__ __device__ constexpr uint64_t slot_words(int n) { return ((pow3(n) + 7) / 8 + 15) / 16 * 4; }

// n <= 4 by one warp, from the definitions (at most 81 cubes): a cube is an
// implicant when every minterm it covers is in ON or DC, a prime when it is
// an implicant and none of its one-digit extensions (a 0/1 digit made '*')
// is.  Cube q = lane + 32 k; its bit in the bitmap is bit q.
__device__ __forceinline__ void tiny_one(int n, const uint8_t *on, const uint8_t *dc, uint32_t *out,
                                         unsigned long long *count)
{
    const int lane = (int)threadIdx.x & 31;
    const int N3 = (int)pow3(n);
    uint32_t imp[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = lane + 32 * k;
        bool is = false;
        if (q < N3) {
            int base = 0, stars = 0, x = q;
            for (int i = 0; i < n; ++i, x /= 3) {
                const int d = x % 3;
                if (d == 2) stars |= 1 << i;
                else base |= d << i;
            }
            is = true;
            for (int sub = stars;; sub = (sub - 1) & stars) {   // every subset of the '*' digits
                const int m = base | sub;
                const uint32_t cell = on[m >> 3] | (dc ? dc[m >> 3] : 0u);
                if (!((cell >> (m & 7)) & 1u)) is = false;
                if (sub == 0) break;
            }
        }
        imp[k] = __ballot_sync(0xffffffffu, is);
    }
    auto implicant = [&](int q) -> bool { return (imp[q >> 5] >> (q & 31)) & 1u; };
    uint32_t pw[3];
    unsigned long long bits = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = lane + 32 * k;
        bool pr = false;
        if (q < N3 && implicant(q)) {
            pr = true;
            int x = q, w = 1;
            for (int i = 0; i < n; ++i, x /= 3, w *= 3) {
                const int d = x % 3;
                if (d != 2 && implicant(q + (2 - d) * w)) pr = false;
            }
        }
        pw[k] = __ballot_sync(0xffffffffu, pr);
        bits += __popc(pw[k]);
    }
    static_assert(slot_words(4) == 4, "n <= 4: a 16-byte bitmap slot");
    if (lane < 4) out[lane] = lane < 3 ? pw[lane] : 0u;
    if (lane == 0 && bits) atomicAdd(count, bits);
}

// 5 <= n <= 13 by one thread group, the whole function in S.
template <int HL, int D, typename Sync>
__device__ __forceinline__ void whole_one(const QueueArgs &a, uint32_t id, uint4 *S, int lt, int tg, const Sync &sync)
{
    constexpr int R = (int)pow3(HL);
    const uint32_t *on = reinterpret_cast<const uint32_t *>(a.arena + a.tt_off[id]);
    const uint64_t dco = a.dc_off[id];
    const uint32_t *dc = dco == ~0ull ? nullptr : reinterpret_cast<const uint32_t *>(a.arena + dco);
    uint32_t *out = reinterpret_cast<uint32_t *>(a.bitmaps + a.bm_off[id]);
    load_rows<HL, 0>(S, on, dc, 0, lt, tg);
    sync();
    merge_all<HL, 0, D>(S, lt, tg, sync);
    reduce_all<HL, 0, D>(S, lt, tg, sync);
    add_count(a.count + id, chunk_pack<R, true>(S, out, lt, tg));
    constexpr uint64_t NP = ((uint64_t)R * pow3(kChunkDigits) + 31) / 32;
    for (uint64_t w = NP + lt; w < slot_words(HL + kChunkDigits); w += tg) out[w] = 0u;   // at most three words
}

template <int D, typename Sync>
__device__ __forceinline__ void queue_one(const QueueArgs &a, int n, uint32_t id, uint4 *S, int lt, int tg,
                                          const Sync &sync)
{
    switch (n) {
    case 5: whole_one<0, D>(a, id, S, lt, tg, sync); break;
    case 6: whole_one<1, D>(a, id, S, lt, tg, sync); break;
    case 7: whole_one<2, D>(a, id, S, lt, tg, sync); break;
    case 8: whole_one<3, D>(a, id, S, lt, tg, sync); break;
    case 9: whole_one<4, D>(a, id, S, lt, tg, sync); break;
    case 10: whole_one<5, D>(a, id, S, lt, tg, sync); break;
    case 11: whole_one<6, D>(a, id, S, lt, tg, sync); break;
    case 12: whole_one<7, D>(a, id, S, lt, tg, sync); break;
    case 13: whole_one<8, D>(a, id, S, lt, tg, sync); break;
    case 14: {
        const uint32_t *on = reinterpret_cast<const uint32_t *>(a.arena + a.tt_off[id]);
        const uint64_t dco = a.dc_off[id];
        const uint32_t *dc = dco == ~0ull ? nullptr : reinterpret_cast<const uint32_t *>(a.arena + dco);
        uint32_t *out = reinterpret_cast<uint32_t *>(a.bitmaps + a.bm_off[id]);
        uint4 *T = a.scratch + (size_t)blockIdx.x * 2 * pow3(8);
        fn_thirds_one<D>(on, dc, out, a.count + id, (pow3(14) + 31) / 32, slot_words(14), S, T, lt, tg, sync);
        break;
    }
    default: break;
    }
}

__global__ void __launch_bounds__(kQueueThreads, 1) fn_queue_kernel(const __grid_constant__ QueueArgs a)
{
    extern __shared__ uint4 qsmem[];
    __shared__ uint32_t item[32];
    const int tid = (int)threadIdx.x;
    for (uint32_t c = 0; c < a.nclass; ++c) {
        const QueueClass k = a.cls[c];
        const int tg = (int)k.tg, sub = tid / tg, lt = tid - sub * tg;
        if (sub < (int)k.groups) {
            const GroupSync sync{1 + sub, tg};
            uint4 *S = qsmem + (size_t)sub * (queue_fn_smem_d((int)k.n) / 16);
            for (;;) {
                if (lt == 0) item[sub] = atomicAdd(a.ctr + c, 1u);
                sync();
                const uint32_t i = item[sub];
                if (i >= k.count) break;
                const uint32_t id = a.fn[k.first + i];
                if (k.n <= 4) {
                    const uint64_t dco = a.dc_off[id];
                    tiny_one((int)k.n, a.arena + a.tt_off[id], dco == ~0ull ? nullptr : a.arena + dco,
                             reinterpret_cast<uint32_t *>(a.bitmaps + a.bm_off[id]), a.count + id);
                } else if (k.digits >= 3) {
                    queue_one<3>(a, (int)k.n, id, S, lt, tg, sync);
                } else {
                    queue_one<2>(a, (int)k.n, id, S, lt, tg, sync);
                }
                sync();   // every thread has read item[sub] and is done with S
            }
        }
        __syncthreads();   // the next n splits the CTA (and its shared memory) its own way
    }
}

uint64_t queue_fn_smem(int n) { return queue_fn_smem_d(n); }

cudaError_t launch_fn_queue(const BatchArgs &b, const QueueSetup &q, cudaStream_t s)
{
    if (q.nclass == 0 || q.nclass > kFnMaxN + 1 || !q.ctr || q.ctas == 0 || q.smem > kFnMaxSmem)
        return cudaErrorInvalidValue;
    QueueArgs a{};
    a.fn = b.fn;
    a.tt_off = b.tt_off;
    a.dc_off = b.dc_off;
    a.bm_off = b.bm_off;
    a.arena = b.arena;
    a.bitmaps = b.bitmaps;
    a.count = b.count;
    a.ctr = q.ctr;
    a.scratch = static_cast<uint4 *>(b.scratch);
    a.nclass = q.nclass;
    for (uint32_t c = 0; c < q.nclass; ++c) {
        const QueueClass &k = q.cls[c];
        // the shapes the kernel takes: a warp per function below n = 5, the
        // whole CTA (with a scratch slot) at n = 14, named barriers 1 .. 15
        if (k.n > (uint32_t)kFnMaxN || k.tg < 32 || k.tg % 32 || k.groups == 0 || k.tg * k.groups > kQueueThreads)
            return cudaErrorInvalidValue;
        if ((k.n < (uint32_t)kFnMinN && k.tg != 32) || (k.n == 14 && (k.tg != kQueueThreads || !b.scratch ||
                                                                       b.scratch_ctas < q.ctas)))
            return cudaErrorInvalidValue;
        if (k.tg > 32 && k.groups > 15) return cudaErrorInvalidValue;
        if (k.digits != 2 && k.digits != 3) return cudaErrorInvalidValue;
        if (k.groups * queue_fn_smem((int)k.n) > q.smem) return cudaErrorInvalidValue;
        a.cls[c] = k;
    }
    cudaError_t e = cudaFuncSetAttribute(fn_queue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem);
    if (e != cudaSuccess) return e;
    fn_queue_kernel<<<q.ctas, kQueueThreads, q.smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fn_batch(int n, const BatchArgs &b, const FnConfig &c, cudaStream_t s)
{
    if (!fn_config_ok(n, c)) return cudaErrorInvalidValue;
    if (b.nfun == 0) return cudaSuccess;
    FnArgs a{};
    a.fn = b.fn;
    a.nfun = b.nfun;
    a.tg = (uint32_t)c.tg;
    a.fpc = (uint32_t)c.fpc;
    a.tt_off = b.tt_off;
    a.dc_off = b.dc_off;
    a.bm_off = b.bm_off;
    a.arena = b.arena;
    a.bitmaps = b.bitmaps;
    a.count = b.count;
    a.out_words = bitmap_words(n);
    a.out_alloc_words = bitmap_alloc_bytes(n) / 4;
    const size_t smem = fn_smem_bytes(n, c.fpc, c.ctas);
    if (n == 14 && c.ctas == 1) {
        // persistent: at most one CTA per scratch slot
        if (!b.scratch || b.scratch_ctas == 0) return cudaErrorInvalidValue;
        a.scratch = static_cast<uint4 *>(b.scratch);
        const uint32_t ctas = b.nfun < b.scratch_ctas ? b.nfun : b.scratch_ctas;
        return c.digits >= 3 ? launch_thirds<3>(a, ctas, smem, s) : launch_thirds<2>(a, ctas, smem, s);
    }
    const uint32_t groups = (b.nfun + c.fpc - 1) / c.fpc;   // CTAs, or clusters
    return c.digits >= 3 ? launch_fn_d<3>(n, c.ctas, a, groups, smem, s)
                         : launch_fn_d<2>(n, c.ctas, a, groups, smem, s);
}

}  // namespace dqmc
