/*
 * dqmc_oracle.c -- CPU oracle for the dense ternary prime-implicant sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  The CUDA library never
 * links, includes or calls it, and this file includes nothing of the CUDA
 * library: the two share no code, headers or tables.
 *
 * What it computes (arXiv 2302.10083, "DenseQMC"):
 *   - a cube s in {0,1,*}^n is stored at index rho(s) = sum_i 3^(i-1) rho(s_i),
 *     with rho(0)=0, rho(1)=1, rho(*)=2 (Section 4.2, the notation rho);
 *   - variable x_i is digit i; a truth-table minterm t = sum_i 2^(i-1) x_i;
 *   - the support I = ON u DC (don't-cares widen the implicants; a prime that
 *     covers only don't-care minterms is kept);
 *   - an implicant is a cube all of whose minterms are in I, a prime implicant
 *     is an implicant with no proper super-cube that is an implicant
 *     (Section 2, Definitions of implicant and prime).
 *
 * oracle_sweep follows Algorithm 3 (Section 4.1): the state S holds one byte per
 * cube; MergeAll visits every digit i = 1..n and every triple (s, t, u) that
 * differs only in digit i (values 0, 1, *) and applies Merge; ReduceAll visits
 * the same triples in the same order and applies Reduce.  Merge and Reduce are
 * the two maps of the Definition in Section 4.1:
 *   Merge (c0, c1, c*) -> (c0, c1, c* OR (c0 AND c1))
 *   Reduce(c0, c1, c*) -> (c0 AND NOT c*, c1 AND NOT c*, c*)
 * The triples of one digit are independent (Section 4.1), so they are split
 * across OpenMP threads; nothing else is reordered or fused.
 * oracle_sweep_packed runs the same passes with one bit per cube, for sizes
 * whose byte state does not fit in host memory.
 *
 * oracle_is_implicant / oracle_is_prime are the plain definitions, evaluated
 * for one cube by enumerating its minterms; they serve as the pointwise check at
 * sizes the sweep cannot hold in host memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

uint64_t oracle_pow3(int n)
{
    uint64_t p = 1;
    for (int i = 0; i < n; ++i) p *= 3u;
    return p;
}

static int tt_bit(const uint8_t *bits, uint64_t t)
{
    return (bits[t >> 3] >> (t & 7)) & 1;
}

/* I(t) = ON(t) or DC(t); dc may be NULL. */
static int support_bit(const uint8_t *on, const uint8_t *dc, uint64_t t)
{
    return tt_bit(on, t) | (dc ? tt_bit(dc, t) : 0);
}

/* rho of the binary cube whose digit i is bit i-1 of t. */
static uint64_t rho_of_minterm(int n, uint64_t t)
{
    uint64_t r = 0, w = 1;
    for (int i = 0; i < n; ++i) {
        if ((t >> i) & 1) r += w;
        w *= 3u;
    }
    return r;
}

/* threads > 0 sets the thread count for one call; the previous count is
 * returned and put back by restore_threads when the call ends. */
static int set_threads(int threads)
{
#ifdef _OPENMP
    const int prev = omp_get_max_threads();
    if (threads > 0) omp_set_num_threads(threads);
    return prev;
#else
    (void)threads;
    return 1;
#endif
}

static void restore_threads(int prev)
{
#ifdef _OPENMP
    omp_set_num_threads(prev);
#else
    (void)prev;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Algorithm 3, one byte per cube.  S must hold 3^n bytes.
 * counts (may be NULL) receives [Merge triples visited, Reduce triples visited].
 */
void oracle_sweep(int n, const uint8_t *on, const uint8_t *dc, uint8_t *S,
                  int threads, uint64_t *counts)
{
    const uint64_t N = oracle_pow3(n);
    const uint64_t T = (uint64_t)1 << n;
    const int prev_threads = set_threads(threads);

    /* Load the input: S = indicator of the support embedded in {0,1,*}^n. */
    memset(S, 0, N);
    for (uint64_t t = 0; t < T; ++t)
        S[rho_of_minterm(n, t)] = (uint8_t)support_bit(on, dc, t);

    const uint64_t triples = (n > 0) ? N / 3u : 0; /* per digit: 3^(n-1) */
    uint64_t merges = 0, reduces = 0;

    /* MergeAll: for i = 1..n, every s with s_i = 0, t = s with 1, u = s with *. */
    uint64_t d = 1; /* 3^(i-1) */
    for (int i = 1; i <= n; ++i) {
        const uint64_t dd = d;
        #pragma omp parallel for schedule(static) reduction(+:merges)
        for (uint64_t k = 0; k < triples; ++k) {
            const uint64_t b = (k / dd) * 3u * dd; /* base of the group of 3^i cells */
            const uint64_t c = k % dd;             /* offset inside the 0-part */
            const uint64_t is = b + c, it = is + dd, iu = is + 2u * dd;
            /* Merge(c0, c1, c*) = (c0, c1, c* | (c0 & c1)) */
            S[iu] = (uint8_t)(S[iu] | (S[is] & S[it]));
            merges += 1;
        }
        d *= 3u;
    }

    /* ReduceAll: same triples, same order, Reduce instead of Merge. */
    d = 1;
    for (int i = 1; i <= n; ++i) {
        const uint64_t dd = d;
        #pragma omp parallel for schedule(static) reduction(+:reduces)
        for (uint64_t k = 0; k < triples; ++k) {
            const uint64_t b = (k / dd) * 3u * dd;
            const uint64_t c = k % dd;
            const uint64_t is = b + c, it = is + dd, iu = is + 2u * dd;
            /* Reduce(c0, c1, c*) = (c0 & !c*, c1 & !c*, c*) */
            const uint8_t z = S[iu];
            S[is] = (uint8_t)(S[is] & !z);
            S[it] = (uint8_t)(S[it] & !z);
            reduces += 1;
        }
        d *= 3u;
    }

    if (counts) {
        counts[0] = merges;
        counts[1] = reduces;
    }
    restore_threads(prev_threads);
}

/* Dense LSB-first bitmap of the byte state: bit rho set iff S[rho] != 0. */
void oracle_bitmap(int n, const uint8_t *S, uint8_t *out)
{
    const uint64_t N = oracle_pow3(n);
    memset(out, 0, (N + 7) / 8);
    for (uint64_t r = 0; r < N; ++r)
        if (S[r]) out[r >> 3] |= (uint8_t)(1u << (r & 7));
}

uint64_t oracle_count(int n, const uint8_t *S)
{
    const uint64_t N = oracle_pow3(n);
    uint64_t c = 0;
    for (uint64_t r = 0; r < N; ++r) c += (S[r] != 0);
    return c;
}

/* (mask, value) of the cube at rho: mask bit i-1 set iff digit i is 0 or 1,
 * value bit i-1 = digit i for those digits. */
void oracle_encode(int n, uint64_t rho, uint32_t *mask, uint32_t *value)
{
    uint32_t m = 0, v = 0;
    for (int i = 0; i < n; ++i) {
        const uint64_t digit = rho % 3u;
        rho /= 3u;
        if (digit != 2) {
            m |= 1u << i;
            if (digit == 1) v |= 1u << i;
        }
    }
    *mask = m;
    *value = v;
}

/* Cubes with S[rho] != 0 in ascending rho, as pairs (mask, value).  Writes at
 * most cap pairs, returns the total number of set cubes. */
uint64_t oracle_list(int n, const uint8_t *S, uint32_t *pairs, uint64_t cap)
{
    const uint64_t N = oracle_pow3(n);
    uint64_t k = 0;
    for (uint64_t r = 0; r < N; ++r) {
        if (!S[r]) continue;
        if (k < cap) oracle_encode(n, r, &pairs[2 * k], &pairs[2 * k + 1]);
        ++k;
    }
    return k;
}

/* Plain definition: every minterm covered by the cube at rho is in I. */
int oracle_is_implicant(int n, const uint8_t *on, const uint8_t *dc, uint64_t rho)
{
    uint64_t fixed = 0;      /* bits of the binary digits */
    int stars[32];
    int w = 0;
    for (int i = 0; i < n; ++i) {
        const uint64_t digit = rho % 3u;
        rho /= 3u;
        if (digit == 2) stars[w++] = i;
        else if (digit == 1) fixed |= (uint64_t)1 << i;
    }
    const uint64_t combos = (uint64_t)1 << w;
    for (uint64_t a = 0; a < combos; ++a) {
        uint64_t t = fixed;
        for (int k = 0; k < w; ++k)
            if ((a >> k) & 1) t |= (uint64_t)1 << stars[k];
        if (!support_bit(on, dc, t)) return 0;
    }
    return 1;
}

/* Plain definition: an implicant none of whose one-digit extensions (a 0/1
 * digit replaced by *) is an implicant.  Every proper super-cube contains such
 * an extension, so this is the same as "no proper super-cube is an implicant". */
int oracle_is_prime(int n, const uint8_t *on, const uint8_t *dc, uint64_t rho)
{
    if (!oracle_is_implicant(n, on, dc, rho)) return 0;
    uint64_t w = 1, r = rho;
    for (int i = 0; i < n; ++i) {
        const uint64_t digit = r % 3u;
        r /= 3u;
        if (digit != 2) {
            const uint64_t ext = rho + (2u - digit) * w; /* digit i -> * */
            if (oracle_is_implicant(n, on, dc, ext)) return 0;
        }
        w *= 3u;
    }
    return 1;
}

/* Pointwise primality for many cubes (OpenMP over the list). */
void oracle_is_prime_many(int n, const uint8_t *on, const uint8_t *dc,
                          const uint64_t *rhos, uint64_t count, uint8_t *out, int threads)
{
    const int prev_threads = set_threads(threads);
    #pragma omp parallel for schedule(dynamic, 64)
    for (uint64_t k = 0; k < count; ++k)
        out[k] = (uint8_t)oracle_is_prime(n, on, dc, rhos[k]);
    restore_threads(prev_threads);
}

/*
 * Packed mode: the same Algorithm 3 with one BIT per cube, for sizes whose
 * byte state does not fit in host memory.  S holds ceil(3^n/64) words; cube
 * rho is bit rho%64 of word rho/64.  Within one digit i every triple is
 * independent (Section 4.1), and a pass writes only one kind of cell: Merge
 * writes the cells whose digit i is *, reading their 0 and 1 siblings; Reduce
 * writes the cells whose digit i is 0 or 1, reading their * sibling.  So the
 * words are split across threads, each thread updates the cells of its own
 * words, and every cell it reads is one that no thread writes in that pass.
 */
/* Words are read and written whole with relaxed atomics: a word another
 * thread is storing keeps the bits read here (only its other kind of cell
 * changes), and the atomics make that well defined. */
static int pk_get(const uint64_t *S, uint64_t r)
{
    return (int)((__atomic_load_n(&S[r >> 6], __ATOMIC_RELAXED) >> (r & 63)) & 1u);
}

/* Digit i (weight d = 3^(i-1)) of cell r, and the position of r inside its
 * run of d cells with that digit. */
static void pk_digit_at(uint64_t r, uint64_t d, unsigned *digit, uint64_t *pos)
{
    *digit = (unsigned)((r / d) % 3u);
    *pos = r % d;
}

void oracle_sweep_packed(int n, const uint8_t *on, const uint8_t *dc, uint64_t *S, int threads)
{
    const uint64_t N = oracle_pow3(n);
    const uint64_t W = (N + 63) / 64;
    const uint64_t T = (uint64_t)1 << n;
    const int prev_threads = set_threads(threads);

    /* Load the input: bit rho(t) = I(t) for every minterm t. */
    memset(S, 0, W * sizeof(uint64_t));
    for (uint64_t t = 0; t < T; ++t)
        if (support_bit(on, dc, t)) {
            const uint64_t r = rho_of_minterm(n, t);
            S[r >> 6] |= (uint64_t)1 << (r & 63);
        }

    /* MergeAll: for i = 1..n, every * cell u |= (its 0 sibling) & (its 1 sibling). */
    uint64_t d = 1;
    for (int i = 1; i <= n; ++i) {
        const uint64_t dd = d;
        #pragma omp parallel for schedule(static)
        for (uint64_t w = 0; w < W; ++w) {
            const uint64_t r0 = 64 * w, r1 = (r0 + 64 < N) ? r0 + 64 : N;
            unsigned digit;
            uint64_t pos;
            pk_digit_at(r0, dd, &digit, &pos);
            uint64_t word = __atomic_load_n(&S[w], __ATOMIC_RELAXED);
            for (uint64_t r = r0; r < r1; ++r) {
                if (digit == 2u && pk_get(S, r - 2 * dd) && pk_get(S, r - dd))
                    word |= (uint64_t)1 << (r - r0);
                if (++pos == dd) {   /* next cell starts the next run of digit i */
                    pos = 0;
                    digit = (digit + 1u) % 3u;
                }
            }
            __atomic_store_n(&S[w], word, __ATOMIC_RELAXED);
        }
        d *= 3u;
    }

    /* ReduceAll: same digits, same order: every 0 or 1 cell &= !(its * sibling). */
    d = 1;
    for (int i = 1; i <= n; ++i) {
        const uint64_t dd = d;
        #pragma omp parallel for schedule(static)
        for (uint64_t w = 0; w < W; ++w) {
            const uint64_t r0 = 64 * w, r1 = (r0 + 64 < N) ? r0 + 64 : N;
            unsigned digit;
            uint64_t pos;
            pk_digit_at(r0, dd, &digit, &pos);
            uint64_t word = __atomic_load_n(&S[w], __ATOMIC_RELAXED);
            for (uint64_t r = r0; r < r1; ++r) {
                if (digit != 2u && pk_get(S, r + (2u - digit) * dd))
                    word &= ~((uint64_t)1 << (r - r0));
                if (++pos == dd) {
                    pos = 0;
                    digit = (digit + 1u) % 3u;
                }
            }
            __atomic_store_n(&S[w], word, __ATOMIC_RELAXED);
        }
        d *= 3u;
    }
    restore_threads(prev_threads);
}

/* The packed state as the dense LSB-first bitmap: byte k holds cubes 8k..8k+7. */
void oracle_packed_bitmap(int n, const uint64_t *S, uint8_t *out)
{
    const uint64_t bytes = (oracle_pow3(n) + 7) / 8;
    for (uint64_t k = 0; k < bytes; ++k)
        out[k] = (uint8_t)(S[k >> 3] >> (8 * (k & 7)));
}

/* The set cubes of a packed state in ascending rho, as (mask, value) pairs
 * (oracle_encode); writes at most cap pairs, returns the number of set cubes. */
uint64_t oracle_packed_list(int n, const uint64_t *S, uint32_t *pairs, uint64_t cap)
{
    const uint64_t W = (oracle_pow3(n) + 63) / 64;
    uint64_t k = 0;
    for (uint64_t w = 0; w < W; ++w)
        for (uint64_t x = S[w]; x; x &= x - 1) {   /* the set bits of word w, lowest first */
            const uint64_t rho = 64 * w + (uint64_t)__builtin_ctzll(x);
            if (k < cap) oracle_encode(n, rho, &pairs[2 * k], &pairs[2 * k + 1]);
            ++k;
        }
    return k;
}
