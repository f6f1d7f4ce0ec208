/*
 * dqmc.h -- C ABI of libdqmc.so, the GB300 (sm_103a) dense ternary
 * prime-implicant sweep of DenseQMC (arXiv 2302.10083).
 *
 * Problem (Section 1, "The Quine-McCluskey method", step 1; Section 2,
 * Definitions of implicant and prime): given the truth table of
 * f : {0,1}^n -> {0,1}, find every prime implicant of f.  Don't-cares are an
 * extension: implicants are taken over the support I = ON u DC, and a prime
 * whose minterms are all don't-cares is kept.
 *
 * Conventions (bind every entry point):
 *  - Variable x_i (i = 1..n) is ternary digit i with weight 3^(i-1); a cube
 *    s in {0,1,*}^n has index rho(s) = sum_i 3^(i-1) rho(s_i) with rho(0)=0,
 *    rho(1)=1, rho(*)=2 (Section 4.2, the notation rho).
 *  - Truth tables: ceil(2^n / 8) bytes, LSB first; minterm t = sum_i 2^(i-1) x_i
 *    is bit t & 7 of byte t >> 3.  Bits t >= 2^n of the last byte are ignored.
 *  - Prime bitmap: dense, unpadded, LSB first; bit rho(s) (byte rho >> 3, bit
 *    rho & 7) is 1 iff s is a prime implicant.  dqmc_bitmap_bytes(n) =
 *    ceil(3^n / 8) bytes; bits >= 3^n of the last byte are 0.
 *  - List: pairs of uint32 (mask, value) in ascending rho: mask bit i-1 is 1
 *    iff s_i is 0 or 1, value bit i-1 = s_i for those digits, else 0.  Cube s
 *    covers minterm t iff (t & mask) == value.  out_pairs[2k] = mask,
 *    out_pairs[2k+1] = value.
 *  - 0 <= n <= DQMC_MAX_N.  n = 0 has one cube (the empty product), prime iff
 *    f = 1.
 *
 * Errors: every call returns DQMC_OK (0) or a negative status and never
 * aborts.  DQMC_EINVAL for a bad argument (n > DQMC_MAX_N, NULL on_bits, a
 * workspace that is too small or misaligned), DQMC_ENOMEM when device memory
 * cannot be had, DQMC_ETRUNC when a list does not fit in `cap` pairs (the
 * first cap pairs and the true count are still written), DQMC_ECUDA for a CUDA
 * runtime error (the call clears it; the context stays usable), DQMC_ETIMEOUT
 * when a bounded device wait gave up.
 *
 * Ownership: the caller owns every buffer it passes.  Host entry points copy
 * inputs to the device and results back; the device memory they use comes from
 * a per-device cache owned by the library (released by dqmc_release()).  The
 * *_dev entry points allocate nothing: the caller passes a device workspace of
 * at least dqmc_workspace_bytes(n) bytes and every device pointer.
 *
 * Thread safety: host entry points serialise on a per-device lock; *_dev
 * entry points only enqueue work on the given stream and may be called
 * concurrently with different workspaces.
 */
#ifndef DQMC_H
#define DQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    DQMC_OK = 0,
    DQMC_EINVAL = -1,
    DQMC_ENOMEM = -2,
    DQMC_ETRUNC = -3,
    DQMC_ECUDA = -4,
    DQMC_ETIMEOUT = -5
};

/* Largest n handled: the padded state of n = 25 (3^20 rows of 32 bytes,
 * 111.6 GB) holds its own bitmap (105.9 GB) when the bitmap is written over it
 * (the host entry points do so at n = 25), well inside the 288 GB of one
 * GB300. */
#define DQMC_MAX_N 25

/* Human-readable text for a status code (static storage, never NULL). */
const char *dqmc_strerror(int status);

/* Library version as major*10000 + minor*100 + patch. */
int dqmc_version(void);

/* ceil(3^n / 8): bytes of the prime bitmap of an n-variable function
 * (0 for n > DQMC_MAX_N). */
uint64_t dqmc_bitmap_bytes(uint32_t n);

/* Bytes a device bitmap buffer must have for the *_dev calls: the bitmap
 * rounded up to a multiple of 16; the padding is written as zeros. */
uint64_t dqmc_bitmap_alloc_bytes(uint32_t n);

/* Device workspace needed by dqmc_primes_dev / dqmc_list_dev for this n
 * (0 for n > DQMC_MAX_N).  It holds the padded ternary state (3^(n-5) rows of
 * 32 bytes for n >= 13), a control block (error word, tile tickets, one
 * look-back word per bitmap tile) and the list scan counters. */
uint64_t dqmc_workspace_bytes(uint32_t n);

/* ------------------------------------------------------------------ host API
 * Host buffers in and out; synchronous.  dc_bits may be NULL (no don't-cares). */

/* Prime bitmap of f (Algorithm 3 of Section 4.1 computed on the device; the
 * result is the set of Section 2's prime implicants).  out_prime_bitmap:
 * caller-owned, dqmc_bitmap_bytes(n) bytes; NULL computes and discards it. */
int dqmc_primes(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
                uint8_t *out_prime_bitmap);

/* Number of prime implicants (the popcount of the bitmap). */
int dqmc_count(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
               uint64_t *out_count);

/* The primes as (mask, value) pairs in ascending rho (the output extraction
 * step of Algorithm 4, Section 4.2).  out_pairs: caller-owned, 2*cap uint32.
 * *out_count receives the number of primes even when it exceeds cap
 * (status DQMC_ETRUNC, first cap pairs written).  When out_pairs is pinned
 * host memory the device can address (cudaHostAlloc / cudaHostRegister,
 * 8-byte aligned), the kernels write the list into it directly (over
 * NVLink-C2C on a Grace-based node) and no copy follows the sweep; otherwise
 * the list goes through a device buffer and one copy. */
int dqmc_list(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
              uint32_t *out_pairs, uint64_t cap, uint64_t *out_count);

/* Flags of the *_ex entry points. */
enum {
    /* Sweep the complement: the prime implicants of not-f, whose implicants
     * are taken over (not ON) u DC (a don't-care of f is one of not-f too).
     * Their disjunction is the complete sum of not-f, so De Morgan turns them
     * into the clauses of f's prime CNF: clause k is the OR over the literals
     * of prime k with each literal negated (Section 1, the DNF / CNF
     * duality of the Quine-McCluskey problem). */
    DQMC_COMPLEMENT = 1
};

/* dqmc_primes / dqmc_count with flags (0 or DQMC_COMPLEMENT; any other bit:
 * DQMC_EINVAL).  out_prime_bitmap and out_count may each be NULL. */
int dqmc_primes_ex(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
                   uint32_t flags, uint8_t *out_prime_bitmap, uint64_t *out_count);

/* dqmc_list with flags (as dqmc_primes_ex). */
int dqmc_list_ex(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
                 uint32_t flags, uint32_t *out_pairs, uint64_t cap,
                 uint64_t *out_count);

/* Largest n of dqmc_sparse_list: 2n code bits plus the control flag fit
 * 64 bits. */
#define DQMC_SPARSE_MAX_N 30

/* SparseQMC on the GPU (Section 5, "SparseQMC"; Algorithm 1 level by level):
 * the same primes as dqmc_list, found from the support's minterms upward
 * (level w = the implicants with w wildcards, as a list and a hash set with
 * linear probing; a new implicant is made only at a position with no
 * wildcard before it, then every merge pair of it is flagged redundant; the
 * unflagged cubes of a level are prime).  Its work and memory follow the
 * number of implicants, not 3^n, so it suits sparse functions (the paper
 * finds it faster than the dense sweep up to about 50-60% density) and n up
 * to DQMC_SPARSE_MAX_N.  flags: 0 or DQMC_COMPLEMENT.  out_pairs: caller-owned,
 * 2*cap uint32, (mask, value) pairs in ascending rho as dqmc_list;
 * *out_count receives the number of primes (DQMC_ETRUNC when it exceeds cap).
 * Device memory is allocated for the call and freed before it returns
 * (DQMC_ENOMEM when the levels do not fit).  Synchronous. */
int dqmc_sparse_list(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
                     uint32_t flags, uint32_t *out_pairs, uint64_t cap,
                     uint64_t *out_count);

/* Largest n of dqmc_cover (two 32-bit words per minterm of device state). */
#define DQMC_COVER_MAX_N 26

/* The second step of the Quine-McCluskey method (Section 1: choose a subset
 * of the prime implicants covering the function; a SetCover instance, so a
 * heuristic): the essential primes (each the only one covering some ON
 * minterm), then, while an ON minterm is uncovered, the prime covering the
 * most uncovered ON minterms (ties: the lowest index).  Don't-care minterms
 * need no cover.  This is not part of the paper's method.
 * pairs: the primes as (mask, value) uint32 pairs (count of them), e.g. from
 * dqmc_list or dqmc_sparse_list.  out_sel: caller-owned, count uint32,
 * receives the selected primes' indexes in ascending order; *out_nsel their
 * number.  DQMC_EINVAL if the given cubes do not cover the ON-set.  Device
 * memory is allocated for the call and freed before it returns.
 * Synchronous. */
int dqmc_cover(uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
               const uint32_t *pairs, uint64_t count, uint32_t *out_sel,
               uint64_t *out_nsel);

/* Free the device buffers cached by the host API on the current device.  It
 * waits for a host call in progress on that device; a later call allocates
 * them again.  The device's stream and count word stay until exit. */
void dqmc_release(void);

/* ---------------------------------------------------------------- device API
 * All pointers are device pointers (cudaMalloc / torch data_ptr), 16-byte
 * aligned.  Work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 * default stream) and the call returns without waiting.  d_work must be at
 * least dqmc_workspace_bytes(n) bytes, 256-byte aligned, and must not be used
 * by another call that overlaps on the device.  Inputs are read-only. */

/* The prime bitmap, as dqmc_primes (Algorithm 3 of Section 4.1: MergeAll,
 * then ReduceAll; the set cells are Section 2's prime implicants).
 * d_on, d_dc: ceil(2^n/8)-byte truth tables (d_dc may be NULL).
 * d_bitmap: dqmc_bitmap_alloc_bytes(n) bytes, receives the prime bitmap.  For
 * n >= 13 it may be d_work itself: the bitmap is then written over the state
 * at the start of the workspace (the state is larger: 32 bytes per 243 cells),
 * so one array holds the sweep (111.6 GB at n = 25 instead of 217.5 GB; the
 * paper's single in-place array, Table 1), and the bitmap stays there until
 * the workspace is used again.  Any other overlap with d_work is DQMC_EINVAL.
 * d_count: one uint64, receives the number of primes (may be NULL). */
int dqmc_primes_dev(uint32_t n, const void *d_on, const void *d_dc,
                    void *d_bitmap, uint64_t *d_count,
                    void *d_work, uint64_t work_bytes, void *stream);

/* Same sweep, then compaction of the bitmap into (mask, value) pairs in
 * ascending rho (the output extraction step of Algorithm 4, Section 4.2).
 * d_pairs: 2*cap uint32 (may be NULL when cap = 0).  d_count: one uint64,
 * receives the number of primes (required).  Pairs at index >= cap are not
 * written; the caller compares *d_count with cap after the stream completes. */
int dqmc_list_dev(uint32_t n, const void *d_on, const void *d_dc,
                  void *d_bitmap, uint32_t *d_pairs, uint64_t cap,
                  uint64_t *d_count, void *d_work, uint64_t work_bytes,
                  void *stream);

/* dqmc_primes_dev and dqmc_list_dev with flags (0 or DQMC_COMPLEMENT; any
 * other bit: DQMC_EINVAL).  With DQMC_COMPLEMENT the first pass reads the
 * same truth tables and forms the support (not ON) u DC on the fly: no other
 * input is read or written. */
int dqmc_primes_dev_ex(uint32_t n, const void *d_on, const void *d_dc,
                       uint32_t flags, void *d_bitmap, uint64_t *d_count,
                       void *d_work, uint64_t work_bytes, void *stream);
int dqmc_list_dev_ex(uint32_t n, const void *d_on, const void *d_dc,
                     uint32_t flags, void *d_bitmap, uint32_t *d_pairs,
                     uint64_t cap, uint64_t *d_count, void *d_work,
                     uint64_t work_bytes, void *stream);

/* Synchronises `stream`, then reports how the last sweep that used d_work
 * ended: DQMC_OK; DQMC_ETIMEOUT when a bounded device wait of the sweep (the
 * bitmap pass waiting for its tile's bulk copies, or the list's look-back
 * waiting for the tiles before it) gave up after one second; DQMC_ECUDA when
 * a kernel found an index out of bounds and skipped the access.  In both
 * error cases the outputs are not valid: once the error word is set, the
 * bitmap pass's tiles leave without loading or writing anything (a tile whose
 * copies did not land waits a second bounded time for them before it leaves).
 * The next sweep on the workspace clears the word.  Device waits never spin
 * unbounded. */
int dqmc_dev_status(uint32_t n, const void *d_work, uint64_t work_bytes, void *stream);

/* For callers that cannot allocate device memory (an application whose own
 * pool owns the device memory, or code on a latency path where an allocation,
 * which may synchronise the device, is not acceptable).  Same result as
 * dqmc_primes_dev, without a workspace argument: the workspace is a static
 * device array of 2 MiB inside the library (held by every GPU that loads the
 * library until the process exits), so only n <= 15 is accepted; larger n
 * returns DQMC_EINVAL.  Nothing is allocated: no cudaMalloc, no cudaFree.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents (each sweep clears
 * what must start at zero); calls that overlap on the GPU, on any stream or
 * thread, race on it and must be serialised by the caller.  d_on, d_dc,
 * d_bitmap, d_count and stream as for dqmc_primes_dev.  The array's device
 * address is cached per device for the life of the process, so resetting a
 * device (cudaDeviceReset) after the first call on it is not supported.  The
 * paper has no counterpart: this is a deployment convenience. */
int dqmc_primes_dev_static(uint32_t n, const void *d_on, const void *d_dc,
                           void *d_bitmap, uint64_t *d_count, void *stream);

/* dqmc_dev_status for the static workspace of the current device: synchronises
 * `stream`, then reports how the last dqmc_primes_dev_static sweep on this
 * device ended (DQMC_OK, DQMC_ETIMEOUT or DQMC_ECUDA as for dqmc_dev_status;
 * the error word lives in the static array, which the caller cannot address).
 * n as given to that sweep (n > 15: DQMC_EINVAL).  Allocates nothing.  The
 * paper has no counterpart. */
int dqmc_dev_status_static(uint32_t n, void *stream);

/* Compaction alone (the output extraction step of Algorithm 4, Section 4.2):
 * (mask, value) pairs, in ascending rho, of the set bits of an existing dense
 * bitmap of an n-variable function.  d_work as above (only its scan part is
 * used).  d_count: one uint64 (required). */
int dqmc_compact_dev(uint32_t n, const void *d_bitmap, uint32_t *d_pairs,
                     uint64_t cap, uint64_t *d_count, void *d_work,
                     uint64_t work_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_H */
