/* dqmc_batch.h -- many independent small functions in one CUDA-graph launch.
 *
 * Each function of the batch is swept exactly as dqmc_primes sweeps a single
 * function (DenseQMC, arXiv 2302.10083, Algorithm 3 in Section 4.1: MergeAll,
 * then ReduceAll; output as in Algorithm 4, Section 4.2).  The paper runs one
 * function at a time and has no counterpart to batching; the arithmetic and
 * the results are unchanged by it.
 *
 * How: functions are grouped by n, and each n is swept by one of two paths
 * (its launch configuration, below):
 *   DQMC_BATCH_PATH_SMEM   (5 <= n <= 14) a function's whole state stays in
 *       shared memory from truth table to bitmap: fns_per_cta functions per
 *       CTA, threads_per_fn threads each, the high digits merged and reduced
 *       digits_per_step at a time; or one function per cluster of
 *       ctas_per_fn = 3 (n = 13, 14) or 9 (n = 14) CTAs, the top one or two
 *       high digits spread over the cluster (distributed shared memory); for
 *       n = 14, ctas_per_fn = 1 is one CTA per SM taking functions in turn
 *       and their three top-digit thirds one after the other (the '*' third
 *       parked in a workspace slot);
 *   DQMC_BATCH_PATH_TILES  n <= 12: one CTA per function (the kernel of the
 *       single-function sweep); n = 13, 14: the streaming pass kernels, one
 *       launch per pass for all functions of that n, each function with its
 *       own device state in a library-owned workspace.
 * The library captures the launches into a CUDA graph (one branch per n) and
 * launches the graph; a later call with the same functions, buffers and
 * configurations launches the same graph again.  dqmc_batch_autotune times
 * every launchable configuration of each n on a given batch and keeps the
 * fastest.
 */
#ifndef DQMC_BATCH_H
#define DQMC_BATCH_H

#include <stdint.h>

#include "dqmc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest n a batch function may have. */
#define DQMC_BATCH_MAX_N 14

/* Paths of one n (dqmc_batch_config.path). */
#define DQMC_BATCH_PATH_SMEM 0
#define DQMC_BATCH_PATH_TILES 1

/* Launch configuration of the functions of one n.  For the TILES path the
 * other fields are ignored (reported as 256, 1, 2, 1).  SMEM needs
 * 5 <= n <= 14, threads_per_fn a multiple of 32 (>= 32),
 * 1 <= fns_per_cta <= 15, digits_per_step 2 or 3,
 * threads_per_fn * fns_per_cta <= 1024, ctas_per_fn 1, 3 (n = 13, 14) or
 * 9 (n = 14) with fns_per_cta = 1 when it is above 1 or n = 14, and
 * fns_per_cta * 3^(n-5-c) * 32 bytes of shared memory per CTA <= 227 KB,
 * c = 0, 1, 2 for 1, 3, 9 CTAs per function (c = 1 for n = 14 on one CTA).
 * The server (dqmc_server.h) runs n = 14 on nine-CTA clusters when the
 * table says one CTA. */
typedef struct {
    uint32_t path;
    uint32_t threads_per_fn;   /* threads per function (per CTA of a cluster) */
    uint32_t fns_per_cta;
    uint32_t digits_per_step;
    uint32_t ctas_per_fn;
} dqmc_batch_config;

/* Sweep nfun functions on the current CUDA device, enqueued on `stream`
 * (a cudaStream_t; NULL = legacy default stream).
 *
 * Host arrays, nfun entries each (read during the call only):
 *   n[f]       variables of function f, 0 <= n[f] <= DQMC_BATCH_MAX_N;
 *   tt_off[f]  byte offset in d_tt_arena of f's ON truth table
 *              (ceil(2^n / 8) bytes, the layout of dqmc_primes' on_bits);
 *              a multiple of 4 when n[f] >= 5;
 *   dc_off     NULL (no don't-cares anywhere) or, per function, the byte
 *              offset of its DC table in d_tt_arena, UINT64_MAX for none;
 *              same alignment as tt_off;
 *   bm_off[f]  byte offset in d_out_bitmaps of f's prime bitmap, a multiple
 *              of 16.  The slot is dqmc_bitmap_alloc_bytes(n[f]) bytes: the
 *              dense bitmap of dqmc_primes (bit rho set iff cube rho is a
 *              prime), then zero bytes up to the slot's end.  Slots must not
 *              overlap one another or the tables.
 * Device buffers (caller-owned, on the current device):
 *   d_tt_arena     the truth tables, 4-byte aligned;
 *   d_out_count    nfun uint64, f's number of prime implicants;
 *   d_out_bitmaps  the bitmap slots, 16-byte aligned.
 *
 * The library owns the workspace (the function tables; device states and
 * control blocks of the n = 13, 14 functions on the TILES path; when the batch
 * has n = 14 functions, one 210 KB slot per SM for the one-CTA thirds) and
 * the graph;
 * both stay allocated until dqmc_batch_release.  Calls must not overlap on
 * the device (they share that workspace): order them on one stream, or
 * synchronise between them.  The call returns once the graph is enqueued;
 * the outputs are ready when `stream` reaches that point.
 *
 * Returns DQMC_OK; DQMC_EINVAL for nfun > 2^24, a null array or buffer, an n
 * above DQMC_BATCH_MAX_N or a misaligned offset or pointer; DQMC_ENOMEM when
 * the workspace does not fit; DQMC_ECUDA for another CUDA error.  nfun = 0
 * returns DQMC_OK and does nothing. */
int dqmc_batch_run(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                   const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps, const uint64_t *bm_off,
                   void *stream);

/* dqmc_batch_run in one persistent launch (captured in the graph after the
 * zeroing of the counts and of one queue counter per n): one CTA of 1024
 * threads per SM takes the batch's n in turn, largest first, splitting its
 * threads and shared memory into groups of that n's shape, and each group
 * takes whole functions one at a time from the n's queue (n <= 4: one warp
 * per function, cubes tested against the definitions; 5 <= n <= 13: the
 * n's SMEM shape from the launch table when it is one CTA per function,
 * else the built-in one, as many functions at once as the CTA's threads and
 * shared memory hold; n = 14: the whole CTA, the thirds of the top digit in
 * turn).  Same arguments, rules, workspace, results and errors as
 * dqmc_batch_run; the two share the cached graph, so switching between them
 * captures a new one. */
int dqmc_batch_run_one_launch(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                              const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps,
                              const uint64_t *bm_off, void *stream);

/* Bytes of device workspace a batch with these n's takes (function tables,
 * control blocks and states of the n = 13, 14 functions on the TILES path,
 * the n = 14 scratch slots), sized for the configurations set now and the
 * current device's SM count (160 slots when no device answers).  0 if an n
 * is out of range. */
uint64_t dqmc_batch_workspace_bytes(uint32_t nfun, const uint32_t *n);

/* The configuration used for functions of n variables (process-wide; the
 * built-in defaults until set or tuned).  DQMC_EINVAL for n above
 * DQMC_BATCH_MAX_N or a null pointer. */
int dqmc_batch_get_config(uint32_t n, dqmc_batch_config *out);

/* Set it.  DQMC_EINVAL if the configuration breaks a rule above.  The next
 * dqmc_batch_run captures a new graph. */
int dqmc_batch_set_config(uint32_t n, const dqmc_batch_config *cfg);

/* Autotuner: for every n present in the batch (same arguments and rules as
 * dqmc_batch_run), time each launchable configuration (the TILES path and
 * every SMEM shape with threads_per_fn in 32..1024, fns_per_cta in
 * {1,2,3,4,6,8}, digits_per_step 2 and 3, ctas_per_fn 1, 3, 9): one untimed run, then the mean of
 * `reps` runs, each a launch of that n's functions alone on `stream`, timed
 * with CUDA events.  The fastest becomes that n's configuration.  Blocks
 * until done.  out_ms (NULL, or DQMC_BATCH_MAX_N + 1 floats) gets each n's
 * best time in ms, -1 for n not in the batch.  The output buffers are
 * overwritten by the trial runs; call dqmc_batch_run for the results.
 * DQMC_EINVAL as for dqmc_batch_run, or reps outside 1..1000. */
int dqmc_batch_autotune(uint32_t nfun, const uint32_t *n, const uint64_t *tt_off, const void *d_tt_arena,
                        const uint64_t *dc_off, uint64_t *d_out_count, void *d_out_bitmaps, const uint64_t *bm_off,
                        uint32_t reps, void *stream, float *out_ms);

/* Free the current device's batch workspace and graph (after the work that
 * uses them is done).  Returns DQMC_OK or DQMC_ECUDA. */
int dqmc_batch_release(void);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_BATCH_H */
