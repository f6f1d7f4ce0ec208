/* dqmc_batch.h -- many independent small functions in one CUDA-graph launch.
 *
 * Each function of the batch is swept exactly as dqmc_primes sweeps a single
 * function (DenseQMC, arXiv 2302.10083, Algorithm 3 in Section 4.1: MergeAll,
 * then ReduceAll; output as in Algorithm 4, Section 4.2).  The paper runs one
 * function at a time and has no counterpart to batching; the arithmetic and
 * the results are unchanged by it.
 *
 * How: functions are grouped by n.  Functions with n <= 12 are swept by one
 * CTA each, with the whole state in shared memory; functions with n = 13 and
 * 14 by the streaming pass kernels, one launch per pass for all functions of
 * that n, each function with its own device state in a library-owned
 * workspace.  The library captures the whole sequence into a CUDA graph and
 * launches the graph; a later call with the same functions and buffers
 * launches the same graph again.
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
 * The library owns the workspace (device states of the n = 13, 14
 * functions, per-class control blocks, the function tables) and the graph;
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

/* Bytes of device workspace a batch with these n's takes (function tables,
 * control blocks, states of the n = 13, 14 functions).  0 if an n is out of
 * range. */
uint64_t dqmc_batch_workspace_bytes(uint32_t nfun, const uint32_t *n);

/* Free the current device's batch workspace and graph (after the work that
 * uses them is done).  Returns DQMC_OK or DQMC_ECUDA. */
int dqmc_batch_release(void);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_BATCH_H */
