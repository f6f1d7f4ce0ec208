/* dqmc_server.h -- a serving loop for prime-implicant jobs on one GPU.
 *
 * Each job is one function, swept exactly as dqmc_primes sweeps it (DenseQMC,
 * arXiv 2302.10083, Algorithm 3 in Section 4.1; output as in Algorithm 4,
 * Section 4.2).  The paper has no counterpart to serving; the arithmetic and
 * each job's result are the same as a dqmc_primes call on that function.
 *
 * The server owns one block of device memory (its HBM budget) and a
 * scheduler thread.  Jobs wait in a queue until their footprint fits in the
 * budget: the device copy of their truth tables, their state (n >= 15) and
 * their bitmap.  Admitted jobs run while others are still running:
 *   * jobs with n <= 14 that are waiting together are swept by one batched
 *     launch per n (whole functions in shared memory, the launch shapes of
 *     dqmc_batch_get_config; a cluster of nine CTAs per function at n = 14,
 *     so that no job needs a workspace);
 *   * jobs with n >= 15 run on their own CUDA stream (several at a time).
 * When a job's kernels are done, its state and tables are freed at once and
 * the next jobs are admitted; its bitmap stays in device memory until the
 * client frees the job (or at once, for DQMC_JOB_DISCARD_BITMAP).
 *
 * Errors: if a launch cannot be enqueued, the server keeps that CUDA error
 * (DQMC_ECUDA or DQMC_ENOMEM) and returns it from submit, query, wait and
 * destroy; the jobs of that launch and every job still queued are marked
 * done with no result, and nothing more is started.
 */
#ifndef DQMC_SERVER_H
#define DQMC_SERVER_H

#include <stdint.h>

#include "dqmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dqmc_server dqmc_server;

/* Server modes. */
#define DQMC_SERVER_CONCURRENT 0   /* continuous batching, several jobs in flight */
#define DQMC_SERVER_SERIAL 1       /* one job at a time, in arrival order (the
                                      one-by-one baseline) */

/* Job flags. */
#define DQMC_JOB_DISCARD_BITMAP 1u /* free the bitmap when the job is done;
                                      only the count is kept */

/* Job states. */
#define DQMC_JOB_QUEUED 0
#define DQMC_JOB_RUNNING 1
#define DQMC_JOB_DONE 2

/* Create a server on the current CUDA device.  hbm_bytes of device memory
 * are allocated now and shared by all jobs; streams (1..32) CUDA streams run
 * the n >= 15 jobs; mode is DQMC_SERVER_CONCURRENT or DQMC_SERVER_SERIAL.
 * Returns DQMC_OK (and *out), DQMC_EINVAL, DQMC_ENOMEM or DQMC_ECUDA. */
int dqmc_server_create(uint64_t hbm_bytes, uint32_t streams, int mode, dqmc_server **out);

/* Wait for every admitted and queued job, stop the scheduler and free the
 * server's memory.  Device pointers returned by dqmc_server_query become
 * invalid. */
int dqmc_server_destroy(dqmc_server *s);

/* Device memory a job of n variables takes while it runs (tables, state,
 * bitmap, count); 0 for n > DQMC_MAX_N. */
uint64_t dqmc_server_job_bytes(uint32_t n, int with_dc);

/* Queue one job: n variables, truth tables in host memory in the layout of
 * dqmc_primes (on_bits required, dc_bits may be NULL), copied during the
 * call.  *job receives the job's id.  Does not wait for the GPU.
 * DQMC_EINVAL for n > DQMC_MAX_N, a null argument, or a job whose footprint
 * exceeds the whole budget. */
int dqmc_server_submit(dqmc_server *s, uint32_t n, const uint8_t *on_bits, const uint8_t *dc_bits,
                       uint32_t flags, uint64_t *job);

/* A job's state (DQMC_JOB_*).  Once done: *count = its number of prime
 * implicants, *d_bitmap = its dense prime bitmap in device memory
 * (dqmc_bitmap_alloc_bytes(n) bytes; NULL when discarded), valid until the
 * job is freed.  Times are steady-clock nanoseconds: submission and
 * completion (completion = the host learning that the job's last kernel is
 * done).  Any output pointer may be NULL.  DQMC_EINVAL for an unknown job. */
int dqmc_server_query(dqmc_server *s, uint64_t job, int *state, uint64_t *count, const void **d_bitmap,
                      uint64_t *t_submit_ns, uint64_t *t_done_ns);

/* Copy a done job's dense prime bitmap (dqmc_bitmap_bytes(n) bytes) into
 * host memory out (cap bytes).  DQMC_EINVAL if the job is unknown, not done,
 * discarded, or cap is too small. */
int dqmc_server_copy_bitmap(dqmc_server *s, uint64_t job, uint8_t *out, uint64_t cap);

/* Block until the job is done or timeout_ms passes (DQMC_ETIMEOUT). */
int dqmc_server_wait(dqmc_server *s, uint64_t job, uint32_t timeout_ms);

/* Forget a done job and free its bitmap.  DQMC_EINVAL if unknown or not done. */
int dqmc_server_free_job(dqmc_server *s, uint64_t job);

/* Counters: out[0] jobs submitted, [1] done, [2] batched launches, [3] jobs
 * that ran in a batch, [4] device bytes in use now, [5] peak device bytes,
 * [6] most jobs running at one time, [7] budget. */
int dqmc_server_stats(dqmc_server *s, uint64_t out[8]);

/* Load generator for the serving benchmark: submit job j at t_arrive_s[j]
 * seconds after the call starts (steady clock; arrival times ascending),
 * each with DQMC_JOB_DISCARD_BITMAP, then wait for all of them.  Per job:
 * count_out[j] = its prime count, latency_s_out[j] = completion time minus
 * arrival time.  *span_s = last completion minus first arrival.  Jobs are
 * freed before return. */
int dqmc_server_replay(dqmc_server *s, uint32_t njobs, const double *t_arrive_s, const uint32_t *n,
                       const uint8_t *const *on_bits, const uint8_t *const *dc_bits, uint64_t *count_out,
                       double *latency_s_out, double *span_s);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_SERVER_H */
