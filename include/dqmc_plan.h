/*
 * dqmc_plan.h -- introspection of the pass plan libdqmc.so runs for a given n.
 *
 * The plan is the device schedule of Algorithm 3 (arXiv 2302.10083, Section
 * 4.1): MergeAll over every digit, then ReduceAll over every digit.  Merge
 * order and Reduce order are both free (the triples of one digit are
 * independent, and Section 6 notes that the Reduce layers can be swapped), so
 * the library merges the high digits in groups from the lowest up and
 * reduces them in groups; this call reports which groups, in which passes.
 * Host-only: it launches nothing and needs no GPU.
 */
#ifndef DQMC_PLAN_H
#define DQMC_PLAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Writes a NUL-terminated JSON description of the plan for n variables into
 * buf (at most cap bytes, truncated if needed) and returns the full length of
 * the JSON text, or DQMC_EINVAL (-1) for n > DQMC_MAX_N.  buf may be NULL when
 * cap is 0 (to query the length).  Fields:
 *   n; C (chunk digits, min(n, 5)); H (high digits, n - C);
 *   state_rows (32-byte rows of device state; 0 when one tile holds the whole
 *     function); out_tiles (tiles of the bitmap pass);
 *   passes[], one per kernel launch, each with
 *     kind: "whole" (n <= 12, one CTA per function) or "super" (a streaming
 *       pass over tiles of 3^7 rows);
 *     n_sb: tiles; sb: [digit, radix] of each high digit fixed per tile, in the
 *       order the tile index enumerates them (radix 2 while the digit is not
 *       merged yet, else 3);
 *     window (both kinds), step_size, n_steps, groups ("super" only): the
 *       launch shape (one launch of n_sb tiles: window = step_size = n_sb,
 *       n_steps = groups = 1);
 *     phases[] (one): load ("tt": truth table, "sparse": the rows whose group
 *       digits are 0/1, "full": every row); a, K (group digits a .. a+K-1);
 *       B (inner digits 0 .. B-1, carried for contiguous rows); merge, reduce
 *       (0/1: the pass merges / reduces its group digits); chunk_mask (bit i:
 *       the pass reduces chunk digit i); out (the pass writes the bitmap, the
 *       count and the list); nbr_a, nbr_K (bitmap pass: high digits nbr_a ..
 *       nbr_a+nbr_K-1 are reduced there too, each cell against its '*'
 *       neighbours in those digits read from the state as the previous pass
 *       left it; nbr_K = 0: none); tiles; fix (unused, empty). */
int dqmc_plan_json(uint32_t n, char *buf, uint64_t cap);

/* Number of passes (kernel launches of the sweep) for n variables, or
 * DQMC_EINVAL for n > DQMC_MAX_N. */
int dqmc_plan_passes(uint32_t n);

/* Bytes pass `pass` must move by its design: 32 bytes per state row it reads
 * and per state row it writes, plus the truth tables it reads and the bitmap
 * bytes it writes.  0 for a bad n or pass. */
uint64_t dqmc_pass_bytes(uint32_t n, int pass, int with_dc);

/* Enqueue pass `pass` alone (arguments as dqmc_list_dev).  Running passes
 * 0 .. dqmc_plan_passes(n)-1 in order on one stream is exactly dqmc_list_dev
 * (d_pairs != NULL) or dqmc_primes_dev (d_pairs == NULL, cap 0); pass 0 also
 * zeroes *d_count and the workspace's control block.  The last pass writes the
 * bitmap, the count and (if asked) the list.  Lets a caller put CUDA events
 * between the kernels of the sweep. */
int dqmc_sweep_pass_dev(uint32_t n, int pass, const void *d_on, const void *d_dc,
                        void *d_bitmap, uint32_t *d_pairs, uint64_t cap,
                        uint64_t *d_count, void *d_work, uint64_t work_bytes,
                        void *stream);

/* Enqueue passes first .. last-1 (0 <= first < last <= dqmc_plan_passes(n);
 * arguments as dqmc_list_dev), the same as calling dqmc_sweep_pass_dev for
 * each in turn.  Returns DQMC_EINVAL for a bad range. */
int dqmc_sweep_passes_dev(uint32_t n, int first, int last, const void *d_on, const void *d_dc, void *d_bitmap,
                          uint32_t *d_pairs, uint64_t cap, uint64_t *d_count, void *d_work, uint64_t work_bytes,
                          void *stream);

/* Self-test of the bounded device waits (no GPU fault, nothing hangs): zeroes
 * the control block of d_work, then runs one device wait on a counter that no
 * kernel ever sets, with a limit of wait_ns nanoseconds (at most 10^9).  A
 * following dqmc_dev_status() must return DQMC_ETIMEOUT, and the next sweep
 * on the same workspace runs normally.  n >= 13 (a workspace with a control
 * block).  Returns DQMC_OK once enqueued. */
int dqmc_selftest_timeout(uint32_t n, void *d_work, uint64_t work_bytes,
                          uint64_t wait_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_PLAN_H */
