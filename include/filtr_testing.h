/* filtr_testing.h -- test hooks of the GB300 alignment library (not for
 * production use).  They exercise failure paths without faulting the GPU. */
#ifndef FILTR_TESTING_H
#define FILTR_TESTING_H

#include "filtr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Run the intra-pair long kernel of filtr_align_long on (q, M) x (r, N) (DEVICE
 * codes, full matrix or band per params, traceback ignored) with the first row
 * strip never publishing its progress, so every later strip's bounded wait runs
 * out after timeout_ns nanoseconds.  Returns FILTR_ERR_TIMEOUT when the
 * timeout path works (every warp stopped and the context stays usable);
 * M must exceed 512 rows (at least two strips). */
filtr_status filtr_test_long_timeout(filtr_ctx *ctx, const filtr_params *params, const uint8_t *q,
                                     uint32_t M, const uint8_t *r, uint32_t N,
                                     uint64_t timeout_ns);

/* Make filtr_align_long use the checkpointed X-drop traceback (state of every
 * `interval`-th antidiagonal kept, segments recomputed backwards) even when
 * the whole traceback would fit; interval 0 restores the automatic choice. */
filtr_status filtr_test_set_checkpoint(filtr_ctx *ctx, int32_t interval);

/* With on != 0, the checkpointed X-drop traceback skips its single pass (every
 * segment's traceback kept in the workspace and walked once) and takes the
 * path it otherwise falls back to when that pool runs out: a forward sweep
 * without traceback, then each segment recomputed backwards and walked. */
filtr_status filtr_test_force_recompute(filtr_ctx *ctx, int32_t on);

/* Group width W (1, 2, 4, 8, 16 or 32: a window of 256 W slots, run by W warps,
 * except that the int16x2 sweep runs W = 2 as one warp of 16-slot threads) at
 * which filtr_align_batch first runs X-drop / Z-drop pairs (those that outgrow
 * it are rerun wider); 0 restores the default.  Results do not depend on it. */
filtr_status filtr_test_set_first_width(filtr_ctx *ctx, int32_t warps);

/* Which planner filtr_align_batch uses for tiled batches: 0 the default (the
 * device planner from a few hundred pairs, see filtr_stats.device_plan), 1 the
 * host planner always, 2 the device planner for every batch it can serve
 * (not X-drop, not one launch per pair; batches whose traceback needs more than
 * one wave still fall back to the host).  Results do not depend on it. */
filtr_status filtr_test_set_device_plan(filtr_ctx *ctx, int32_t mode);

/* Entries of each per-warp shared-memory wavefront ring of filtr_search_batch's
 * score pass (a power of two from 32 to 4096; 0 restores the default).
 * Wavefronts wider than the ring continue in global memory, so results do not
 * depend on it; it trades shared memory (occupancy) against load latency. */
filtr_status filtr_test_set_search_ring(filtr_ctx *ctx, int32_t entries);

/* Cell width of the antidiagonal (X-drop / Z-drop) sweep: 0 the default (two
 * cells per register for affine pairs whose threshold leaves room, int32
 * otherwise), 1 int32 always, 2 two cells per register with the base score
 * never moved, so pairs whose scores drift more than about 16,000 from where
 * they started leave the 16-bit range and are rerun in int32
 * (filtr_stats.pairs_xd16_rerun counts them).  Results do not depend on it. */
filtr_status filtr_test_set_packed_sweep(filtr_ctx *ctx, int32_t mode);

/* Run filtr_align_batch's host planner, with no device and the default shape
 * costs, on n pairs of lengths q_len[p] x r_len[p] (HOST arrays) under params.
 * Each wave's traceback may use tb_budget_words 32-bit words.  Outputs are HOST
 * arrays the caller allocates:
 *   order[n]       : the planned pairs in launch order (waves, then the groups
 *                    of one kernel shape inside a wave, each cost-descending),
 *                    then the pairs with nothing to evaluate;
 *   wave[n]        : per pair id, its wave (UINT32_MAX: nothing to evaluate);
 *   tb_off[n], tb_words[n] : per pair id, its traceback area inside its wave's
 *                    (words; 0 with traceback off);
 *   kernel[n]      : per pair id, family << 16 | R << 8 | warps (family 0 the
 *                    int32 tile, 1 the antidiagonal sweep, 3 the int16x2 tile;
 *                    R rows per lane of a tile or slots per lane of the sweep;
 *                    warps the sweep's first group width);
 *   wave_info[3n]  : per wave, its traceback words, then the first and one past
 *                    the last position of its pairs in order;
 *   counts[3]      : planned pairs, waves, pairs with nothing to evaluate.
 * FILTR_ERR_NOMEM when one pair's traceback exceeds tb_budget_words;
 * FILTR_ERR_INVALID for bad parameters or NULL arrays. */
filtr_status filtr_test_plan_host(const filtr_params *params, uint32_t n, const uint32_t *q_len,
                                  const uint32_t *r_len, uint64_t tb_budget_words, uint32_t *order,
                                  uint32_t *wave, uint64_t *tb_off, uint64_t *tb_words,
                                  uint32_t *kernel, uint64_t *wave_info, uint32_t *counts);

#ifdef __cplusplus
}
#endif
#endif /* FILTR_TESTING_H */
