/*
 * faco_batch.h -- many independent colonies on one GPU (libfaco.so).
 *
 * The paper runs one colony at a time and parallelises over its ants
 * (Sec. 5, OpenMP over ants); it has no batched form.  A batch runs `count`
 * independent colonies -- each exactly the colony of faco.h for its own
 * instance and seed -- through the same kernel launches: one launch of the
 * per-ant kernels covers every ant of every colony, one launch of each
 * colony kernel (iteration best, source, Eq. 2 rows, prefix sums) covers
 * every colony, and a whole iteration budget is replayed as one CUDA graph.
 * Small instances, which would leave most of the GPU idle one at a time,
 * then share it.
 *
 * Results: colony i of a batch is bit-identical to
 *   faco_create_ex(coords_xy[i], ns[i], k, p_i, ...) followed by the same
 *   faco_iterate(ants, budget) calls,
 * where p_i is *p with seed = seeds[i] (or p->seed when seeds is NULL).
 * The kernel choice per colony (a block of eight warps per ant on a segment
 * table in shared memory, or one warp per ant on explicit arrays compiled
 * for 2, 4 or 8 resident blocks of four ants per SM; chosen per size class
 * by a timing autotuner or fixed with faco_batch_set_plan) changes only the
 * speed, never a result.
 *
 * Conventions are those of faco.h: int status returns, int32 (x, y)
 * coordinates in [0, 2^24), int64 lengths, work enqueued on p->stream (NULL
 * = a stream the batch owns); faco_batch_iterate only enqueues, the other
 * calls synchronise.  A batch owns its device memory (one arena for the
 * colonies, one for the ants of the current ant count).
 */
#ifndef FACO_BATCH_H
#define FACO_BATCH_H

#include "faco.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct faco_batch faco_batch;

/* Largest instance a batch accepts (visited bits of one ant and of the
 * nearest-neighbour tour stay in shared memory). */
#define FACO_BATCH_MAX_N 262144

/* Creates `count` colonies (1..65535).  coords_xy[i] is a host array of
 * ns[i] (x, y) pairs, copied; ns[i] in 3..FACO_BATCH_MAX_N.  k as in
 * faco_create (2..32, clamped to n-1 per colony); when k > 16 every
 * instance needs n > 17 (one roulette width per batch).  p: NULL = defaults;
 * p->keep_ant_tours and p->keep_pre_ls must be 0 and p->seg_cap -1 (tables
 * sized per colony from shared memory) or 0 (explicit arrays for every
 * ant).  seeds: NULL, or `count` seeds replacing p->seed per colony.
 * Enqueues the set-up of Alg 2 for every colony (candidate lists, nearest-
 * neighbour tour, its local search, limits, tau = tau_max) without a host
 * synchronisation; coordinates are range-checked on the host first.
 * Errors: FACO_E_ARG, FACO_E_SIZE (an n above FACO_BATCH_MAX_N),
 * FACO_E_NOMEM, FACO_E_CUDA. */
int faco_batch_create(const int32_t* const* coords_xy, const int32_t* ns, int32_t count, int32_t k,
                      const faco_params* p, const uint64_t* seeds, faco_batch** out);

/* Enqueues `budget` iterations of every colony with `ants` ants each
 * (Alg 2 main loop).  The first call for an ant count allocates its
 * buffers and, unless a plan is fixed, times both per-ant kernels on each
 * size class of the batch (the per-ant kernels write only per-ant buffers,
 * so the trial launches change no colony state); the budget is then
 * captured once as a CUDA graph and replayed with one launch.  Errors:
 * FACO_E_ARG, FACO_E_NOMEM, FACO_E_CUDA. */
int faco_batch_iterate(faco_batch* b, int32_t ants, int32_t budget);

/* Waits for the enqueued work; FACO_E_CAPACITY / FACO_E_CUDA when a colony
 * raised a device error flag (FACO_E_TIMEOUT is reserved: no kernel of this
 * version waits on the device). */
int faco_batch_sync(faco_batch* b);

/* Global-best tour (ns[i] entries, len >= ns[i]; NULL to skip) and length of
 * colony i.  Synchronises.  Errors: FACO_E_ARG, FACO_E_SIZE. */
int faco_batch_best(faco_batch* b, int32_t i, int32_t* tour, int32_t len, int64_t* length_out);

/* Every colony's global-best tour, concatenated in colony order (sum of ns
 * entries; NULL to skip) and the `count` lengths (NULL to skip).  One
 * device gather, then one copy each.  Synchronises. */
int faco_batch_tours(faco_batch* b, int32_t* tours, int64_t* lengths);

/* Counters of colony i as faco_stats_get reports them for one colony
 * (kernel_launches counts the batch's launches). */
int faco_batch_stats(faco_batch* b, int32_t i, faco_stats* s);

/* Pheromone of colony i, [n][k'] in candidate-list order. */
int faco_batch_tau(faco_batch* b, int32_t i, float* tau);

/* Kernel plan: mode -1 = autotune per size class (default); 0 = segment-
 * table blocks for every colony whose table fits (the others: mode 1);
 * 1, 2, 3 = one warp per ant on explicit arrays, the kernel compiled for
 * 2, 4, 8 resident blocks of four ants per SM (fewer registers per thread
 * as the residency grows).  Takes effect at the next faco_batch_iterate
 * (re-planned and re-captured; the ant counters restart from zero).
 * Errors: FACO_E_ARG. */
int faco_batch_set_plan(faco_batch* b, int32_t mode);

/* The plan in use: `count` entries with the codes of faco_batch_set_plan;
 * -1 before the first faco_batch_iterate. */
int faco_batch_get_plan(faco_batch* b, int32_t* variants);

/* The kernel tuner's measurements on the current device (host data; the
 * tuner runs inside the first faco_batch_iterate of a batch whose size
 * classes are new to the process, and inside the server).  One row of 9
 * doubles per tuned (size class, ants, roulette width, goal): the class
 * (0: n < 512; c >= 1: 512 * 4^(c-1) <= n < 512 * 4^c), ants per
 * iteration, roulette width (16 or 32), goal (0
 * batch throughput, 1 one request's latency), the chosen code (0 segment
 * table, 1/2/3 arrays at 2/4/8 resident blocks per SM), then the four
 * codes' timings in ms -- one iteration of up to 64 colonies of the class,
 * scaled for goal 0 by the share of the GPU's resident ant slots the class
 * holds; -1 where a code was not tried.  Writes min(max_rows, recorded)
 * rows and the recorded count into *count.  Errors: FACO_E_ARG. */
int faco_batch_tuner_report(double* rows, int32_t max_rows, int32_t* count);

void faco_batch_destroy(faco_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* FACO_BATCH_H */
