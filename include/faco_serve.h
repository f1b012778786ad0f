/*
 * faco_serve.h -- a request server over the batched colonies (libfaco.so).
 *
 * The paper has no serving form; it solves one instance per run.  A server
 * accepts TSP instances of uneven sizes as they arrive and keeps every
 * admitted instance's state -- lists, pheromone, source and best tours,
 * ant buffers -- resident in device memory until its iteration budget is
 * spent.  Admission is by device memory: each request needs a fixed number
 * of bytes (faco_server_request_bytes), taken from one pool allocated when
 * the server is created; requests wait in arrival order until the pool has
 * room.  A scheduler thread inside the library runs continuous batching:
 *   - an admitted request's set-up (candidate lists, initial tour and its
 *     local search, Alg 2 set-up) runs on a set-up stream while the GPU
 *     keeps iterating the active requests;
 *   - active requests are grouped into cohorts by roulette width (k <= 16
 *     or not) and size (n <= 4096, <= 32768, larger); each cohort iterates
 *     in rounds of its own on a stream of its own, so cohorts proceed at
 *     their own pace and their kernels share the GPU;
 *   - a round is one iteration (Alg 2 main loop body) of every request of
 *     the cohort, with the same launches as a faco_batch; a request joins
 *     at the next round after its set-up completes and leaves the round in
 *     which its budget is spent;
 *   - its global-best tour and length are then copied to host memory and
 *     its device memory returns to the pool.
 *
 * Results: a request's tour and length are bit-identical to
 *   faco_create_ex(coords, n, k, p', ...); faco_iterate(c, ants, budget);
 * with p' = the server's parameters with seed = the request's seed -- alone
 * or in any mix of other requests.
 *
 * Threads: faco_server_submit, _poll, _wait, _release and _stats may be
 * called from any host thread.  Times are host steady-clock nanoseconds.
 */
#ifndef FACO_SERVE_H
#define FACO_SERVE_H

#include "faco.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct faco_server faco_server;

#define FACO_PENDING 1 /* positive status of faco_server_poll / _wait: not done yet */

typedef struct {
  int64_t submitted;       /* requests accepted by faco_server_submit           */
  int64_t completed;       /* requests finished (successfully or not)           */
  int64_t queued;          /* waiting for memory                                */
  int64_t setting_up;      /* admitted, set-up in flight                        */
  int64_t active;          /* iterating                                         */
  int64_t peak_active;     /* largest number of requests iterating at once      */
  int64_t rounds;          /* iteration rounds run (all cohorts)                */
  int64_t kernel_launches; /* kernels launched by the server so far             */
  int64_t pool_bytes;      /* device bytes of the pool                          */
  int64_t pool_in_use;     /* bytes held by admitted requests                   */
} faco_server_stats;

/* Creates a server with a device pool of `device_bytes` (allocated now) and
 * the parameters `p` (NULL = defaults; keep_ant_tours, keep_pre_ls must be 0,
 * seg_cap -1 or 0; p->stream is ignored: the server owns its streams) and
 * starts its scheduler thread on the current device.  Errors: FACO_E_ARG,
 * FACO_E_NOMEM (the pool), FACO_E_CUDA. */
int faco_server_create(size_t device_bytes, const faco_params* p, faco_server** out);

/* Device bytes a request of this shape holds while admitted. */
int64_t faco_server_request_bytes(int32_t n, int32_t k, int32_t ants, const faco_params* p);

/* Queues a request: host coordinates (copied; n pairs in [0, 2^24)), list
 * length k (2..32), `ants` per iteration, iteration `budget` (>= 1) and
 * Philox seed.  Does not wait for the GPU.  *ticket identifies it.  Errors:
 * FACO_E_ARG, FACO_E_SIZE (n above 262144), FACO_E_NOMEM (the request can
 * never fit the pool), FACO_E_STATE (the server is shutting down). */
int faco_server_submit(faco_server* s, const int32_t* coords_xy, int32_t n, int32_t k, int32_t ants,
                       int32_t budget, uint64_t seed, uint64_t* ticket);

/* FACO_PENDING while the request runs; then its final status (FACO_OK or an
 * error) with, when non-NULL, its tour (len >= n, else FACO_E_SIZE), length
 * and submit / completion times.  Unknown or released ticket: FACO_E_ARG. */
int faco_server_poll(faco_server* s, uint64_t ticket, int32_t* tour, int32_t len, int64_t* length_out,
                     int64_t* t_submit_ns, int64_t* t_done_ns);

/* Blocks until the request is done or `timeout_ms` passes (then
 * FACO_PENDING); returns its final status like faco_server_poll. */
int faco_server_wait(faco_server* s, uint64_t ticket, int32_t timeout_ms);

/* Forgets a finished request's host-side result.  FACO_E_STATE if it is
 * not finished, FACO_E_ARG if unknown. */
int faco_server_release(faco_server* s, uint64_t ticket);

int faco_server_stats_get(faco_server* s, faco_server_stats* st);

/* Test hook (host only; needs no GPU): replays a script of `count`
 * operations on a pool of `pool_bytes` (at most 2^26) with the server's
 * allocator -- first fit in 256-byte granules, freed ranges merged with
 * free neighbours.  ops[2i] > 0: take that many bytes; ops[2i] == 0: give
 * back the range taken by operation ops[2i+1] (an earlier, still held
 * take).  out[2i] = the offset taken (-1: no room; 0 for a give-back),
 * out[2i+1] = bytes in use after the operation.  FACO_E_ARG on a malformed
 * script. */
int faco_test_pool(int64_t pool_bytes, const int64_t* ops, int32_t count, int64_t* out);

/* Drops the requests still waiting for memory (their status becomes
 * FACO_E_STATE), lets the admitted ones run to the end of their budgets,
 * stops the scheduler and frees everything; results are then gone. */
void faco_server_destroy(faco_server* s);

#ifdef __cplusplus
}
#endif
#endif /* FACO_SERVE_H */
