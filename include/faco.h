/*
 * faco.h -- C ABI of the GB300 Focused ACO library (libfaco.so).
 *
 * Method: R. Skinderowicz, "Improving Ant Colony Optimization Efficiency for
 * Solving Large TSP Instances", Applied Soft Computing 2022 (arXiv
 * 2203.02228).  One colony = one symmetric Euclidean TSP instance with
 * integer coordinates and EUC_2D costs (Sec. 2.1).  Every step of the
 * per-iteration path -- focused construction (Sec. 4.3, Alg 2), the
 * checklist-seeded 2-opt / Or-opt local search (Sec. 4.4, Alg 3), the
 * iteration-best / global-best selection with trail limits (Sec. 4.5) and
 * the pheromone update on candidate edges (Eq. 2, Sec. 4.2) -- runs in CUDA
 * kernels for sm_103a.  There is no CPU fallback: without a usable GPU every
 * call that needs one returns FACO_E_CUDA.
 *
 * Conventions
 *   - Every function returns an int status: FACO_OK (0) or a negative error.
 *   - Coordinates are int32 pairs (x, y), row-major [n][2], each in
 *     [0, 2^24).  Out-of-range values are rejected, never clamped.
 *   - Node ids are 0..n-1 in input order.  Tour lengths are int64.
 *   - A faco_ctx owns all device memory of its colony.  One context must not
 *     be used from two host threads at once; distinct contexts are
 *     independent.
 *   - Work is enqueued on the stream given in faco_params.stream (NULL = a
 *     non-blocking stream the context creates and owns).  faco_iterate only
 *     enqueues (a CUDA graph replay per iteration); faco_sync,
 *     faco_best and the faco_get_* calls synchronise that stream.  Device
 *     faults of enqueued work surface at the next synchronising call.
 */
#ifndef FACO_H
#define FACO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FACO_OK = 0,
  FACO_E_ARG = -1,       /* invalid argument (null pointer, size, range)  */
  FACO_E_SIZE = -2,      /* caller buffer too small                       */
  FACO_E_NOMEM = -3,     /* device or host allocation failed              */
  FACO_E_CUDA = -4,      /* CUDA runtime error (no device, launch, fault) */
  FACO_E_TIMEOUT = -5,   /* a bounded device-side wait gave up; reserved: */
                         /* no kernel of this version waits on the       */
                         /* device, so no call returns it                */
  FACO_E_STATE = -6,     /* call not valid in the context's state         */
  FACO_E_CAPACITY = -7   /* a fixed device capacity was exceeded          */
};

/* Parameters; faco_params_default fills the paper's defaults. */
typedef struct {
  uint64_t seed;          /* Philox4x32-10 key (default 1)                        */
  float rho;              /* pheromone retention of Eq. 2, in (0,1) (default 0.5; */
                          /* Sec. 5.3 uses 0.5 with local search)                 */
  int32_t min_new_edges;  /* Table 2 (default 8); >= n gives plain MMAS walks     */
  int32_t bl_size;        /* backup list length, Table 2 (default 64)             */
  double p_best;          /* tau_min formula of Sec. 4.5, in (0,1) (default 0.05) */
  double p_source_gb;     /* probability the source is the global best,          */
                          /* Sec. 5.2 (default 0.01)                              */
  int32_t oropt;          /* 1: Or-opt after a failed 2-opt scan (default 1)      */
  int32_t verify_pass;    /* 1: re-queue popped nodes until a clean round (1)     */
  int32_t keep_ant_tours; /* 1: keep every ant's last tour for faco_get_ant_tours */
  int32_t keep_pre_ls;    /* 1: also keep tours before local search (tests)       */
  int32_t seg_cap;        /* per-ant tour table in shared memory, in segments:   */
                          /* -1 = sized from shared memory (default), 0 = every  */
                          /* ant on explicit n-entry arrays, 8..4096 = that size */
                          /* (an ant whose table fills up is redone on arrays;   */
                          /* results are identical in every case)                */
  int32_t local_search;   /* 1: every new tour gets the local search (FACO+LS,   */
                          /* default); 0: base FACO, tours kept as constructed   */
                          /* (the min_new_edges study, Figs. 1 and 3, uses it    */
                          /* with rho = 0.9); the initial tour's local search is */
                          /* part of the set-up either way                       */
  int32_t init_3opt;      /* 1: the initial tour's local search (Alg 2 set-up)   */
                          /* also tries 3-opt segment exchanges after 2-opt and  */
                          /* Or-opt (Sec. 4.3, "2-opt and 3-opt"); default 0     */
  void* stream;           /* cudaStream_t to enqueue on (NULL = own stream)       */
} faco_params;

typedef struct faco_ctx faco_ctx;

/* Colony state and counters; the per-ant counters are sums over all ants and
 * all iterations run with the current ant count. */
typedef struct {
  int64_t iteration;       /* iterations completed                         */
  int64_t best_length;     /* global-best tour length                      */
  int64_t initial_length;  /* length of the initial tour                   */
  int64_t source_length;   /* length of the current source solution        */
  int32_t n, k, bl;        /* size and effective list lengths              */
  int32_t ants;            /* ants of the last iteration                   */
  int64_t aco_steps;       /* select_next_node calls (sum over ants)       */
  int64_t new_edges;       /* counted new edges (sum)                      */
  int64_t backup_picks;    /* picks from backup lists (sum)                */
  int64_t global_picks;    /* global nearest-unvisited fallbacks (sum)     */
  int64_t ls_pops;         /* local-search queue pops (sum)                */
  int64_t moves_2opt;      /* applied 2-opt moves (sum)                    */
  int64_t moves_or;        /* applied Or-opt moves (sum)                   */
  int64_t flip_elems;      /* elements moved by reversals (sum)            */
  int64_t kernel_launches; /* kernels this context has launched so far     */
  int64_t redone_ants;     /* ants whose segment table filled up and that  */
                           /* were rebuilt on explicit arrays (sum)        */
  int32_t seg_cap;         /* segments per ant table (0: arrays only)      */
  int32_t pad;
} faco_stats;

/* Fills *p with the defaults listed above.  Errors: FACO_E_ARG if p is NULL. */
int faco_params_default(faco_params* p);

/* Creates a colony from host coordinates with default parameters.
 * coords_xy: host array of n (x,y) pairs, copied; the caller keeps it.
 * k: candidate list length (Sec. 4.1; clamped to n-1, must be 2..32).
 * Builds the candidate/backup lists (k + bl nearest by exact distance,
 * ties by index), eta = 1/d, the initial tour (nearest neighbour from node
 * 0, then the local search with every node queued), the trail limits from
 * its length, tau = tau_max and source = initial tour (Alg 2 set-up).
 * Synchronous.  Errors: FACO_E_ARG (n < 3, k out of range, coordinate out
 * of range, NULL), FACO_E_NOMEM, FACO_E_CUDA. */
int faco_create(const int32_t* coords_xy, int32_t n, int32_t k, faco_ctx** out);

/* As faco_create with explicit parameters (p may be NULL = defaults). */
int faco_create_ex(const int32_t* coords_xy, int32_t n, int32_t k, const faco_params* p,
                   faco_ctx** out);

/* As faco_create_ex, but coords_xy is DEVICE memory (n int2, 8-byte
 * aligned) that stays owned by the caller and is read during the call only.
 * The range check runs on the device. */
int faco_create_device(const int32_t* coords_xy, int32_t n, int32_t k, const faco_params* p,
                       faco_ctx** out);

/* Enqueues `budget` FACO iterations (Alg 2 main loop) with `ants` ants each:
 * construction + local search per ant, iteration best, global best and
 * limits, source choice, pheromone update.  The iteration is captured once
 * per ant count into a CUDA graph and replayed.  Asynchronous.
 * Errors: FACO_E_ARG (ants < 1, budget < 0), FACO_E_NOMEM, FACO_E_CUDA. */
int faco_iterate(faco_ctx* c, int32_t ants, int32_t budget);

/* Synchronises the context's stream and reports device-side error flags.
 * Errors: FACO_E_CUDA, FACO_E_CAPACITY (FACO_E_TIMEOUT is reserved for a
 * bounded device wait; no kernel of this version has one). */
int faco_sync(faco_ctx* c);

/* Copies the global-best tour (host array of len >= n node ids) and its
 * length.  tour may be NULL to read the length only.  Synchronous.
 * Errors: FACO_E_SIZE if len < n, FACO_E_ARG, FACO_E_CUDA. */
int faco_best(faco_ctx* c, int32_t* tour, int32_t len, int64_t* length_out);

/* Device-side variant: enqueues copies of the global-best tour into
 * tour_dev (n int32) and its length into length_dev (one int64), both
 * device memory owned by the caller.  Asynchronous. */
int faco_best_device(faco_ctx* c, int32_t* tour_dev, int64_t* length_dev);

/* Counters; synchronous. */
int faco_stats_get(faco_ctx* c, faco_stats* s);

/* Kernel timing.  While enabled, faco_iterate brackets the per-ant kernel
 * (construction + local search) of every iteration with a pair of CUDA
 * events on the context's stream: the iteration is then replayed as two
 * graphs (ants, colony update) with the events between them.
 * faco_profile_read synchronises, returns the summed duration in
 * milliseconds and the number of bracketed launches since the last read,
 * and resets both.  Errors: FACO_E_ARG, FACO_E_CUDA. */
int faco_profile_enable(faco_ctx* c, int on);
int faco_profile_read(faco_ctx* c, double* ants_ms, int64_t* launches);

/* Frees every resource of the context (NULL is accepted). */
void faco_destroy(faco_ctx* c);

/* Static English text for a status code. */
const char* faco_strerror(int status);

/* ---- inspection (tests and diagnostics; all synchronous, host buffers) ---- */

/* cand/backup/eta: n*k, n*bl, n*k entries; any may be NULL. */
int faco_get_lists(faco_ctx* c, int32_t* cand, int32_t* backup, float* eta);
/* tau: n*k entries, node-major, slot order of the candidate list. */
int faco_get_tau(faco_ctx* c, float* tau);
/* out4: tau_max, tau_min (double), tau_max, tau_min (as stored in FP32). */
int faco_get_limits(faco_ctx* c, double* out4);
/* Current source solution / initial tour (n entries, may be NULL). */
int faco_get_source(faco_ctx* c, int32_t* route, int64_t* length_out);
int faco_get_initial(faco_ctx* c, int32_t* route, int64_t* length_out);
/* Per-iteration history, 4 int64 per iteration: iteration-best length,
 * iteration-best ant, global-best length, 1 if the next source is the
 * global best.  Copies min(max_iters, iterations done) rows, returns the
 * count through *rows. */
int faco_get_history(faco_ctx* c, int64_t* hist, int64_t max_iters, int64_t* rows);
/* Tours (ants*n) and lengths (ants) of the last iteration's ants; needs
 * keep_ant_tours.  pre_* need keep_pre_ls (tours before local search and
 * their checklists: ants*n entries, counts in nchecks). */
int faco_get_ant_tours(faco_ctx* c, int32_t* tours, int64_t* lens);
int faco_get_ant_pre(faco_ctx* c, int32_t* tours, int64_t* lens, int32_t* checklists,
                     int32_t* nchecks);
/* Per-ant counters (ants x 24 int64).  Columns 0-10 accumulate over the
 * iterations run with the current ant count: select_next_node calls, new
 * edges, backup picks, global picks, checklist length, queue pops, 2-opt
 * moves, Or-opt moves, reversed elements, verify rounds, redone on arrays.
 * Columns 11-18 are device timer readings (ns) of the last iteration: start,
 * duration, construction, nearest-unvisited scans, local-search evaluation,
 * pop confirmation, move application, endpoint queueing.  19-23: zero. */
int faco_get_ant_stats(faco_ctx* c, int64_t* stats);

/* ---- candidate lists without device allocation --------------------------
 * The paper has no counterpart to this call; it exists for callers that may
 * not let a library allocate device memory -- applications whose memory
 * manager owns the whole device (a fixed pool in a serving process, a
 * framework's caching allocator), or loops that cannot afford the device
 * synchronisation that cudaMalloc/cudaFree imply.
 *
 * Builds the same candidate lists, backup lists and eta = 1/d as
 * faco_create (k + bl nearest other nodes by exact distance, ties by index)
 * for n device-resident (x, y) pairs, into caller-owned device buffers:
 * cand_dev and eta_dev with n * k' entries, backup_dev with n * bl' entries
 * (k' = min(k, n-1), bl' = min(bl, n-1-k'); backup_dev may be NULL when
 * bl' = 0).  It calls no allocating routine: its scratch (the point grid)
 * is a fixed array inside the library, reserved on every GPU that loads
 * the library until the process exits; n may be at most 262144
 * (FACO_E_SIZE above).  Every call looks up that array's device address
 * afresh, so the call stays valid after a cudaDeviceReset (which unloads
 * the library's module and may place the array elsewhere when it is loaded
 * again); it synchronises its stream, so it cannot run inside a stream
 * capture.  All calls share
 * the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The call
 * synchronises `stream` (a cudaStream_t, NULL = legacy default stream)
 * once, to size the grid.  Errors: FACO_E_ARG (sizes, NULL buffers,
 * coordinates outside [0, 2^24)), FACO_E_SIZE (n > 262144), FACO_E_CUDA. */
int faco_lists_noalloc(const int32_t* coords_dev, int32_t n, int32_t k, int32_t bl, int32_t* cand_dev,
                       int32_t* backup_dev, float* eta_dev, void* stream);

/* ---- L2 bandwidth probe (diagnostics) --------------------------------------
 * The paper has no counterpart.  Measures the L2 read bandwidth of the
 * current device: a buffer of `bytes` (1 MiB .. 1 GiB; pick one well inside
 * the L2, e.g. 48 MiB) is filled, read once to bring it into L2, then read
 * `reps` times (1..100000) by 4 blocks per SM with 16-byte L1-bypassing
 * loads; *gbs = bytes * reps / the timed kernel's CUDA-event duration, in
 * GB/s.  Allocates and frees its own device buffers and stream; synchronous.
 * Errors: FACO_E_ARG, FACO_E_NOMEM, FACO_E_CUDA. */
int faco_l2_probe(size_t bytes, int32_t reps, double* gbs);

/* ---- device self-test hook (used by the test-suite) ----------------------
 * Runs one of the library's device primitives on `count` inputs copied from
 * host memory and copies the results back (synchronous, default stream):
 *   what 0  Philox draw     in: uint32[count][4] (idx, ant, iter, tag), seed;
 *                           out: uint32[count]
 *   what 1  EUC_2D cost     in: int32[count][4] (x1, y1, x2, y2); out: int32[count]
 *   what 2  Eq. 1 roulette  in: float[count][width+1] (weights, u01), width 16
 *                           or 32; out: int32[count] (selected slot)
 * Errors: FACO_E_ARG, FACO_E_CUDA. */
int faco_test_device(int what, const void* in, size_t in_bytes, void* out, size_t out_bytes,
                     int count, int width, uint64_t seed);

#ifdef __cplusplus
}
#endif
#endif /* FACO_H */
