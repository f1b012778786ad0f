/*
 * faco_oracle.h -- plain CPU oracle for Focused ACO (FACO), Skinderowicz,
 * "Improving Ant Colony Optimization Efficiency for Solving Large TSP
 * Instances", Applied Soft Computing 2022 (arXiv 2203.02228).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Every function follows the paper's step order and notation; where the
 * paper is silent the reading adopted is stated beside the code.
 */
#ifndef FACO_ORACLE_H
#define FACO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint64_t seed;          /* Philox key (low word, high word)                  */
  float rho;              /* pheromone retention rho of Eq. 2                  */
  int32_t min_new_edges;  /* Table 2: 8                                        */
  int32_t bl_size;        /* Table 2: 64                                       */
  double p_best;          /* tau_min formula of Sec. 4.5 (paper silent: 0.05)  */
  double p_source_gb;     /* Sec. 5.2: source = global best with 1 %           */
  int32_t oropt;          /* 1: Or-opt after a failed 2-opt scan (own def.)    */
  int32_t verify_pass;    /* 1: re-scan visited nodes until no move is found   */
  int32_t threads;        /* OpenMP threads over ants (1 = serial)             */
  int32_t keep_pre_ls;    /* 1: keep each ant's tour before local search       */
  int32_t local_search;   /* 1: each new tour gets the local search (FACO+LS); */
                          /* 0: base FACO, the tour is kept as constructed     */
                          /* (the study of min_new_edges, Figs. 1 and 3)       */
  int32_t init_3opt;      /* 1: the initial tour's local search also tries     */
                          /* 3-opt segment exchanges (Sec. 4.3; see            */
                          /* orc_local_search_ex)                              */
} orc_params;

typedef struct orc_colony orc_colony;

enum { ORC_OK = 0, ORC_E_ARG = -1, ORC_E_NOMEM = -3 };

/* Per-ant counters recorded by the oracle (index into the stats row). */
enum {
  ORC_ST_ACO_STEPS = 0,   /* select_next_node calls                         */
  ORC_ST_NEW_EDGES,       /* counted new edges (closing edge not counted)   */
  ORC_ST_BACKUP,          /* picks from the backup list                     */
  ORC_ST_GLOBAL,          /* picks by the global shortest-edge fallback     */
  ORC_ST_CHECKLIST,       /* checklist length handed to local search       */
  ORC_ST_POPS,            /* queue pops in local search                     */
  ORC_ST_MOVES_2OPT,      /* applied 2-opt moves                            */
  ORC_ST_MOVES_OR,        /* applied Or-opt moves                           */
  ORC_ST_FLIP_ELEMS,      /* total elements moved by reversals              */
  ORC_ST_VERIFY_ROUNDS,   /* verify rounds started                          */
  ORC_ST_MOVES_3OPT,      /* applied 3-opt segment exchanges                */
  ORC_NSTATS = 16
};

/* ---- primitives ---------------------------------------------------- */
uint64_t orc_isqrt(uint64_t m);
int32_t orc_euc2d(const int32_t* xy, int32_t a, int32_t b);
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_draw(uint64_t seed, uint32_t idx, uint32_t ant, uint32_t iter, uint32_t tag);
float orc_u01(uint32_t x);
void orc_params_default(orc_params* p);

/* K nearest other nodes of each listed node, ordered by (squared distance,
 * index); out is nrows x K. */
void orc_knn_rows(const int32_t* xy, int32_t n, int32_t K, const int32_t* rows,
                  int32_t nrows, int32_t threads, int32_t* out);

/* Roulette selection of Eq. 1 over one candidate row (alpha = beta = 1).
 * w[s] are the weights tau*eta (0 for visited / padding); returns the slot. */
int32_t orc_roulette(const float* w, int32_t width, float u01);

/* 2-opt (+ optional Or-opt) local search of Alg. 3 on an explicit route.
 * route/pos are updated in place; queue holds the initial checklist.
 * Returns the total gain (old length - new length); stats may be NULL. */
int64_t orc_local_search(const int32_t* xy, int32_t n, const int32_t* cand, int32_t k,
                         int32_t oropt, int32_t verify, int32_t* route, int32_t* pos,
                         const int32_t* queue, int32_t nqueue, int64_t* stats);
/* orc_local_search with, when three_opt = 1, a third move type tried from a
 * node whose 2-opt and Or-opt scans found nothing: the 3-opt segment
 * exchange (see or3_eval in the source). */
int64_t orc_local_search_ex(const int32_t* xy, int32_t n, const int32_t* cand, int32_t k,
                            int32_t oropt, int32_t verify, int32_t three_opt, int32_t* route,
                            int32_t* pos, const int32_t* queue, int32_t nqueue, int64_t* stats);

void orc_nn_tour(const int32_t* xy, int32_t n, const int32_t* cand, int32_t k,
                 const int32_t* backup, int32_t bl, int32_t* route);

int64_t orc_tour_length(const int32_t* xy, int32_t n, const int32_t* route);

/* ---- the colony ---------------------------------------------------- */
int orc_create(const int32_t* xy, int32_t n, int32_t k, const orc_params* p, orc_colony** out);
void orc_destroy(orc_colony* c);
/* Runs `iters` FACO iterations (Alg. 2 main loop) with `ants` ants.
 * hist (iters x 4 int64, may be NULL): it-best length, it-best ant,
 * global-best length, 1 if the next source is the global best.
 * ant_len_hist (iters x ants, may be NULL): every ant's length after LS. */
int orc_iterate(orc_colony* c, int32_t ants, int32_t iters, int64_t* hist, int64_t* ant_len_hist);

int32_t orc_n(const orc_colony* c);
int32_t orc_k(const orc_colony* c);
int32_t orc_bl(const orc_colony* c);
int64_t orc_iteration(const orc_colony* c);
void orc_get_lists(const orc_colony* c, int32_t* cand, int32_t* backup, float* eta);
void orc_get_tau(const orc_colony* c, float* tau);
void orc_get_limits(const orc_colony* c, double* out4); /* tmax_d, tmin_d, tmax_f, tmin_f */
int64_t orc_get_source(const orc_colony* c, int32_t* route);
int64_t orc_get_best(const orc_colony* c, int32_t* route);
int64_t orc_get_initial(const orc_colony* c, int32_t* route);
/* Last iteration: tours after LS (ants x n), lengths, stats (ants x ORC_NSTATS),
 * and, if keep_pre_ls, tours/lengths before LS plus checklists. */
int32_t orc_last_ants(const orc_colony* c);
void orc_get_ant_tours(const orc_colony* c, int32_t* tours, int64_t* lens);
void orc_get_ant_stats(const orc_colony* c, int64_t* stats);
int orc_get_ant_pre(const orc_colony* c, int32_t* tours, int64_t* lens,
                    int32_t* checklists /* ants x n */, int32_t* nchecks);
/* Overwrites the pheromone and the source (a test hook for fixed-point checks). */
int orc_set_state(orc_colony* c, const float* tau, const int32_t* src_route);
/* OpenMP threads used by later orc_iterate calls (>= 1); results do not
 * depend on it (ants are independent within an iteration). */
int orc_set_threads(orc_colony* c, int32_t threads);

#ifdef __cplusplus
}
#endif
#endif
