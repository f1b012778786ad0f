/*
 * faco_oracle.c -- plain CPU oracle for Focused ACO (FACO).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and
 * the CPU-baseline leg of the benchmark.  Slow and literal on purpose.  It
 * shares no code with the CUDA library.
 *
 * Paper: R. Skinderowicz, "Improving Ant Colony Optimization Efficiency for
 * Solving Large TSP Instances", Applied Soft Computing 2022.
 *   Sec. 2.1        problem model, Eq. 1 (random-proportional rule),
 *                   Eq. 2 (pheromone update with limits)
 *   Sec. 4.1        candidate lists and backup lists
 *   Sec. 4.2        pheromone kept only for candidate edges
 *   Sec. 4.3, Alg 2 focused construction, source solution, main loop
 *   Sec. 4.4, Alg 3 checklist-seeded 2-opt with neighbour lists
 *   Sec. 4.5        pheromone trail limits
 *   Table 2         parameter defaults
 *
 * Readings where the paper is silent (each decided the same way in the GPU
 * library, which implements them independently):
 *   - cost d_ij: TSPLIB EUC_2D, round-half-up of the Euclidean distance of
 *     integer coordinates, computed exactly in integers;
 *   - alpha = beta = 1: the weight of a candidate is tau*eta in FP32;
 *   - eta = 1/d as an IEEE FP32 division (d = 0 maps to eta = 1);
 *   - neighbour order: (squared distance, node index) ascending;
 *   - roulette: inclusive Kogge-Stone scan over 16 (or 32) zero-padded
 *     slots, r = u01 * total, first slot with positive weight whose prefix
 *     exceeds r, else the last slot with positive weight;
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (draw/4, ant, iteration, stream tag), word = draw % 4;
 *     draw 0 of an ant picks the start node, draw k the roulette that
 *     fills route position k; tag 1 / draw 0 is the colony's source pick;
 *   - completion (Alg 2): from the current end x follow the source's
 *     successor while it is unvisited, then its predecessor while that is
 *     unvisited; afterwards the ACO rule resumes (the literal pseudocode's
 *     backward loop can never run, see the note in construct());
 *   - new edge: (u,v) is new iff v is neither successor nor predecessor of
 *     u in the source; the closing edge is neither counted nor checked;
 *   - the checklist holds v of every new edge; the LS queue is a FIFO with
 *     an in-queue bit (a node already queued is not queued twice);
 *   - 2-opt flip: reverse the forward span x..y, or its complement when the
 *     span is longer than half the tour;
 *   - verify pass: when the queue runs dry after a round that applied a
 *     move, every node popped in that round is queued again;
 *   - Or-opt (not in the paper; asked for beside 2-opt): tried from a node
 *     whose 2-opt scan found nothing, segment lengths 1..3 (definition at
 *     or_opt_eval());
 *   - pheromone: one fused max(tmin, min(tmax, fmaf(rho, tau, delta))) per
 *     stored entry, delta = (float)(1/L_source) on source edges;
 *   - limits: tmax = 1/(L_gb (1-rho)), tmin = tmax * c,
 *     c = (1 - p^(1/n)) / ((cl_size - 1) p^(1/n)), p_best = 0.05;
 *   - initial tour: nearest neighbour from node 0 (candidate list, backup
 *     list, then global nearest), then the same local search with every
 *     node queued in tour order; with init_3opt it also tries the 3-opt
 *     segment exchange of or3_eval() (Sec. 4.3's "2-opt and 3-opt").
 */
#include "faco_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* EUC_2D cost (Sec. 2.1: d_ij is the cost of edge (i,j))              */
/* ------------------------------------------------------------------ */

/* Largest r with r*r <= m, by the classic digit-by-digit method. */
uint64_t orc_isqrt(uint64_t m) {
  uint64_t r = 0;
  uint64_t bit = (uint64_t)1 << 62;
  while (bit > m) bit >>= 2;
  while (bit != 0) {
    if (m >= r + bit) {
      m -= r + bit;
      r = (r >> 1) + bit;
    } else {
      r >>= 1;
    }
    bit >>= 2;
  }
  return r;
}

static uint64_t sq_dist(const int32_t* xy, int32_t a, int32_t b) {
  int64_t dx = (int64_t)xy[2 * a] - xy[2 * b];
  int64_t dy = (int64_t)xy[2 * a + 1] - xy[2 * b + 1];
  return (uint64_t)(dx * dx + dy * dy);
}

/* nint(sqrt(m)): sqrt(m) >= r + 1/2  <=>  m - r^2 > r for integer m. */
int32_t orc_euc2d(const int32_t* xy, int32_t a, int32_t b) {
  uint64_t m = sq_dist(xy, a, b);
  uint64_t r = orc_isqrt(m);
  return (int32_t)(r + ((m - r * r) > r ? 1 : 0));
}

int64_t orc_tour_length(const int32_t* xy, int32_t n, const int32_t* route) {
  int64_t L = 0;
  for (int32_t i = 0; i < n; ++i) L += orc_euc2d(xy, route[i], route[(i + 1) % n]);
  return L;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                   */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* Weyl key schedule */
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint32_t orc_draw(uint64_t seed, uint32_t idx, uint32_t ant, uint32_t iter, uint32_t tag) {
  uint32_t ctr[4] = {idx >> 2, ant, iter, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[idx & 3u];
}

/* Top 24 bits scaled by 2^-24: exact in FP32, in [0, 1). */
float orc_u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

/* ------------------------------------------------------------------ */
/* Parameters                                                          */
/* ------------------------------------------------------------------ */

void orc_params_default(orc_params* p) {
  p->seed = 1;
  p->rho = 0.5f;           /* Sec. 5.3: rho = 0.5 with the LS       */
  p->min_new_edges = 8;    /* Table 2                               */
  p->bl_size = 64;         /* Table 2                               */
  p->p_best = 0.05;        /* paper silent; MMAS convention         */
  p->p_source_gb = 0.01;   /* Sec. 5.2: global best used with 1 %   */
  p->oropt = 1;
  p->verify_pass = 1;
  p->threads = 1;
  p->keep_pre_ls = 0;
  p->local_search = 1;
  p->init_3opt = 0;
}

/* ------------------------------------------------------------------ */
/* Candidate and backup lists (Sec. 4.1): brute-force nearest nodes    */
/* ------------------------------------------------------------------ */

static int key_less(uint64_t ma, int32_t a, uint64_t mb, int32_t b) {
  return ma < mb || (ma == mb && a < b);
}

static void knn_one(const int32_t* xy, int32_t n, int32_t K, int32_t u, uint64_t* bm,
                    int32_t* bi) {
  int32_t cnt = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (v == u) continue;
    uint64_t m = sq_dist(xy, u, v);
    if (cnt == K && !key_less(m, v, bm[K - 1], bi[K - 1])) continue;
    int32_t j = cnt < K ? cnt++ : K - 1;
    while (j > 0 && key_less(m, v, bm[j - 1], bi[j - 1])) {
      bm[j] = bm[j - 1];
      bi[j] = bi[j - 1];
      --j;
    }
    bm[j] = m;
    bi[j] = v;
  }
}

void orc_knn_rows(const int32_t* xy, int32_t n, int32_t K, const int32_t* rows, int32_t nrows,
                  int32_t threads, int32_t* out) {
  if (threads < 1) threads = 1;
#pragma omp parallel num_threads(threads)
  {
    uint64_t* bm = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(K > 0 ? K : 1));
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
#pragma omp for schedule(dynamic, 64)
    for (int32_t r = 0; r < nrows; ++r) {
      knn_one(xy, n, K, rows[r], bm, bi);
      memcpy(out + (size_t)r * K, bi, sizeof(int32_t) * (size_t)K);
    }
    free(bm);
    free(bi);
  }
}

/* ------------------------------------------------------------------ */
/* Roulette of Eq. 1 (alpha = beta = 1)                                */
/* ------------------------------------------------------------------ */

int32_t orc_roulette(const float* w, int32_t width, float u01) {
  float cur[32], nxt[32];
  for (int32_t i = 0; i < width; ++i) cur[i] = w[i];
  /* inclusive Kogge-Stone scan: level `off` adds the value `off` slots left */
  for (int32_t off = 1; off < width; off <<= 1) {
    for (int32_t i = 0; i < width; ++i) nxt[i] = (i >= off) ? cur[i - off] + cur[i] : cur[i];
    for (int32_t i = 0; i < width; ++i) cur[i] = nxt[i];
  }
  float total = cur[width - 1];
  float r = u01 * total;
  for (int32_t i = 0; i < width; ++i)
    if (w[i] > 0.0f && cur[i] > r) return i;
  for (int32_t i = width - 1; i >= 0; --i)
    if (w[i] > 0.0f) return i;
  return -1;
}

/* ------------------------------------------------------------------ */
/* Colony state                                                        */
/* ------------------------------------------------------------------ */

struct orc_colony {
  int32_t n, k, bl;
  orc_params prm;
  int32_t* xy;
  int32_t* cand;   /* n x k  */
  int32_t* backup; /* n x bl */
  float* eta;      /* n x k  */
  float* tau;      /* n x k  */
  double c_min;
  double tmax_d, tmin_d;
  float tmax, tmin;
  int32_t *src_route, *src_pos;
  int64_t src_len;
  int32_t *gb_route, *gb_pos;
  int64_t gb_len;
  int32_t* init_route;
  int64_t init_len;
  int64_t iter;
  /* last iteration */
  int32_t ants_cap, ants_last;
  int32_t* ant_routes;
  int64_t* ant_len;
  int64_t* ant_stats;
  int32_t* pre_routes;
  int64_t* pre_len;
  int32_t* pre_check;
  int32_t* pre_ncheck;
};

/* ------------------------------------------------------------------ */
/* Local search (Sec. 4.4, Alg 3)                                      */
/* ------------------------------------------------------------------ */

typedef struct {
  const int32_t* xy;
  int32_t n;
  const int32_t* cand;
  int32_t k;
  int32_t* route;
  int32_t* pos;
  uint8_t* inq;
  int32_t* q; /* ring of n entries */
  int32_t qh, qn;
  int32_t* log;
  int64_t nlog, caplog;
  int64_t* st;
} ls_state;

static int32_t succ_of(const ls_state* S, int32_t x) { return S->route[(S->pos[x] + 1) % S->n]; }
static int32_t pred_of(const ls_state* S, int32_t x) {
  return S->route[(S->pos[x] + S->n - 1) % S->n];
}
static int64_t dist(const ls_state* S, int32_t a, int32_t b) { return orc_euc2d(S->xy, a, b); }

static void q_push(ls_state* S, int32_t x) {
  if (S->inq[x]) return;
  S->inq[x] = 1;
  S->q[(S->qh + S->qn) % S->n] = x;
  S->qn++;
}

static int32_t q_pop(ls_state* S) {
  int32_t x = S->q[S->qh];
  S->qh = (S->qh + 1) % S->n;
  S->qn--;
  S->inq[x] = 0;
  return x;
}

static void log_add(ls_state* S, int32_t x) {
  if (S->nlog == S->caplog) {
    S->caplog = S->caplog ? 2 * S->caplog : 1024;
    S->log = (int32_t*)realloc(S->log, sizeof(int32_t) * (size_t)S->caplog);
  }
  S->log[S->nlog++] = x;
}

/* Reverse the forward cyclic span x..y; when it holds more than half of the
 * tour, reverse the complementary span instead (same cycle, fewer writes). */
static void flip(ls_state* S, int32_t x, int32_t y) {
  int32_t n = S->n;
  int32_t i = S->pos[x], j = S->pos[y];
  int32_t L = ((j - i) % n + n) % n + 1;
  if (2 * L > n) {
    int32_t i2 = (j + 1) % n, j2 = (i + n - 1) % n;
    i = i2;
    j = j2;
    L = n - L;
  }
  for (int32_t t = 0; t < L / 2; ++t) {
    int32_t ia = (i + t) % n, ib = ((j - t) % n + n) % n;
    int32_t va = S->route[ia], vb = S->route[ib];
    S->route[ia] = vb;
    S->pos[vb] = ia;
    S->route[ib] = va;
    S->pos[va] = ib;
  }
  if (S->st) S->st[ORC_ST_FLIP_ELEMS] += L;
}

/* Exchange tour edges {n1,n2},{n3,n4} for {n1,n3},{n2,n4}.  When n1->n2 is a
 * forward edge this is Alg 3's move (w,x,y,z) = (n1,n2,n3,n4), flip n2..n3;
 * otherwise it is (n2,n1,n4,n3), flip n1..n4. */
static void move_2opt(ls_state* S, int32_t n1, int32_t n2, int32_t n3, int32_t n4) {
  if (succ_of(S, n1) == n2)
    flip(S, n2, n3);
  else
    flip(S, n1, n4);
}

/* Or-opt (own definition; the paper applies only 2-opt in the main loop).
 * Segment s = a..e of length l in 1..3 following a forward, p = pred(a),
 * q = succ(e).  For every b in NN(a) in list order and for the two tour
 * edges (u,v) at b -- first (b, succ b), then (pred b, b) -- with u and v
 * outside {p, q} and outside the segment, the segment is moved between u
 * and v, first reversed (u,e..a,v), then (for l >= 2) kept (u,a..e,v).
 * gain = d(p,a) + d(e,q) + d(u,v) - d(p,q) - d(u,s1) - d(s2,v).
 * The first strictly largest gain in the order (l, b, edge, orientation)
 * wins.  Returns the gain (0 = no move) and the move in mv[0..6] =
 * {p,a,e,q,u,v,kept}. */
static int64_t or_opt_eval(ls_state* S, int32_t a, int32_t mv[7]) {
  int32_t n = S->n;
  int64_t best = 0;
  if (n < 8) return 0;
  for (int32_t l = 1; l <= 3; ++l) {
    int32_t seg[3];
    seg[0] = a;
    for (int32_t t = 1; t < l; ++t) seg[t] = succ_of(S, seg[t - 1]);
    int32_t e = seg[l - 1];
    int32_t p = pred_of(S, a), q = succ_of(S, e);
    int64_t removed = dist(S, p, a) + dist(S, e, q) - dist(S, p, q);
    for (int32_t s = 0; s < S->k; ++s) {
      int32_t b = S->cand[(size_t)a * S->k + s];
      for (int32_t side = 0; side < 2; ++side) {
        int32_t u = side == 0 ? b : pred_of(S, b);
        int32_t v = side == 0 ? succ_of(S, b) : b;
        int bad = (u == p || u == q || v == p || v == q);
        for (int32_t t = 0; t < l; ++t) bad |= (u == seg[t] || v == seg[t]);
        if (bad) continue;
        for (int32_t kept = 0; kept < (l >= 2 ? 2 : 1); ++kept) {
          int32_t s1 = kept ? a : e, s2 = kept ? e : a;
          int64_t g = removed + dist(S, u, v) - dist(S, u, s1) - dist(S, s2, v);
          if (g > best) {
            best = g;
            mv[0] = p; mv[1] = a; mv[2] = e; mv[3] = q; mv[4] = u; mv[5] = v; mv[6] = kept;
          }
        }
      }
    }
  }
  return best;
}

/* Apply an Or-opt move as successive edge exchanges:
 *   {p,a},{u,v} -> {p,u},{a,v};  {p,u},{q,e} -> {p,q},{u,e};
 *   and, to keep the orientation, {u,e},{a,v} -> {u,a},{e,v}. */
static void or_opt_apply(ls_state* S, const int32_t mv[7]) {
  int32_t p = mv[0], a = mv[1], e = mv[2], q = mv[3], u = mv[4], v = mv[5];
  move_2opt(S, p, a, u, v);
  move_2opt(S, p, u, q, e);
  if (mv[6]) move_2opt(S, u, e, a, v);
}

/* Alg 3 for one popped node a: best improving 2-opt move over NN(a), first
 * the successor-side loop, then the predecessor-side loop; strict '>'. */
static int64_t two_opt_eval(ls_state* S, int32_t a, int32_t mv[4]) {
  int64_t gain = 0;
  int32_t a_succ = succ_of(S, a), a_pred = pred_of(S, a);
  const int32_t* nn = S->cand + (size_t)a * S->k;
  int64_t d_as = dist(S, a, a_succ);
  for (int32_t s = 0; s < S->k; ++s) {
    int32_t b = nn[s];
    int32_t b_succ = succ_of(S, b);
    int64_t d_ab = dist(S, a, b);
    if (d_as > d_ab) {
      int64_t c_old = d_as + dist(S, b, b_succ);
      int64_t c_new = d_ab + dist(S, a_succ, b_succ);
      if (c_old - c_new > gain) {
        gain = c_old - c_new;
        mv[0] = a; mv[1] = a_succ; mv[2] = b; mv[3] = b_succ;
      }
    }
  }
  int64_t d_ap = dist(S, a_pred, a);
  for (int32_t s = 0; s < S->k; ++s) {
    int32_t b = nn[s];
    int32_t b_pred = pred_of(S, b);
    int64_t d_ab = dist(S, a, b);
    if (d_ap > d_ab) {
      int64_t c_old = d_ap + dist(S, b_pred, b);
      int64_t c_new = d_ab + dist(S, a_pred, b_pred);
      if (c_old - c_new > gain) {
        gain = c_old - c_new;
        mv[0] = a_pred; mv[1] = a; mv[2] = b_pred; mv[3] = b;
      }
    }
  }
  return gain;
}

/* 3-opt segment exchange for the initial tour (Sec. 4.3: the initial
 * solution is improved by 2-opt and 3-opt following Bentley; the paper
 * gives no further detail, so the move and its search are a reading).
 * Three tour edges (a,t2), (b,b'), (c,c') are replaced by (a,b'), (b,c'),
 * (c,t2): walking from a towards t2, the tour is a [t2 .. b] [b' .. c] c'
 * and becomes a [b' .. c] [t2 .. b] c' -- the two sections swap places,
 * neither is reversed (the one reconnection of three edges that is not a
 * 2-opt move or a reversal).  Neighbour lists with Bentley's positive
 * partial gains: t2 = succ(a) (dir 0) or pred(a) (dir 1); b' runs over
 * NN(a) with g1 = d(a,t2) - d(a,b') > 0, b is b''s neighbour before it in
 * the walking direction; c' runs over NN(b) with g2 = g1 + d(b,b') -
 * d(b,c') > 0, c is c''s neighbour before it; the move is valid when, in
 * walking order from a, 1 <= r(b) < r(c) <= n - 2.  gain = g2 + d(c,c') -
 * d(c,t2).  The first strictly largest gain in the order (dir, b', c')
 * wins.  mv = {a, t2, b, b', c, c'}. */
static int64_t or3_eval(ls_state* S, int32_t a, int32_t mv[6]) {
  int32_t n = S->n;
  int64_t best = 0;
  if (n < 8) return 0;
  for (int32_t dir = 0; dir < 2; ++dir) {
    int32_t t2 = dir == 0 ? succ_of(S, a) : pred_of(S, a);
    int64_t d_at2 = dist(S, a, t2);
    for (int32_t i = 0; i < S->k; ++i) {
      int32_t b1 = S->cand[(size_t)a * S->k + i]; /* b' */
      int64_t g1 = d_at2 - dist(S, a, b1);
      if (g1 <= 0) continue;
      int32_t b = dir == 0 ? pred_of(S, b1) : succ_of(S, b1);
      for (int32_t j = 0; j < S->k; ++j) {
        int32_t c1 = S->cand[(size_t)b * S->k + j]; /* c' */
        int64_t g2 = g1 + dist(S, b, b1) - dist(S, b, c1);
        if (g2 <= 0) continue;
        int32_t c = dir == 0 ? pred_of(S, c1) : succ_of(S, c1);
        /* positions counted from a in the walking direction */
        int32_t rb = dir == 0 ? S->pos[b] - S->pos[a] : S->pos[a] - S->pos[b];
        int32_t rc = dir == 0 ? S->pos[c] - S->pos[a] : S->pos[a] - S->pos[c];
        rb = (rb % n + n) % n;
        rc = (rc % n + n) % n;
        if (!(rb >= 1 && rb < rc && rc <= n - 2)) continue;
        int64_t g = g2 + dist(S, c, c1) - dist(S, c, t2);
        if (g > best) {
          best = g;
          mv[0] = a; mv[1] = t2; mv[2] = b; mv[3] = b1; mv[4] = c; mv[5] = c1;
        }
      }
    }
  }
  return best;
}

/* The segment exchange as three edge exchanges:
 *   {a,t2},{b,b'} -> {a,b},{t2,b'};  {a,b},{c,c'} -> {a,c},{b,c'};
 *   {a,c},{b',t2} -> {a,b'},{c,t2}. */
static void or3_apply(ls_state* S, const int32_t mv[6]) {
  int32_t a = mv[0], t2 = mv[1], b = mv[2], b1 = mv[3], c = mv[4], c1 = mv[5];
  move_2opt(S, a, t2, b, b1);
  move_2opt(S, a, b, c, c1);
  move_2opt(S, a, c, b1, t2);
}

int64_t orc_local_search_ex(const int32_t* xy, int32_t n, const int32_t* cand, int32_t k,
                            int32_t oropt, int32_t verify, int32_t three_opt, int32_t* route,
                            int32_t* pos, const int32_t* queue, int32_t nqueue, int64_t* stats) {
  ls_state S;
  memset(&S, 0, sizeof S);
  S.xy = xy; S.n = n; S.cand = cand; S.k = k; S.route = route; S.pos = pos; S.st = stats;
  S.inq = (uint8_t*)calloc((size_t)n, 1);
  S.q = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t i = 0; i < nqueue; ++i) q_push(&S, queue[i]);

  int64_t total_gain = 0;
  int32_t changes = 0;
  int32_t moves_in_round = 0;
  for (;;) {
    while (S.qn > 0 && changes < n) {
      int32_t a = q_pop(&S);
      log_add(&S, a);
      if (stats) stats[ORC_ST_POPS]++;
      int32_t mv[7];
      int64_t g = two_opt_eval(&S, a, mv);
      if (g > 0) {
        /* (w,x,y,z) = mv: flip x..y, queue w,x,y,z */
        flip(&S, mv[1], mv[2]);
        for (int t = 0; t < 4; ++t) q_push(&S, mv[t]);
        total_gain += g;
        changes++;
        moves_in_round++;
        if (stats) stats[ORC_ST_MOVES_2OPT]++;
        continue;
      }
      if (oropt) {
        g = or_opt_eval(&S, a, mv);
        if (g > 0) {
          or_opt_apply(&S, mv);
          for (int t = 0; t < 6; ++t) q_push(&S, mv[t]);
          total_gain += g;
          changes++;
          moves_in_round++;
          if (stats) stats[ORC_ST_MOVES_OR]++;
          continue;
        }
      }
      if (three_opt) {
        g = or3_eval(&S, a, mv);
        if (g > 0) {
          or3_apply(&S, mv);
          for (int t = 0; t < 6; ++t) q_push(&S, mv[t]);
          total_gain += g;
          changes++;
          moves_in_round++;
          if (stats) stats[ORC_ST_MOVES_3OPT]++;
        }
      }
    }
    if (changes >= n || !verify || moves_in_round == 0) break;
    /* verify round: queue again every node popped since the last round */
    if (stats) stats[ORC_ST_VERIFY_ROUNDS]++;
    int64_t nl = S.nlog;
    S.nlog = 0;
    int32_t* old = S.log;
    int64_t oldcap = S.caplog;
    S.log = NULL;
    S.caplog = 0;
    for (int64_t i = 0; i < nl; ++i) q_push(&S, old[i]);
    free(old);
    (void)oldcap;
    moves_in_round = 0;
  }
  free(S.inq);
  free(S.q);
  free(S.log);
  return total_gain;
}

int64_t orc_local_search(const int32_t* xy, int32_t n, const int32_t* cand, int32_t k,
                         int32_t oropt, int32_t verify, int32_t* route, int32_t* pos,
                         const int32_t* queue, int32_t nqueue, int64_t* stats) {
  return orc_local_search_ex(xy, n, cand, k, oropt, verify, 0, route, pos, queue, nqueue, stats);
}

/* ------------------------------------------------------------------ */
/* Focused construction (Sec. 4.3, Alg 2 inner loop)                   */
/* ------------------------------------------------------------------ */

/* select_next_node: Eq. 1 over the unvisited candidates, else the first
 * unvisited node of the backup list, else the unvisited node with the
 * shortest edge (highest eta; ties by exact distance, then index). */
static int32_t select_next(const orc_colony* C, int32_t u, const uint8_t* visited, uint32_t word,
                           int64_t* st) {
  int32_t k = C->k;
  int32_t width = k <= 16 ? 16 : 32;
  float w[32];
  int any = 0;
  for (int32_t s = 0; s < width; ++s) {
    w[s] = 0.0f;
    if (s < k && !visited[C->cand[(size_t)u * k + s]]) {
      w[s] = C->tau[(size_t)u * k + s] * C->eta[(size_t)u * k + s];
      if (w[s] > 0.0f) any = 1; /* tau >= tau_min > 0 and eta > 0 */
    }
  }
  if (any) {
    int32_t s = orc_roulette(w, width, orc_u01(word));
    return C->cand[(size_t)u * k + s];
  }
  for (int32_t j = 0; j < C->bl; ++j) {
    int32_t v = C->backup[(size_t)u * C->bl + j];
    if (!visited[v]) {
      if (st) st[ORC_ST_BACKUP]++;
      return v;
    }
  }
  int32_t best = -1;
  uint64_t bm = 0;
  for (int32_t v = 0; v < C->n; ++v) {
    if (visited[v]) continue;
    uint64_t m = sq_dist(C->xy, u, v);
    if (best < 0 || key_less(m, v, bm, best)) {
      best = v;
      bm = m;
    }
  }
  if (st) st[ORC_ST_GLOBAL]++;
  return best;
}

/* One ant's focused tour (Alg 2).  Note on the completion loops: read
 * literally, the backward loop starts from the predecessor of the node that
 * stopped the forward loop, i.e. from an already-visited node, and never
 * runs.  The reading adopted: from the current end x, follow succ(source, x)
 * while unvisited, then pred(source, x) while unvisited. */
static int32_t construct(const orc_colony* C, int32_t ant, uint32_t iter, int32_t* route,
                         uint8_t* visited, int32_t* check, int64_t* st) {
  int32_t n = C->n;
  const int32_t* sr = C->src_route;
  const int32_t* sp = C->src_pos;
  uint64_t seed = C->prm.seed;
  memset(visited, 0, (size_t)n);
  uint32_t x0 = orc_draw(seed, 0, (uint32_t)ant, iter, 0);
  int32_t start = (int32_t)(((uint64_t)x0 * (uint64_t)n) >> 32);
  route[0] = start;
  visited[start] = 1;
  int32_t k = 1, new_edges = 0, nc = 0;
  while (k < n) {
    int32_t u = route[k - 1];
    uint32_t word = orc_draw(seed, (uint32_t)k, (uint32_t)ant, iter, 0);
    int32_t v = select_next(C, u, visited, word, st);
    if (st) st[ORC_ST_ACO_STEPS]++;
    route[k++] = v;
    visited[v] = 1;
    int32_t su = sr[(sp[u] + 1) % n], pu = sr[(sp[u] + n - 1) % n];
    if (v != su && v != pu) {
      new_edges++;
      check[nc++] = v;
    }
    if (new_edges >= C->prm.min_new_edges) {
      int32_t x = v;
      for (;;) { /* forward along the source */
        int32_t y = sr[(sp[x] + 1) % n];
        if (visited[y]) break;
        route[k++] = y;
        visited[y] = 1;
        x = y;
      }
      for (;;) { /* backward along the source */
        int32_t y = sr[(sp[x] + n - 1) % n];
        if (visited[y]) break;
        route[k++] = y;
        visited[y] = 1;
        x = y;
      }
    }
  }
  if (st) {
    st[ORC_ST_NEW_EDGES] = new_edges;
    st[ORC_ST_CHECKLIST] = nc;
  }
  return nc;
}

/* ------------------------------------------------------------------ */
/* Pheromone limits (Sec. 4.5) and update (Eq. 2)                      */
/* ------------------------------------------------------------------ */

static void set_limits(orc_colony* C, int64_t L_gb) {
  C->tmax_d = 1.0 / ((double)L_gb * (1.0 - (double)C->prm.rho));
  C->tmin_d = C->tmax_d * C->c_min;
  C->tmax = (float)C->tmax_d;
  C->tmin = (float)C->tmin_d;
}

static void update_pheromone(orc_colony* C) {
  int32_t n = C->n, k = C->k;
  float delta = (float)(1.0 / (double)C->src_len);
  float rho = C->prm.rho;
  for (int32_t u = 0; u < n; ++u) {
    int32_t su = C->src_route[(C->src_pos[u] + 1) % n];
    int32_t pu = C->src_route[(C->src_pos[u] + n - 1) % n];
    for (int32_t s = 0; s < k; ++s) {
      int32_t v = C->cand[(size_t)u * k + s];
      float dep = (v == su || v == pu) ? delta : 0.0f;
      float t = fmaf(rho, C->tau[(size_t)u * k + s], dep);
      t = t < C->tmax ? t : C->tmax; /* min{tau_max, .} */
      t = t > C->tmin ? t : C->tmin; /* max{tau_min, .} */
      C->tau[(size_t)u * k + s] = t;
    }
  }
}

static void set_positions(int32_t n, const int32_t* route, int32_t* pos) {
  for (int32_t i = 0; i < n; ++i) pos[route[i]] = i;
}

/* ------------------------------------------------------------------ */
/* Create: lists, eta, initial tour, limits, tau = tau_max            */
/* ------------------------------------------------------------------ */

/* Nearest-neighbour heuristic from node 0 (Sec. 4.3: the initial solution):
 * the first unvisited node of the candidate list, else of the backup list,
 * else the globally nearest unvisited node by (squared distance, index). */
void orc_nn_tour(const int32_t* xy, int32_t n, const int32_t* cand, int32_t k,
                 const int32_t* backup, int32_t bl, int32_t* route) {
  uint8_t* vis = (uint8_t*)calloc((size_t)n, 1);
  route[0] = 0;
  vis[0] = 1;
  for (int32_t i = 1; i < n; ++i) {
    int32_t u = route[i - 1], v = -1;
    for (int32_t s = 0; s < k && v < 0; ++s)
      if (!vis[cand[(size_t)u * k + s]]) v = cand[(size_t)u * k + s];
    for (int32_t j = 0; j < bl && v < 0; ++j)
      if (!vis[backup[(size_t)u * bl + j]]) v = backup[(size_t)u * bl + j];
    if (v < 0) {
      uint64_t bm = 0;
      for (int32_t w = 0; w < n; ++w) {
        if (vis[w]) continue;
        uint64_t m = sq_dist(xy, u, w);
        if (v < 0 || key_less(m, w, bm, v)) {
          v = w;
          bm = m;
        }
      }
    }
    route[i] = v;
    vis[v] = 1;
  }
  free(vis);
}

int orc_create(const int32_t* xy, int32_t n, int32_t k, const orc_params* p, orc_colony** out) {
  if (!xy || !out || n < 3 || k < 2) return ORC_E_ARG;
  orc_params prm;
  if (p)
    prm = *p;
  else
    orc_params_default(&prm);
  if (prm.threads < 1) prm.threads = 1;
  for (int32_t i = 0; i < 2 * n; ++i)
    if (xy[i] < 0 || xy[i] >= (1 << 24)) return ORC_E_ARG;
  orc_colony* C = (orc_colony*)calloc(1, sizeof(orc_colony));
  if (!C) return ORC_E_NOMEM;
  C->n = n;
  C->k = k < n - 1 ? k : n - 1;
  C->bl = prm.bl_size < n - 1 - C->k ? prm.bl_size : n - 1 - C->k;
  if (C->bl < 0) C->bl = 0;
  C->prm = prm;
  C->xy = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)n);
  memcpy(C->xy, xy, sizeof(int32_t) * 2 * (size_t)n);

  int32_t K = C->k + C->bl;
  int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* nn = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * (size_t)(K > 0 ? K : 1));
  for (int32_t i = 0; i < n; ++i) rows[i] = i;
  orc_knn_rows(C->xy, n, K, rows, n, prm.threads, nn);
  C->cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * C->k);
  C->backup = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * (C->bl > 0 ? C->bl : 1));
  C->eta = (float*)malloc(sizeof(float) * (size_t)n * C->k);
  C->tau = (float*)malloc(sizeof(float) * (size_t)n * C->k);
  for (int32_t u = 0; u < n; ++u) {
    for (int32_t s = 0; s < C->k; ++s) {
      int32_t v = nn[(size_t)u * K + s];
      C->cand[(size_t)u * C->k + s] = v;
      int32_t d = orc_euc2d(C->xy, u, v);
      C->eta[(size_t)u * C->k + s] = d > 0 ? 1.0f / (float)d : 1.0f; /* eta = 1/d */
    }
    for (int32_t j = 0; j < C->bl; ++j) C->backup[(size_t)u * C->bl + j] = nn[(size_t)u * K + C->k + j];
  }
  free(nn);

  /* initial tour: nearest neighbour from node 0, then local search */
  C->init_route = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  orc_nn_tour(C->xy, n, C->cand, C->k, C->backup, C->bl, C->init_route);
  set_positions(n, C->init_route, pos);
  for (int32_t i = 0; i < n; ++i) rows[i] = C->init_route[i];
  orc_local_search_ex(C->xy, n, C->cand, C->k, prm.oropt, prm.verify_pass, prm.init_3opt, C->init_route,
                      pos, rows, n, NULL);
  free(rows);
  free(pos);
  C->init_len = orc_tour_length(C->xy, n, C->init_route);

  /* Alg 2: global best := initial, limits, tau := tau_max, source := gb */
  C->gb_route = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  C->gb_pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  C->src_route = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  C->src_pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  memcpy(C->gb_route, C->init_route, sizeof(int32_t) * (size_t)n);
  set_positions(n, C->gb_route, C->gb_pos);
  C->gb_len = C->init_len;
  memcpy(C->src_route, C->gb_route, sizeof(int32_t) * (size_t)n);
  memcpy(C->src_pos, C->gb_pos, sizeof(int32_t) * (size_t)n);
  C->src_len = C->gb_len;
  double pr = pow(prm.p_best, 1.0 / (double)n);
  C->c_min = (1.0 - pr) / ((double)(C->k - 1) * pr);
  set_limits(C, C->gb_len);
  for (size_t i = 0; i < (size_t)n * C->k; ++i) C->tau[i] = C->tmax;
  C->iter = 0;
  *out = C;
  return ORC_OK;
}

void orc_destroy(orc_colony* C) {
  if (!C) return;
  free(C->xy); free(C->cand); free(C->backup); free(C->eta); free(C->tau);
  free(C->src_route); free(C->src_pos); free(C->gb_route); free(C->gb_pos);
  free(C->init_route);
  free(C->ant_routes); free(C->ant_len); free(C->ant_stats);
  free(C->pre_routes); free(C->pre_len); free(C->pre_check); free(C->pre_ncheck);
  free(C);
}

/* ------------------------------------------------------------------ */
/* Main loop (Alg 2)                                                   */
/* ------------------------------------------------------------------ */

static void ensure_ants(orc_colony* C, int32_t ants) {
  if (ants <= C->ants_cap) return;
  size_t n = (size_t)C->n;
  C->ant_routes = (int32_t*)realloc(C->ant_routes, sizeof(int32_t) * n * ants);
  C->ant_len = (int64_t*)realloc(C->ant_len, sizeof(int64_t) * ants);
  C->ant_stats = (int64_t*)realloc(C->ant_stats, sizeof(int64_t) * ORC_NSTATS * ants);
  if (C->prm.keep_pre_ls) {
    C->pre_routes = (int32_t*)realloc(C->pre_routes, sizeof(int32_t) * n * ants);
    C->pre_len = (int64_t*)realloc(C->pre_len, sizeof(int64_t) * ants);
    C->pre_check = (int32_t*)realloc(C->pre_check, sizeof(int32_t) * n * ants);
    C->pre_ncheck = (int32_t*)realloc(C->pre_ncheck, sizeof(int32_t) * ants);
  }
  C->ants_cap = ants;
}

int orc_iterate(orc_colony* C, int32_t ants, int32_t iters, int64_t* hist, int64_t* ant_len_hist) {
  if (!C || ants < 1 || iters < 0) return ORC_E_ARG;
  ensure_ants(C, ants);
  C->ants_last = ants;
  int32_t n = C->n;
  for (int32_t it = 0; it < iters; ++it) {
    C->iter++;
    uint32_t iter = (uint32_t)C->iter;
#pragma omp parallel num_threads(C->prm.threads)
    {
      uint8_t* visited = (uint8_t*)malloc((size_t)n);
      int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      int32_t* check = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
      for (int32_t a = 0; a < ants; ++a) {
        int32_t* route = C->ant_routes + (size_t)a * n;
        int64_t* st = C->ant_stats + (size_t)a * ORC_NSTATS;
        memset(st, 0, sizeof(int64_t) * ORC_NSTATS);
        int32_t nc = construct(C, a, iter, route, visited, check, st);
        if (C->prm.keep_pre_ls) {
          memcpy(C->pre_routes + (size_t)a * n, route, sizeof(int32_t) * (size_t)n);
          memcpy(C->pre_check + (size_t)a * n, check, sizeof(int32_t) * (size_t)nc);
          C->pre_ncheck[a] = nc;
          C->pre_len[a] = orc_tour_length(C->xy, n, route);
        }
        int64_t L0 = orc_tour_length(C->xy, n, route);
        int64_t g = 0;
        if (C->prm.local_search) {  /* base FACO (no LS) keeps the constructed tour */
          set_positions(n, route, pos);
          g = orc_local_search(C->xy, n, C->cand, C->k, C->prm.oropt, C->prm.verify_pass, route, pos,
                               check, nc, st);
        }
        C->ant_len[a] = L0 - g;
      }
      free(visited);
      free(pos);
      free(check);
    }
    /* iteration best: shortest tour, lowest ant index on ties */
    int32_t best = 0;
    for (int32_t a = 1; a < ants; ++a)
      if (C->ant_len[a] < C->ant_len[best]) best = a;
    int32_t* ib = C->ant_routes + (size_t)best * n;
    if (C->ant_len[best] < C->gb_len) {
      memcpy(C->gb_route, ib, sizeof(int32_t) * (size_t)n);
      set_positions(n, C->gb_route, C->gb_pos);
      C->gb_len = C->ant_len[best];
      set_limits(C, C->gb_len);
    }
    /* source: global best with probability p_source_gb, else iteration best */
    float u = orc_u01(orc_draw(C->prm.seed, 0, 0, iter, 1));
    int use_gb = (double)u < C->prm.p_source_gb;
    if (use_gb) {
      memcpy(C->src_route, C->gb_route, sizeof(int32_t) * (size_t)n);
      C->src_len = C->gb_len;
    } else {
      memcpy(C->src_route, ib, sizeof(int32_t) * (size_t)n);
      C->src_len = C->ant_len[best];
    }
    set_positions(n, C->src_route, C->src_pos);
    update_pheromone(C);
    if (hist) {
      hist[4 * it + 0] = C->ant_len[best];
      hist[4 * it + 1] = best;
      hist[4 * it + 2] = C->gb_len;
      hist[4 * it + 3] = use_gb;
    }
    if (ant_len_hist) memcpy(ant_len_hist + (size_t)it * ants, C->ant_len, sizeof(int64_t) * ants);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Accessors                                                           */
/* ------------------------------------------------------------------ */

int32_t orc_n(const orc_colony* C) { return C->n; }
int32_t orc_k(const orc_colony* C) { return C->k; }
int32_t orc_bl(const orc_colony* C) { return C->bl; }
int64_t orc_iteration(const orc_colony* C) { return C->iter; }

void orc_get_lists(const orc_colony* C, int32_t* cand, int32_t* backup, float* eta) {
  size_t n = (size_t)C->n;
  if (cand) memcpy(cand, C->cand, sizeof(int32_t) * n * C->k);
  if (backup && C->bl > 0) memcpy(backup, C->backup, sizeof(int32_t) * n * C->bl);
  if (eta) memcpy(eta, C->eta, sizeof(float) * n * C->k);
}

void orc_get_tau(const orc_colony* C, float* tau) {
  memcpy(tau, C->tau, sizeof(float) * (size_t)C->n * C->k);
}

void orc_get_limits(const orc_colony* C, double* out4) {
  out4[0] = C->tmax_d;
  out4[1] = C->tmin_d;
  out4[2] = C->tmax;
  out4[3] = C->tmin;
}

int64_t orc_get_source(const orc_colony* C, int32_t* route) {
  if (route) memcpy(route, C->src_route, sizeof(int32_t) * (size_t)C->n);
  return C->src_len;
}

int64_t orc_get_best(const orc_colony* C, int32_t* route) {
  if (route) memcpy(route, C->gb_route, sizeof(int32_t) * (size_t)C->n);
  return C->gb_len;
}

int64_t orc_get_initial(const orc_colony* C, int32_t* route) {
  if (route) memcpy(route, C->init_route, sizeof(int32_t) * (size_t)C->n);
  return C->init_len;
}

int32_t orc_last_ants(const orc_colony* C) { return C->ants_last; }

void orc_get_ant_tours(const orc_colony* C, int32_t* tours, int64_t* lens) {
  if (tours) memcpy(tours, C->ant_routes, sizeof(int32_t) * (size_t)C->n * C->ants_last);
  if (lens) memcpy(lens, C->ant_len, sizeof(int64_t) * C->ants_last);
}

void orc_get_ant_stats(const orc_colony* C, int64_t* stats) {
  memcpy(stats, C->ant_stats, sizeof(int64_t) * ORC_NSTATS * C->ants_last);
}

int orc_get_ant_pre(const orc_colony* C, int32_t* tours, int64_t* lens, int32_t* checklists,
                    int32_t* nchecks) {
  if (!C->prm.keep_pre_ls || !C->pre_routes) return ORC_E_ARG;
  size_t n = (size_t)C->n;
  if (tours) memcpy(tours, C->pre_routes, sizeof(int32_t) * n * C->ants_last);
  if (lens) memcpy(lens, C->pre_len, sizeof(int64_t) * C->ants_last);
  if (checklists) memcpy(checklists, C->pre_check, sizeof(int32_t) * n * C->ants_last);
  if (nchecks) memcpy(nchecks, C->pre_ncheck, sizeof(int32_t) * C->ants_last);
  return ORC_OK;
}

int orc_set_state(orc_colony* C, const float* tau, const int32_t* src_route) {
  if (tau) memcpy(C->tau, tau, sizeof(float) * (size_t)C->n * C->k);
  if (src_route) {
    memcpy(C->src_route, src_route, sizeof(int32_t) * (size_t)C->n);
    set_positions(C->n, C->src_route, C->src_pos);
    C->src_len = orc_tour_length(C->xy, C->n, C->src_route);
  }
  return ORC_OK;
}

int orc_set_threads(orc_colony* C, int32_t threads) {
  if (!C || threads < 1) return ORC_E_ARG;
  C->prm.threads = threads;
  return ORC_OK;
}
