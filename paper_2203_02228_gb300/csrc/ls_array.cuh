// ls_array.cuh -- warp-cooperative local search on an explicit tour array.
//
// Sec. 4.4, Alg 3: pop a node a from the checklist FIFO, scan its
// nearest-neighbour list for the best improving 2-opt move (successor side
// first, then predecessor side, strict '>'), flip the tour section, queue
// the four endpoints.  The scan is one warp: with k <= 16, lanes 0..15 take
// the successor-side moves of NN(a)[lane] and lanes 16..31 the
// predecessor-side moves; the warp arg-max with ties to the lowest order
// index is exactly the first strict maximum of the sequential loops.
//
// Readings shared with the oracle (decided independently there):
//   flip       reverse the forward span x..y, or the complementary span when
//              2*len > n (same cycle, opposite orientation);
//   queue      FIFO with an in-queue bit; a queued node is not queued twice;
//   verify     when the queue runs dry after a round that applied a move,
//              every node popped in that round is queued again (first-pop
//              order) and the search continues; stop after a clean round,
//              or after n applied moves (Alg 3's limit);
//   Or-opt     tried from a only when its 2-opt scan found nothing: move the
//              segment a..e (1..3 nodes following a) between the ends (u,v)
//              of a tour edge at b in NN(a) -- (b, succ b) then (pred b, b)
//              -- reversed first, then kept; u, v outside the segment and
//              {pred a, succ e}; applied as two or three edge exchanges.
#pragma once

#include <climits>

#include "common.cuh"

namespace faco {

struct ArrTour {
  int n;
  int32_t* route;
  int32_t* pos;
};

struct LsEnv {
  int n, k, oropt, verify;
  const int2* xy;
  const int32_t* cand;
  int32_t* queue;   // n entries, ring
  uint8_t* flags;   // n entries, zero on entry and on exit
  int32_t* logb;    // n entries
};

struct LsStats {
  int64_t pops, moves2, movesor, flip, verify;
};

static __device__ __forceinline__ int arr_succ(const ArrTour& T, int x) {
  const int p = T.pos[x] + 1;
  return T.route[p == T.n ? 0 : p];
}

static __device__ __forceinline__ int arr_pred(const ArrTour& T, int x) {
  const int p = T.pos[x] - 1;
  return T.route[p < 0 ? T.n - 1 : p];
}

// Reverse the forward span x..y (or its complement when longer than n/2).
static __device__ __noinline__ void arr_flip(ArrTour& T, int x, int y, LsStats& S) {
  const int n = T.n, lane = lane_id();
  int i = T.pos[x], j = T.pos[y];
  int L = j - i;
  if (L < 0) L += n;
  L += 1;
  if (2 * L > n) {
    const int i2 = (j + 1 == n) ? 0 : j + 1;
    const int j2 = (i == 0) ? n - 1 : i - 1;
    i = i2;
    j = j2;
    L = n - L;
  }
  const int half = L >> 1;
  constexpr int U = 4;
  for (int t0 = 0; t0 < half; t0 += 32 * U) {
    int ia[U], ib[U], va[U], vb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + lane + 32 * u;
      ia[u] = -1;
      if (t < half) {
        ia[u] = i + t;
        if (ia[u] >= n) ia[u] -= n;
        ib[u] = j - t;
        if (ib[u] < 0) ib[u] += n;
        va[u] = T.route[ia[u]];
        vb[u] = T.route[ib[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (ia[u] >= 0) {
        T.route[ia[u]] = vb[u];
        T.route[ib[u]] = va[u];
        T.pos[vb[u]] = ia[u];
        T.pos[va[u]] = ib[u];
      }
    }
  }
  __syncwarp();
  S.flip += L;
}

// Exchange tour edges {n1,n2},{n3,n4} for {n1,n3},{n2,n4}: with n1->n2 a
// forward edge this is the Alg 3 move (n1,n2,n3,n4) -> flip n2..n3,
// otherwise the move (n2,n1,n4,n3) -> flip n1..n4.
static __device__ __forceinline__ void arr_move2(ArrTour& T, int n1, int n2, int n3, int n4, LsStats& S) {
  if (arr_succ(T, n1) == n2)
    arr_flip(T, n2, n3, S);
  else
    arr_flip(T, n1, n4, S);
}

// Best improving 2-opt move from a; returns the gain (0: none) and the move
// (w,x,y,z) with w->x and y->z removed, flip x..y.
static __device__ __noinline__ int64_t arr_eval_2opt(const LsEnv& E, const ArrTour& T, int a, int mv[4]) {
  const int n = E.n, k = E.k, lane = lane_id();
  const int apos = T.pos[a];
  const int a_succ = T.route[apos + 1 == n ? 0 : apos + 1];
  const int a_pred = T.route[apos == 0 ? n - 1 : apos - 1];
  const int2 xa = E.xy[a], xs = E.xy[a_succ], xp = E.xy[a_pred];
  const int d_as = euc2d(xa, xs), d_ap = euc2d(xp, xa);
  int64_t best = 0;
  int bidx = INT_MAX;
  const int passes = k <= 16 ? 1 : 2;
  for (int pass = 0; pass < passes; ++pass) {
    const int side = k <= 16 ? (lane >> 4) : pass;
    const int s = k <= 16 ? (lane & 15) : lane;
    int64_t g = 0;
    if (s < k) {
      const int b = E.cand[(size_t)a * k + s];
      const int bp = T.pos[b];
      const int bn = side == 0 ? T.route[bp + 1 == n ? 0 : bp + 1] : T.route[bp == 0 ? n - 1 : bp - 1];
      const int2 xb = E.xy[b], xbn = E.xy[bn];
      const int d_ab = euc2d(xa, xb);
      if (side == 0) {
        if (d_as > d_ab) g = (int64_t)d_as + euc2d(xb, xbn) - d_ab - euc2d(xs, xbn);
      } else {
        if (d_ap > d_ab) g = (int64_t)d_ap + euc2d(xbn, xb) - d_ab - euc2d(xp, xbn);
      }
    }
    int idx = side * k + s;
    if (!(g > 0)) {
      g = 0;
      idx = INT_MAX;
    }
    warp_max_gain(g, idx);
    if (g > best) {
      best = g;
      bidx = idx;
    }
  }
  if (best > 0) {
    const int side = bidx / k, s = bidx % k;
    const int b = E.cand[(size_t)a * k + s];
    if (side == 0) {
      mv[0] = a; mv[1] = a_succ; mv[2] = b; mv[3] = arr_succ(T, b);
    } else {
      mv[0] = a_pred; mv[1] = a; mv[2] = arr_pred(T, b); mv[3] = b;
    }
  }
  return best;
}

// Best improving Or-opt move from a (definition in the file comment).
// mv = {p, a, e, q, u, v, kept}.
static __device__ __noinline__ int64_t arr_eval_or(const LsEnv& E, const ArrTour& T, int a, int mv[7]) {
  const int n = E.n, k = E.k, lane = lane_id();
  if (n < 8) return 0;
  const int apos = T.pos[a];
  auto at = [&](int off) {
    int p = apos + off;
    if (p >= n) p -= n;
    if (p < 0) p += n;
    return T.route[p];
  };
  const int p = at(-1), s1 = at(1), s2 = at(2), s3 = at(3);
  const int2 xa = E.xy[a], xp = E.xy[p], x1 = E.xy[s1], x2 = E.xy[s2], x3 = E.xy[s3];
  const int d_pa = euc2d(xp, xa);
  // l = 1: e = a, q = s1;  l = 2: e = s1, q = s2;  l = 3: e = s2, q = s3
  const int64_t rem1 = (int64_t)d_pa + euc2d(xa, x1) - euc2d(xp, x1);
  const int64_t rem2 = (int64_t)d_pa + euc2d(x1, x2) - euc2d(xp, x2);
  const int64_t rem3 = (int64_t)d_pa + euc2d(x2, x3) - euc2d(xp, x3);
  int64_t lbest = 0;
  int lidx = INT_MAX;
  const int passes = k <= 16 ? 1 : 2;
  for (int pass = 0; pass < passes; ++pass) {
    const int side = k <= 16 ? (lane >> 4) : pass;
    const int s = k <= 16 ? (lane & 15) : lane;
    if (s < k) {
      const int b = E.cand[(size_t)a * k + s];
      const int bp = T.pos[b];
      int u, v;
      if (side == 0) {
        u = b;
        v = T.route[bp + 1 == n ? 0 : bp + 1];
      } else {
        u = T.route[bp == 0 ? n - 1 : bp - 1];
        v = b;
      }
      const int2 xu = E.xy[u], xv = E.xy[v];
      const int d_uv = euc2d(xu, xv);
      const int d_ua = euc2d(xu, xa), d_av = euc2d(xa, xv);
#pragma unroll
      for (int l = 1; l <= 3; ++l) {
        const int q = l == 1 ? s1 : (l == 2 ? s2 : s3);
        bool bad = (u == p || v == p || u == q || v == q || u == a || v == a);
        if (l >= 2) bad |= (u == s1 || v == s1);
        if (l >= 3) bad |= (u == s2 || v == s2);
        if (bad) continue;
        const int64_t rem = l == 1 ? rem1 : (l == 2 ? rem2 : rem3);
        const int2 xe = l == 1 ? xa : (l == 2 ? x1 : x2);
        // reversed: u-e ... a-v
        {
          const int64_t g = rem + d_uv - euc2d(xu, xe) - d_av;
          const int idx = (((l - 1) * k + s) * 2 + side) * 2 + 0;
          if (g > lbest || (g == lbest && g > 0 && idx < lidx)) {
            lbest = g;
            lidx = idx;
          }
        }
        if (l >= 2) {  // kept: u-a ... e-v
          const int64_t g = rem + d_uv - d_ua - euc2d(xe, xv);
          const int idx = (((l - 1) * k + s) * 2 + side) * 2 + 1;
          if (g > lbest || (g == lbest && g > 0 && idx < lidx)) {
            lbest = g;
            lidx = idx;
          }
        }
      }
    }
  }
  if (!(lbest > 0)) {
    lbest = 0;
    lidx = INT_MAX;
  }
  warp_max_gain(lbest, lidx);
  if (lbest > 0) {
    const int kept = lidx & 1, side = (lidx >> 1) & 1, rest = lidx >> 2;
    const int s = rest % k, l = rest / k + 1;
    const int b = E.cand[(size_t)a * k + s];
    int u, v;
    if (side == 0) {
      u = b;
      v = arr_succ(T, b);
    } else {
      u = arr_pred(T, b);
      v = b;
    }
    mv[0] = p; mv[1] = a; mv[2] = l == 1 ? a : (l == 2 ? s1 : s2);
    mv[3] = l == 1 ? s1 : (l == 2 ? s2 : s3); mv[4] = u; mv[5] = v; mv[6] = kept;
  }
  return lbest;
}

// FIFO push by lane 0 (the caller broadcasts qn afterwards).
static __device__ __forceinline__ void ls_push0(const LsEnv& E, int x, int qh, int& qn) {
  const uint8_t f = E.flags[x];
  if (!(f & 1)) {
    E.flags[x] = f | 1;
    int t = qh + qn;
    if (t >= E.n) t -= E.n;
    E.queue[t] = x;
    ++qn;
  }
}

// Runs the search from the checklist init[0..ninit) (distinct nodes).
// Returns the total gain (old length - new length).
static __device__ __noinline__ int64_t ls_array_run(const LsEnv& E, ArrTour& T, const int32_t* init,
                                             int ninit, LsStats& S) {
  const int n = E.n, lane = lane_id();
  for (int i = lane; i < ninit; i += 32) {
    const int x = init[i];
    E.queue[i] = x;
    E.flags[x] = 1;
  }
  __syncwarp();
  int qh = 0, qn = ninit, nlog = 0, changes = 0, moves_round = 0;
  int64_t total = 0;
  for (;;) {
    while (qn > 0 && changes < n) {
      const int a = E.queue[qh];
      qh = (qh + 1 == n) ? 0 : qh + 1;
      --qn;
      const uint8_t f = E.flags[a];
      __syncwarp();
      if (lane == 0) {
        E.flags[a] = (uint8_t)((f & ~1) | 2);
        if (!(f & 2)) E.logb[nlog] = a;
      }
      if (!(f & 2)) ++nlog;
      __syncwarp();
      S.pops++;
      int mv[7];
      int64_t g = arr_eval_2opt(E, T, a, mv);
      if (g > 0) {
        arr_flip(T, mv[1], mv[2], S);
        if (lane == 0)
          for (int t = 0; t < 4; ++t) ls_push0(E, mv[t], qh, qn);
        qn = __shfl_sync(kFull, qn, 0);
        __syncwarp();
        total += g;
        ++changes;
        ++moves_round;
        S.moves2++;
        continue;
      }
      if (E.oropt) {
        g = arr_eval_or(E, T, a, mv);
        if (g > 0) {
          arr_move2(T, mv[0], mv[1], mv[4], mv[5], S);  // {p,a},{u,v} -> {p,u},{a,v}
          arr_move2(T, mv[0], mv[4], mv[3], mv[2], S);  // {p,u},{q,e} -> {p,q},{u,e}
          if (mv[6]) arr_move2(T, mv[4], mv[2], mv[1], mv[5], S);  // {u,e},{a,v} -> {u,a},{e,v}
          if (lane == 0)
            for (int t = 0; t < 6; ++t) ls_push0(E, mv[t], qh, qn);
          qn = __shfl_sync(kFull, qn, 0);
          __syncwarp();
          total += g;
          ++changes;
          ++moves_round;
          S.movesor++;
        }
      }
    }
    if (changes >= n || !E.verify || moves_round == 0) break;
    // verify round: queue again every node popped in the last round
    S.verify++;
    for (int i = lane; i < nlog; i += 32) {
      const int x = E.logb[i];
      E.queue[i] = x;
      E.flags[x] = 1;
    }
    __syncwarp();
    qh = 0;
    qn = nlog;
    nlog = 0;
    moves_round = 0;
  }
  // leave the flags clean for the next search
  for (int t = lane; t < qn; t += 32) {
    int i = qh + t;
    if (i >= n) i -= n;
    E.flags[E.queue[i]] = 0;
  }
  for (int i = lane; i < nlog; i += 32) E.flags[E.logb[i]] = 0;
  __syncwarp();
  return total;
}

}  // namespace faco
