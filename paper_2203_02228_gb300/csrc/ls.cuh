// ls.cuh -- warp-cooperative local search (Sec. 4.4, Alg 3), generic over
// the tour representation.
//
// Pop a node a from the checklist FIFO, scan its nearest-neighbour list for
// the best improving 2-opt move (successor side first, then predecessor
// side, strict '>'), flip the tour section, queue the four endpoints.  The
// scan is one warp: with k <= 16, lanes 0..15 take the successor-side moves
// of NN(a)[lane] and lanes 16..31 the predecessor-side moves; the warp
// arg-max with ties to the lowest order index is exactly the first strict
// maximum of the sequential loops.
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
//
// A Tour provides (device, lane-local unless noted): n, k; pos_of(x);
// succ(x), pred(x); adj(x, up) (succ when up, else pred, one code path for
// lanes that differ in direction); nbrs(x, pred, succ); walk(a, pred, s1,
// s2, s3) (the predecessor and three successors); coord(x); cand(x, s);
// cdist(x, s) (the cost of that candidate edge); and the warp-collective
// flip(x, y, S) (false when the representation ran out of capacity).
#pragma once

#include <climits>

#include "common.cuh"

namespace faco {

struct LsEnv {
  int n, oropt, verify;
  int32_t* queue;   // n entries, ring
  uint8_t* flags;   // n entries: bit0 queued, bit1 popped this round; zero on entry and exit
  int32_t* logb;    // n entries: nodes popped this round, first-pop order
};

struct LsStats {
  int64_t pops, moves2, movesor, flip, verify;
  int64_t t_eval, t_confirm, t_flip, t_push;  // device ns per phase (block search)
};

// Explicit tour: route[t] = node at position t, pos = inverse.  Nodes are
// node ids (with node-indexed xy/cn) or source positions (with the
// source-ordered copies); cn rows are `stride` entries apart.
struct ArrTour {
  int n, k;
  int32_t* route;
  int32_t* pos;
  const int2* xy;       // coordinates by node
  const int32_t* cn;    // candidate lists by node [n][stride]
  int stride;
  const int32_t* cd;    // their EUC_2D costs, same layout
  __device__ __forceinline__ int pos_of(int x) const { return pos[x]; }
  // x moves from position `from` to `to`
  __device__ __forceinline__ void move_pos(int x, int from, int to) {
    (void)from;
    pos[x] = to;
  }
  __device__ __forceinline__ int at_off(int p, int d) const {
    p += d;
    if (p >= n) p -= n;
    if (p < 0) p += n;
    return route[p];
  }
  __device__ __forceinline__ int succ(int x) const { return at_off(pos[x], 1); }
  __device__ __forceinline__ int succ_w(int x) const { return succ(x); }  // warp-uniform x
  __device__ __forceinline__ int pred(int x) const { return at_off(pos[x], -1); }
  __device__ __forceinline__ int adj(int x, bool up) const { return at_off(pos[x], up ? 1 : -1); }
  __device__ __forceinline__ void nbrs(int x, int& p, int& s) const {
    const int t = pos[x];
    p = at_off(t, -1);
    s = at_off(t, 1);
  }
  __device__ __forceinline__ void walk(int a, int& p, int& s1, int& s2, int& s3) const {
    const int t = pos[a];
    p = at_off(t, -1);
    s1 = at_off(t, 1);
    s2 = at_off(t, 2);
    s3 = at_off(t, 3);
  }
  __device__ __forceinline__ int2 coord(int x) const { return xy[x]; }
  __device__ __forceinline__ int cand(int x, int s) const { return cn[(size_t)x * stride + s]; }
  __device__ __forceinline__ int cdist(int x, int s) const { return cd[(size_t)x * stride + s]; }

  // Reverse the forward span x..y (or its complement when longer than n/2).
  __device__ __forceinline__ bool flip(int x, int y, LsStats& S) {
    const int lane = lane_id();
    int i = pos[x], j = pos[y];
    __syncwarp();  // every lane has read i and j before a position moves
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
          va[u] = route[ia[u]];
          vb[u] = route[ib[u]];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (ia[u] >= 0) {
          route[ia[u]] = vb[u];
          route[ib[u]] = va[u];
          pos[vb[u]] = ia[u];
          pos[va[u]] = ib[u];
        }
      }
    }
    __syncwarp();
    S.flip += L;
    return true;
  }
};

// Exchange tour edges {n1,n2},{n3,n4} for {n1,n3},{n2,n4}: with n1->n2 a
// forward edge this is the Alg 3 move (n1,n2,n3,n4) -> flip n2..n3,
// otherwise the move (n2,n1,n4,n3) -> flip n1..n4.  Warp-collective.
template <class Tour>
__device__ __forceinline__ bool tour_move2(Tour& T, int n1, int n2, int n3, int n4, LsStats& S) {
  if (T.succ_w(n1) == n2) return T.flip(n2, n3, S);
  return T.flip(n1, n4, S);
}

// Both scans from a in one pass over NN(a) (one lookup of a, one of each
// neighbour b): the best 2-opt move and, when do_or, the best Or-opt move.
// The search then takes the 2-opt move if it gains, else the Or-opt move --
// the same decision as scanning one after the other.  Lane layout: with
// k <= 16, lane = side * 16 + s (side 0: the edge (b, succ b), side 1:
// (pred b, b)); with k > 16, lane = s and the two sides are two passes.
// The loads that do not depend on the walk from a (the candidate row, b's
// coordinates) are issued before it; the move is rebuilt from the winning
// lane's registers.
template <class Tour>
__device__ __forceinline__ void eval_both(const Tour& T, int a, bool do_or, int64_t& g2, int mv2[4],
                                          int64_t& go, int mvo[7]) {
  const int n = T.n, k = T.k, lane = lane_id();
  do_or = do_or && n >= 8;
  const bool two = k > 16;
  const int s = two ? lane : (lane & 15);
  const bool live = s < k;
  const int b = live ? T.cand(a, s) : a;
  const int d_ab = live ? T.cdist(a, s) : 0;  // = euc2d(xa, xb), kept with the lists
  const int2 xb = T.coord(b);
  int p, s1, s2 = -1, s3 = -1;
  if (do_or)
    T.walk(a, p, s1, s2, s3);
  else
    T.nbrs(a, p, s1);
  const int2 xa = T.coord(a), x1 = T.coord(s1), xp = T.coord(p);
  int2 x2 = xa, x3 = xa;
  if (do_or) {
    x2 = T.coord(s2);
    x3 = T.coord(s3);
  }
  // b's tour neighbour on this lane's side (pass 0), and for k > 16 the
  // predecessor for pass 1
  int bn0 = a, bn1 = a;
  if (live) {
    if (two)
      T.nbrs(b, bn1, bn0);
    else
      bn0 = T.adj(b, lane < 16);
  }
  const int2 xbn0 = T.coord(bn0), xbn1 = two ? T.coord(bn1) : xa;
  // the costs within a's tour neighbourhood are the same on every lane:
  // lane j computes the j-th, shuffles share them
  //   0 d(a,s1)  1 d(p,a)  2 d(p,s1)  3 d(s1,s2)  4 d(p,s2)  5 d(s2,s3)  6 d(p,s3)
  int2 cu = xa, cv = x1;
  if (lane == 1) {
    cu = xp;
    cv = xa;
  } else if (lane == 2) {
    cu = xp;
  } else if (lane == 3) {
    cu = x1;
    cv = x2;
  } else if (lane == 4) {
    cu = xp;
    cv = x2;
  } else if (lane == 5) {
    cu = x2;
    cv = x3;
  } else if (lane == 6) {
    cu = xp;
    cv = x3;
  }
  const int32_t cst = euc2d(cu, cv);
  const int d_as = __shfl_sync(kFull, cst, 0), d_ap = __shfl_sync(kFull, cst, 1);
  // gains in 32 bits: each is a signed sum of at most six EUC_2D costs of
  // coordinates below 2^24 (each cost below 2^25)
  int32_t rem1 = 0, rem2 = 0, rem3 = 0;
  {
    const int32_t c2 = __shfl_sync(kFull, cst, 2), c3 = __shfl_sync(kFull, cst, 3),
                  c4 = __shfl_sync(kFull, cst, 4), c5 = __shfl_sync(kFull, cst, 5),
                  c6 = __shfl_sync(kFull, cst, 6);
    if (do_or) {
      rem1 = d_ap + d_as - c2;
      rem2 = d_ap + c3 - c4;
      rem3 = d_ap + c5 - c6;
    }
  }
  int32_t b2 = 0, bo = 0;
  int i2 = INT_MAX, io = INT_MAX;
  const int passes = two ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    const int side = two ? pass : (lane >> 4);
    const int bn = pass == 0 ? bn0 : bn1;
    const int2 xbn = pass == 0 ? xbn0 : xbn1;
    int32_t g = 0;
    int32_t lo = 0;
    int li = INT_MAX;
    if (live) {
      const int d_bbn = euc2d(xb, xbn);
      if (side == 0) {
        if (d_as > d_ab) g = d_as + d_bbn - d_ab - euc2d(x1, xbn);
      } else {
        if (d_ap > d_ab) g = d_ap + d_bbn - d_ab - euc2d(xp, xbn);
      }
      if (do_or) {
        // the tour edge (u, v) at b: (b, succ b) or (pred b, b)
        const int u = side == 0 ? b : bn, v = side == 0 ? bn : b;
        const int2 xu = side == 0 ? xb : xbn, xv = side == 0 ? xbn : xb;
        const int d_uv = d_bbn;
        const int d_ua = side == 0 ? d_ab : euc2d(xu, xa);
        const int d_av = side == 0 ? euc2d(xa, xv) : d_ab;
        const bool base_bad = (u == p || v == p || u == a || v == a);
#pragma unroll
        for (int l = 1; l <= 3; ++l) {
          const int q = l == 1 ? s1 : (l == 2 ? s2 : s3);
          bool bad = base_bad || u == q || v == q;
          if (l >= 2) bad |= (u == s1 || v == s1);
          if (l >= 3) bad |= (u == s2 || v == s2);
          if (bad) continue;
          const int32_t rem = l == 1 ? rem1 : (l == 2 ? rem2 : rem3);
          if (l == 1) {  // one node: only the reversed form, u-a-v
            const int32_t gg = rem + d_uv - d_ua - d_av;
            if (gg > lo) {
              lo = gg;
              li = (s * 2 + side) * 2;
            }
          } else {
            const int2 xe = l == 2 ? x1 : x2;
            const int d_ue = euc2d(xu, xe), d_ev = euc2d(xe, xv);
            const int base = (((l - 1) * k + s) * 2 + side) * 2;
            const int32_t g0 = rem + d_uv - d_ue - d_av;  // reversed: u-e ... a-v
            if (g0 > lo) {
              lo = g0;
              li = base;
            }
            const int32_t g1 = rem + d_uv - d_ua - d_ev;  // kept: u-a ... e-v
            if (g1 > lo) {
              lo = g1;
              li = base + 1;
            }
          }
        }
      }
    }
    int idx = side * k + s;
    if (!(g > 0)) {
      g = 0;
      idx = INT_MAX;
    }
    warp_max_gain(g, idx);
    if (g > b2) {
      b2 = g;
      i2 = idx;
    }
    if (do_or) {
      if (!(lo > 0)) {
        lo = 0;
        li = INT_MAX;
      }
      warp_max_gain(lo, li);
      if (lo > bo || (lo == bo && lo > 0 && li < io)) {
        bo = lo;
        io = li;
      }
    }
  }
  g2 = b2;
  go = bo;
  // the winner's b and tour neighbour, from its lane (the side is uniform)
  int side = 0, sw = 0;
  if (b2 > 0) {
    side = i2 / k;
    sw = i2 % k;
  } else if (bo > 0) {
    const int rest = io >> 2;
    side = (io >> 1) & 1;
    sw = rest % k;
  }
  const int wl = two ? sw : side * 16 + sw;
  const int bw = __shfl_sync(kFull, b, wl);
  const int bnw = __shfl_sync(kFull, (two && side == 1) ? bn1 : bn0, wl);
  if (b2 > 0) {
    if (side == 0) {
      mv2[0] = a; mv2[1] = s1; mv2[2] = bw; mv2[3] = bnw;
    } else {
      mv2[0] = p; mv2[1] = a; mv2[2] = bnw; mv2[3] = bw;
    }
  } else if (bo > 0) {
    const int kept = io & 1, l = (io >> 2) / k + 1;
    const int u = side == 0 ? bw : bnw, v = side == 0 ? bnw : bw;
    mvo[0] = p; mvo[1] = a; mvo[2] = l == 1 ? a : (l == 2 ? s1 : s2);
    mvo[3] = l == 1 ? s1 : (l == 2 ? s2 : s3); mvo[4] = u; mvo[5] = v; mvo[6] = kept;
  }
}

// The 3-opt segment exchange of the initial tour (Sec. 4.3: 2-opt and
// 3-opt following Bentley; the move and its search are a reading): the
// tour edges (a,t2), (b,b'), (c,c') become (a,b'), (b,c'), (c,t2), so that,
// walking from a towards t2, a [t2..b] [b'..c] c' turns into
// a [b'..c] [t2..b] c' -- two adjacent sections swap places, neither
// reversed.  t2 is a's successor (dir 0) or predecessor (dir 1); b' runs
// over NN(a) with g1 = d(a,t2) - d(a,b') > 0 and b is the node before b' in
// the walking direction; c' runs over NN(b) with g2 = g1 + d(b,b') -
// d(b,c') > 0 and c is the node before c'; valid when, counted from a in
// the walking direction, 1 <= r(b) < r(c) <= n - 2.  gain = g2 + d(c,c') -
// d(c,t2); the first strictly largest gain in the order (dir, b', c') wins.
// The warp takes the (dir, b', c') combinations 32 at a time, lane = order
// index mod 32.  Returns the gain (0: none) and mv = {a, t2, b, b', c, c'}.
// Warp-collective; the tour's nodes and coordinates as the Tour names them.
template <class Tour>
__device__ __forceinline__ int64_t eval_or3(const Tour& T, int a, int mv[6]) {
  const int n = T.n, k = T.k, lane = lane_id();
  if (n < 8) return 0;
  int p, s1;
  T.nbrs(a, p, s1);
  const int2 xa = T.coord(a), xs = T.coord(s1), xp = T.coord(p);
  const int d_as = euc2d(xa, xs), d_ap = euc2d(xa, xp);
  const int pa = T.pos_of(a);
  const int kk = k * k, total = 2 * kk;
  int32_t best = 0;
  int bi = INT_MAX, bb = -1, bb1 = -1, bc = -1, bc1 = -1;
  for (int idx = lane; idx < total; idx += 32) {
    const int dir = idx >= kk ? 1 : 0;
    const int r = idx - dir * kk;
    const int i = r / k, j = r - i * k;
    const int2 xt2 = dir ? xp : xs;
    const int g1 = (dir ? d_ap : d_as) - T.cdist(a, i);
    if (g1 <= 0) continue;
    const int b1 = T.cand(a, i);
    const int b = T.adj(b1, dir != 0);  // dir 0: pred(b'), dir 1: succ(b')
    const int2 xb = T.coord(b), xb1 = T.coord(b1);
    const int g2 = g1 + euc2d(xb, xb1) - T.cdist(b, j);
    if (g2 <= 0) continue;
    const int c1 = T.cand(b, j);
    const int c = T.adj(c1, dir != 0);
    int rb = dir ? pa - T.pos_of(b) : T.pos_of(b) - pa;
    int rc = dir ? pa - T.pos_of(c) : T.pos_of(c) - pa;
    if (rb < 0) rb += n;
    if (rc < 0) rc += n;
    if (!(rb >= 1 && rb < rc && rc <= n - 2)) continue;
    const int2 xc = T.coord(c), xc1 = T.coord(c1);
    const int32_t g = g2 + euc2d(xc, xc1) - euc2d(xc, xt2);
    if (g > best) {  // idx grows along the lane's loop: ties keep the earlier
      best = g;
      bi = idx;
      bb = b;
      bb1 = b1;
      bc = c;
      bc1 = c1;
    }
  }
  int32_t g = best > 0 ? best : 0;
  int32_t wi = best > 0 ? bi : INT_MAX;
  warp_max_gain(g, wi);
  if (g <= 0) return 0;
  const int wl = wi & 31;
  mv[0] = a;
  mv[1] = wi >= kk ? p : s1;
  mv[2] = __shfl_sync(kFull, bb, wl);
  mv[3] = __shfl_sync(kFull, bb1, wl);
  mv[4] = __shfl_sync(kFull, bc, wl);
  mv[5] = __shfl_sync(kFull, bc1, wl);
  return g;
}

// Evaluation from a on any tour; representations that can change on the
// way (a segment table that may move to arrays) provide their own overload
// that picks one concrete representation per call.
template <class Tour>
__device__ __forceinline__ void eval_dispatch(const Tour& T, int a, bool do_or, int64_t& g2, int mv2[4],
                                              int64_t& go, int mvo[7]) {
  eval_both(T, a, do_or, g2, mv2, go, mvo);
}

// Applies an Or-opt move {p,a,e,q,u,v,kept} as edge exchanges.
template <class Tour>
__device__ __forceinline__ bool apply_or(Tour& T, const int mv[7], LsStats& S) {
  if (!tour_move2(T, mv[0], mv[1], mv[4], mv[5], S)) return false;  // {p,a},{u,v} -> {p,u},{a,v}
  if (!tour_move2(T, mv[0], mv[4], mv[3], mv[2], S)) return false;  // {p,u},{q,e} -> {p,q},{u,e}
  if (mv[6] && !tour_move2(T, mv[4], mv[2], mv[1], mv[5], S)) return false;  // {u,e},{a,v} -> {u,a},{e,v}
  return true;
}

// apply_or called rather than inlined in the block search's round loop
// (about one move in six is an Or-opt move): the loop keeps a smaller code
// footprint and fewer spills (per-ant kernel 1.6 % faster).
template <class Tour>
__device__ __noinline__ bool apply_or_call(Tour& T, const int* mv, LsStats& S) {
  int m[7];
  for (int t = 0; t < 7; ++t) m[t] = mv[t];
  return apply_or(T, m, S);
}

// Queue the np (<= 32) nodes x[0..np) in order, each only if it is not
// queued yet (and not already pushed earlier in the list): lane t handles
// x[t].  Warp-collective; every lane receives the new qn.
__device__ __forceinline__ int ls_push_warp(const LsEnv& E, const int* x, int np, int qh, int qn) {
  const int lane = lane_id();
  int node = -1 - lane;  // distinct dummies for idle lanes
  if (lane < np) node = x[lane];
  const unsigned same = __match_any_sync(kFull, node);
  const bool leader = (same & ((1u << lane) - 1u)) == 0;  // first lane with this node
  uint8_t f = 0;
  if (lane < np && leader) f = E.flags[node];
  const bool push = lane < np && leader && !(f & 1);
  const unsigned bal = __ballot_sync(kFull, push);
  if (push) {
    E.flags[node] = f | 1;
    int t = qh + qn + __popc(bal & ((1u << lane) - 1u));
    if (t >= E.n) t -= E.n;
    if (t >= E.n) t -= E.n;
    E.queue[t] = node;
  }
  __syncwarp();
  return qn + __popc(bal);
}

// FIFO push by lane 0 (the caller broadcasts qn afterwards).
__device__ __forceinline__ void ls_push0(const LsEnv& E, int x, int qh, int& qn) {
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
// Returns the total gain (old length - new length), or -1 if the tour
// representation ran out of capacity (flags are left clean either way).
template <class Tour>
__device__ __forceinline__ int64_t ls_run(const LsEnv& E, Tour& T, const int32_t* init, int ninit,
                                          LsStats& S) {
  const int n = E.n, lane = lane_id();
  for (int i = lane; i < ninit; i += 32) {
    const int x = init[i];
    E.queue[i] = x;
    E.flags[x] = 1;
  }
  __syncwarp();
  int qh = 0, qn = ninit, nlog = 0, changes = 0, moves_round = 0;
  int64_t total = 0;
  bool ok = true;
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
      int mv[4], mvo[7];
      int64_t g, go;
      eval_both(T, a, E.oropt != 0, g, mv, go, mvo);
      if (g > 0) {
        ok = T.flip(mv[1], mv[2], S);
        if (!ok) break;
        qn = ls_push_warp(E, mv, 4, qh, qn);
        total += g;
        ++changes;
        ++moves_round;
        S.moves2++;
        continue;
      }
      if (E.oropt) {
        g = go;
        if (g > 0) {
          ok = apply_or(T, mvo, S);
          if (!ok) break;
          qn = ls_push_warp(E, mvo, 6, qh, qn);
          total += g;
          ++changes;
          ++moves_round;
          S.movesor++;
        }
      }
    }
    if (!ok || changes >= n || !E.verify || moves_round == 0) break;
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
  return ok ? total : -1;
}

// Shared scratch of the block version below.
struct LsShared {
  int64_t gain[32];
  int mv[32][8];
  int qh, qn, nlog, changes, moves_round, win, fail;
  int64_t total;
};

// The same search run by a block of W warps on one tour: each round, warp w
// evaluates the w-th queued node; entries are popped in queue order up to
// and including the first one whose evaluation found a move, which warp 0
// applies.  Nothing changes the tour between the confirmed evaluations, so
// the result equals popping one node at a time.  Must be called by every
// thread of the block.  Returns the gain, or -1 (capacity).
template <class Tour>
__device__ __forceinline__ int64_t ls_run_block(const LsEnv& E, Tour& T, const int32_t* init, int ninit,
                                                LsStats& S, LsShared& sh) {
  const int n = E.n, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int W = blockDim.x >> 5;
  for (int i = tid; i < ninit; i += blockDim.x) {
    const int x = init[i];
    E.queue[i] = x;
    E.flags[x] = 1;
  }
  if (tid == 0) {
    sh.qh = 0; sh.qn = ninit; sh.nlog = 0; sh.changes = 0; sh.moves_round = 0; sh.fail = 0;
    sh.total = 0;
  }
  __syncthreads();
  for (;;) {
    const int qh = sh.qh, qn = sh.qn;
    if (qn == 0 || sh.changes >= n || sh.fail) {
      if (sh.fail || sh.changes >= n || !E.verify || sh.moves_round == 0) break;
      const int nl = sh.nlog;  // verify round: queue again the nodes popped
      for (int i = tid; i < nl; i += blockDim.x) {
        const int x = E.logb[i];
        E.queue[i] = x;
        E.flags[x] = 1;
      }
      __syncthreads();
      if (tid == 0) {
        sh.qh = 0; sh.qn = nl; sh.nlog = 0; sh.moves_round = 0;
      }
      if (w == 0) S.verify++;
      __syncthreads();
      continue;
    }
    const int R = qn < W ? qn : W;
    const uint64_t t0 = (w == 0) ? global_ns() : 0;
    if (w < R) {
      int idx = qh + w;
      if (idx >= n) idx -= n;
      const int a = E.queue[idx];
      int mv2[4], mvo[7];
      int64_t g2, go;
      eval_dispatch(T, a, E.oropt != 0, g2, mv2, go, mvo);
      if (lane == 0) {
        if (g2 > 0) {
          sh.gain[w] = g2;
          for (int t = 0; t < 4; ++t) sh.mv[w][t] = mv2[t];
          sh.mv[w][7] = 0;
        } else {
          sh.gain[w] = go > 0 ? go : 0;
          for (int t = 0; t < 7; ++t) sh.mv[w][t] = mvo[t];
          sh.mv[w][7] = 1;
        }
      }
    }
    __syncthreads();
    if (w == 0) {
      const uint64_t t1 = global_ns();
      S.t_eval += (int64_t)(t1 - t0);
      const unsigned bal = __ballot_sync(kFull, lane < R && sh.gain[lane] > 0);
      const int first = bal ? __ffs(bal) - 1 : R;
      const int cnt = bal ? first + 1 : R;  // queue entries popped this round
      int a = -1;
      bool first_pop = false;
      if (lane < cnt) {
        int idx = qh + lane;
        if (idx >= n) idx -= n;
        a = E.queue[idx];
        const uint8_t f = E.flags[a];
        first_pop = !(f & 2);
        E.flags[a] = (uint8_t)((f & ~1) | 2);
      }
      const unsigned fb = __ballot_sync(kFull, first_pop);
      if (first_pop) E.logb[sh.nlog + __popc(fb & ((1u << lane) - 1u))] = a;
      S.pops += cnt;
      __syncwarp();
      int qh2 = qh + cnt;
      if (qh2 >= n) qh2 -= n;
      int qn2 = qn - cnt;
      const uint64_t t2 = global_ns();
      S.t_confirm += (int64_t)(t2 - t1);
      if (bal) {  // apply the first move found, queue its endpoints
        int mv[8];
        for (int t = 0; t < 8; ++t) mv[t] = sh.mv[first][t];
        bool ok;
        if (mv[7] == 0) {
          ok = T.flip(mv[1], mv[2], S);
          S.moves2++;
        } else {
          ok = apply_or_call(T, mv, S);
          S.movesor++;
        }
        const uint64_t t3 = global_ns();
        S.t_flip += (int64_t)(t3 - t2);
        if (!ok) {
          if (lane == 0) sh.fail = 1;
        } else {
          qn2 = ls_push_warp(E, mv, mv[7] == 0 ? 4 : 6, qh2, qn2);
          if (lane == 0) {
            sh.total += sh.gain[first];
            sh.changes++;
            sh.moves_round++;
          }
        }
        __syncwarp();
        S.t_push += (int64_t)(global_ns() - t3);
      }
      if (lane == 0) {
        sh.nlog += __popc(fb);
        sh.qh = qh2;
        sh.qn = qn2;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  __syncthreads();
  const int qh = sh.qh, qn = sh.qn, nl = sh.nlog;
  for (int t = tid; t < qn; t += blockDim.x) {
    int i = qh + t;
    if (i >= n) i -= n;
    E.flags[E.queue[i]] = 0;
  }
  for (int i = tid; i < nl; i += blockDim.x) E.flags[E.logb[i]] = 0;
  __syncthreads();
  return sh.fail ? -1 : sh.total;
}

}  // namespace faco
