// seg.cuh -- an ant's tour held as runs of the source solution.
//
// After focused construction (Alg 2) an ant's tour is a concatenation of a
// few runs of the source solution; the local search (Alg 3) then changes
// the tour by reversals.  Instead of materialising route[]/pos[] arrays of
// n entries per ant, a warp keeps the tour as a table of segments in shared
// memory: segment id covers source positions [lo, lo+len) and ant positions
// [off, off+len), traversed upwards (rev = 0) or downwards (rev = 1) in the
// source.  Nodes are named by their source position.  Two orders index the
// table: A (ids by ant position, A[0] at position 0) and B (ids by lo).
// Segments never straddle ant position 0 nor the source's end, so every
// lookup is a binary search; the inverse orders (rankA, rankB: the rank of
// each id) make every lookup by id direct.  A reversal of ant positions
// i..j splits the segments at i and j+1, reverses that part of A and flips
// each segment's direction -- exactly the array reversal, entry for entry,
// in O(segments).
// Neighbouring segments that continue each other are merged back.  When the
// table is full the operation reports failure and the caller redoes the ant
// with explicit arrays (same result, more memory traffic).
#pragma once

#include "common.cuh"
#include "ls.cuh"

namespace faco {

struct Seg {
  int32_t lo, len, off, rev;
};

// Shared-memory table of one warp.
struct SegTab {
  Seg* sg;           // [cap] segments by id (ids 0..S-1)
  uint16_t* A;       // [cap] ids in ant order
  uint16_t* B;       // [cap] ids in source order
  int32_t* offA;     // [cap] sg[A[r]].off
  int32_t* loB;      // [cap] sg[B[r]].lo
  uint16_t* tmp;     // [2 * cap + 2] scratch
  uint16_t* rankA;   // [cap] rank in A of each id
  uint16_t* rankB;   // [cap] rank in B of each id
  int32_t* S;        // segment count (shared)
  int cap;
};

// bytes of shared memory per segment, and per table of `cap` segments
constexpr size_t kSegBytes = sizeof(Seg) + 6 * sizeof(uint16_t) + 2 * sizeof(int32_t);
__host__ __device__ constexpr size_t segtab_bytes(int cap) {
  return (size_t)cap * kSegBytes + 2 * sizeof(uint16_t) + 16;
}

__device__ __forceinline__ SegTab segtab_at(char* base, int cap) {
  SegTab T;
  T.sg = reinterpret_cast<Seg*>(base);
  char* p = base + (size_t)cap * sizeof(Seg);
  T.offA = reinterpret_cast<int32_t*>(p);
  p += (size_t)cap * sizeof(int32_t);
  T.loB = reinterpret_cast<int32_t*>(p);
  p += (size_t)cap * sizeof(int32_t);
  T.A = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * sizeof(uint16_t);
  T.B = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * sizeof(uint16_t);
  T.tmp = reinterpret_cast<uint16_t*>(p);
  p += (size_t)(2 * cap + 2) * sizeof(uint16_t);
  T.rankA = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * sizeof(uint16_t);
  T.rankB = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * sizeof(uint16_t);
  T.S = reinterpret_cast<int32_t*>((reinterpret_cast<uintptr_t>(p) + 3) & ~uintptr_t(3));
  T.cap = cap;
  return T;
}

// Table capacity once the visited bits in front of a table of `cap`
// segments are free (the local search does not need them): the same
// shared memory, whole multiples of 32 segments added.
__host__ __device__ constexpr int segtab_cap_ls(size_t vis_bytes, int cap) {
  return cap + (int)((vis_bytes / kSegBytes) & ~(size_t)31);
}

// Moves the table `from` (placed after the visited bits) to `to` (placed at
// the start of the same shared memory, larger capacity), with the whole
// block.  Every array lies lower in `to` than in `from`, by at least the
// room gained, so copying each array in increasing index order -- all of a
// chunk's reads before its writes -- never overwrites an entry not yet
// read.  The scratch array is not copied.
__device__ __forceinline__ void seg_relayout(const SegTab& from, const SegTab& to) {
  const int S = *from.S;
  const int t = threadIdx.x, T = blockDim.x;
  __syncthreads();
  for (int c = 0; c < S; c += T) {
    const int r = c + t;
    Seg v{0, 0, 0, 0};
    if (r < S) v = from.sg[r];
    __syncthreads();
    if (r < S) to.sg[r] = v;
    __syncthreads();
  }
  for (int c = 0; c < S; c += T) {
    const int r = c + t;
    int32_t a = 0, b = 0;
    if (r < S) {
      a = from.offA[r];
      b = from.loB[r];
    }
    __syncthreads();
    if (r < S) {
      to.offA[r] = a;
      to.loB[r] = b;
    }
    __syncthreads();
  }
  for (int c = 0; c < S; c += T) {
    const int r = c + t;
    uint16_t a = 0, b = 0, k = 0, kb = 0;
    if (r < S) {
      a = from.A[r];
      b = from.B[r];
      k = from.rankA[r];
      kb = from.rankB[r];
    }
    __syncthreads();
    if (r < S) {
      to.A[r] = a;
      to.B[r] = b;
      to.rankA[r] = k;
      to.rankB[r] = kb;
    }
    __syncthreads();
  }
  if (t == 0) *to.S = S;
  __syncthreads();
}

// Largest r in [0, S) with key[r] <= v (key ascending, key[0] <= v).
__device__ __forceinline__ int bsearch_le(const int32_t* key, int S, int v) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key[mid] <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The same search by a whole warp for one (warp-uniform) value: each level
// compares 32 keys spaced evenly over the remaining range and keeps the
// last one <= v, so a table of up to 1,024 keys takes two shared-memory
// round trips instead of ten dependent ones.  Every lane gets the rank.
__device__ __forceinline__ int bsearch_le_warp(const int32_t* key, int S, int v) {
  const int lane = lane_id();
  int lo = 0, len = S;  // the answer lies in [lo, lo + len); key[lo] <= v
  while (len > 1) {
    const int st = (len + 31) >> 5;
    const bool le = lane * st < len && key[lo + lane * st] <= v;
    const unsigned b = __ballot_sync(kFull, le);
    const int L = b ? 31 - __clz(b) : 0;
    lo += L * st;
    len = min(st, len - L * st);
  }
  return lo;
}

// Insert id (source start lo) at index r of B/loB, arrays of S entries;
// rankB follows (warp-collective).
__device__ __forceinline__ void ins_B(const SegTab& T, int S, int r, int id, int32_t lo) {
  const int lane = lane_id();
  for (int e = S - 1; e >= r; e -= 32) {
    const int idx = e - lane;
    uint16_t v = 0;
    int32_t k = 0;
    if (idx >= r) {
      v = T.B[idx];
      k = T.loB[idx];
    }
    __syncwarp();
    if (idx >= r) {
      T.B[idx + 1] = v;
      T.loB[idx + 1] = k;
      T.rankB[v] = (uint16_t)(idx + 1);
    }
    __syncwarp();
  }
  if (lane == 0) {
    T.B[r] = (uint16_t)id;
    T.loB[r] = lo;
    T.rankB[id] = (uint16_t)r;
  }
  __syncwarp();
}

// Rebuild the search keys and the inverse orders from the orders
// (warp-collective).
__device__ __forceinline__ void segtab_keys(const SegTab& T) {
  const int S = *T.S;
  for (int r = lane_id(); r < S; r += 32) {
    const int ida = T.A[r], idb = T.B[r];
    T.offA[r] = T.sg[ida].off;
    T.rankA[ida] = (uint16_t)r;
    T.loB[r] = T.sg[idb].lo;
    T.rankB[idb] = (uint16_t)r;
  }
  __syncwarp();
}

// The two inserts of a split in one pass: (idA, keyA) at index rA of
// A/offA and (idB, keyB) at index rB of B/loB, both arrays of S entries;
// rankA and rankB follow (warp-collective).
__device__ __forceinline__ void ins2_both(const SegTab& T, int S, int rA, int idA, int32_t keyA, int rB, int idB,
                                          int32_t keyB) {
  const int lane = lane_id();
  const int lo = rA < rB ? rA : rB;
  for (int e = S - 1; e >= lo; e -= 32) {
    const int idx = e - lane;
    uint16_t va = 0, vb = 0;
    int32_t ka = 0, kb = 0;
    if (idx >= rA) {
      va = T.A[idx];
      ka = T.offA[idx];
    }
    if (idx >= rB) {
      vb = T.B[idx];
      kb = T.loB[idx];
    }
    __syncwarp();
    if (idx >= rA) {
      T.A[idx + 1] = va;
      T.offA[idx + 1] = ka;
      T.rankA[va] = (uint16_t)(idx + 1);
    }
    if (idx >= rB) {
      T.B[idx + 1] = vb;
      T.loB[idx + 1] = kb;
      T.rankB[vb] = (uint16_t)(idx + 1);
    }
    __syncwarp();
  }
  if (lane == 0) {
    T.A[rA] = (uint16_t)idA;
    T.offA[rA] = keyA;
    T.rankA[idA] = (uint16_t)rA;
    T.B[rB] = (uint16_t)idB;
    T.loB[rB] = keyB;
    T.rankB[idB] = (uint16_t)rB;
  }
  __syncwarp();
}

// The two removals of a merge in one pass: index rA of A/offA and index rB
// of B/loB, arrays of S entries; rankA and rankB follow (warp-collective).
__device__ __forceinline__ void del_both(const SegTab& T, int S, int rA, int rB) {
  const int lane = lane_id();
  for (int e = (rA < rB ? rA : rB) + 1; e < S; e += 32) {
    const int idx = e + lane;
    const bool da = idx > rA && idx < S, db = idx > rB && idx < S;
    uint16_t va = 0, vb = 0;
    int32_t ka = 0, kb = 0;
    if (da) {
      va = T.A[idx];
      ka = T.offA[idx];
    }
    if (db) {
      vb = T.B[idx];
      kb = T.loB[idx];
    }
    __syncwarp();
    if (da) {
      T.A[idx - 1] = va;
      T.offA[idx - 1] = ka;
      T.rankA[va] = (uint16_t)(idx - 1);
    }
    if (db) {
      T.B[idx - 1] = vb;
      T.loB[idx - 1] = kb;
      T.rankB[vb] = (uint16_t)(idx - 1);
    }
    __syncwarp();
  }
}

// Ensure a segment starts at ant position t (0 < t < n), given the id of
// the segment that holds t.  Keys and ranks are current on entry and on
// exit.  Returns the id of the segment that starts at t (id itself when t
// is already its first position, else the new id, which takes the part
// from t on), or -1 when the table is full.
static __device__ __noinline__ int seg_split(const SegTab& T, int t, int id) {
  const int S = *T.S;
  const Seg s = T.sg[id];
  if (s.off == t) return id;
  if (S >= T.cap) return -1;
  const int d = t - s.off;
  const int nid = S;
  const int r = T.rankA[id], rb = T.rankB[id];
  __syncwarp();
  if (lane_id() == 0) {
    if (!s.rev) {
      T.sg[nid] = Seg{s.lo + d, s.len - d, t, 0};
      T.sg[id].len = d;
    } else {
      T.sg[nid] = Seg{s.lo, s.len - d, t, 1};
      T.sg[id].lo = s.lo + s.len - d;
      T.sg[id].len = d;
    }
  }
  __syncwarp();
  if (!s.rev) {
    ins2_both(T, S, r + 1, nid, t, rb + 1, nid, s.lo + d);
  } else {  // nid keeps the low end: it goes before id, whose lo moved up
    ins2_both(T, S, r + 1, nid, t, rb, nid, s.lo);
    if (lane_id() == 0) T.loB[rb + 1] = s.lo + s.len - d;
  }
  if (lane_id() == 0) *T.S = S + 1;
  __syncwarp();
  return nid;
}

// Merge ant ranks r and r+1 if the second continues the first in the
// source (r + 1 > 0, so never across ant position 0).  Keys and ranks stay
// current.
static __device__ __noinline__ void seg_merge_at(const SegTab& T, int r) {
  const int S = *T.S;
  if (r < 0 || r + 1 >= S) return;
  const int ia = T.A[r], ib = T.A[r + 1];
  const Seg a = T.sg[ia], b = T.sg[ib];
  if (!(a.rev == b.rev && (a.rev ? (b.lo + b.len == a.lo) : (a.lo + a.len == b.lo)))) return;
  const int rbb = T.rankB[ib];
  __syncwarp();
  if (lane_id() == 0) {
    T.sg[ia].len = a.len + b.len;
    if (a.rev) T.sg[ia].lo = b.lo;
  }
  __syncwarp();
  del_both(T, S, r + 1, rbb);
  if (a.rev && lane_id() == 0) T.loB[rbb] = b.lo;  // a slid down to b's rank and took its lo
  __syncwarp();
  // free id ib: move the last id into its slot
  const int last = S - 1;
  if (ib != last) {
    const Seg sl = T.sg[last];
    const int ra = T.rankA[last], rl = T.rankB[last];
    __syncwarp();
    if (lane_id() == 0) {
      T.sg[ib] = sl;
      T.A[ra] = (uint16_t)ib;
      T.rankA[ib] = (uint16_t)ra;
      T.B[rl] = (uint16_t)ib;
      T.rankB[ib] = (uint16_t)rl;
    }
  }
  if (lane_id() == 0) *T.S = S - 1;
  __syncwarp();
}

// Tour over the segment table (nodes = source positions).
struct SegTour {
  int n, k, kw;
  SegTab T;
  const int2* xy;       // coordinates by source position
  const int32_t* cn;    // candidate source positions by source position [n][kw]
  const int32_t* cd;    // their EUC_2D costs, same layout

  // Lookups stay in [0, n) even if the table were inconsistent (which would
  // be a library bug: it is flagged and shows up as a wrong tour, not as an
  // out-of-range access).
  __device__ __forceinline__ int pos_of(int q) const {
    const int r = bsearch_le(T.loB, *T.S, q);
    const Seg s = T.sg[T.B[r]];
    const int t = s.off + (s.rev ? s.lo + s.len - 1 - q : q - s.lo);
    return (unsigned)t < (unsigned)n ? t : 0;
  }
  // pos_of and succ for a warp-uniform argument (warp-collective)
  __device__ __forceinline__ int pos_of_w(int q) const {
    const int r = bsearch_le_warp(T.loB, *T.S, q);
    const Seg s = T.sg[T.B[r]];
    const int t = s.off + (s.rev ? s.lo + s.len - 1 - q : q - s.lo);
    return (unsigned)t < (unsigned)n ? t : 0;
  }
  __device__ __forceinline__ int succ_w(int q) const {
    int id = T.B[bsearch_le_warp(T.loB, *T.S, q)];
    return step_up(q, id);
  }
  // pos_of for two warp-uniform nodes, with the segments that hold them
  // (warp-collective): the two searches of B go level by level together,
  // so that their shared-memory round trips overlap.
  __device__ __forceinline__ void pos_id2_w(int q1, int q2, int& t1, int& id1, int& t2, int& id2) const {
    const int lane = lane_id(), S = *T.S;
    int lo1 = 0, len1 = S, lo2 = 0, len2 = S;
    while (len1 > 1 || len2 > 1) {
      const int st1 = (len1 + 31) >> 5, st2 = (len2 + 31) >> 5;
      const bool le1 = len1 > 1 && lane * st1 < len1 && T.loB[lo1 + lane * st1] <= q1;
      const bool le2 = len2 > 1 && lane * st2 < len2 && T.loB[lo2 + lane * st2] <= q2;
      const unsigned b1 = __ballot_sync(kFull, le1), b2 = __ballot_sync(kFull, le2);
      if (len1 > 1) {
        const int L = b1 ? 31 - __clz(b1) : 0;
        lo1 += L * st1;
        len1 = min(st1, len1 - L * st1);
      }
      if (len2 > 1) {
        const int L = b2 ? 31 - __clz(b2) : 0;
        lo2 += L * st2;
        len2 = min(st2, len2 - L * st2);
      }
    }
    id1 = T.B[lo1];
    id2 = T.B[lo2];
    const Seg s1 = T.sg[id1], s2 = T.sg[id2];
    t1 = s1.off + (s1.rev ? s1.lo + s1.len - 1 - q1 : q1 - s1.lo);
    t2 = s2.off + (s2.rev ? s2.lo + s2.len - 1 - q2 : q2 - s2.lo);
    if ((unsigned)t1 >= (unsigned)n) t1 = 0;
    if ((unsigned)t2 >= (unsigned)n) t2 = 0;
  }
  __device__ __forceinline__ int at(int t) const {
    const int r = bsearch_le(T.offA, *T.S, t);
    const Seg s = T.sg[T.A[r]];
    const int d = t - s.off;
    const int q = s.rev ? s.lo + s.len - 1 - d : s.lo + d;
    return (unsigned)q < (unsigned)n ? q : 0;
  }
  __device__ __forceinline__ int2 coord(int q) const { return xy[q]; }
  __device__ __forceinline__ int cand(int q, int s) const { return cn[(size_t)q * kw + s]; }
  __device__ __forceinline__ int cdist(int q, int s) const { return cd[(size_t)q * kw + s]; }

  // Segment id holding source position q.
  __device__ __forceinline__ int locate(int q) const { return T.B[bsearch_le(T.loB, *T.S, q)]; }
  // Next / previous node in ant order from q (in segment id); id follows.
  __device__ __forceinline__ int step_up(int q, int& id) const {
    const Seg s = T.sg[id];
    const int d = s.rev ? s.lo + s.len - 1 - q : q - s.lo;
    if (d < s.len - 1) return s.rev ? q - 1 : q + 1;
    int r = T.rankA[id] + 1;
    if (r == *T.S) r = 0;
    id = T.A[r];
    const Seg t = T.sg[id];
    return t.rev ? t.lo + t.len - 1 : t.lo;
  }
  __device__ __forceinline__ int step_dn(int q, int& id) const {
    const Seg s = T.sg[id];
    const int d = s.rev ? s.lo + s.len - 1 - q : q - s.lo;
    if (d > 0) return s.rev ? q + 1 : q - 1;
    int r = T.rankA[id] - 1;
    if (r < 0) r = *T.S - 1;
    id = T.A[r];
    const Seg t = T.sg[id];
    return t.rev ? t.lo : t.lo + t.len - 1;
  }
  __device__ __forceinline__ int succ(int q) const {
    int id = locate(q);
    return step_up(q, id);
  }
  __device__ __forceinline__ int pred(int q) const {
    int id = locate(q);
    return step_dn(q, id);
  }
  // succ(q) when up, else pred(q): one lookup whatever the direction
  __device__ __forceinline__ int adj(int q, bool up) const {
    const int id = locate(q);
    const Seg s = T.sg[id];
    const int d = s.rev ? s.lo + s.len - 1 - q : q - s.lo;  // q's offset in ant order
    if (up ? d < s.len - 1 : d > 0) return (up != (bool)s.rev) ? q + 1 : q - 1;
    int r = T.rankA[id] + (up ? 1 : -1);
    if (r == *T.S) r = 0;
    if (r < 0) r = *T.S - 1;
    const Seg t = T.sg[T.A[r]];
    // first node in ant order of the next segment, or last of the previous
    return (up == (bool)t.rev) ? t.lo + t.len - 1 : t.lo;
  }
  __device__ __forceinline__ void nbrs(int q, int& p, int& s) const {
    const int id = locate(q);
    int i1 = id, i2 = id;
    p = step_dn(q, i1);
    s = step_up(q, i2);
  }
  __device__ __forceinline__ void walk(int a, int& p, int& s1, int& s2, int& s3) const {
    const int id = locate(a);
    int i1 = id, i2 = id;
    p = step_dn(a, i1);
    s1 = step_up(a, i2);
    s2 = step_up(s1, i2);
    s3 = step_up(s2, i2);
  }

  // Reverse the forward span x..y, or its complement when longer than n/2
  // (the array rule, entry for entry).  false: the table is full.
  __device__ __noinline__ bool flip(int x, int y, LsStats& St) {
    const int lane = lane_id();
    int px, hx, py, hy;
    pos_id2_w(x, y, px, hx, py, hy);
    // the position after y and the segment that holds it: y's own, unless
    // y ends it (then the next one in ant order)
    const int cy = (py + 1 == n) ? 0 : py + 1;
    int hcy = hy;
    if (cy != 0) {
      const Seg sy = T.sg[hy];
      if (cy >= sy.off + sy.len) hcy = T.A[T.rankA[hy] + 1];
    }
    __syncwarp();  // every lane has read the table before any lane rewrites a segment
    // the span i..j and the segments holding its cuts i and j1 = j + 1
    // (positions 0 and n need no cut): x..y, or y+1..x-1
    int i = px, j = py, hi = hx, j1 = cy, hj = hcy;
    int L = j - i;
    if (L < 0) L += n;
    L += 1;
    if (2 * L > n) {
      i = cy;
      hi = hcy;
      j = (px == 0) ? n - 1 : px - 1;
      j1 = px;
      hj = hx;
      L = n - L;
    }
    if (L <= 1) {
      St.flip += L;
      return true;
    }
    // a reversal adds at most three segments (two cuts, one at position 0):
    // refuse before touching the table, which then still holds the tour
    if (*T.S + 3 > T.cap) return false;
    St.flip += L;
    int si = -1, sj = -1;  // the segments that start at i and at j1
    if (i != 0) {
      si = seg_split(T, i, hi);
      if (si < 0) return false;
      // both cuts in one segment: the part from i on now holds j1
      if (hj == hi && si != hi && j1 >= i) hj = si;
    }
    if (j1 != 0) {
      sj = seg_split(T, j1, hj);
      if (sj < 0) return false;
    }
    const int S = *T.S;
    const int ri = (i == 0) ? 0 : T.rankA[si];
    const int rj = (j1 == 0) ? S - 1 : T.rankA[sj] - 1;
    if (i <= j) {
      // contiguous ranks ri..rj: new off = i + j + 1 - off - len, direction
      // flips, and the ranks reverse.  Lane m takes the pair of ranks
      // (ri + m, rj - m) in one pass: the pairs, their ids and their
      // segments are disjoint, so no lane reads what another writes.
      const int c = rj - ri + 1, h = (c + 1) >> 1;
      for (int m = lane; m < h; m += 32) {
        const int ra = ri + m, rb = rj - m;
        const int ida = T.A[ra], idb = T.A[rb];
        const Seg sa = T.sg[ida], sb = T.sg[idb];
        const int offa = i + j + 1 - sa.off - sa.len, offb = i + j + 1 - sb.off - sb.len;
        T.sg[ida].off = offa;
        T.sg[ida].rev = sa.rev ^ 1;
        T.A[rb] = (uint16_t)ida;
        T.offA[rb] = offa;
        T.rankA[ida] = (uint16_t)rb;
        if (rb != ra) {
          T.sg[idb].off = offb;
          T.sg[idb].rev = sb.rev ^ 1;
          T.A[ra] = (uint16_t)idb;
          T.offA[ra] = offb;
          T.rankA[idb] = (uint16_t)ra;
        }
      }
      __syncwarp();
      seg_merge_at(T, rj);      // the span's right end and its old right neighbour
      seg_merge_at(T, ri - 1);  // its left neighbour and the span's new left end
      return true;
    } else {
      // the span wraps: ranks ri..S-1 then 0..rj; lay the reversed list
      // out from position i, cutting the segment that crosses position 0
      const int clo = rj + 1, chi = S - ri, c = clo + chi;
      // R[m] = A[rj - m] (m < clo), A[S - 1 - (m - clo)] (m >= clo)
      for (int m = lane; m < c; m += 32) T.tmp[m] = m < clo ? T.A[rj - m] : T.A[S - 1 - (m - clo)];
      __syncwarp();
      // new offsets: R laid out from position i (a prefix sum of the lengths,
      // 32 segments at a time), wrapped below n; the segment that crosses
      // position n (straddle) and how many start below n (nhi)
      int straddle = -1, cut = 0, nhi = 0, carry = 0;
      for (int m0 = 0; m0 < c; m0 += 32) {
        const int m = m0 + lane;
        int len = 0;
        if (m < c) len = T.sg[T.tmp[m]].len;
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const int at = i + carry + incl - len;  // first position of segment m
        if (m < c) {
          Seg& s = T.sg[T.tmp[m]];
          s.rev ^= 1;
          s.off = at >= n ? at - n : at;
        }
        const unsigned bs = __ballot_sync(kFull, m < c && at < n && at + len > n);
        if (bs) {
          const int l = __ffs(bs) - 1;
          straddle = m0 + l;
          cut = n - __shfl_sync(kFull, at, l);
        }
        nhi += __popc(__ballot_sync(kFull, m < c && at < n));
        carry += __shfl_sync(kFull, incl, 31);
      }
      __syncwarp();
      int S2 = S;
      int nid = -1;
      if (straddle >= 0) {
        if (S >= T.cap) return false;
        const int id = T.tmp[straddle];
        const Seg s = T.sg[id];
        nid = S;
        const int rb = T.rankB[id];
        __syncwarp();
        if (lane == 0) {
          // id keeps ant positions [s.off, n); nid takes [0, s.len - cut)
          if (!s.rev) {
            T.sg[nid] = Seg{s.lo + cut, s.len - cut, 0, 0};
            T.sg[id].len = cut;
          } else {
            T.sg[nid] = Seg{s.lo, s.len - cut, 0, 1};
            T.sg[id].lo = s.lo + s.len - cut;
            T.sg[id].len = cut;
          }
        }
        __syncwarp();
        if (!s.rev) {
          ins_B(T, S, rb + 1, nid, s.lo + cut);
        } else {  // nid keeps the low end: it goes before id, whose lo moved up
          ins_B(T, S, rb, nid, s.lo);
          if (lane == 0) T.loB[rb + 1] = s.lo + s.len - cut;
          __syncwarp();
        }
        S2 = S + 1;
      }
      // new A: [nid] + wrapped part of R + middle A[clo..ri) + unwrapped part of R
      // R is ordered by new position: the unwrapped part (offsets >= i) comes
      // first in R, the wrapped part after it.
      // nhi: R entries placed in [i, n), up to and including the straddler
      // assemble into the tail of tmp: tmp[c..c+S2)
      uint16_t* out = T.tmp + c;
      const int mid = ri - clo;
      const int head = (nid >= 0) ? 1 : 0;
      const int nlo = c - nhi;
      if (lane == 0 && nid >= 0) out[0] = (uint16_t)nid;
      for (int m = lane; m < nlo; m += 32) out[head + m] = T.tmp[nhi + m];
      for (int m = lane; m < mid; m += 32) out[head + nlo + m] = T.A[clo + m];
      for (int m = lane; m < nhi; m += 32) out[head + nlo + mid + m] = T.tmp[m];
      __syncwarp();
      for (int m = lane; m < S2; m += 32) {
        const int id = out[m];
        T.A[m] = (uint16_t)id;
        T.offA[m] = T.sg[id].off;
        T.rankA[id] = (uint16_t)m;
      }
      __syncwarp();
      if (lane == 0) *T.S = S2;
      __syncwarp();
      // Merges: reversing a run of segments keeps every pair inside it as
      // (un)mergeable as it was, and the table held no mergeable pair except
      // across position 0.  New pairs: the span's right end with the middle
      // (r1), the middle with the span's left end (r2), and the pair that
      // crossed position 0 (R[clo-1], R[clo]), now inside the span (r3; none
      // when the new cut at position 0 falls between them).  Highest rank
      // first, so that no merge moves a rank still to be merged.
      const int r1 = head + nlo - 1, r2 = r1 + mid;
      int r3 = -1;
      if (clo < nhi)
        r3 = r2 + clo;  // both in the part placed from position i
      else if (clo - 1 >= nhi)
        r3 = head + clo - 1 - nhi;  // both in the part wrapped below position i
      else if (head)
        r3 = 0;  // the cut split R[clo-1]: its tail (nid) precedes R[clo]
      if (r3 > r2) seg_merge_at(T, r3);
      seg_merge_at(T, r2);
      seg_merge_at(T, r1);
      if (r3 >= 0 && r3 < r1) seg_merge_at(T, r3);
      return true;
    }
  }
};

// A segment tour that moves to explicit arrays the first time its table is
// full: the table (which still holds the tour) is written out as
// route[t] = source position, pos = inverse, and the search goes on there
// with the same node names, queue and counters.
struct HybTour {
  int n, k;
  SegTour sg;
  ArrTour ar;       // over source positions (XYsrc, Csrc), used once *mode != 0
  int32_t* mode;    // shared flag: 0 = table, 1 = arrays

  __device__ __forceinline__ bool arrays() const { return *mode != 0; }
  __device__ __forceinline__ int pos_of(int x) const { return arrays() ? ar.pos_of(x) : sg.pos_of(x); }
  __device__ __forceinline__ int succ(int x) const { return arrays() ? ar.succ(x) : sg.succ(x); }
  __device__ __forceinline__ int succ_w(int x) const { return arrays() ? ar.succ(x) : sg.succ_w(x); }
  __device__ __forceinline__ int pred(int x) const { return arrays() ? ar.pred(x) : sg.pred(x); }
  __device__ __forceinline__ int adj(int x, bool up) const { return arrays() ? ar.adj(x, up) : sg.adj(x, up); }
  __device__ __forceinline__ void nbrs(int x, int& p, int& s) const {
    if (arrays())
      ar.nbrs(x, p, s);
    else
      sg.nbrs(x, p, s);
  }
  __device__ __forceinline__ void walk(int a, int& p, int& s1, int& s2, int& s3) const {
    if (arrays())
      ar.walk(a, p, s1, s2, s3);
    else
      sg.walk(a, p, s1, s2, s3);
  }
  __device__ __forceinline__ int2 coord(int x) const { return sg.coord(x); }
  __device__ __forceinline__ int cand(int x, int s) const { return sg.cand(x, s); }
  __device__ __forceinline__ int cdist(int x, int s) const { return sg.cdist(x, s); }

  __device__ __noinline__ void to_arrays() {
    const int S = *sg.T.S;
    for (int r = 0; r < S; ++r) {
      const Seg s = sg.T.sg[sg.T.A[r]];
      for (int d = lane_id(); d < s.len; d += 32) {
        const int q = s.rev ? s.lo + s.len - 1 - d : s.lo + d;
        ar.route[s.off + d] = q;
        ar.pos[q] = s.off + d;
      }
    }
    __syncwarp();
    if (lane_id() == 0) *mode = 1;
    __syncwarp();
  }

  static __device__ __noinline__ bool flip_arrays(ArrTour& A, int x, int y, LsStats& S) { return A.flip(x, y, S); }
  // warp-collective; never fails
  __device__ __forceinline__ bool flip(int x, int y, LsStats& S) {
    if (!arrays()) {
      if (sg.flip(x, y, S)) return true;
      to_arrays();
    }
    return flip_arrays(ar, x, y, S);
  }
};

// Evaluation on the representation the hybrid tour holds now (uniform
// across the block): the table path and the array path stay separate
// code, instead of a branch in every lookup.
// The array representation serves only ants whose table filled up: its
// evaluation and reversal stay out of line, so that the table's hot loop
// keeps its registers and a smaller code footprint (spill stores of the
// per-ant kernel 620 -> 220 bytes, the kernel 3-4 % faster).
static __device__ __noinline__ void eval_arrays(const ArrTour& T, int a, bool do_or, int64_t& g2, int* mv2,
                                                int64_t& go, int* mvo) {
  int m2[4], mo[7];
  eval_both(T, a, do_or, g2, m2, go, mo);
  for (int t = 0; t < 4; ++t) mv2[t] = m2[t];
  for (int t = 0; t < 7; ++t) mvo[t] = mo[t];
}
__device__ __forceinline__ void eval_dispatch(const HybTour& T, int a, bool do_or, int64_t& g2, int mv2[4],
                                              int64_t& go, int mvo[7]) {
  if (T.arrays())
    eval_arrays(T.ar, a, do_or, g2, mv2, go, mvo);
  else
    eval_both(T.sg, a, do_or, g2, mv2, go, mvo);
}

}  // namespace faco
