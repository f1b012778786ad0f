// nearest.cuh -- the nearest unvisited node, the last fallback of the
// construction step (Sec. 4.3: when the candidate and backup lists are
// exhausted, the node with the highest heuristic value, i.e. the shortest
// edge).  Exact arg-min of (squared distance, node id) over the unvisited
// nodes, found by scanning rings of grid cells around u until the best key
// is strictly below the squared distance to anything outside the scanned
// block (warp-cooperative: one lane per cell of a ring).
#pragma once

#include <climits>

#include "common.cuh"

namespace faco {

// Returns the node, or -1 when `max_rings` rings did not settle it (the
// caller then scans everything); `handle` receives the chosen record's x
// field.  recs[cstart[c] .. cstart[c+1]) are the records (x = handle,
// (y, z) = coordinates, w = node id) of cell c; visited(rec) tells whether
// the record's node is visited.  The points of up to 32 cells of a ring
// are spread over the lanes (a warp prefix sum over the cell sizes), so a
// dense cell does not serialise one lane.
template <class Visited>
__device__ __forceinline__ int ring_nearest(const int4* recs, const Grid& g, const int32_t* cstart, int2 xu,
                                            int max_rings, Visited visited, int& handle) {
  const int lane = lane_id();
  const int cx = (xu.x - g.minx) / g.cs, cy = (xu.y - g.miny) / g.cs;
  uint64_t bk = ~0ull;
  int32_t bi = INT_MAX;
  int bh = -1;
  for (int r = 0; r <= max_rings; ++r) {
    const int cnt = r == 0 ? 1 : 8 * r;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const int c = c0 + lane;
      int st = 0, len = 0;
      if (c < cnt) {
        int dx = 0, dy = 0;
        if (r > 0) {
          if (c <= 2 * r) {
            dx = c - r;
            dy = -r;
          } else if (c <= 4 * r + 1) {
            dx = c - (3 * r + 1);
            dy = r;
          } else if (c <= 6 * r) {
            dx = -r;
            dy = c - (5 * r + 1);
          } else {
            dx = r;
            dy = c - 7 * r;
          }
        }
        const int x = cx + dx, y = cy + dy;
        if (x >= 0 && x < g.gx && y >= 0 && y < g.gy) {
          const int cell = y * g.gx + x;
          st = cstart[cell];
          len = cstart[cell + 1] - st;
        }
      }
      int incl = len;  // inclusive prefix sum of the cell sizes over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      const int excl_st = st - (incl - len);  // record index = excl_st(owner) + t
      // two points per lane in flight: the record loads of a step do not
      // wait for each other
      constexpr int U = 2;
      for (int t0 = 0; t0 < total; t0 += 32 * U) {
        int4 P[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int t = t0 + 32 * u + lane;
          // owner lane of point t: the first lane whose inclusive sum exceeds t
          int o = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1)
            if (__shfl_sync(kFull, incl, o + step - 1) <= t) o += step;
          const int base = __shfl_sync(kFull, excl_st, o);
          P[u] = t < total ? recs[base + t] : make_int4(-1, 0, 0, INT_MAX);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (P[u].x >= 0 && !visited(P[u])) {
            const uint64_t m = sqdist(xu, make_int2(P[u].y, P[u].z));
            if (m < bk || (m == bk && P[u].w < bi)) {
              bk = m;
              bi = P[u].w;
              bh = P[u].x;
            }
          }
        }
      }
    }
    uint64_t wk = bk;
    int32_t wi = bi;
    warp_min_key(wk, wi);
    const bool lin = cx - r <= 0, rin = cx + r >= g.gx - 1, din = cy - r <= 0, uin = cy + r >= g.gy - 1;
    bool done = lin && rin && din && uin;
    if (!done && wi != INT_MAX) {
      int64_t dmin = INT64_MAX;
      if (!lin) dmin = min(dmin, (int64_t)xu.x - ((int64_t)g.minx + (int64_t)(cx - r) * g.cs) + 1);
      if (!rin) dmin = min(dmin, ((int64_t)g.minx + (int64_t)(cx + r + 1) * g.cs) - xu.x);
      if (!din) dmin = min(dmin, (int64_t)xu.y - ((int64_t)g.miny + (int64_t)(cy - r) * g.cs) + 1);
      if (!uin) dmin = min(dmin, ((int64_t)g.miny + (int64_t)(cy + r + 1) * g.cs) - xu.y);
      done = wk < (uint64_t)(dmin * dmin);
    }
    if (done) {
      if (wi == INT_MAX) return -1;
      const unsigned own = __ballot_sync(kFull, bi == wi && bk == wk);
      handle = __shfl_sync(kFull, bh, __ffs(own) - 1);
      return wi;
    }
  }
  return -1;
}

}  // namespace faco
