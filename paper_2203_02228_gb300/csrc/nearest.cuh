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
// caller then scans everything).  visited(v) tells whether node v is
// visited.
template <class Visited>
__device__ __forceinline__ int ring_nearest(const int2* xy, const Grid& g, const int32_t* cstart,
                                            const int32_t* cpts, int2 xu, int max_rings,
                                            Visited visited) {
  const int lane = lane_id();
  const int cx = (xu.x - g.minx) / g.cs, cy = (xu.y - g.miny) / g.cs;
  uint64_t bk = ~0ull;
  int32_t bi = INT_MAX;
  for (int r = 0; r <= max_rings; ++r) {
    const int cnt = r == 0 ? 1 : 8 * r;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const int c = c0 + lane;
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
          const int e = cstart[cell + 1];
          for (int j = cstart[cell]; j < e; ++j) {
            const int v = cpts[j];
            if (visited(v)) continue;
            const uint64_t m = sqdist(xu, xy[v]);
            if (m < bk || (m == bk && v < bi)) {
              bk = m;
              bi = v;
            }
          }
        }
      }
    }
    uint64_t wk = bk;
    int32_t wi = bi;
    warp_min_key(wk, wi);
    const bool lin = cx - r <= 0, rin = cx + r >= g.gx - 1, din = cy - r <= 0, uin = cy + r >= g.gy - 1;
    if (lin && rin && din && uin) return wi == INT_MAX ? -1 : wi;
    if (wi != INT_MAX) {
      int64_t dmin = INT64_MAX;
      if (!lin) dmin = min(dmin, (int64_t)xu.x - ((int64_t)g.minx + (int64_t)(cx - r) * g.cs) + 1);
      if (!rin) dmin = min(dmin, ((int64_t)g.minx + (int64_t)(cx + r + 1) * g.cs) - xu.x);
      if (!din) dmin = min(dmin, (int64_t)xu.y - ((int64_t)g.miny + (int64_t)(cy - r) * g.cs) + 1);
      if (!uin) dmin = min(dmin, ((int64_t)g.miny + (int64_t)(cy + r + 1) * g.cs) - xu.y);
      if (wk < (uint64_t)(dmin * dmin)) return wi;
    }
  }
  return -1;
}

}  // namespace faco
