// A* paths of the pick-place base (Sec. IV-A: the base moves between
// locations along A* paths whose waypoints a PID controller tracks).
//
// The graph is the visibility graph of the plane minus the base footprints
// of the static bodies (their slabs with a horizontal normal) grown by
// base_infl along every slab normal.  Its corners (pushed 1 mm out) and their
// mutual visibility are built once per scene on the host (DevScene::corner,
// corner_vis); a query adds the start and the goal, whose edges are tested
// here in FP32 against the grown footprints -- a footprint holding the
// endpoint is tested ungrown, or skipped if even that holds it.  A* uses the
// straight-line distance to the goal as its heuristic and breaks ties by the
// lower node index (corners, then start, then goal).  Without a path the
// goal is the only waypoint.  One thread plans alone, in registers and local
// memory: at most CEM_MAX_CORNERS + 2 nodes.
#pragma once
#include "internal.h"

namespace cem {

constexpr int kMaxWaypoints = CEM_MAX_CORNERS + 2;

// is (x, y) strictly inside the footprint of body g grown by r?
__device__ __forceinline__ bool footprint_holds(const DevScene& s, int g, float r, float x, float y) {
  bool any = false;
  for (int i = 0; i < s.geom_nslab[g]; ++i) {
    const float* sl = s.slab[g][i];
    if (sl[2] != 0.0f) continue;
    any = true;
    const float lo = fabsf(sl[3]) < 1e6f ? sl[3] - r : sl[3];
    const float hi = fabsf(sl[4]) < 1e6f ? sl[4] + r : sl[4];
    const float p = sl[0] * x + sl[1] * y;
    if (!(p > lo && p < hi)) return false;
  }
  return any;
}

// does the open segment a -> b cross the interior of body g's footprint
// grown by r?  (the segment parameter clipped against every slab)
__device__ __forceinline__ bool footprint_crossed(const DevScene& s, int g, float r, float ax, float ay, float bx,
                                                  float by) {
  float t0 = 0.0f, t1 = 1.0f;
  bool any = false;
  for (int i = 0; i < s.geom_nslab[g]; ++i) {
    const float* sl = s.slab[g][i];
    if (sl[2] != 0.0f) continue;
    any = true;
    const float lo = (fabsf(sl[3]) < 1e6f ? sl[3] - r : sl[3]) + 1e-6f;
    const float hi = (fabsf(sl[4]) < 1e6f ? sl[4] + r : sl[4]) - 1e-6f;
    const float p0 = sl[0] * ax + sl[1] * ay, dp = sl[0] * (bx - ax) + sl[1] * (by - ay);
    if (fabsf(dp) < 1e-12f) {
      if (p0 <= lo || p0 >= hi) return false;
      continue;
    }
    const float ta = (lo - p0) / dp, tb = (hi - p0) / dp;
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
    if (t0 >= t1) return false;
  }
  return any && t0 < t1;
}

// is q visible from endpoint p?
__device__ __forceinline__ bool endpoint_sees(const DevScene& s, float px, float py, float qx, float qy) {
  for (int g = 0; g < s.n_geoms; ++g) {
    if (!(s.geom_flags[g] & 1)) continue;
    float r = s.base_infl;
    if (footprint_holds(s, g, r, px, py)) {
      r = 0.0f;
      if (footprint_holds(s, g, 0.0f, px, py)) continue;
    }
    if (footprint_crossed(s, g, r, px, py, qx, qy)) return false;
  }
  return true;
}

// A* from (sx, sy) to (gx, gy) given the corners each endpoint sees;
// writes the waypoints (wx, wy), ending with the goal, returns their number
static __device__ __noinline__ int astar_base_path(const DevScene& s, float sx, float sy, float gx, float gy,
                                                   uint64_t sees_s, uint64_t sees_g, float* wx, float* wy) {
  const int C = s.n_corners, S = C, Gn = C + 1, V = C + 2;
  const bool direct = endpoint_sees(s, sx, sy, gx, gy) && endpoint_sees(s, gx, gy, sx, sy);
  float g[kMaxWaypoints], h[kMaxWaypoints];  // cost so far, straight-line distance to the goal
  for (int i = 0; i < C; ++i)
    h[i] = sqrtf((s.corner[i][0] - gx) * (s.corner[i][0] - gx) + (s.corner[i][1] - gy) * (s.corner[i][1] - gy));
  h[S] = sqrtf((sx - gx) * (sx - gx) + (sy - gy) * (sy - gy));
  h[Gn] = 0.0f;
  int8_t parent[kMaxWaypoints];
  for (int i = 0; i < V; ++i) {
    g[i] = INFINITY;
    parent[i] = -1;
  }
  uint64_t open = 1ull << S, closed = 0;
  g[S] = 0.0f;
  bool found = false;
  for (;;) {
    int u = -1;
    float fu = INFINITY;
    for (uint64_t m = open; m; m &= m - 1ull) {
      const int i = __ffsll((long long)m) - 1;
      const float f = g[i] + h[i];
      if (f < fu) {
        fu = f;
        u = i;
      }
    }
    if (u < 0) break;
    if (u == Gn) {
      found = true;
      break;
    }
    open &= ~(1ull << u);
    closed |= 1ull << u;
    const float xu = u < C ? s.corner[u][0] : sx, yu = u < C ? s.corner[u][1] : sy;
    // neighbours of u: corners it sees, and the goal
    uint64_t nb = u < C ? s.corner_vis[u] : sees_s;
    const bool to_goal = u < C ? ((sees_g >> u) & 1ull) != 0 : direct;
    if (to_goal) nb |= 1ull << Gn;
    nb &= ~closed;
    for (uint64_t m = nb; m; m &= m - 1ull) {
      const int v = __ffsll((long long)m) - 1;
      const float xv = v < C ? s.corner[v][0] : gx, yv = v < C ? s.corner[v][1] : gy;
      const float c = g[u] + sqrtf((xv - xu) * (xv - xu) + (yv - yu) * (yv - yu));
      if (c < g[v]) {
        g[v] = c;
        parent[v] = (int8_t)u;
        open |= 1ull << v;
      }
    }
  }
  if (!found) {
    wx[0] = gx;
    wy[0] = gy;
    return 1;
  }
  int n = 0;
  for (int v = Gn; v != S; v = parent[v]) ++n;
  int k = n;
  for (int v = Gn; v != S; v = parent[v]) {
    --k;
    wx[k] = v < C ? s.corner[v][0] : gx;
    wy[k] = v < C ? s.corner[v][1] : gy;
  }
  return n;
}

}  // namespace cem

namespace cem {

// is corner i visible from endpoint (px, py)?  One compiled copy, so the
// solo and the warp-cooperative queries decide every edge identically.
static __device__ __noinline__ bool sees_corner(const DevScene& s, float px, float py, int i) {
  return endpoint_sees(s, px, py, s.corner[i][0], s.corner[i][1]);
}

// corners visible from (px, py), tested by one thread
__device__ __forceinline__ uint64_t corners_seen(const DevScene& s, float px, float py) {
  uint64_t m = 0;
  for (int i = 0; i < s.n_corners; ++i)
    if (sees_corner(s, px, py, i)) m |= 1ull << i;
  return m;
}

// the corner masks of lane `owner`'s endpoints, computed by all `lanes`
// (each active lane takes every nact-th corner) and OR-reduced
__device__ __forceinline__ void corners_seen_warp(const DevScene& s, unsigned lanes, float sx, float sy, float gx,
                                                  float gy, uint64_t& ms, uint64_t& mg) {
  const int lane = threadIdx.x & 31;
  const int rank = __popc(lanes & ((1u << lane) - 1u)), nact = __popc(lanes);
  uint32_t s_lo = 0, s_hi = 0, g_lo = 0, g_hi = 0;
  for (int i = rank; i < s.n_corners; i += nact) {
    const uint32_t bit = 1u << (i & 31);
    if (sees_corner(s, sx, sy, i)) {
      if (i < 32) s_lo |= bit;
      else s_hi |= bit;
    }
    if (sees_corner(s, gx, gy, i)) {
      if (i < 32) g_lo |= bit;
      else g_hi |= bit;
    }
  }
  s_lo = __reduce_or_sync(lanes, s_lo);
  s_hi = __reduce_or_sync(lanes, s_hi);
  g_lo = __reduce_or_sync(lanes, g_lo);
  g_hi = __reduce_or_sync(lanes, g_hi);
  ms = (uint64_t)s_lo | ((uint64_t)s_hi << 32);
  mg = (uint64_t)g_lo | ((uint64_t)g_hi << 32);
}

// the whole path query by one thread
static __device__ __noinline__ int plan_base_path(const DevScene& s, float sx, float sy, float gx, float gy, float* wx,
                                                  float* wy) {
  return astar_base_path(s, sx, sy, gx, gy, corners_seen(s, sx, sy), corners_seen(s, gx, gy), wx, wy);
}

}  // namespace cem
