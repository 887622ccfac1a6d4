// Oracle: base path planning for moveTo in pick-place scenes (Sec. IV-A: A*
// computes collision-free paths for the mobile base, a PID controller tracks
// the waypoints).  FP64, plain loops.  Test infrastructure only.
//
// Readings (the paper gives no planner detail beyond "A*" and "waypoints"):
//  * the configuration space of the base is the plane minus each static
//    body's footprint (its slabs with a horizontal normal) grown by the
//    base's half-diagonal r along every slab normal;
//  * A* (Hart, Nilsson, Raphael 1968) runs on the visibility graph of that
//    space: the corners of the grown footprints (pushed 1 mm outwards, kept
//    when outside every grown footprint), the start and the goal; an edge
//    exists when the open segment enters no grown footprint; the heuristic
//    is the straight-line distance to the goal (admissible, consistent), ties
//    go to the lower node index (corners in geometry and slab order, then
//    the start, then the goal);
//  * a footprint that contains the start (or goal) is used ungrown for the
//    edges of that endpoint, and ignored if even its ungrown form contains
//    it (a base already pressed against a table must still be able to leave);
//  * no path: the goal itself is the only waypoint.
#include "oracle.h"

#include <cmath>
#include <cstring>

#include "plan2d.h"

namespace {

constexpr double kPush = 1e-3;   // corner offset out of its footprint (m)
constexpr double kMargin = 1e-9; // interior tolerance of the segment test

bool finite_bound(double v) { return std::fabs(v) < 1e6; }

}  // namespace

// Footprints of the static bodies the base collides with, grown by r and
// ungrown.
void base_footprints(const or_scene& s, double r, BaseGraph& G) {
  G.n_obs = 0;
  for (int gi = 0; gi < s.n_geoms; ++gi) {
    if (!s.geom_base[gi]) continue;
    Footprint f{}, f0{};
    for (int i = 0; i < s.geom_nslab[gi]; ++i) {
      const double* sl = s.slab[gi][i];
      if (sl[2] != 0.0) continue;  // not a wall of the footprint
      f.nx[f.n] = f0.nx[f0.n] = sl[0];
      f.ny[f.n] = f0.ny[f0.n] = sl[1];
      f0.lo[f0.n] = sl[3];
      f0.hi[f0.n] = sl[4];
      f.lo[f.n] = finite_bound(sl[3]) ? sl[3] - r : sl[3];
      f.hi[f.n] = finite_bound(sl[4]) ? sl[4] + r : sl[4];
      ++f.n;
      ++f0.n;
    }
    if (f.n == 0) continue;
    G.grown[G.n_obs] = f;
    G.bare[G.n_obs] = f0;
    ++G.n_obs;
  }
}

bool footprint_contains(const Footprint& f, double x, double y) {
  for (int i = 0; i < f.n; ++i) {
    const double p = f.nx[i] * x + f.ny[i] * y;
    if (!(p > f.lo[i] && p < f.hi[i])) return false;
  }
  return true;
}

// Does the open segment a -> b pass through the footprint's interior?
// (Liang-Barsky clipping of the parameter interval against every slab.)
bool segment_enters(const Footprint& f, double ax, double ay, double bx, double by) {
  double t0 = 0.0, t1 = 1.0;
  for (int i = 0; i < f.n; ++i) {
    const double s0 = f.nx[i] * ax + f.ny[i] * ay;
    const double d = f.nx[i] * (bx - ax) + f.ny[i] * (by - ay);
    const double lo = f.lo[i] + kMargin, hi = f.hi[i] - kMargin;
    if (std::fabs(d) < 1e-15) {
      if (!(s0 > lo && s0 < hi)) return false;
      continue;
    }
    double ta = (lo - s0) / d, tb = (hi - s0) / d;
    if (ta > tb) {
      const double t = ta;
      ta = tb;
      tb = t;
    }
    if (ta > t0) t0 = ta;
    if (tb < t1) t1 = tb;
    if (t0 >= t1) return false;
  }
  return t0 < t1;
}

void base_graph(const or_scene& s, BaseGraph& G) {
  std::memset(&G, 0, sizeof(G));
  const double r = s.base_infl;
  base_footprints(s, r, G);
  // corners: intersections of boundary lines of two different slabs of one
  // footprint that satisfy the footprint's other slabs
  for (int k = 0; k < G.n_obs; ++k) {
    const Footprint& f = G.grown[k];
    for (int i = 0; i < f.n; ++i)
      for (int j = i + 1; j < f.n; ++j)
        for (int si = 0; si < 2; ++si)
          for (int sj = 0; sj < 2; ++sj) {
            const double ci = si ? f.hi[i] : f.lo[i], cj = sj ? f.hi[j] : f.lo[j];
            if (!finite_bound(ci) || !finite_bound(cj)) continue;
            const double det = f.nx[i] * f.ny[j] - f.ny[i] * f.nx[j];
            if (std::fabs(det) < 1e-12) continue;
            double x = (ci * f.ny[j] - cj * f.ny[i]) / det;
            double y = (f.nx[i] * cj - f.nx[j] * ci) / det;
            bool on = true;
            for (int m = 0; m < f.n && on; ++m) {
              if (m == i || m == j) continue;
              const double p = f.nx[m] * x + f.ny[m] * y;
              on = p >= f.lo[m] - 1e-9 && p <= f.hi[m] + 1e-9;
            }
            if (!on) continue;
            // push out along the sum of the two outward normals
            double ox = (si ? f.nx[i] : -f.nx[i]) + (sj ? f.nx[j] : -f.nx[j]);
            double oy = (si ? f.ny[i] : -f.ny[i]) + (sj ? f.ny[j] : -f.ny[j]);
            const double on2 = std::sqrt(ox * ox + oy * oy);
            x += kPush * ox / on2;
            y += kPush * oy / on2;
            bool free = true;
            for (int q = 0; q < G.n_obs && free; ++q) free = !footprint_contains(G.grown[q], x, y);
            if (!free || G.nc >= OR_MAX_CORNERS) continue;
            G.cx[G.nc] = x;
            G.cy[G.nc] = y;
            ++G.nc;
          }
  }
  for (int a = 0; a < G.nc; ++a)
    for (int b = a + 1; b < G.nc; ++b) {
      bool vis = true;
      for (int q = 0; q < G.n_obs && vis; ++q) vis = !segment_enters(G.grown[q], G.cx[a], G.cy[a], G.cx[b], G.cy[b]);
      if (vis) {
        G.vis[a] |= 1ull << b;
        G.vis[b] |= 1ull << a;
      }
    }
}

// Visible from endpoint (px, py) to (qx, qy)?  Footprints that contain the
// endpoint are taken ungrown, or skipped if that contains it too.
static bool endpoint_sees(const BaseGraph& G, double px, double py, double qx, double qy) {
  for (int k = 0; k < G.n_obs; ++k) {
    const Footprint* f = &G.grown[k];
    if (footprint_contains(*f, px, py)) {
      f = &G.bare[k];
      if (footprint_contains(*f, px, py)) continue;
    }
    if (segment_enters(*f, px, py, qx, qy)) return false;
  }
  return true;
}

int plan_path(const BaseGraph& G, double sx, double sy, double gx, double gy, double* wx, double* wy, int cap) {
  const int C = G.nc, S = C, Gn = C + 1, V = C + 2;
  double X[OR_MAX_CORNERS + 2], Y[OR_MAX_CORNERS + 2];
  for (int i = 0; i < C; ++i) {
    X[i] = G.cx[i];
    Y[i] = G.cy[i];
  }
  X[S] = sx;
  Y[S] = sy;
  X[Gn] = gx;
  Y[Gn] = gy;
  // visibility of the start and the goal (an edge from the start is tested
  // from the start's side, an edge to the goal from the goal's side)
  bool sv[OR_MAX_CORNERS + 2], gv[OR_MAX_CORNERS + 2];
  for (int i = 0; i < C; ++i) {
    sv[i] = endpoint_sees(G, sx, sy, X[i], Y[i]);
    gv[i] = endpoint_sees(G, gx, gy, X[i], Y[i]);
  }
  sv[Gn] = endpoint_sees(G, sx, sy, gx, gy) && endpoint_sees(G, gx, gy, sx, sy);
  auto visible = [&](int a, int b) {
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (b < C) return ((G.vis[a] >> b) & 1ull) != 0;
    if (a == S && b == Gn) return sv[Gn];
    if (b == S) return sv[a];
    if (b == Gn) return a == S ? sv[Gn] : gv[a];
    return false;
  };
  double g[OR_MAX_CORNERS + 2];
  int parent[OR_MAX_CORNERS + 2];
  bool open[OR_MAX_CORNERS + 2], closed[OR_MAX_CORNERS + 2];
  for (int i = 0; i < V; ++i) {
    g[i] = INFINITY;
    parent[i] = -1;
    open[i] = closed[i] = false;
  }
  g[S] = 0.0;
  open[S] = true;
  bool found = false;
  for (;;) {
    int u = -1;
    double fu = INFINITY;
    for (int i = 0; i < V; ++i) {
      if (!open[i]) continue;
      const double f = g[i] + std::hypot(X[i] - gx, Y[i] - gy);
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
    open[u] = false;
    closed[u] = true;
    for (int v = 0; v < V; ++v) {
      if (closed[v] || v == u || !visible(u, v)) continue;
      const double c = g[u] + std::hypot(X[v] - X[u], Y[v] - Y[u]);
      if (c < g[v]) {
        g[v] = c;
        parent[v] = u;
        open[v] = true;
      }
    }
  }
  if (!found) {
    wx[0] = gx;
    wy[0] = gy;
    return 1;
  }
  int chain[OR_MAX_CORNERS + 2], n = 0;
  for (int v = Gn; v != S; v = parent[v]) chain[n++] = v;
  int k = 0;
  for (int i = n - 1; i >= 0 && k < cap; --i, ++k) {
    wx[k] = X[chain[i]];
    wy[k] = Y[chain[i]];
  }
  return k;
}

extern "C" int or_base_corners(const or_scene* s, double* xy, int cap) {
  BaseGraph G;
  base_graph(*s, G);
  const int n = G.nc < cap ? G.nc : cap;
  for (int i = 0; i < n; ++i) {
    xy[2 * i] = G.cx[i];
    xy[2 * i + 1] = G.cy[i];
  }
  return G.nc;
}

extern "C" int or_plan_path(const or_scene* s, double sx, double sy, double gx, double gy, double* xy, int cap) {
  BaseGraph G;
  base_graph(*s, G);
  double wx[OR_MAX_CORNERS + 2], wy[OR_MAX_CORNERS + 2];
  const int n = plan_path(G, sx, sy, gx, gy, wx, wy, OR_MAX_CORNERS + 2);
  const int m = n < cap ? n : cap;
  for (int i = 0; i < m; ++i) {
    xy[2 * i] = wx[i];
    xy[2 * i + 1] = wy[i];
  }
  return n;
}
