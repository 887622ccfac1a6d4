// Oracle: the "Evaluate" step of Algorithm 1 -- roll each parameter vector
// out through the plan's controllers and the rigid-body dynamics
// x_{t+1} = f(x_t, a_i) (Eq. 1b) and score it with the plan cost of
// Problem 2 (Sec. III-B).  FP64, one sample at a time, no blocking, no
// reordering.  Test infrastructure only.
//
// The paper runs this step in IsaacGym and does not define f; the model
// here is the library's documented reading:
//   * semi-implicit Euler: v <- v + a dt, then x <- x + v dt;
//   * ground friction as an implicit Coulomb clamp on the trial velocity
//     (a sliding body decelerates at mu g and never reverses);
//   * one penalty contact per (body, geometry) pair: separating-axis
//     minimum overlap gives normal and depth, F_n = max(0, k d - c v_n);
//   * Coulomb friction between bodies as one Jacobi impulse per contact,
//     capped by mu F_n dt and by the impulse that stops the sliding;
//   * action costs of Sec. IV-A: 1 per time step while the action has not
//     succeeded (here: seconds), the next action starts the step after
//     success (Problem 1), plus the end cost of each task.
#include "oracle.h"
#include "plan2d.h"
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

// ------------------------------------------------------------------ reals
// R is double for rollouts and Cnt for the flop tally (every +,-,*,/ and
// math call on a Cnt is counted; comparisons, abs, min and max are not).
namespace {
thread_local or_ops g_ops;
// test switch: run the exact base-block contact test on every step (the
// broad phase's skip is exact, so results must not change)
std::atomic<int> g_exhaustive_contacts{0};

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}
  explicit operator double() const { return v; }
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops.div; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
inline Cnt Sqrt(Cnt a) { ++g_ops.sqrt; return Cnt(std::sqrt(a.v)); }
inline Cnt Sin(Cnt a) { ++g_ops.transc; return Cnt(std::sin(a.v)); }
inline Cnt Cos(Cnt a) { ++g_ops.transc; return Cnt(std::cos(a.v)); }
inline Cnt Atan2(Cnt y, Cnt x) { ++g_ops.transc; return Cnt(std::atan2(y.v, x.v)); }
inline Cnt Acos(Cnt a) { ++g_ops.transc; return Cnt(std::acos(a.v)); }
inline Cnt Abs(Cnt a) { return Cnt(std::fabs(a.v)); }
inline Cnt Min(Cnt a, Cnt b) { return Cnt(std::fmin(a.v, b.v)); }
inline Cnt Max(Cnt a, Cnt b) { return Cnt(std::fmax(a.v, b.v)); }
inline double Val(Cnt a) { return a.v; }

inline double Sqrt(double a) { return std::sqrt(a); }
inline double Sin(double a) { return std::sin(a); }
inline double Cos(double a) { return std::cos(a); }
inline double Atan2(double y, double x) { return std::atan2(y, x); }
inline double Acos(double a) { return std::acos(a); }
inline double Abs(double a) { return std::fabs(a); }
inline double Min(double a, double b) { return std::fmin(a, b); }
inline double Max(double a, double b) { return std::fmax(a, b); }
inline double Val(double a) { return a; }

// The footprint's mean radius is a constant of the rectangle: the midpoint
// integral (or_mean_radius, 4e6 square roots) runs once per (a, b) for the
// whole process and is then looked up, so a rollout call times the dynamics,
// not this integral.  The value is the same either way.
double mean_radius_cached(double a, double b) {
  static std::mutex mu;
  static std::map<std::pair<double, double>, double> memo;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find({a, b});
    if (it != memo.end()) return it->second;
  }
  const double r = or_mean_radius(a, b);
  std::lock_guard<std::mutex> lock(mu);
  memo[{a, b}] = r;
  return r;
}

// Scene-derived constants computed once per call (not per step).
struct Prep {
  double Ib, Ik, rbar_b, rbar_k;
  BaseGraph base;  // planner graph (pick-place with the A* base controller)
};

Prep prepare(const or_scene& s) {
  Prep p{};
  // Inertia of a box about its centre: m (w^2 + l^2) / 12 with full sides.
  p.Ib = s.base_mass * (4 * s.base_half[0] * s.base_half[0] + 4 * s.base_half[1] * s.base_half[1]) / 12.0;
  p.Ik = s.block_mass * (4 * s.block_half[0] * s.block_half[0] + 4 * s.block_half[1] * s.block_half[1]) / 12.0;
  p.rbar_b = mean_radius_cached(s.base_half[0], s.base_half[1]);
  p.rbar_k = s.kind == OR_PUSH ? mean_radius_cached(s.block_half[0], s.block_half[1]) : 0.0;
  if (s.kind == OR_PICKPLACE && s.base_ctrl == 1) base_graph(s, p.base);
  return p;
}

void clamp_theta(const or_scene& s, const double* in, double* out) {
  for (int d = 0; d < s.D; ++d) out[d] = std::min(std::max(in[d], s.lo[d]), s.hi[d]);
}

// Time at which an action succeeded during step k (state advanced from
// t_k to t_{k+1}): the first crossing of the tolerance, linearly
// interpolated between the two distances (cost_step = 0), or the end of
// the step (cost_step = 1, the paper's "1 per unfinished step").
template <class R>
R success_time(const or_scene& s, int k, R d_prev, R d_new) {
  if (s.cost_step) return R((k + 1) * s.dt);
  R frac = R(0.0);
  if (d_prev > R(s.eps)) frac = (d_prev - R(s.eps)) / (d_prev - d_new);
  frac = Min(Max(frac, R(0.0)), R(1.0));
  return (R(k) + frac) * R(s.dt);
}

// ------------------------------------------------------------ planar bodies
template <class R>
struct Body2 {
  R x, y, psi, vx, vy, w;
};

// Implicit Coulomb clamp of a body sliding on the ground (normal force m g):
// translational capacity mu g dt per step, rotational capacity
// mu m g rbar dt / I, where rbar is the mean distance of the footprint's area
// from its centre.  Stick if the trial speed is within capacity.
template <class R>
void ground_clamp(Body2<R>& b, double mu, double g, double dt, double m, double I, double rbar) {
  R cap = R(mu * g * dt);
  R sp = Sqrt(b.vx * b.vx + b.vy * b.vy);
  if (sp <= cap) {
    b.vx = R(0.0); b.vy = R(0.0);
  } else {
    R f = R(1.0) - cap / sp;
    b.vx = b.vx * f; b.vy = b.vy * f;
  }
  R wcap = R(mu * m * g * rbar * dt / I);
  if (Abs(b.w) <= wcap) b.w = R(0.0);
  else b.w = b.w > R(0.0) ? b.w - wcap : b.w + wcap;
}

template <class R>
bool inside_obb(R px, R py, R cx, R cy, R c, R s, double hx, double hy) {
  R rx = px - cx, ry = py - cy;
  R u = rx * c + ry * s, w = ry * c - rx * s;
  return Abs(u) <= R(hx) && Abs(w) <= R(hy);
}

// Separating-axis test of two oriented rectangles A (base) and B (block).
// Axes in order A.u, A.w, B.u, B.w; the minimum-overlap axis (first one on
// ties) gives the normal, oriented from A to B, and the depth.  The contact
// point is the mean of the incident body's corners that lie inside the
// reference body (the body owning the axis), each weighted by its
// penetration below the reference face along the normal, so that a corner
// entering contact starts with zero weight; if no incident corner is inside,
// the roles are swapped; if still none, the midpoint of the centres.
template <class R>
bool sat_rect(const Body2<R>& A, double ahx, double ahy, const Body2<R>& B, double bhx, double bhy,
              R& nx, R& ny, R& depth, R& qx, R& qy) {
  R ca = Cos(A.psi), sa = Sin(A.psi), cb = Cos(B.psi), sb = Sin(B.psi);
  R axx[4] = {ca, -sa, cb, -sb};
  R axy[4] = {sa, ca, sb, cb};
  R dx = B.x - A.x, dy = B.y - A.y;
  int best = -1;
  R best_ov = R(0.0);
  for (int k = 0; k < 4; ++k) {
    R ux = axx[k], uy = axy[k];
    R ra = R(ahx) * Abs(ca * ux + sa * uy) + R(ahy) * Abs(ca * uy - sa * ux);
    R rb = R(bhx) * Abs(cb * ux + sb * uy) + R(bhy) * Abs(cb * uy - sb * ux);
    R sproj = dx * ux + dy * uy;
    R ov = ra + rb - Abs(sproj);
    if (ov <= R(0.0)) return false;
    if (best < 0 || ov < best_ov) {
      best = k; best_ov = ov;
      nx = sproj >= R(0.0) ? ux : -ux;
      ny = sproj >= R(0.0) ? uy : -uy;
    }
  }
  depth = best_ov;
  // reference faces along the normal: A's face at c_A.n + r_A(n) (outward +n),
  // B's face at c_B.n - r_B(n) (outward -n)
  R ra_n = R(ahx) * Abs(ca * nx + sa * ny) + R(ahy) * Abs(ca * ny - sa * nx);
  R rb_n = R(bhx) * Abs(cb * nx + sb * ny) + R(bhy) * Abs(cb * ny - sb * nx);
  R faceA = A.x * nx + A.y * ny + ra_n;
  R faceB = B.x * nx + B.y * ny - rb_n;
  // corners of the incident rectangle inside the reference one, weighted by
  // their penetration; ref_is_A selects the sign of the penetration
  auto weighted = [&](bool ref_is_A, R& mx, R& my, R& wsum, R& px_sum, R& py_sum) -> int {
    const Body2<R>& inc = ref_is_A ? B : A;
    const Body2<R>& ref = ref_is_A ? A : B;
    R ci = ref_is_A ? cb : ca, si = ref_is_A ? sb : sa;
    R cr = ref_is_A ? ca : cb, sr = ref_is_A ? sa : sb;
    double ihx = ref_is_A ? bhx : ahx, ihy = ref_is_A ? bhy : ahy;
    double rhx = ref_is_A ? ahx : bhx, rhy = ref_is_A ? ahy : bhy;
    int cnt = 0;
    mx = R(0.0); my = R(0.0); wsum = R(0.0); px_sum = R(0.0); py_sum = R(0.0);
    for (int i = 0; i < 4; ++i) {
      double su = (i & 1) ? 1.0 : -1.0, sw = (i & 2) ? 1.0 : -1.0;
      R px = inc.x + R(su * ihx) * ci - R(sw * ihy) * si;
      R py = inc.y + R(su * ihx) * si + R(sw * ihy) * ci;
      if (inside_obb(px, py, ref.x, ref.y, cr, sr, rhx, rhy)) {
        R pn = px * nx + py * ny;
        R w = Max(ref_is_A ? faceA - pn : pn - faceB, R(0.0));
        mx = mx + w * px; my = my + w * py; wsum = wsum + w;
        px_sum = px_sum + px; py_sum = py_sum + py;
        ++cnt;
      }
    }
    return cnt;
  };
  R mx, my, ws, psx, psy;
  const bool refA = best < 2;
  int cnt = weighted(refA, mx, my, ws, psx, psy);
  if (cnt == 0) cnt = weighted(!refA, mx, my, ws, psx, psy);
  if (cnt == 0) {
    qx = (A.x + B.x) * R(0.5); qy = (A.y + B.y) * R(0.5);
  } else if (ws > R(0.0)) {
    qx = mx / ws; qy = my / ws;
  } else {
    qx = psx / R((double)cnt); qy = psy / R((double)cnt);
  }
  return true;
}

template <class R>
R cross2(R ax, R ay, R bx, R by) { return ax * by - ay * bx; }

// reach (1 action) and push (move + push) tasks.
template <class R>
void planar_rollout(const or_scene& s, const Prep& pp, const double* th, int T, R& J_out, int& cls_out,
                    double* trace) {
  const bool has_block = s.kind == OR_PUSH;
  const double dt = s.dt, g = s.g;
  const double mb = s.base_mass, mk = s.block_mass;
  Body2<R> b{R(s.base_start[0]), R(s.base_start[1]), R(s.base_start[2]), R(s.base_v0[0]), R(s.base_v0[1]), R(s.base_v0[2])};
  Body2<R> k{R(s.block_start[0]), R(s.block_start[1]), R(s.block_start[2]), R(s.block_v0[0]), R(s.block_v0[1]), R(s.block_v0[2])};
  const int L = s.n_act;
  int a = 0, loaded = -1;
  R gx = R(0.0), gy = R(0.0), kp = R(0.0), kd = R(0.0), rx = R(0.0), ry = R(0.0);
  double yaw_t = 0.0;
  R t_done = R(T * dt), viol = R(0.0);
  for (int step = 0; step < T; ++step) {
    const int ai = a < L ? a : L - 1;
    if (ai != loaded) {  // controller parameters of the active action
      const int o = s.act_off[ai];
      gx = R(s.act_nom[ai][0]) + R(th[o]);
      gy = R(s.act_nom[ai][1]) + R(th[o + 1]);
      kp = R(th[o + 2]);
      kd = R(2.0) * Sqrt(kp);
      rx = s.act_ref_target[ai] ? gx : R(s.act_nom[ai][0]);
      ry = s.act_ref_target[ai] ? gy : R(s.act_nom[ai][1]);
      yaw_t = s.act_yaw[ai];
      loaded = ai;
    }
    R d_prev = R(0.0);
    if (a < L) d_prev = Sqrt((b.x - rx) * (b.x - rx) + (b.y - ry) * (b.y - ry));
    // controller: PD on position (unit-mass law scaled by m) and on yaw
    R fx = R(mb) * (kp * (gx - b.x) - kd * b.vx);
    R fy = R(mb) * (kp * (gy - b.y) - kd * b.vy);
    R tq = R(pp.Ib) * (R(s.yaw_kp) * (R(yaw_t) - b.psi) - R(s.yaw_kd) * b.w);
    R fkx = R(0.0), fky = R(0.0), tk = R(0.0);
    bool hit = false;
    R nx = R(0.0), ny = R(0.0), dep = R(0.0), qx = R(0.0), qy = R(0.0), Fn = R(0.0);
    R rax = R(0.0), ray = R(0.0), rbx = R(0.0), rby = R(0.0);
    if (has_block) {
      // broad phase: the rectangles can only touch if the block's bounding
      // circle reaches the base rectangle (tested in the base frame); the
      // skip is exact (a block outside that slab cannot overlap the base),
      // so it changes no result, only the operations the counter sees
      R cdx = k.x - b.x, cdy = k.y - b.y;
      R cbp = Cos(b.psi), sbp = Sin(b.psi);
      const double rk = std::sqrt(s.block_half[0] * s.block_half[0] + s.block_half[1] * s.block_half[1]);
      if (g_exhaustive_contacts.load(std::memory_order_relaxed) ||
          (Abs(cdx * cbp + cdy * sbp) < R(s.base_half[0] + rk) && Abs(cdy * cbp - cdx * sbp) < R(s.base_half[1] + rk)))
        hit = sat_rect(b, s.base_half[0], s.base_half[1], k, s.block_half[0], s.block_half[1], nx, ny, dep, qx, qy);
      if (hit) {
        rax = qx - b.x; ray = qy - b.y; rbx = qx - k.x; rby = qy - k.y;
        // relative velocity of the block's contact point w.r.t. the base's
        R vrx = (k.vx - k.w * rby) - (b.vx - b.w * ray);
        R vry = (k.vy + k.w * rbx) - (b.vy + b.w * rax);
        R vn = vrx * nx + vry * ny;
        Fn = Max(R(0.0), R(s.k_contact) * dep - R(s.c_contact) * vn);
        fkx = Fn * nx; fky = Fn * ny;
        fx = fx - fkx; fy = fy - fky;
        tq = tq - cross2(rax, ray, fkx, fky);
        tk = cross2(rbx, rby, fkx, fky);
        R over = Fn - R(s.force_limit);
        if (over > R(0.0)) viol = viol + over * R(dt);
      }
    }
    // trial velocities
    b.vx = b.vx + R(dt / mb) * fx;
    b.vy = b.vy + R(dt / mb) * fy;
    b.w = b.w + R(dt / pp.Ib) * tq;
    if (has_block) {
      k.vx = k.vx + R(dt / mk) * fkx;
      k.vy = k.vy + R(dt / mk) * fky;
      k.w = k.w + R(dt / pp.Ik) * tk;
      if (hit && Fn > R(0.0)) {  // Coulomb friction impulse at the contact
        R tx = -ny, ty = nx;
        R vrx = (k.vx - k.w * rby) - (b.vx - b.w * ray);
        R vry = (k.vy + k.w * rbx) - (b.vy + b.w * rax);
        R vt = vrx * tx + vry * ty;
        R ca = cross2(rax, ray, tx, ty), cb = cross2(rbx, rby, tx, ty);
        R inv_m = R(1.0 / mb) + R(1.0 / mk) + ca * ca / R(pp.Ib) + cb * cb / R(pp.Ik);
        R jm = Min(R(s.contact_mu * dt) * Fn, Abs(vt) / inv_m);
        R jt = vt > R(0.0) ? -jm : jm;  // impulse on the block along t
        R jx = jt * tx, jy = jt * ty;
        k.vx = k.vx + jx / R(mk); k.vy = k.vy + jy / R(mk);
        k.w = k.w + cross2(rbx, rby, jx, jy) / R(pp.Ik);
        b.vx = b.vx - jx / R(mb); b.vy = b.vy - jy / R(mb);
        b.w = b.w - cross2(rax, ray, jx, jy) / R(pp.Ib);
      }
      ground_clamp(k, s.block_mu, g, dt, mk, pp.Ik, pp.rbar_k);
    }
    ground_clamp(b, s.base_mu, g, dt, mb, pp.Ib, pp.rbar_b);
    // positions
    b.x = b.x + b.vx * R(dt); b.y = b.y + b.vy * R(dt); b.psi = b.psi + b.w * R(dt);
    if (has_block) {
      k.x = k.x + k.vx * R(dt); k.y = k.y + k.vy * R(dt); k.psi = k.psi + k.w * R(dt);
    }
    // success of the active action; the next one starts at the next step
    if (a < L) {
      R d_new = Sqrt((b.x - rx) * (b.x - rx) + (b.y - ry) * (b.y - ry));
      if (d_new <= R(s.eps)) {
        R ts = success_time(s, step, d_prev, d_new);
        if (a == L - 1) t_done = ts;
        ++a;
      }
    }
    if (trace) {
      double* o = trace + (size_t)step * OR_TRACE_W;
      const double v[13] = {Val(b.x), Val(b.y), Val(b.psi), Val(b.vx), Val(b.vy), Val(b.w),
                            Val(k.x), Val(k.y), Val(k.psi), Val(k.vx), Val(k.vy), Val(k.w), (double)a};
      for (int i = 0; i < OR_TRACE_W; ++i) o[i] = i < 13 ? v[i] : 0.0;
    }
  }
  const bool complete = a == L;
  bool goal;
  R J;
  if (!has_block) {
    R ex = b.x - R(s.goal_center[0]), ey = b.y - R(s.goal_center[1]);
    R dist = Sqrt(ex * ex + ey * ey);
    goal = dist <= R(s.eps);
    J = R(s.w_time) * t_done + R(s.w_goal) * dist;
  } else {
    R ex = Max(Abs(k.x - R(s.goal_center[0])) - R(s.goal_half[0]), R(0.0));
    R ey = Max(Abs(k.y - R(s.goal_center[1])) - R(s.goal_half[1]), R(0.0));
    R dist = Sqrt(ex * ex + ey * ey);
    goal = Abs(k.x - R(s.goal_center[0])) <= R(s.goal_half[0]) && Abs(k.y - R(s.goal_center[1])) <= R(s.goal_half[1]);
    J = R(s.w_time) * t_done + R(s.w_goal) * dist + R(s.w_viol) * viol;
  }
  J_out = J;
  cls_out = complete ? (goal ? 0 : 1) : 2;
  if (!std::isfinite(Val(J))) cls_out = 3;
}

// -------------------------------------------------------------- pick-place
// Minimum-overlap contact of an axis-aligned mover against one static convex
// body given as slabs (projection intervals).  Movers: the object cube
// (3-D, half size h on every axis) or the base footprint (2-D, only slabs
// with n_z == 0).  Returns the outward normal and depth.
template <class R>
bool slab_contact(const or_scene& s, int gidx, bool planar, R px, R py, R pz, double hx, double hy,
                  double hz, R& nx, R& ny, R& nz, R& depth) {
  bool any = false;
  R best = R(0.0);
  for (int i = 0; i < s.geom_nslab[gidx]; ++i) {
    const double* sl = s.slab[gidx][i];
    if (planar && sl[2] != 0.0) continue;
    R r = R(hx * std::fabs(sl[0]) + hy * std::fabs(sl[1]) + hz * std::fabs(sl[2]));
    R sp = R(sl[0]) * px + R(sl[1]) * py + R(sl[2]) * pz;
    R ov_pos = R(sl[4]) - (sp - r);  // push out through the 'hi' side
    R ov_neg = (sp + r) - R(sl[3]);  // push out through the 'lo' side
    if (ov_pos <= R(0.0) || ov_neg <= R(0.0)) return false;
    R ov = Min(ov_pos, ov_neg);
    if (!any || ov < best) {
      best = ov; any = true;
      const double sg = ov_pos <= ov_neg ? 1.0 : -1.0;
      nx = R(sg * sl[0]); ny = R(sg * sl[1]); nz = R(sg * sl[2]);
    }
  }
  depth = best;
  return any;
}

// Analytic inverse kinematics of the 2-link arm in its vertical plane
// (elbow up).  Targets out of reach are pulled onto the reachable shell.
template <class R>
void arm_ik(const or_scene& s, R bx, R by, R tx, R ty, R tz, R& beta, R& q1, R& q2) {
  R dx = tx - bx, dy = ty - by;
  beta = Atan2(dy, dx);
  R rr = Sqrt(dx * dx + dy * dy);
  R zz = tz - R(s.arm_z);
  const double l1 = s.arm_l1, l2 = s.arm_l2;
  R rho = Sqrt(rr * rr + zz * zz);
  const double rmax = l1 + l2 - 1e-3, rmin = std::fabs(l1 - l2) + 1e-3;
  if (rho > R(rmax)) {
    R f = R(rmax) / rho; rr = rr * f; zz = zz * f; rho = R(rmax);
  } else if (rho < R(rmin)) {
    R f = R(rmin) / Max(rho, R(1e-9)); rr = rr * f; zz = zz * f; rho = R(rmin);
  }
  R c2 = (rho * rho - R(l1 * l1 + l2 * l2)) / R(2.0 * l1 * l2);
  c2 = Min(Max(c2, R(-1.0)), R(1.0));
  q2 = -Acos(c2);
  q1 = Atan2(zz, rr) - Atan2(R(l2) * Sin(q2), R(l1) + R(l2) * Cos(q2));
}

template <class R>
void arm_fk(const or_scene& s, R bx, R by, R beta, R q1, R q2, R& ex, R& ey, R& ez) {
  R q12 = q1 + q2;
  R r = R(s.arm_l1) * Cos(q1) + R(s.arm_l2) * Cos(q12);
  ez = R(s.arm_z) + R(s.arm_l1) * Sin(q1) + R(s.arm_l2) * Sin(q12);
  ex = bx + r * Cos(beta);
  ey = by + r * Sin(beta);
}

template <class R>
void pickplace_final(const or_scene& s, R bx, R by, R ox, R oy, R oz, bool attached, bool complete, R t_done,
                     R& J_out, int& cls_out);

// Velocity of the end effector: the base's velocity plus the arm's, the
// time derivative of the forward kinematics at fixed azimuth, with the
// shoulder-to-tip radius r = l1 cos q1 + l2 cos(q1 + q2) and height
// z = l1 sin q1 + l2 sin(q1 + q2):
//   dr/dt = -(l1 sin q1 dq1 + l2 sin(q1 + q2) (dq1 + dq2)),
//   dz/dt = l1 cos q1 dq1 + l2 cos(q1 + q2) (dq1 + dq2),
//   v = (bvx + dr/dt cos beta, bvy + dr/dt sin beta, dz/dt).
// The azimuth beta is set kinematically when a grasp or place starts, so
// it has no rate; its jumps move the end effector but give it no speed.
template <class R>
void arm_ee_velocity(const or_scene& s, R bvx, R bvy, R beta, R q1, R q2, R dq1, R dq2, R& vx, R& vy, R& vz) {
  const R w1 = dq1, w12 = dq1 + dq2;
  const R dr = -(R(s.arm_l1) * Sin(q1) * w1 + R(s.arm_l2) * Sin(q1 + q2) * w12);
  vz = R(s.arm_l1) * Cos(q1) * w1 + R(s.arm_l2) * Cos(q1 + q2) * w12;
  vx = bvx + dr * Cos(beta);
  vy = bvy + dr * Sin(beta);
}

template <class R>
void pickplace_rollout(const or_scene& s, const Prep& pp, const double* th, int T, R& J_out, int& cls_out,
                       double* trace) {
  const double dt = s.dt, m = s.base_mass, mo = s.obj_mass, h = s.obj_half;
  R bx = R(s.base_start[0]), by = R(s.base_start[1]), bvx = R(s.base_v0[0]), bvy = R(s.base_v0[1]);
  R q1 = R(s.arm_home[0]), q2 = R(s.arm_home[1]), dq1 = R(0.0), dq2 = R(0.0), beta = R(0.0);
  R q1t = q1, q2t = q2;
  R ox = R(s.obj_start[0]), oy = R(s.obj_start[1]), oz = R(s.obj_start[2]);
  R ovx = R(s.obj_v0[0]), ovy = R(s.obj_v0[1]), ovz = R(s.obj_v0[2]);
  bool attached = false;
  R offx = R(0.0), offy = R(0.0), offz = R(0.0);
  R ex, ey, ez;
  arm_fk(s, bx, by, beta, q1, q2, ex, ey, ez);
  const int L = s.n_act;
  int a = 0, loaded = -1;
  R gx = bx, gy = by, kp = R(0.0), kd = R(0.0);      // base PD target and gains
  R mgx = bx, mgy = by, mkp = R(0.0), mkd = R(0.0);  // last moveTo target and gains
  R rx = R(0.0), ry = R(0.0);                         // moveTo success reference
  R caz = R(1.0), saz = R(0.0), hgrip = R(0.0);       // grasp parameters
  R ptx = R(0.0), pty = R(0.0), ptz = R(0.0);         // place target
  R t_done = R(T * dt);
  // A* base controller: waypoints of the current moveTo and the integral term
  double wpx[OR_MAX_CORNERS + 2], wpy[OR_MAX_CORNERS + 2];
  int nwp = 0, wi = 0;
  R Ix = R(0.0), Iy = R(0.0);
  const bool astar = s.base_ctrl == 1;
  for (int step = 0; step < T; ++step) {
    const int ai = a < L ? a : L - 1;
    const int kind = s.act_kind[ai];
    if (ai != loaded) {
      const int o = s.act_off[ai];
      if (kind == OR_MOVE) {
        mgx = R(s.act_nom[ai][0]) + R(th[o]);
        mgy = R(s.act_nom[ai][1]) + R(th[o + 1]);
        mkp = R(th[o + 2]);
        mkd = R(2.0) * Sqrt(mkp);
        rx = s.act_ref_target[ai] ? mgx : R(s.act_nom[ai][0]);
        ry = s.act_ref_target[ai] ? mgy : R(s.act_nom[ai][1]);
        if (astar) {  // plan from where the base is now
          nwp = plan_path(pp.base, Val(bx), Val(by), Val(mgx), Val(mgy), wpx, wpy, OR_MAX_CORNERS + 2);
          wi = 0;
          Ix = Iy = R(0.0);
        }
      } else if (kind == OR_GRASP) {
        caz = Cos(R(th[o])); saz = Sin(R(th[o]));
        hgrip = R(th[o + 1]);
        kp = R(s.grasp_kp); kd = R(2.0) * Sqrt(kp);
      } else if (kind == OR_PLACE) {
        ptx = R(s.act_nom[ai][0]) + R(th[o]);
        pty = R(s.act_nom[ai][1]) + R(th[o + 1]);
        ptz = R(s.act_nom[ai][2]) + R(th[o + 2]);
      }
      loaded = ai;
    }
    // targets of this step
    R tx = R(0.0), ty = R(0.0), tz = R(0.0);
    R fix = R(0.0), fiy = R(0.0);  // integral force term per unit mass
    if (kind == OR_MOVE) {
      gx = mgx; gy = mgy; kp = mkp; kd = mkd;
      if (astar) {
        // advance past every waypoint already within the switching radius
        while (wi < nwp - 1 && std::hypot(Val(bx) - wpx[wi], Val(by) - wpy[wi]) < s.wp_switch) ++wi;
        if (wi < nwp - 1) {  // an intermediate waypoint: PD towards it
          gx = R(wpx[wi]); gy = R(wpy[wi]);
          Ix = Iy = R(0.0);
        } else {  // the goal: PID, integrating the error near it
          const R ex_ = mgx - bx, ey_ = mgy - by;
          if (Val(Sqrt(ex_ * ex_ + ey_ * ey_)) < s.pid_irad) {
            Ix = Min(Max(Ix + ex_ * R(dt), R(-s.pid_imax)), R(s.pid_imax));
            Iy = Min(Max(Iy + ey_ * R(dt), R(-s.pid_imax)), R(s.pid_imax));
          } else {
            Ix = Iy = R(0.0);
          }
          fix = R(s.pid_ki) * kp * Ix;
          fiy = R(s.pid_ki) * kp * Iy;
        }
      }
    } else if (kind == OR_GRASP) {
      tx = ox; ty = oy; tz = oz + hgrip;
      gx = ox - R(s.grasp_reach) * caz;
      gy = oy - R(s.grasp_reach) * saz;
    } else {  // place: the base holds the last moveTo target
      tx = ptx; ty = pty; tz = ptz;
      gx = mgx; gy = mgy; kp = mkp; kd = mkd;
    }
    R d_prev = R(0.0);
    if (a < L) {
      if (kind == OR_MOVE) d_prev = Sqrt((bx - rx) * (bx - rx) + (by - ry) * (by - ry));
      else d_prev = Sqrt((ex - tx) * (ex - tx) + (ey - ty) * (ey - ty) + (ez - tz) * (ez - tz));
    }
    if (kind != OR_MOVE) arm_ik(s, bx, by, tx, ty, tz, beta, q1t, q2t);
    // base: PD + penalty contacts against the static footprints
    R fx = R(m) * (kp * (gx - bx) - kd * bvx);
    R fy = R(m) * (kp * (gy - by) - kd * bvy);
    if (astar && kind == OR_MOVE) {
      fx = fx + R(m) * fix;
      fy = fy + R(m) * fiy;
    }
    for (int gi = 0; gi < s.n_geoms; ++gi) {
      if (!s.geom_base[gi]) continue;
      R nx, ny, nz, dep;
      if (slab_contact(s, gi, true, bx, by, R(0.0), s.base_half[0], s.base_half[1], 0.0, nx, ny, nz, dep)) {
        R vn = bvx * nx + bvy * ny;
        R Fn = Max(R(0.0), R(s.k_contact) * dep - R(s.c_contact) * vn);
        fx = fx + Fn * nx; fy = fy + Fn * ny;
      }
    }
    bvx = bvx + R(dt / m) * fx;
    bvy = bvy + R(dt / m) * fy;
    {  // ground friction of the base (yaw is locked)
      R cap = R(s.base_mu * s.g * dt);
      R sp = Sqrt(bvx * bvx + bvy * bvy);
      if (sp <= cap) { bvx = R(0.0); bvy = R(0.0); }
      else { R f = R(1.0) - cap / sp; bvx = bvx * f; bvy = bvy * f; }
    }
    bx = bx + bvx * R(dt); by = by + bvy * R(dt);
    // arm: joint-space PD (computed-torque double integrator)
    R dd1 = R(s.arm_kp) * (q1t - q1) - R(s.arm_kd) * dq1;
    R dd2 = R(s.arm_kp) * (q2t - q2) - R(s.arm_kd) * dq2;
    dq1 = dq1 + R(dt) * dd1; dq2 = dq2 + R(dt) * dd2;
    q1 = q1 + R(dt) * dq1; q2 = q2 + R(dt) * dq2;
    R nex, ney, nez;
    arm_fk(s, bx, by, beta, q1, q2, nex, ney, nez);
    // object
    if (attached) {
      ox = nex + offx; oy = ney + offy; oz = nez + offz;
      arm_ee_velocity(s, bvx, bvy, beta, q1, q2, dq1, dq2, ovx, ovy, ovz);
    } else {
      R cnx[OR_MAX_GEOM], cny[OR_MAX_GEOM], cnz[OR_MAX_GEOM], cfn[OR_MAX_GEOM];
      int nc = 0;
      R fsx = R(0.0), fsy = R(0.0), fsz = R(0.0);
      for (int gi = 0; gi < s.n_geoms; ++gi) {
        if (!s.geom_obj[gi]) continue;
        R nx, ny, nz, dep;
        if (slab_contact(s, gi, false, ox, oy, oz, h, h, h, nx, ny, nz, dep)) {
          R vn = ovx * nx + ovy * ny + ovz * nz;
          R Fn = Max(R(0.0), R(s.k_contact) * dep - R(s.c_contact) * vn);
          if (Fn > R(0.0)) {
            cnx[nc] = nx; cny[nc] = ny; cnz[nc] = nz; cfn[nc] = Fn; ++nc;
            fsx = fsx + Fn * nx; fsy = fsy + Fn * ny; fsz = fsz + Fn * nz;
          }
        }
      }
      ovx = ovx + R(dt / mo) * fsx;
      ovy = ovy + R(dt / mo) * fsy;
      ovz = ovz + R(dt / mo) * fsz - R(s.g * dt);
      // Jacobi Coulomb impulses, all from the same trial velocity
      R jx = R(0.0), jy = R(0.0), jz = R(0.0);
      for (int c = 0; c < nc; ++c) {
        R vn = ovx * cnx[c] + ovy * cny[c] + ovz * cnz[c];
        R tx_ = ovx - vn * cnx[c], ty_ = ovy - vn * cny[c], tz_ = ovz - vn * cnz[c];
        R vt = Sqrt(tx_ * tx_ + ty_ * ty_ + tz_ * tz_);
        if (vt > R(0.0)) {
          R jm = Min(R(s.obj_mu * dt) * cfn[c], R(mo) * vt / R((double)nc));
          R f = jm / (R(mo) * vt);
          jx = jx - f * tx_; jy = jy - f * ty_; jz = jz - f * tz_;
        }
      }
      ovx = ovx + jx; ovy = ovy + jy; ovz = ovz + jz;
      ox = ox + ovx * R(dt); oy = oy + ovy * R(dt); oz = oz + ovz * R(dt);
    }
    // success of the active action
    if (a < L) {
      R d_new;
      bool ok;
      if (kind == OR_MOVE) {
        d_new = Sqrt((bx - rx) * (bx - rx) + (by - ry) * (by - ry));
        ok = d_new <= R(s.eps);
      } else {
        d_new = Sqrt((nex - tx) * (nex - tx) + (ney - ty) * (ney - ty) + (nez - tz) * (nez - tz));
        ok = d_new <= R(s.eps);
        if (kind == OR_GRASP) ok = ok && Abs(hgrip) <= R(s.grip_tol);
      }
      if (ok) {
        R ts = success_time(s, step, d_prev, d_new);
        if (a == L - 1) t_done = ts;
        if (kind == OR_GRASP) {
          attached = true;
          offx = ox - nex; offy = oy - ney; offz = oz - nez;
        } else if (kind == OR_PLACE) {
          attached = false;  // released with the end-effector velocity
        }
        ++a;
      }
    }
    ex = nex; ey = ney; ez = nez;
    if (trace) {
      double* o = trace + (size_t)step * OR_TRACE_W;
      const double v[20] = {Val(bx), Val(by), Val(bvx), Val(bvy), Val(q1), Val(q2), Val(dq1),
                            Val(dq2), Val(beta), Val(ox), Val(oy), Val(oz), Val(ovx), Val(ovy),
                            Val(ovz), attached ? 1.0 : 0.0, (double)a, Val(ex), Val(ey), Val(ez)};
      for (int i = 0; i < OR_TRACE_W; ++i) o[i] = v[i];
    }
  }
  pickplace_final(s, bx, by, ox, oy, oz, attached, a == L, t_done, J_out, cls_out);
}

// End of a pick-place rollout (Problem 2, Sec. IV-A): the goal psi_g and the
// plan cost from the final state.  The goal holds when every flagged part
// does: the object at rest in its region and not held (goal_obj_region),
// the object held (goal_obj_held), the base inside its region
// (goal_base_region).  J = w_time t_done + w_obj d_obj + w_base d_base with
// the Euclidean distances of object and base to their boxes (a held-object
// goal counts d_obj = 0 if held, 1 if not).  Class 0: every action
// succeeded and the goal holds; 1: every action succeeded, goal false; 2:
// an action unfinished; 3: non-finite cost.
template <class R>
void pickplace_final(const or_scene& s, R bx, R by, R ox, R oy, R oz, bool attached, bool complete, R t_done,
                     R& J_out, int& cls_out) {
  bool goal = true;
  R d_obj = R(0.0), d_base = R(0.0);
  if (s.goal_obj_region) {
    R e0 = Abs(ox - R(s.obj_region_c[0])), e1 = Abs(oy - R(s.obj_region_c[1])), e2 = Abs(oz - R(s.obj_region_c[2]));
    goal = goal && !attached && e0 <= R(s.obj_region_h[0]) && e1 <= R(s.obj_region_h[1]) && e2 <= R(s.obj_region_h[2]);
    R x0 = Max(e0 - R(s.obj_region_h[0]), R(0.0)), x1 = Max(e1 - R(s.obj_region_h[1]), R(0.0));
    R x2 = Max(e2 - R(s.obj_region_h[2]), R(0.0));
    d_obj = Sqrt(x0 * x0 + x1 * x1 + x2 * x2);
  }
  if (s.goal_obj_held) {
    goal = goal && attached;
    d_obj = attached ? R(0.0) : R(1.0);
  }
  if (s.goal_base_region) {
    R e0 = Abs(bx - R(s.base_region_c[0])), e1 = Abs(by - R(s.base_region_c[1]));
    goal = goal && e0 <= R(s.base_region_h[0]) && e1 <= R(s.base_region_h[1]);
    R x0 = Max(e0 - R(s.base_region_h[0]), R(0.0)), x1 = Max(e1 - R(s.base_region_h[1]), R(0.0));
    d_base = Sqrt(x0 * x0 + x1 * x1);
  }
  R J = R(s.w_time) * t_done + R(s.w_obj) * d_obj + R(s.w_base) * d_base;
  J_out = J;
  cls_out = complete ? (goal ? 0 : 1) : 2;
  if (!std::isfinite(Val(J))) cls_out = 3;
}

// ---------------------------------------------------------------- quadratic
template <class R>
void quadratic_cost(const or_scene& s, const double* th, R& J_out, int& cls_out) {
  R J = R(0.0);
  for (int i = 0; i < s.D; ++i) {
    R ri = R(0.0);
    for (int j = 0; j < s.D; ++j) ri = ri + R(s.A[i * s.D + j]) * (R(th[j]) - R(s.theta_star[j]));
    J = J + (R(th[i]) - R(s.theta_star[i])) * ri;
  }
  J_out = J;
  cls_out = std::isfinite(Val(J)) ? 0 : 3;
}

template <class R>
void rollout_one(const or_scene& s, const Prep& pp, const double* theta, int T, R& J, int& cls, double* trace) {
  double th[OR_MAX_D];
  clamp_theta(s, theta, th);
  switch (s.kind) {
    case OR_QUAD: quadratic_cost(s, th, J, cls); break;
    case OR_REACH:
    case OR_PUSH: planar_rollout(s, pp, th, T, J, cls, trace); break;
    case OR_PICKPLACE: pickplace_rollout(s, pp, th, T, J, cls, trace); break;
    default: J = R(NAN); cls = 3;
  }
}
}  // namespace

extern "C" void or_pickplace_final(const or_scene* s, const double* state, int complete, double t_done,
                                   double* J, int* cls) {
  pickplace_final<double>(*s, state[0], state[1], state[9], state[10], state[11], state[15] != 0.0,
                          complete != 0, t_done, *J, *cls);
}

extern "C" double or_mean_radius(double a, double b) {
  // mean of sqrt(x^2 + y^2) over [0,a] x [0,b] by the midpoint rule
  const int M = 2000;
  double acc = 0.0;
  for (int i = 0; i < M; ++i) {
    double x = (i + 0.5) * a / M;
    double row = 0.0;
    for (int j = 0; j < M; ++j) {
      double y = (j + 0.5) * b / M;
      row += std::sqrt(x * x + y * y);
    }
    acc += row;
  }
  return acc / ((double)M * M);
}

extern "C" void or_rollout(const or_scene* s, const double* theta, int N, double* J, uint8_t* cls,
                           int nthreads) {
  const Prep pp = prepare(*s);
  int nt = nthreads > 0 ? nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
  nt = std::max(1, std::min(nt, N));
  auto work = [&](int t0) {
    for (int n = t0; n < N; n += nt) {
      double Jn;
      int c;
      rollout_one<double>(*s, pp, theta + (size_t)n * s->D, s->T, Jn, c, nullptr);
      J[n] = Jn;
      cls[n] = (uint8_t)c;
    }
  };
  if (nt == 1) {
    work(0);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(work, t);
  for (auto& th : pool) th.join();
}

extern "C" void or_rollout_trace(const or_scene* s, const double* theta, int steps, double* states) {
  const Prep pp = prepare(*s);
  double J;
  int c;
  std::memset(states, 0, sizeof(double) * (size_t)steps * OR_TRACE_W);
  rollout_one<double>(*s, pp, theta, steps, J, c, states);
}

extern "C" int or_rollout_count(const or_scene* s, const double* theta, or_ops* ops) {
  const Prep pp = prepare(*s);
  g_ops = or_ops{0, 0, 0, 0, 0};
  Cnt J;
  int c;
  rollout_one<Cnt>(*s, pp, theta, s->T, J, c, nullptr);
  ops->add += g_ops.add;
  ops->mul += g_ops.mul;
  ops->div += g_ops.div;
  ops->sqrt += g_ops.sqrt;
  ops->transc += g_ops.transc;
  return s->kind == OR_QUAD ? 1 : s->T;
}

// Domain randomisation (Sec. IV-C: plans made robust to bounded uncertainty
// in friction or mass).  Environment m of CE iteration `iter` scales every
// friction coefficient by s_mu = 1 + dmu (2 u0 - 1) and the manipulated
// body's mass by s_m = 1 + dm (2 u1 - 1), with (u0, u1) from the first two
// words of the Philox block (m, 256, iter, problem) under key `seed` and
// u = (word + 1) 2^-32.  All samples of an iteration share the environments.
extern "C" void or_set_exhaustive_contacts(int on) { g_exhaustive_contacts.store(on ? 1 : 0); }

extern "C" void or_dr_factors(uint64_t seed, uint32_t iter, uint32_t problem, int M, double dmu, double dm,
                              double* smu, double* sm) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int m = 0; m < M; ++m) {
    const uint32_t ctr[4] = {(uint32_t)m, 256u, iter, problem};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    const double u0 = ((double)r[0] + 1.0) * 0x1p-32, u1 = ((double)r[1] + 1.0) * 0x1p-32;
    smu[m] = 1.0 + dmu * (2.0 * u0 - 1.0);
    sm[m] = 1.0 + dm * (2.0 * u1 - 1.0);
  }
}

// Every sample in each of the M environments: J = mean over environments,
// class = the worst (largest) class over environments, so a plan counts as
// feasible only if it succeeds in all of them.
extern "C" void or_rollout_dr(const or_scene* s, const double* theta, int N, int M, double dmu, double dm,
                              uint64_t seed, uint32_t iter, uint32_t problem, double* J, uint8_t* cls,
                              int nthreads) {
  std::vector<double> smu(M), sm(M), Jm(N);
  std::vector<uint8_t> cm(N);
  or_dr_factors(seed, iter, problem, M, dmu, dm, smu.data(), sm.data());
  for (int n = 0; n < N; ++n) {
    J[n] = 0.0;
    cls[n] = 0;
  }
  for (int m = 0; m < M; ++m) {
    or_scene e = *s;
    e.base_mu *= smu[m];
    e.block_mu *= smu[m];
    e.contact_mu *= smu[m];
    e.obj_mu *= smu[m];
    e.block_mass *= sm[m];
    e.obj_mass *= sm[m];
    or_rollout(&e, theta, N, Jm.data(), cm.data(), nthreads);
    for (int n = 0; n < N; ++n) {
      J[n] += Jm[n];
      cls[n] = std::max(cls[n], cm[n]);
    }
  }
  for (int n = 0; n < N; ++n) {
    J[n] /= (double)M;
    if (!std::isfinite(J[n])) cls[n] = 3;
  }
}
