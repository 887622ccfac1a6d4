// Evaluate step of Algorithm 1 (Sec. III-B): every sample's plan is rolled
// out through its controllers and the rigid-body dynamics x_{t+1} =
// f(x_t, a_i) (Eq. 1b, Problem 2) for T steps and scored with the plan cost.
//
// Dynamics (the paper uses IsaacGym and does not define f; this is the
// library's model): semi-implicit Euler; ground friction as an implicit
// Coulomb clamp of the trial velocity; one penalty contact per (body,
// geometry) pair from the separating-axis minimum overlap,
// F_n = max(0, k depth - c v_n); Coulomb friction between bodies as one
// Jacobi impulse per contact capped by mu F_n dt and by the impulse that
// stops sliding.  Action cost (Sec. IV-A): time until the action succeeds;
// the next action starts at the step after success (Problem 1).
//
// GB300 mapping: one thread per rollout, the whole state in registers, the
// scene (geometry, constants, skeleton) staged once per block in shared
// memory, the T-step loop fused in one launch, nothing per step written to
// HBM.  The kernel reads N*D*4 bytes and writes N*5 bytes, so it is bound by
// the FP32 pipe and by instruction latency, not by HBM.
#include "internal.h"
#include "philox.cuh"
#include "plan.cuh"

namespace cem {
namespace {

constexpr int TW = CEM_TRACE_W;

// parameter i clamped to its bounds; a NaN stays NaN (its rollout then ends
// with a non-finite cost, class 3)
__device__ __forceinline__ float theta_at(const DevScene& s, const float* __restrict__ row, int i) {
  i = CEM_DIDX(i, s.D, 7);
  const float x = row[i];
  return isnan(x) ? x : fminf(fmaxf(x, s.lo[i]), s.hi[i]);
}

// time at which an action succeeded inside step k (state t_k -> t_{k+1})
__device__ __forceinline__ float success_time(const DevScene& s, int k, float d_prev, float d_new) {
  if (s.cost_step) return (float)(k + 1) * s.dt;
  float frac = 0.0f;
  if (d_prev > s.eps) frac = (d_prev - s.eps) / (d_prev - d_new);
  frac = fminf(fmaxf(frac, 0.0f), 1.0f);
  return ((float)k + frac) * s.dt;
}

struct B2 {
  float x, y, psi, vx, vy, w;
};

// Implicit Coulomb clamp of the trial velocity (branch-free): stick if the
// speed is within mu g dt, else remove mu g dt along the velocity; the same
// for the spin with capacity mu m g rbar dt / I.
__device__ __forceinline__ void ground_clamp(B2& b, float cap, float cap2, float wcap) {
  const float v2 = b.vx * b.vx + b.vy * b.vy;
  const float f = v2 > cap2 ? 1.0f - cap * rsqrtf(v2) : 0.0f;
  b.vx *= f;
  b.vy *= f;
  b.w = fabsf(b.w) <= wcap ? 0.0f : b.w - copysignf(wcap, b.w);
}

// Contact point of the rectangle pair in the reference body's frame: the
// incident body's corners that lie inside the reference rectangle, each
// weighted by its penetration along the normal.  Inputs (all in the
// reference frame): the incident centre d, the incident axes u_i, w_i, the
// normal n, the reference half sizes and the reference support r_n along n.
// ref_is_A: penetration below A's face (r_n - p.n), else above B's face
// (p.n + r_n).  Returns how many corners are inside.
__device__ __forceinline__ int corners_local(float dx, float dy, float uix, float uiy, float wix, float wiy, float ihx,
                                             float ihy, float rhx, float rhy, float nlx, float nly, float r_n,
                                             bool ref_is_A, float& mx, float& my, float& ws, float& px_sum,
                                             float& py_sum) {
  int cnt = 0;
  mx = my = ws = px_sum = py_sum = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float su = (i & 1) ? ihx : -ihx, sw = (i & 2) ? ihy : -ihy;
    const float px = dx + su * uix + sw * wix;
    const float py = dy + su * uiy + sw * wiy;
    if (fabsf(px) <= rhx && fabsf(py) <= rhy) {
      const float pn = px * nlx + py * nly;
      const float w = fmaxf(ref_is_A ? r_n - pn : pn + r_n, 0.0f);
      mx += w * px;
      my += w * py;
      ws += w;
      px_sum += px;
      py_sum += py;
      ++cnt;
    }
  }
  return cnt;
}

// SAT of rectangle A (base) against rectangle B (block) with the relative
// rotation (c, s) = (cos, sin)(psi_B - psi_A): the support of a box along
// the other box's axes needs only |c| and |s|.  Axes in order A.u, A.w, B.u,
// B.w; the minimum overlap (first on ties) gives the normal (A -> B) and the
// depth.  Contact point: penetration-weighted mean of the incident corners
// inside the reference body (roles swapped if none; midpoint last).
// sine and cosine of a yaw angle: wrapped into [-pi, pi], where the hardware
// unit is accurate to ~5e-7 (a spinning block's yaw grows without bound)
__device__ __forceinline__ void yaw_sincos(float psi, float* sn, float* cs) {
  const float w = psi - 6.28318530717958648f * rintf(psi * 0.159154943091895336f);
  __sincosf(w, sn, cs);
}

// (sa, ca): A's yaw sine and cosine, already at hand in the caller
__device__ __forceinline__ bool sat_rect(const B2& A, float sa, float ca, float ahx, float ahy, const B2& B, float bhx,
                                         float bhy, float& nx, float& ny, float& depth, float& qx, float& qy) {
  float sb, cb;
  yaw_sincos(B.psi, &sb, &cb);
  const float c = ca * cb + sa * sb, s = ca * sb - sa * cb;
  const float ac = fabsf(c), as = fabsf(s);
  const float dx = B.x - A.x, dy = B.y - A.y;
  const float dAx = dx * ca + dy * sa, dAy = dy * ca - dx * sa;  // B's centre in A's frame
  const float dBx = dx * cb + dy * sb, dBy = dy * cb - dx * sb;  // same vector in B's frame
  const float ov0 = ahx + bhx * ac + bhy * as - fabsf(dAx);
  const float ov1 = ahy + bhx * as + bhy * ac - fabsf(dAy);
  const float ov2 = ahx * ac + ahy * as + bhx - fabsf(dBx);
  const float ov3 = ahx * as + ahy * ac + bhy - fabsf(dBy);
  if (ov0 <= 0.0f || ov1 <= 0.0f || ov2 <= 0.0f || ov3 <= 0.0f) return false;
  int best = 0;
  float ov = ov0;
  if (ov1 < ov) { best = 1; ov = ov1; }
  if (ov2 < ov) { best = 2; ov = ov2; }
  if (ov3 < ov) { best = 3; ov = ov3; }
  depth = ov;
  // normal in world and in both local frames (sg = side of B along the axis)
  float nAx, nAy, nBx, nBy;
  if (best == 0) {
    const float sg = dAx >= 0.0f ? 1.0f : -1.0f;
    nx = sg * ca; ny = sg * sa; nAx = sg; nAy = 0.0f; nBx = sg * c; nBy = -sg * s;
  } else if (best == 1) {
    const float sg = dAy >= 0.0f ? 1.0f : -1.0f;
    nx = -sg * sa; ny = sg * ca; nAx = 0.0f; nAy = sg; nBx = sg * s; nBy = sg * c;
  } else if (best == 2) {
    const float sg = dBx >= 0.0f ? 1.0f : -1.0f;
    nx = sg * cb; ny = sg * sb; nAx = sg * c; nAy = sg * s; nBx = sg; nBy = 0.0f;
  } else {
    const float sg = dBy >= 0.0f ? 1.0f : -1.0f;
    nx = -sg * sb; ny = sg * cb; nAx = -sg * s; nAy = sg * c; nBx = 0.0f; nBy = sg;
  }
  const float rA_n = ahx * fabsf(nAx) + ahy * fabsf(nAy);  // A's support along n
  const float rB_n = bhx * fabsf(nBx) + bhy * fabsf(nBy);
  // B's corners in A's frame use B's axes (c, s), (-s, c); A's corners in
  // B's frame use A's axes (c, -s), (s, c) and A's centre at -dB
  float mx, my, ws, psx, psy;
  bool in_A = best < 2;  // frame of the points being accumulated
  int cnt = in_A ? corners_local(dAx, dAy, c, s, -s, c, bhx, bhy, ahx, ahy, nAx, nAy, rA_n, true, mx, my, ws, psx, psy)
                 : corners_local(-dBx, -dBy, c, -s, s, c, ahx, ahy, bhx, bhy, nBx, nBy, rB_n, false, mx, my, ws, psx,
                                 psy);
  if (cnt == 0) {
    in_A = !in_A;
    cnt = in_A ? corners_local(dAx, dAy, c, s, -s, c, bhx, bhy, ahx, ahy, nAx, nAy, rA_n, true, mx, my, ws, psx, psy)
               : corners_local(-dBx, -dBy, c, -s, s, c, ahx, ahy, bhx, bhy, nBx, nBy, rB_n, false, mx, my, ws, psx,
                               psy);
  }
  if (cnt == 0) {
    qx = (A.x + B.x) * 0.5f;
    qy = (A.y + B.y) * 0.5f;
    return true;
  }
  float lx, ly;
  if (ws > 0.0f) {
    const float inv = __fdividef(1.0f, ws);  // fast reciprocal (2 ulp; 0 < ws, far below 2^126)
    lx = mx * inv;
    ly = my * inv;
  } else {
    const float inv = cnt == 1 ? 1.0f : cnt == 2 ? 0.5f : cnt == 4 ? 0.25f : (1.0f / 3.0f);
    lx = psx * inv;
    ly = psy * inv;
  }
  if (in_A) {
    qx = A.x + lx * ca - ly * sa;
    qy = A.y + lx * sa + ly * ca;
  } else {
    qx = B.x + lx * cb - ly * sb;
    qy = B.y + lx * sb + ly * cb;
  }
  return true;
}

__device__ __forceinline__ float cross2(float ax, float ay, float bx, float by) { return ax * by - ay * bx; }

__device__ __forceinline__ void put_trace(float* tr, int step, const float* v, int nv) {
  float* o = tr + (size_t)step * TW;
#pragma unroll
  for (int i = 0; i < TW; ++i) o[i] = i < nv ? v[i] : 0.0f;
}

// ------------------------------------------------------------- reach / push
// The success test compares squared distances; the square roots are taken
// only at the step that succeeds (for the interpolated crossing time).
// The rollout functions are compiled once (noinline) and called by every
// rollout kernel, so the single-problem, traced and batched launches execute
// the same instructions and return bit-identical results.
// smu / sm: friction and manipulated-body mass scales of a randomised
// environment (exactly 1 otherwise, which leaves every value unchanged).
template <bool HAS_BLOCK, bool TRACE>
__device__ __noinline__ void planar_rollout(const DevScene& s, const float* __restrict__ row, int T, float smu, float sm,
                                            float& J_out, int& cls_out, float* tr) {
  // loop invariants in registers
  const float dt = s.dt, eps2 = s.eps * s.eps;
  const float mb = s.mb, Ib = s.Ib, dt_mb = s.dt_mb, dt_Ib = s.dt_Ib;
  const float bcap = s.base_cap * smu, bcap2 = bcap * bcap, bwcap = s.base_wcap * smu;
  const float ykp = s.yaw_kp, ykd = s.yaw_kd;
  const float bhx = s.bhx, bhy = s.bhy, khx = s.khx, khy = s.khy;
  // the block's spin capacity mu m g rbar dt / I does not depend on its mass (I is proportional to m)
  const float dt_mk = s.dt_mk / sm, dt_Ik = s.dt_Ik / sm, kcap = s.block_cap * smu, kcap2 = kcap * kcap;
  const float kwcap = s.block_wcap * smu;
  const float kc = s.k_contact, cc = s.c_contact, mu_dt = s.contact_mu * smu * s.dt, flim = s.force_limit;
  const float inv_mb = 1.0f / s.mb, inv_Ib = 1.0f / s.Ib;
  const float inv_mk = HAS_BLOCK ? 1.0f / (s.mk * sm) : 0.0f, inv_Ik = HAS_BLOCK ? 1.0f / (s.Ik * sm) : 0.0f;
  // broad phase: the block's bounding circle (radius rk) against the base
  // rectangle, in the base frame; the hardware sine/cosine is off by < 1e-6,
  // so a 1e-4 m margin keeps the test conservative (it never rejects a pair
  // the exact test would keep)
  const float rk = sqrtf(khx * khx + khy * khy);
  const float reach_u = bhx + rk + 1e-4f, reach_w = bhy + rk + 1e-4f;
  B2 b{s.base_start[0], s.base_start[1], s.base_start[2], s.base_v0[0], s.base_v0[1], s.base_v0[2]};
  B2 k{s.block_start[0], s.block_start[1], s.block_start[2], s.block_v0[0], s.block_v0[1], s.block_v0[2]};
  const int L = s.n_act;
  int a = 0, loaded = -1;
  float gx = 0.f, gy = 0.f, kp = 0.f, kd = 0.f, rx = 0.f, ry = 0.f, yaw_t = 0.f;
  float t_done = (float)T * dt, viol = 0.0f, d2_cur = 0.0f;
  for (int step = 0; step < T; ++step) {
    const int ai = a < L ? a : L - 1;
    if (ai != loaded) {
      const int o = s.act_off[ai];
      gx = s.act_nom[ai][0] + theta_at(s, row, o);
      gy = s.act_nom[ai][1] + theta_at(s, row, o + 1);
      kp = theta_at(s, row, o + 2);
      kd = 2.0f * sqrtf(kp);
      rx = s.act_ref[ai] ? gx : s.act_nom[ai][0];
      ry = s.act_ref[ai] ? gy : s.act_nom[ai][1];
      yaw_t = s.act_yaw[ai];
      loaded = ai;
      d2_cur = (b.x - rx) * (b.x - rx) + (b.y - ry) * (b.y - ry);
    }
    float fx = mb * (kp * (gx - b.x) - kd * b.vx);
    float fy = mb * (kp * (gy - b.y) - kd * b.vy);
    float tq = Ib * (ykp * (yaw_t - b.psi) - ykd * b.w);
    float fkx = 0.f, fky = 0.f, tk = 0.f, Fn = 0.f;
    float rax = 0.f, ray = 0.f, rbx = 0.f, rby = 0.f, nx = 0.f, ny = 0.f;
    bool hit = false;
    if (HAS_BLOCK) {
      const float cdx = k.x - b.x, cdy = k.y - b.y;
      float sbp, cbp;
      yaw_sincos(b.psi, &sbp, &cbp);
      if (fabsf(cdx * cbp + cdy * sbp) < reach_u && fabsf(cdy * cbp - cdx * sbp) < reach_w) {
        float dep, qx, qy;
        hit = sat_rect(b, sbp, cbp, bhx, bhy, k, khx, khy, nx, ny, dep, qx, qy);
        if (hit) {
          rax = qx - b.x;
          ray = qy - b.y;
          rbx = qx - k.x;
          rby = qy - k.y;
          const float vrx = (k.vx - k.w * rby) - (b.vx - b.w * ray);
          const float vry = (k.vy + k.w * rbx) - (b.vy + b.w * rax);
          const float vn = vrx * nx + vry * ny;
          Fn = fmaxf(0.0f, kc * dep - cc * vn);
          fkx = Fn * nx;
          fky = Fn * ny;
          fx -= fkx;
          fy -= fky;
          tq -= cross2(rax, ray, fkx, fky);
          tk = cross2(rbx, rby, fkx, fky);
          const float over = Fn - flim;
          if (over > 0.0f) viol += over * dt;
        }
      }
    }
    b.vx += dt_mb * fx;
    b.vy += dt_mb * fy;
    b.w += dt_Ib * tq;
    if (HAS_BLOCK) {
      k.vx += dt_mk * fkx;
      k.vy += dt_mk * fky;
      k.w += dt_Ik * tk;
      if (hit && Fn > 0.0f) {
        const float tx = -ny, ty = nx;
        const float vrx = (k.vx - k.w * rby) - (b.vx - b.w * ray);
        const float vry = (k.vy + k.w * rbx) - (b.vy + b.w * rax);
        const float vt = vrx * tx + vry * ty;
        const float ca = cross2(rax, ray, tx, ty), cb = cross2(rbx, rby, tx, ty);
        const float inv_m = inv_mb + inv_mk + ca * ca * inv_Ib + cb * cb * inv_Ik;
        // fast division (2 ulp; inv_m is an inverse mass sum of order 1..10):
        // this chain sets the step latency of every warp with a block contact
        const float jm = fminf(mu_dt * Fn, __fdividef(fabsf(vt), inv_m));
        const float jt = vt > 0.0f ? -jm : jm;
        const float jx = jt * tx, jy = jt * ty;
        k.vx += jx * inv_mk;
        k.vy += jy * inv_mk;
        k.w += cross2(rbx, rby, jx, jy) * inv_Ik;
        b.vx -= jx * inv_mb;
        b.vy -= jy * inv_mb;
        b.w -= cross2(rax, ray, jx, jy) * inv_Ib;
      }
      ground_clamp(k, kcap, kcap2, kwcap);
    }
    ground_clamp(b, bcap, bcap2, bwcap);
    b.x += b.vx * dt;
    b.y += b.vy * dt;
    b.psi += b.w * dt;
    if (HAS_BLOCK) {
      k.x += k.vx * dt;
      k.y += k.vy * dt;
      k.psi += k.w * dt;
    }
    if (a < L) {
      const float d2_new = (b.x - rx) * (b.x - rx) + (b.y - ry) * (b.y - ry);
      if (d2_new <= eps2) {
        const float ts = success_time(s, step, sqrtf(d2_cur), sqrtf(d2_new));
        if (a == L - 1) t_done = ts;
        ++a;
      }
      d2_cur = d2_new;
    }
    if (TRACE) {
      const float v[13] = {b.x, b.y, b.psi, b.vx, b.vy, b.w, k.x, k.y, k.psi, k.vx, k.vy, k.w, (float)a};
      put_trace(tr, step, v, 13);
    }
  }
  const bool complete = a == L;
  bool goal;
  float J;
  if (!HAS_BLOCK) {
    const float ex = b.x - s.goal_center[0], ey = b.y - s.goal_center[1];
    const float dist = sqrtf(ex * ex + ey * ey);
    goal = dist <= s.eps;
    J = s.w_time * t_done + s.w_goal * dist;
  } else {
    const float ax = fabsf(k.x - s.goal_center[0]), ay = fabsf(k.y - s.goal_center[1]);
    const float ex = fmaxf(ax - s.goal_half[0], 0.0f), ey = fmaxf(ay - s.goal_half[1], 0.0f);
    const float dist = sqrtf(ex * ex + ey * ey);
    goal = ax <= s.goal_half[0] && ay <= s.goal_half[1];
    J = s.w_time * t_done + s.w_goal * dist + s.w_viol * viol;
  }
  J_out = J;
  cls_out = complete ? (goal ? 0 : 1) : 2;
  if (!isfinite(J)) cls_out = 3;
}

// --------------------------------------------------------------- pick-place
// Minimum-overlap contact of an axis-aligned mover against static geometry g.
// The mover's support along each slab normal is folded into the slab when
// the scene is prepared (DevScene::oslab for the object cube, ::bslab for
// the base footprint's slabs with n_z == 0), so a slab costs one projection
// and two differences: overlap through the 'hi' side hi' - p.n, through the
// 'lo' side p.n - lo'.  The smallest overlap (first on ties) gives the
// outward normal and the depth; any separating slab means no contact.
template <bool PLANAR>
__device__ __forceinline__ bool slab_contact(const DevScene& s, int g, float px, float py, float pz, float& nx,
                                             float& ny, float& nz, float& depth) {
  g = CEM_DIDX(g, s.n_geoms, 6);
  bool any = false;
  float best = 0.0f;
  const int ns = PLANAR ? s.bslab_n[g] : s.geom_nslab[g];
  for (int i = 0; i < ns; ++i) {
    // rounding pinned (no contraction choices left to the compiler): every
    // lane-group width evaluates a contact with the same operations
    float n0, n1, n2, sp, lo, hi;
    if (PLANAR) {
      const float4 sl = *reinterpret_cast<const float4*>(s.bslab[g][i]);
      n0 = sl.x;
      n1 = sl.y;
      n2 = 0.0f;
      sp = __fmaf_rn(n0, px, __fmul_rn(n1, py));
      lo = sl.z;
      hi = sl.w;
    } else {
      const float4 sl = *reinterpret_cast<const float4*>(s.oslab[g][i]);
      n0 = sl.x;
      n1 = sl.y;
      n2 = sl.z;
      sp = __fmaf_rn(n0, px, __fmaf_rn(n1, py, __fmul_rn(n2, pz)));
      lo = sl.w;
      hi = s.oslab[g][i][4];
    }
    const float ov_pos = __fsub_rn(hi, sp);
    const float ov_neg = __fsub_rn(sp, lo);
    if (ov_pos <= 0.0f || ov_neg <= 0.0f) return false;
    const float ov = fminf(ov_pos, ov_neg);
    if (!any || ov < best) {
      best = ov;
      any = true;
      const float sg = ov_pos <= ov_neg ? 1.0f : -1.0f;
      nx = sg * n0;
      ny = sg * n1;
      nz = sg * n2;
    }
  }
  depth = best;
  return any;
}

// A group of G consecutive lanes (G = 1, 8 or 32) sharing one rollout: every
// lane holds the same state and runs the same serial dynamics, the group
// splits the per-geometry contact queries and combines their results with
// warp shuffles.
template <int G>
struct Group {
  unsigned mask;  // the group's lanes
  int rank;       // this lane's index in the group
  __device__ __forceinline__ Group() {
    const int lane = threadIdx.x & 31;
    rank = lane & (G - 1);
    mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - rank));
  }
  __device__ __forceinline__ float from(float v, int src) const { return G == 1 ? v : __shfl_sync(mask, v, src, G); }
  __device__ __forceinline__ uint32_t any_bits(uint32_t v) const { return G == 1 ? v : __reduce_or_sync(mask, v); }
};

// position of the k-th (0-based) set bit of m
__device__ __forceinline__ int nth_bit(uint32_t m, int k) {
  for (int i = 0; i < k; ++i) m &= m - 1u;
  return __ffs(m) - 1;
}

// Penalty force on the base footprint from geometry g: F_n = max(0, k depth -
// c v_n) along the minimum-overlap normal, returned as (cx, cy) = F_n n.
__device__ __forceinline__ bool base_force(const DevScene& s, int g, float bx, float by, float bvx, float bvy,
                                           float kc, float cc, float& cx, float& cy) {
  float nx, ny, nz, dep;
  if (!slab_contact<true>(s, g, bx, by, 0.0f, nx, ny, nz, dep)) return false;
  const float vn = __fmaf_rn(bvx, nx, __fmul_rn(bvy, ny));
  const float Fn = fmaxf(0.0f, __fsub_rn(__fmul_rn(kc, dep), __fmul_rn(cc, vn)));
  cx = __fmul_rn(Fn, nx);
  cy = __fmul_rn(Fn, ny);
  return true;
}

// Normal and F_n of the object against geometry g (false: no overlap).
__device__ __forceinline__ bool obj_force(const DevScene& s, int g, float px, float py, float pz, float vx, float vy,
                                          float vz, float kc, float cc, float& nx, float& ny, float& nz, float& Fn) {
  float dep;
  if (!slab_contact<false>(s, g, px, py, pz, nx, ny, nz, dep)) return false;
  const float vn = __fmaf_rn(vx, nx, __fmaf_rn(vy, ny, __fmul_rn(vz, nz)));
  Fn = fmaxf(0.0f, __fsub_rn(__fmul_rn(kc, dep), __fmul_rn(cc, vn)));
  return true;
}

// Jacobi friction impulse of one of nc object contacts (normal n, force Fn)
// from the trial velocity v: the tangential velocity removed, capped by
// mu F_n dt; returned as the impulse per unit mass to subtract.  With t the
// tangential velocity and j = min(mu dt F_n, m |t| / nc) the impulse, the
// velocity change is (j / (m |t|)) t = min(mu dt F_n / (m |t|), 1 / nc) t,
// formed here from one reciprocal square root and no division.
// The object's friction and mass terms of one (possibly randomised)
// environment: cap = mu dt, its mass, dt / mass, 1 / mass.
struct ObjPhys {
  float cap, mo, dt_mo, inv_mo;
};

__device__ __forceinline__ bool obj_friction(const ObjPhys& op, float nx, float ny, float nz, float Fn, float vx,
                                             float vy, float vz, float inv_nc, float& cx, float& cy, float& cz) {
  const float vn = __fmaf_rn(vx, nx, __fmaf_rn(vy, ny, __fmul_rn(vz, nz)));
  const float tx = __fmaf_rn(-vn, nx, vx), ty = __fmaf_rn(-vn, ny, vy), tz = __fmaf_rn(-vn, nz, vz);
  const float vt2 = __fmaf_rn(tx, tx, __fmaf_rn(ty, ty, __fmul_rn(tz, tz)));
  if (!(vt2 > 0.0f)) return false;
  const float f = fminf(__fmul_rn(__fmul_rn(__fmul_rn(op.cap, Fn), op.inv_mo), rsqrtf(vt2)), inv_nc);
  cx = __fmul_rn(f, tx);
  cy = __fmul_rn(f, ty);
  cz = __fmul_rn(f, tz);
  return true;
}

// Neighbour list of an axis-aligned mover (half sizes hx, hy, hz at p):
// the geometries whose gap to the mover along every world axis they list is
// below `skin`.  A geometry left out has a gap >= skin along some world axis;
// while the mover has moved less than skin along every axis since the build
// that gap stays positive, so the geometry is still separated and its
// contact test would return no contact.  PLANAR: base footprint (x, y only).
// A lane group splits the geometries (lane r tests g = r, r + G, ...) and
// ORs the bits.
template <bool PLANAR, int G>
__device__ __forceinline__ uint32_t near_list(const DevScene& s, int n_geoms, float px, float py, float pz, float hx,
                                              float hy, float hz, float skin, const Group<G>& grp) {
  uint32_t m = 0;
  const int flag = PLANAR ? 1 : 2;
  for (int g = grp.rank; g < n_geoms; g += G) {
    if (!(s.geom_flags[g] & flag)) continue;
    bool far = false;
    const int ns = s.geom_nslab[g];
    for (int i = 0; i < ns && !far; ++i) {
      const float* sl = s.slab[g][i];
      float p, r;
      if (sl[0] == 1.0f && sl[1] == 0.0f && sl[2] == 0.0f) {
        p = px;
        r = hx;
      } else if (sl[0] == 0.0f && sl[1] == 1.0f && sl[2] == 0.0f) {
        p = py;
        r = hy;
      } else if (!PLANAR && sl[0] == 0.0f && sl[1] == 0.0f && sl[2] == 1.0f) {
        p = pz;
        r = hz;
      } else {
        continue;
      }
      far = fmaxf(sl[3] - (p + r), (p - r) - sl[4]) >= skin;
    }
    if (!far) m |= 1u << g;
  }
  return grp.any_bits(m);
}

// Sum of the base's contact forces over the neighbour list `nbr`, added to
// (fx, fy) in ascending geometry order.  G > 1: the k-th neighbour belongs to
// lane k % G, which evaluates it; the sum then takes each contacting
// geometry's force from its owner lane, in the same order and with the same
// roundings as one lane alone.
template <int G>
__device__ __forceinline__ void base_contacts(const DevScene& s, uint32_t nbr, float bx, float by, float bvx,
                                              float bvy, float kc, float cc, const Group<G>& grp, float& fx,
                                              float& fy) {
  if (G == 1) {
    for (uint32_t m = nbr; m; m &= m - 1u) {
      float cx, cy;
      if (base_force(s, __ffs(m) - 1, bx, by, bvx, bvy, kc, cc, cx, cy)) {
        fx = __fadd_rn(fx, cx);
        fy = __fadd_rn(fy, cy);
      }
    }
    return;
  }
  constexpr int SL = (CEM_MAX_GEOMS + G - 1) / G;
  float cx[SL], cy[SL];
  uint32_t hit = 0;
  const int nn = __popc(nbr);
#pragma unroll
  for (int j = 0; j < SL; ++j) {
    cx[j] = cy[j] = 0.0f;
    const int k = grp.rank + j * G;
    if (k < nn) {
      const int g = nth_bit(nbr, k);
      if (base_force(s, g, bx, by, bvx, bvy, kc, cc, cx[j], cy[j])) hit |= 1u << g;
    }
  }
  for (uint32_t m = grp.any_bits(hit); m; m &= m - 1u) {
    const int g = __ffs(m) - 1;
    const int k = __popc(nbr & ((1u << g) - 1u));
    const int j = k / G, src = k & (G - 1);
    float vx = cx[0], vy = cy[0];
#pragma unroll
    for (int i = 1; i < SL; ++i)
      if (j == i) {
        vx = cx[i];
        vy = cy[i];
      }
    fx = __fadd_rn(fx, grp.from(vx, src));
    fy = __fadd_rn(fy, grp.from(vy, src));
  }
}

// 1 / nc, the share of one of nc simultaneous contacts (exact for 1, 2, 4)
__device__ __forceinline__ float contact_share(int nc) {
  return nc == 1 ? 1.0f : nc == 2 ? 0.5f : __frcp_rn((float)nc);
}

// One object step against the static geometry in `nbr` (not attached):
// penalty forces from the pre-step state, the trial velocity with gravity,
// then one Jacobi friction impulse per contact from that trial velocity,
// each summed in ascending geometry order.  Updates the velocity only.
template <int G>
__device__ __forceinline__ void object_contacts(const DevScene& s, const ObjPhys& op, uint32_t nbr, float ox,
                                                float oy, float oz,
                                                float& ovx, float& ovy, float& ovz, float kc, float cc,
                                                const Group<G>& grp) {
  const float pvx = ovx, pvy = ovy, pvz = ovz;
  float fsx = 0.f, fsy = 0.f, fsz = 0.f;
  float jx = 0.f, jy = 0.f, jz = 0.f;
  if (G == 1) {
    // the first two contacts (in ascending geometry order) are kept for the
    // friction pass; a third or later one is evaluated again there
    uint32_t cm = 0;
    int nc = 0;
    float n0x = 0.f, n0y = 0.f, n0z = 0.f, F0 = 0.f, n1x = 0.f, n1y = 0.f, n1z = 0.f, F1 = 0.f;
    for (uint32_t m = nbr; m; m &= m - 1u) {
      const int g = __ffs(m) - 1;
      float nx, ny, nz, Fn;
      if (obj_force(s, g, ox, oy, oz, pvx, pvy, pvz, kc, cc, nx, ny, nz, Fn) && Fn > 0.0f) {
        if (nc == 0) {
          n0x = nx; n0y = ny; n0z = nz; F0 = Fn;
        } else if (nc == 1) {
          n1x = nx; n1y = ny; n1z = nz; F1 = Fn;
        }
        cm |= 1u << g;
        ++nc;
        fsx = __fadd_rn(fsx, __fmul_rn(Fn, nx));
        fsy = __fadd_rn(fsy, __fmul_rn(Fn, ny));
        fsz = __fadd_rn(fsz, __fmul_rn(Fn, nz));
      }
    }
    ovx = __fmaf_rn(op.dt_mo, fsx, pvx);
    ovy = __fmaf_rn(op.dt_mo, fsy, pvy);
    ovz = __fsub_rn(__fmaf_rn(op.dt_mo, fsz, pvz), __fmul_rn(s.g, s.dt));
    if (nc > 0) {
      const float inv_nc = contact_share(nc);
      float cx, cy, cz;
      if (obj_friction(op, n0x, n0y, n0z, F0, ovx, ovy, ovz, inv_nc, cx, cy, cz)) {
        jx = __fsub_rn(jx, cx);
        jy = __fsub_rn(jy, cy);
        jz = __fsub_rn(jz, cz);
      }
      if (nc > 1 && obj_friction(op, n1x, n1y, n1z, F1, ovx, ovy, ovz, inv_nc, cx, cy, cz)) {
        jx = __fsub_rn(jx, cx);
        jy = __fsub_rn(jy, cy);
        jz = __fsub_rn(jz, cz);
      }
      // contacts after the second (identical arithmetic to the first pass)
      uint32_t rest = cm;
      rest &= rest - 1u;
      rest &= rest - 1u;
      for (uint32_t m = rest; m; m &= m - 1u) {
        const int g = __ffs(m) - 1;
        float nx, ny, nz, Fn;
        obj_force(s, g, ox, oy, oz, pvx, pvy, pvz, kc, cc, nx, ny, nz, Fn);
        if (obj_friction(op, nx, ny, nz, Fn, ovx, ovy, ovz, inv_nc, cx, cy, cz)) {
          jx = __fsub_rn(jx, cx);
          jy = __fsub_rn(jy, cy);
          jz = __fsub_rn(jz, cz);
        }
      }
    }
  } else {
    constexpr int SL = (CEM_MAX_GEOMS + G - 1) / G;
    float nx[SL], ny[SL], nz[SL], Fn[SL];
    uint32_t hit = 0;
    const int nn = __popc(nbr);
#pragma unroll
    for (int j = 0; j < SL; ++j) {
      nx[j] = ny[j] = nz[j] = Fn[j] = 0.0f;
      const int k = grp.rank + j * G;
      if (k < nn) {
        const int g = nth_bit(nbr, k);
        if (obj_force(s, g, ox, oy, oz, pvx, pvy, pvz, kc, cc, nx[j], ny[j], nz[j], Fn[j]) && Fn[j] > 0.0f)
          hit |= 1u << g;
      }
    }
    const uint32_t cm = grp.any_bits(hit);
    const int nc = __popc(cm);
    const float inv_nc = contact_share(nc);
    // forces in ascending geometry order, each from its owner lane
    for (uint32_t m = cm; m; m &= m - 1u) {
      const int g = __ffs(m) - 1;
      const int k = __popc(nbr & ((1u << g) - 1u));
      const int j = k / G, src = k & (G - 1);
      float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
      for (int i = 0; i < SL; ++i)
        if (j == i) {
          a = __fmul_rn(Fn[i], nx[i]);
          b = __fmul_rn(Fn[i], ny[i]);
          c = __fmul_rn(Fn[i], nz[i]);
        }
      fsx = __fadd_rn(fsx, grp.from(a, src));
      fsy = __fadd_rn(fsy, grp.from(b, src));
      fsz = __fadd_rn(fsz, grp.from(c, src));
    }
    ovx = __fmaf_rn(op.dt_mo, fsx, pvx);
    ovy = __fmaf_rn(op.dt_mo, fsy, pvy);
    ovz = __fsub_rn(__fmaf_rn(op.dt_mo, fsz, pvz), __fmul_rn(s.g, s.dt));
    // friction: every owner evaluates its contacts, then the ordered sum
    float fx[SL], fy[SL], fz[SL];
    uint32_t fr = 0;
#pragma unroll
    for (int j = 0; j < SL; ++j) {
      fx[j] = fy[j] = fz[j] = 0.0f;
      const int k = grp.rank + j * G;
      if (k < nn) {
        const int g = nth_bit(nbr, k);
        if (((cm >> g) & 1u) && obj_friction(op, nx[j], ny[j], nz[j], Fn[j], ovx, ovy, ovz, inv_nc, fx[j], fy[j], fz[j]))
          fr |= 1u << g;
      }
    }
    for (uint32_t m = grp.any_bits(fr); m; m &= m - 1u) {
      const int g = __ffs(m) - 1;
      const int k = __popc(nbr & ((1u << g) - 1u));
      const int j = k / G, src = k & (G - 1);
      float a = fx[0], b = fy[0], c = fz[0];
#pragma unroll
      for (int i = 1; i < SL; ++i)
        if (j == i) {
          a = fx[i];
          b = fy[i];
          c = fz[i];
        }
      jx = __fsub_rn(jx, grp.from(a, src));
      jy = __fsub_rn(jy, grp.from(b, src));
      jz = __fsub_rn(jz, grp.from(c, src));
    }
  }
  ovx = __fadd_rn(ovx, jx);
  ovy = __fadd_rn(ovy, jy);
  ovz = __fadd_rn(ovz, jz);
}

// Analytic inverse kinematics of the 2-link arm in its vertical plane
// (elbow up), returning the plane's azimuth as (cos, sin) = (dx, dy) / |d|
// (what the forward kinematics uses; the angle itself only for traces).
// With s2 = sin q2 = -sqrt(1 - c2^2) and c2 = cos q2 no trigonometric call is
// needed for the elbow; for equal links the shoulder offset
// atan2(l2 s2, l1 + l2 c2) equals q2 / 2 (tangent half-angle identity).
// Targets out of reach are pulled onto the reachable shell.
template <bool WANT_ANGLE>
__device__ __forceinline__ void arm_ik(const DevScene& s, float bx, float by, float tx, float ty, float tz,
                                       float& beta, float& cbeta, float& sbeta, float& q1, float& q2) {
  const float dx = tx - bx, dy = ty - by;
  const float r2 = dx * dx + dy * dy;
  // horizontal reach and the plane's unit vector from one hardware
  // reciprocal square root (~2 ulp), no square root or division
  float rr = 0.0f;
  if (r2 > 0.0f) {
    const float inv = rsqrtf(r2);
    rr = r2 * inv;
    cbeta = dx * inv;
    sbeta = dy * inv;
  } else {
    cbeta = 1.0f;
    sbeta = 0.0f;
  }
  if (WANT_ANGLE) beta = atan2f(dy, dx);
  float zz = tz - s.arm_z;
  float rho2 = rr * rr + zz * zz;
  const float l1 = s.arm_l1, l2 = s.arm_l2;
  const float rmax = l1 + l2 - 1e-3f, rmin = fabsf(l1 - l2) + 1e-3f;
  if (rho2 > rmax * rmax) {  // pulled onto the reachable shell
    const float f = rmax * rsqrtf(rho2);
    rr *= f;
    zz *= f;
    rho2 = rmax * rmax;
  } else if (rho2 < rmin * rmin) {
    const float f = rmin * rsqrtf(fmaxf(rho2, 1e-18f));
    rr *= f;
    zz *= f;
    rho2 = rmin * rmin;
  }
  float c2 = (rho2 - (l1 * l1 + l2 * l2)) * __frcp_rn(2.0f * l1 * l2);
  c2 = fminf(fmaxf(c2, -1.0f), 1.0f);
  q2 = -acosf(c2);
  const float a = atan2f(zz, rr);
  if (l1 == l2) {
    q1 = a - 0.5f * q2;
  } else {
    const float s2 = -sqrtf(fmaxf(1.0f - c2 * c2, 0.0f));
    q1 = a - atan2f(l2 * s2, l1 + l2 * c2);
  }
}

// Forward kinematics.  Joint angles stay within (-pi, pi), where the
// hardware sine/cosine is accurate to ~5e-7 absolute (~2e-7 m at the end
// effector), far inside the per-step state tolerance.
struct ArmTrig {
  float s1, c1, s12, c12;  // sin / cos of q1 and of q1 + q2
};

__device__ __forceinline__ void arm_fk(const DevScene& s, float bx, float by, float cb, float sb, float q1, float q2,
                                       float& ex, float& ey, float& ez, ArmTrig* trig = nullptr) {
  float s1, c1, s12, c12;
  __sincosf(q1, &s1, &c1);
  __sincosf(q1 + q2, &s12, &c12);
  const float r = s.arm_l1 * c1 + s.arm_l2 * c12;
  ez = s.arm_z + s.arm_l1 * s1 + s.arm_l2 * s12;
  ex = bx + r * cb;
  ey = by + r * sb;
  if (trig) *trig = ArmTrig{s1, c1, s12, c12};
}

// End-effector velocity: the base's plus the arm's (the forward kinematics
// differentiated at fixed azimuth: dr/dt = -(l1 sin q1 dq1 + l2 sin(q1 + q2)
// (dq1 + dq2)), dz/dt = l1 cos q1 dq1 + l2 cos(q1 + q2) (dq1 + dq2)).  The
// azimuth is set kinematically when a grasp or place starts and has no rate.
__device__ __forceinline__ void arm_ee_velocity(const DevScene& s, const ArmTrig& t, float cb, float sb, float bvx,
                                                float bvy, float dq1, float dq2, float& vx, float& vy, float& vz) {
  const float w12 = dq1 + dq2;
  const float dr = -(s.arm_l1 * t.s1 * dq1 + s.arm_l2 * t.s12 * w12);
  vz = s.arm_l1 * t.c1 * dq1 + s.arm_l2 * t.c12 * w12;
  vx = bvx + dr * cb;
  vy = bvy + dr * sb;
}

// ASTAR = false compiles the A* base controller out (its waypoint arrays,
// planning calls and integral state): a scene with the PD base takes that
// instantiation everywhere (pickplace_any), which leaves the body without
// register spills and with a tenth of the stack.
template <int G, bool TRACE, bool ASTAR>
__device__ __noinline__ void pickplace_rollout(const DevScene& s, const float* __restrict__ row, int T, float smu,
                                               float sm, float& J_out, int& cls_out, float* tr) {
  const Group<G> grp;
  const float dt = s.dt, h = s.oh, eps2 = s.eps * s.eps;
  const float mb = s.mb, dt_mb = s.dt_mb, bcap = s.base_cap * smu, bcap2 = bcap * bcap;
  const ObjPhys op{s.obj_cap * smu, s.mo * sm, s.dt_mo / sm, 1.0f / (s.mo * sm)};
  const float kc = s.k_contact, cc = s.c_contact, akp = s.arm_kp, akd = s.arm_kd;
  const int n_geoms = s.n_geoms;
  float bx = s.base_start[0], by = s.base_start[1], bvx = s.base_v0[0], bvy = s.base_v0[1];
  float q1 = s.arm_home[0], q2 = s.arm_home[1], dq1 = 0.f, dq2 = 0.f, beta = 0.f;
  float cbeta = 1.0f, sbeta = 0.0f;
  float q1t = q1, q2t = q2;
  float ox = s.obj_start[0], oy = s.obj_start[1], oz = s.obj_start[2];
  float ovx = s.obj_v0[0], ovy = s.obj_v0[1], ovz = s.obj_v0[2];
  bool attached = false;
  float offx = 0.f, offy = 0.f, offz = 0.f;
  float ex, ey, ez;
  arm_fk(s, bx, by, cbeta, sbeta, q1, q2, ex, ey, ez);
  const int L = s.n_act;
  int a = 0, loaded = -1;
  float gx = bx, gy = by, kp = 0.f, kd = 0.f;
  float mgx = bx, mgy = by, mkp = 0.f, mkd = 0.f;
  float rx = 0.f, ry = 0.f, caz = 1.f, saz = 0.f, hgrip = 0.f, ptx = 0.f, pty = 0.f, ptz = 0.f;
  float t_done = (float)T * dt;
  // Neighbour lists (bit g = geometry g) and the positions they were built
  // at.  A warp rebuilds all its lanes' lists together as soon as one lane
  // needs it (rebuilding early is always valid), so the rebuild loop runs
  // once per event instead of once per lane.  A body left out is at least
  // kSkin away along some axis; a rebuild once any lane has moved kRebuild
  // keeps it at least 1 cm clear (far above FP32 rounding), and the later
  // the rebuild, the fewer of them a warp runs.
  constexpr float kSkin = 0.15f, kRebuild = 0.14f;
  const unsigned lanes = __activemask();
  // A* base controller: waypoints of the current moveTo, integral state
  const bool astar = ASTAR && s.base_ctrl != 0;
  float wpx[kMaxWaypoints], wpy[kMaxWaypoints];
  int nwp = 0, wi = 0;
  float Ix = 0.f, Iy = 0.f;
  bool need_plan = false;
  uint32_t bmask = 0, omask = 0;
  float brx = 1e30f, bry = 1e30f, orx = 1e30f, ory = 1e30f, orz = 1e30f;
  for (int step = 0; step < T; ++step) {
    const int ai = a < L ? a : L - 1;
    const int kind = s.act_kind[ai];
    if (ai != loaded) {
      const int o = s.act_off[ai];
      if (kind == CEM_ACT_MOVE) {
        mgx = s.act_nom[ai][0] + theta_at(s, row, o);
        mgy = s.act_nom[ai][1] + theta_at(s, row, o + 1);
        mkp = theta_at(s, row, o + 2);
        mkd = 2.0f * sqrtf(mkp);
        rx = s.act_ref[ai] ? mgx : s.act_nom[ai][0];
        ry = s.act_ref[ai] ? mgy : s.act_nom[ai][1];
        if (astar) {  // plan from where the base is now, below, with the whole warp's help
          need_plan = true;
          wi = 0;
          Ix = Iy = 0.f;
        }
      } else if (kind == CEM_ACT_GRASP) {
        sincosf(theta_at(s, row, o), &saz, &caz);
        hgrip = theta_at(s, row, o + 1);
        kp = s.grasp_kp;
        kd = 2.0f * sqrtf(kp);
      } else if (kind == CEM_ACT_PLACE) {
        ptx = s.act_nom[ai][0] + theta_at(s, row, o);
        pty = s.act_nom[ai][1] + theta_at(s, row, o + 1);
        ptz = s.act_nom[ai][2] + theta_at(s, row, o + 2);
      }
      loaded = ai;
    }
    if (astar) {
      // every lane that starts a moveTo this step gets its path in turn: all
      // lanes split its corner-visibility tests, then it runs A* on the masks
      // (the lanes of a lane group take their turns one by one, redundantly,
      // so every group width runs this same code)
      unsigned need = __ballot_sync(lanes, need_plan);
      while (need) {
        const int owner = __ffs(need) - 1;
        need &= need - 1u;
        const float sx = __shfl_sync(lanes, bx, owner), sy = __shfl_sync(lanes, by, owner);
        const float qx = __shfl_sync(lanes, mgx, owner), qy = __shfl_sync(lanes, mgy, owner);
        uint64_t ms, mg;
        corners_seen_warp(s, lanes, sx, sy, qx, qy, ms, mg);
        if ((int)(threadIdx.x & 31) == owner) nwp = astar_base_path(s, sx, sy, qx, qy, ms, mg, wpx, wpy);
      }
      need_plan = false;
    }
    float tx = 0.f, ty = 0.f, tz = 0.f;
    float fix = 0.f, fiy = 0.f;  // integral force per unit mass
    if (kind == CEM_ACT_MOVE) {
      gx = mgx;
      gy = mgy;
      kp = mkp;
      kd = mkd;
      if (astar) {
        // past every waypoint already within the switching radius
        while (wi < nwp - 1 && sqrtf((bx - wpx[wi]) * (bx - wpx[wi]) + (by - wpy[wi]) * (by - wpy[wi])) < s.wp_switch)
          ++wi;
        if (wi < nwp - 1) {  // an intermediate waypoint: PD towards it
          gx = wpx[wi];
          gy = wpy[wi];
          Ix = Iy = 0.f;
        } else {  // the goal: PID, integrating the error near it
          const float ex_ = mgx - bx, ey_ = mgy - by;
          if (sqrtf(ex_ * ex_ + ey_ * ey_) < s.pid_irad) {
            Ix = fminf(fmaxf(Ix + ex_ * dt, -s.pid_imax), s.pid_imax);
            Iy = fminf(fmaxf(Iy + ey_ * dt, -s.pid_imax), s.pid_imax);
          } else {
            Ix = Iy = 0.f;
          }
          fix = s.pid_ki * kp * Ix;
          fiy = s.pid_ki * kp * Iy;
        }
      }
    } else if (kind == CEM_ACT_GRASP) {
      tx = ox;
      ty = oy;
      tz = oz + hgrip;
      gx = ox - s.grasp_reach * caz;
      gy = oy - s.grasp_reach * saz;
    } else {
      tx = ptx;
      ty = pty;
      tz = ptz;
      gx = mgx;
      gy = mgy;
      kp = mkp;
      kd = mkd;
    }
    float d2_prev = 0.0f;  // squared distance to the action's target at t_k
    if (a < L) {
      if (kind == CEM_ACT_MOVE) d2_prev = (bx - rx) * (bx - rx) + (by - ry) * (by - ry);
      else d2_prev = (ex - tx) * (ex - tx) + (ey - ty) * (ey - ty) + (ez - tz) * (ez - tz);
    }
    if (kind != CEM_ACT_MOVE) arm_ik<TRACE>(s, bx, by, tx, ty, tz, beta, cbeta, sbeta, q1t, q2t);
    // base: PD + penalty contacts with the static footprints
    float fx = mb * (kp * (gx - bx) - kd * bvx);
    float fy = mb * (kp * (gy - by) - kd * bvy);
    if (astar && kind == CEM_ACT_MOVE) {
      fx += mb * fix;
      fy += mb * fiy;
    }
    if (__any_sync(lanes, fmaxf(fabsf(bx - brx), fabsf(by - bry)) >= kRebuild)) {
      bmask = near_list<true, G>(s, n_geoms, bx, by, 0.0f, s.bhx, s.bhy, 0.0f, kSkin, grp);
      brx = bx;
      bry = by;
    }
    base_contacts<G>(s, bmask, bx, by, bvx, bvy, kc, cc, grp, fx, fy);
    bvx += dt_mb * fx;
    bvy += dt_mb * fy;
    {  // ground friction of the base (yaw is locked)
      const float v2 = bvx * bvx + bvy * bvy;
      const float f = v2 > bcap2 ? 1.0f - bcap * rsqrtf(v2) : 0.0f;
      bvx *= f;
      bvy *= f;
    }
    bx += bvx * dt;
    by += bvy * dt;
    // arm joints
    const float dd1 = akp * (q1t - q1) - akd * dq1;
    const float dd2 = akp * (q2t - q2) - akd * dq2;
    dq1 += dt * dd1;
    dq2 += dt * dd2;
    q1 += dt * dq1;
    q2 += dt * dq2;
    float nex, ney, nez;
    ArmTrig trig;
    arm_fk(s, bx, by, cbeta, sbeta, q1, q2, nex, ney, nez, &trig);
    // object (a warp-wide rebuild of the object lists, see above)
    const bool orebuild = __any_sync(
        lanes, !attached && fmaxf(fmaxf(fabsf(ox - orx), fabsf(oy - ory)), fabsf(oz - orz)) >= kRebuild);
    if (attached) {
      ox = nex + offx;
      oy = ney + offy;
      oz = nez + offz;
      arm_ee_velocity(s, trig, cbeta, sbeta, bvx, bvy, dq1, dq2, ovx, ovy, ovz);
    } else {
      if (orebuild) {
        omask = near_list<false, G>(s, n_geoms, ox, oy, oz, h, h, h, kSkin, grp);
        orx = ox;
        ory = oy;
        orz = oz;
      }
      object_contacts<G>(s, op, omask, ox, oy, oz, ovx, ovy, ovz, kc, cc, grp);
      ox += ovx * dt;
      oy += ovy * dt;
      oz += ovz * dt;
    }
    if (a < L) {
      float d2_new;
      if (kind == CEM_ACT_MOVE) d2_new = (bx - rx) * (bx - rx) + (by - ry) * (by - ry);
      else d2_new = (nex - tx) * (nex - tx) + (ney - ty) * (ney - ty) + (nez - tz) * (nez - tz);
      bool ok = d2_new <= eps2;
      if (kind == CEM_ACT_GRASP) ok = ok && fabsf(hgrip) <= s.grip_tol;
      if (ok) {
        const float ts = success_time(s, step, sqrtf(d2_prev), sqrtf(d2_new));
        if (a == L - 1) t_done = ts;
        if (kind == CEM_ACT_GRASP) {
          attached = true;
          offx = ox - nex;
          offy = oy - ney;
          offz = oz - nez;
        } else if (kind == CEM_ACT_PLACE) {
          attached = false;
        }
        ++a;
      }
    }
    ex = nex;
    ey = ney;
    ez = nez;
    if (TRACE) {
      const float v[20] = {bx,  by,  bvx, bvy, q1,  q2,  dq1, dq2, beta, ox,
                           oy,  oz,  ovx, ovy, ovz, attached ? 1.f : 0.f, (float)a, ex, ey, ez};
      put_trace(tr, step, v, 20);
    }
  }
  const bool complete = a == L;
  bool goal = true;
  float d_obj = 0.f, d_base = 0.f;
  if (s.goal_obj_region) {
    const float e0 = fabsf(ox - s.obj_region_c[0]), e1 = fabsf(oy - s.obj_region_c[1]),
                e2 = fabsf(oz - s.obj_region_c[2]);
    goal = goal && !attached && e0 <= s.obj_region_h[0] && e1 <= s.obj_region_h[1] && e2 <= s.obj_region_h[2];
    const float x0 = fmaxf(e0 - s.obj_region_h[0], 0.f), x1 = fmaxf(e1 - s.obj_region_h[1], 0.f),
                x2 = fmaxf(e2 - s.obj_region_h[2], 0.f);
    d_obj = sqrtf(x0 * x0 + x1 * x1 + x2 * x2);
  }
  if (s.goal_obj_held) {
    goal = goal && attached;
    d_obj = attached ? 0.f : 1.f;
  }
  if (s.goal_base_region) {
    const float e0 = fabsf(bx - s.base_region_c[0]), e1 = fabsf(by - s.base_region_c[1]);
    goal = goal && e0 <= s.base_region_h[0] && e1 <= s.base_region_h[1];
    const float x0 = fmaxf(e0 - s.base_region_h[0], 0.f), x1 = fmaxf(e1 - s.base_region_h[1], 0.f);
    d_base = sqrtf(x0 * x0 + x1 * x1);
  }
  const float J = s.w_time * t_done + s.w_obj * d_obj + s.w_base * d_base;
  J_out = J;
  cls_out = complete ? (goal ? 0 : 1) : 2;
  if (!isfinite(J)) cls_out = 3;
}

// Every launch picks the instantiation by the scene's base controller, so a
// given scene runs the same compiled rollout in the single-problem, batched,
// randomised and traced kernels (and results stay bit-identical across them).
template <int G, bool TRACE>
__device__ __forceinline__ void pickplace_any(const DevScene& s, const float* __restrict__ row, int T, float smu,
                                              float sm, float& J_out, int& cls_out, float* tr) {
  if (s.base_ctrl) pickplace_rollout<G, TRACE, true>(s, row, T, smu, sm, J_out, cls_out, tr);
  else pickplace_rollout<G, TRACE, false>(s, row, T, smu, sm, J_out, cls_out, tr);
}

__device__ __noinline__ void quadratic_cost(const DevScene& s, const float* __restrict__ row, float& J_out, int& cls_out) {
  float e[CEM_MAX_D];
#pragma unroll
  for (int i = 0; i < CEM_MAX_D; ++i) e[i] = i < s.D ? theta_at(s, row, i) - s.theta_star[i] : 0.0f;
  float J = 0.0f;
#pragma unroll
  for (int i = 0; i < CEM_MAX_D; ++i) {
    if (i < s.D) {
      float ri = 0.0f;
#pragma unroll
      for (int j = 0; j < CEM_MAX_D; ++j)
        if (j < s.D) ri += s.A[i * s.D + j] * e[j];
      J += e[i] * ri;
    }
  }
  J_out = J;
  cls_out = isfinite(J) ? 0 : 3;
}

__device__ __forceinline__ void stage_scene(const DevScene* __restrict__ g, DevScene& sh) {
  const int words = (int)(sizeof(DevScene) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(g);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sh);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Occupancy: the planar rollouts fit 80 registers without spilling, so three
// 256-thread CTAs share an SM (12 % faster at N = 196,608 than two); the
// pick-and-place rollout keeps 128 registers (two CTAs): given more it takes
// ~150, and its small CTAs then no longer fit one wave at N = 16384
template <int KIND>
constexpr int rollout_min_ctas() {
  return KIND == CEM_SCENE_PICKPLACE ? 2 : 3;
}

// One rollout per group of G lanes (G > 1 only for pick-and-place); the
// group's first lane writes the result.
template <int KIND, bool TRACE, int G, bool AS = true>
__global__ void __launch_bounds__(256, rollout_min_ctas<KIND>()) rollout_kernel(const DevScene* __restrict__ scene_g,
                                                                                const float* __restrict__ theta, int N,
                                                                                int steps,
                                                      float* __restrict__ J, uint8_t* __restrict__ cls,
                                                      float* __restrict__ trace) {
  __shared__ DevScene s;
  stage_scene(scene_g, s);
  const int n = (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
  if (n >= N) return;
  const float* row = theta + (size_t)n * s.D;
  float* tr = TRACE ? trace + (size_t)n * steps * TW : nullptr;
  const int T = TRACE ? steps : s.T;
  float Jn;
  int c;
  if (KIND == CEM_SCENE_REACH) planar_rollout<false, TRACE>(s, row, T, 1.0f, 1.0f, Jn, c, tr);
  else if (KIND == CEM_SCENE_PUSH) planar_rollout<true, TRACE>(s, row, T, 1.0f, 1.0f, Jn, c, tr);
  else if (KIND == CEM_SCENE_PICKPLACE) {
    if (AS) pickplace_any<G, TRACE>(s, row, T, 1.0f, 1.0f, Jn, c, tr);
    else pickplace_rollout<G, TRACE, false>(s, row, T, 1.0f, 1.0f, Jn, c, tr);  // the scene has the PD base
  }
  else quadratic_cost(s, row, Jn, c);
  if (!TRACE && (G == 1 || (threadIdx.x & (G - 1)) == 0)) {
    J[n] = Jn;
    cls[n] = (uint8_t)c;
  }
}

// Domain-randomised rollouts: M consecutive lanes (M a power of two <= 32)
// roll one sample out in the M environments of the iteration, then combine
// by shuffles: the mean cost (an xor-butterfly sum, identical in every lane)
// and the worst class; the group's first lane writes.
template <int KIND>
__global__ void __launch_bounds__(256, rollout_min_ctas<KIND>()) rollout_dr_kernel(const DevScene* __restrict__ scene_g,
                                                         const float* __restrict__ theta, int N,
                                                         float* __restrict__ J, uint8_t* __restrict__ cls,
                                                         const DrArgs dr) {
  __shared__ DevScene s;
  stage_scene(scene_g, s);
  const int M = dr.M;
  const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int n = t / M, m = t & (M - 1);
  if (n >= N) return;  // all M lanes of a sample leave together
  const uint32_t it = dr.iter_ptr ? *dr.iter_ptr : dr.iter;
  uint32_t r[4];
  philox4x32_10((uint32_t)m, 256u, it, dr.problem, (uint32_t)dr.seed, (uint32_t)(dr.seed >> 32), r);
  const float smu = fmaf(dr.dmu, fmaf(2.0f, u01(r[0]), -1.0f), 1.0f);
  const float sm = fmaf(dr.dm, fmaf(2.0f, u01(r[1]), -1.0f), 1.0f);
  const float* row = theta + (size_t)n * s.D;
  float Jn;
  int c;
  if (KIND == CEM_SCENE_REACH) planar_rollout<false, false>(s, row, s.T, smu, sm, Jn, c, nullptr);
  else if (KIND == CEM_SCENE_PUSH) planar_rollout<true, false>(s, row, s.T, smu, sm, Jn, c, nullptr);
  else pickplace_any<1, false>(s, row, s.T, smu, sm, Jn, c, nullptr);
  const int lane = threadIdx.x & 31;
  const unsigned gmask = M == 32 ? 0xffffffffu : (((1u << M) - 1u) << (lane & ~(M - 1)));
  for (int o = 1; o < M; o <<= 1) {
    Jn += __shfl_xor_sync(gmask, Jn, o);
    c = max(c, __shfl_xor_sync(gmask, c, o));
  }
  if (m == 0) {
    const float mean = Jn * (1.0f / (float)M);
    J[n] = mean;
    cls[n] = (uint8_t)(isfinite(mean) ? c : 3);
  }
}

template <bool TRACE>
cudaError_t dispatch(const DevScene* s_d, int kind, const float* theta, int N, int steps, float* J, uint8_t* cls,
                     float* trace, int block, int tpr, cudaStream_t st, bool astar) {
  if (N <= 0) return cudaSuccess;
  if (block <= 0) block = 128;
  const int grid = (N + block - 1) / block;
  switch (kind) {
    case CEM_SCENE_QUADRATIC:
      rollout_kernel<CEM_SCENE_QUADRATIC, TRACE, 1><<<grid, block, 0, st>>>(s_d, theta, N, steps, J, cls, trace);
      break;
    case CEM_SCENE_REACH:
      rollout_kernel<CEM_SCENE_REACH, TRACE, 1><<<grid, block, 0, st>>>(s_d, theta, N, steps, J, cls, trace);
      break;
    case CEM_SCENE_PUSH:
      rollout_kernel<CEM_SCENE_PUSH, TRACE, 1><<<grid, block, 0, st>>>(s_d, theta, N, steps, J, cls, trace);
      break;
    case CEM_SCENE_PICKPLACE:
      if (!TRACE && (tpr == 8 || tpr == 32)) {
        // block threads: a multiple of 32 carrying block / tpr rollouts
        const int bt = block < 32 ? 32 : block;
        const long long threads = (long long)N * tpr;
        const int g2 = (int)((threads + bt - 1) / bt);
        if (tpr == 8)
          rollout_kernel<CEM_SCENE_PICKPLACE, false, 8><<<g2, bt, 0, st>>>(s_d, theta, N, steps, J, cls, trace);
        else
          rollout_kernel<CEM_SCENE_PICKPLACE, false, 32><<<g2, bt, 0, st>>>(s_d, theta, N, steps, J, cls, trace);
      } else if (astar) {
        rollout_kernel<CEM_SCENE_PICKPLACE, TRACE, 1><<<grid, block, 0, st>>>(s_d, theta, N, steps, J, cls, trace);
      } else {
        rollout_kernel<CEM_SCENE_PICKPLACE, TRACE, 1, false><<<grid, block, 0, st>>>(s_d, theta, N, steps, J, cls, trace);
      }
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Rollout order of a batch (a schedule, not arithmetic): the persistent
// kernel rolls sample perm[k] out on the lane that takes position k, so
// samples that will be in the same action at the same time share a warp
// and its lanes take the same branches.  For a pick-and-place problem with
// the PD base controller the samples are grouped by a cheap forecast from
// theta: first those whose first moveTo can end (its target lies outside
// every obstacle footprint grown by the base, and its gain exceeds mu g /
// eps, below which the PD law stalls short of the target), then those
// whose grip height lies within the grasp tolerance (they can grasp), then
// by the first moveTo's gain (how soon they arrive) in 256 steps over its
// range; every other problem keeps the identity.  One CTA per problem, a
// counting sort over the 1024 forecast bins with shared-memory atomics (the
// order inside a bin may differ from run to run; each sample's result is
// the same wherever it runs).
constexpr int kOrderBins = 1024;
constexpr int kOrderThreads = 1024;
constexpr int kOrderKeep = 8192;

__global__ void __launch_bounds__(kOrderThreads, 1) order_batch_kernel(const DevScene* __restrict__ scenes,
                                                                    const BatchProblem* __restrict__ probs,
                                                                    const float* __restrict__ theta,
                                                                    int32_t* __restrict__ perm) {
  __shared__ int count[kOrderBins];
  __shared__ uint16_t sbin[kOrderKeep];  // the bins of the first kOrderKeep samples, between the two passes
  const BatchProblem pb = probs[blockIdx.x];
  int32_t* out = perm + pb.sample_off;
  const DevScene& s = scenes[blockIdx.x];
  int grasp = -1, first_move = -1;
  if (s.kind == CEM_SCENE_PICKPLACE && s.base_ctrl == 0)
    for (int i = 0; i < s.n_act; ++i) {
      if (first_move < 0 && s.act_kind[i] == CEM_ACT_MOVE) first_move = i;
      if (grasp < 0 && s.act_kind[i] == CEM_ACT_GRASP) grasp = i;
    }
  if (!pb.active || grasp < 0 || first_move < 0) {
    for (int k = threadIdx.x; k < pb.N; k += blockDim.x) out[k] = k;
    return;
  }
  const int gi = s.act_off[grasp] + 1, mo = s.act_off[first_move], ki = mo + 2;
  const float tol = s.grip_tol, klo = s.lo[ki], kspan = s.hi[ki] - s.lo[ki];
  const float kscale = kspan > 0.0f ? 255.0f / kspan : 0.0f;
  const float kp_stall = s.base_cap / (s.dt * s.eps);  // mu g / eps
  auto bin_of = [&](int k) {
    const float* row = theta + pb.theta_off + (size_t)k * pb.D;
    const float grip = fminf(fmaxf(row[gi], s.lo[gi]), s.hi[gi]);
    const float kp = fminf(fmaxf(row[ki], klo), s.hi[ki]);
    const float tx = s.act_nom[first_move][0] + fminf(fmaxf(row[mo], s.lo[mo]), s.hi[mo]);
    const float ty = s.act_nom[first_move][1] + fminf(fmaxf(row[mo + 1], s.lo[mo + 1]), s.hi[mo + 1]);
    bool never = kp < kp_stall;
    for (int g = 0; g < s.n_geoms && !never; ++g) {
      if (!(s.geom_flags[g] & 1) || s.bslab_n[g] == 0) continue;
      bool inside = true;
      for (int j = 0; j < s.bslab_n[g] && inside; ++j) {
        const float v = s.bslab[g][j][0] * tx + s.bslab[g][j][1] * ty;
        inside = v >= s.bslab[g][j][2] && v <= s.bslab[g][j][3];
      }
      never = inside;
    }
    return (never ? 512 : 0) + (fabsf(grip) <= tol ? 0 : 256) + (int)fminf((kp - klo) * kscale, 255.0f);
  };
  for (int b = threadIdx.x; b < kOrderBins; b += blockDim.x) count[b] = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < pb.N; k += blockDim.x) {
    const int b = bin_of(k);
    if (k < kOrderKeep) sbin[k] = (uint16_t)b;
    atomicAdd(&count[b], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive prefix sum: each lane 32 consecutive bins
    const int lane = threadIdx.x;
    int v[kOrderBins / 32], sum = 0;
#pragma unroll
    for (int i = 0; i < kOrderBins / 32; ++i) {
      v[i] = sum;
      sum += count[lane * (kOrderBins / 32) + i];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int base = incl - sum;
#pragma unroll
    for (int i = 0; i < kOrderBins / 32; ++i) count[lane * (kOrderBins / 32) + i] = base + v[i];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < pb.N; k += blockDim.x)
    out[CEM_DIDX(atomicAdd(&count[CEM_DIDX(k < kOrderKeep ? (int)sbin[k] : bin_of(k), kOrderBins, 4)], 1), pb.N, 3)] = k;
}

// Persistent batched rollout: every warp of a resident CTA repeatedly takes
// the next (problem, 32-sample chunk) item from a global queue and rolls the
// chunk out with that problem's scene, staged in the warp's own shared-memory
// slot (reloaded only when the problem changes).  Items come longest horizon
// first, so the tail of the queue is short work.  There are no waits between
// warps or CTAs: a warp that finds the queue empty exits.
constexpr int kMaxBatchWarps = 8;

// The batched pick-and-place rollout: AS = false (a batch without an A*
// base controller) keeps the A* instantiation out of the kernel altogether,
// which made the batch 2-3 % faster than calling it through pickplace_any;
// either way a problem runs the instantiation its single-problem solve runs.
template <int G, bool AS>
__device__ __forceinline__ void pickplace_batch(const DevScene& s, const float* __restrict__ row, float smu, float sm,
                                                float& J_out, int& cls_out) {
  if (AS) pickplace_any<G, false>(s, row, s.T, smu, sm, J_out, cls_out, nullptr);
  else pickplace_rollout<G, false, false>(s, row, s.T, smu, sm, J_out, cls_out, nullptr);
}

template <int G, bool AS>
__global__ void __launch_bounds__(256) rollout_persistent_kernel(const DevScene* __restrict__ scenes,
                                                                 const BatchProblem* __restrict__ probs,
                                                                 const BatchItem* __restrict__ items, int n_items,
                                                                 int* __restrict__ counter,
                                                                 const float* __restrict__ theta,
                                                                 float* __restrict__ J, uint8_t* __restrict__ cls,
                                                                 const Track* __restrict__ tracks, const DrArgs dr,
                                                                 const int32_t* __restrict__ perm,
                                                                 const int32_t* __restrict__ dorder,
                                                                 uint32_t* __restrict__ idur) {
  extern __shared__ __align__(16) unsigned char psm[];  // one DevScene per warp
  DevScene* sc = reinterpret_cast<DevScene*>(psm);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DevScene& s = sc[w];
  int cur = -1;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const int src_it = dorder ? CEM_DIDX(dorder[it], n_items, 1) : it;  // the dispatch order (longest item first)
    const BatchItem item = items[src_it];
    uint64_t t_item = 0;
    if (idur && lane == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_item));
    if (item.problem != cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(scenes + item.problem);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s);
      for (int i = lane; i < (int)(sizeof(DevScene) / 4); i += 32) dst[i] = src[i];
      __syncwarp();
      cur = item.problem;
    }
    const BatchProblem pb = probs[item.problem];
    if (dr.M > 0 && s.kind != CEM_SCENE_QUADRATIC) {
      // domain randomisation: the item's 32 samples in M passes, M lanes per
      // sample (one environment each, of the problem's current iteration),
      // combined as in the single-problem randomised kernel
      const int M = dr.M, per = 32 / M, m = lane & (M - 1);
      const uint32_t itn = tracks[item.problem].iter;
      const unsigned gmask = M == 32 ? 0xffffffffu : (((1u << M) - 1u) << (lane & ~(M - 1)));
      for (int sub = 0; sub < M; ++sub) {
        const int n = item.first + sub * per + lane / M;
        if (n < pb.N) {
          uint32_t r[4];
          philox4x32_10((uint32_t)m, 256u, itn, pb.problem, (uint32_t)dr.seed, (uint32_t)(dr.seed >> 32), r);
          const float smu = fmaf(dr.dmu, fmaf(2.0f, u01(r[0]), -1.0f), 1.0f);
          const float sm = fmaf(dr.dm, fmaf(2.0f, u01(r[1]), -1.0f), 1.0f);
          const float* row = theta + pb.theta_off + (size_t)n * pb.D;
          float Jn;
          int c;
          switch (s.kind) {
            case CEM_SCENE_REACH: planar_rollout<false, false>(s, row, s.T, smu, sm, Jn, c, nullptr); break;
            case CEM_SCENE_PUSH: planar_rollout<true, false>(s, row, s.T, smu, sm, Jn, c, nullptr); break;
            default: pickplace_batch<1, AS>(s, row, smu, sm, Jn, c); break;
          }
          for (int o = 1; o < M; o <<= 1) {
            Jn += __shfl_xor_sync(gmask, Jn, o);
            c = max(c, __shfl_xor_sync(gmask, c, o));
          }
          if (m == 0) {
            const float mean = Jn * (1.0f / (float)M);
            J[pb.sample_off + n] = mean;
            cls[pb.sample_off + n] = (uint8_t)(isfinite(mean) ? c : 3);
          }
        }
        __syncwarp();
      }
    } else if (G > 1 && s.kind == CEM_SCENE_PICKPLACE) {
      // G lanes per rollout: the 32-sample item in G passes of 32 / G
      for (int sub = 0; sub < G; ++sub) {
        const int k = item.first + sub * (32 / G) + lane / G;
        if (k < pb.N) {
          const int n = perm ? CEM_DIDX(perm[pb.sample_off + k], pb.N, 2) : k;
          const float* row = theta + pb.theta_off + (size_t)n * pb.D;
          float Jn;
          int c;
          pickplace_batch<G, AS>(s, row, 1.0f, 1.0f, Jn, c);
          if ((lane & (G - 1)) == 0) {
            J[pb.sample_off + n] = Jn;
            cls[pb.sample_off + n] = (uint8_t)c;
          }
        }
        __syncwarp();
      }
    } else {
      const int k = item.first + lane;
      if (k < pb.N) {
        const int n = perm ? CEM_DIDX(perm[pb.sample_off + k], pb.N, 2) : k;
        const float* row = theta + pb.theta_off + (size_t)n * pb.D;
        float Jn;
        int c;
        switch (s.kind) {
          case CEM_SCENE_REACH: planar_rollout<false, false>(s, row, s.T, 1.0f, 1.0f, Jn, c, nullptr); break;
          case CEM_SCENE_PUSH: planar_rollout<true, false>(s, row, s.T, 1.0f, 1.0f, Jn, c, nullptr); break;
          case CEM_SCENE_PICKPLACE: pickplace_batch<1, AS>(s, row, 1.0f, 1.0f, Jn, c); break;
          default: quadratic_cost(s, row, Jn, c); break;
        }
        J[pb.sample_off + n] = Jn;
        cls[pb.sample_off + n] = (uint8_t)c;
      }
    }
    __syncwarp();
    if (idur && lane == 0) {  // running average of this item's duration (128 ns units): the next dispatch
      uint64_t t_end;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
      const uint32_t d = (uint32_t)min((t_end - t_item) >> 7, (uint64_t)0x7fffffffu);
      idur[src_it] = (idur[src_it] >> 1) + (d >> 1);
    }
  }
}

}  // namespace

#ifdef CEM_DEBUG
CEM_DEBUG_STATUS_ACCESSOR(debug_status_rollout)

namespace {
__global__ void debug_selftest_kernel(int* out) {
  __shared__ int a[3];
  if (threadIdx.x == 0) {
    a[0] = a[1] = a[2] = 0;
    a[CEM_DIDX(5, 3, 99)] = 7;  // clamped to a[2]
    *out = a[2];
  }
}
}  // namespace

cudaError_t debug_selftest_rollout() {
  int* d = nullptr;
  cudaError_t e = dev_malloc(&d, sizeof(int));
  if (e != cudaSuccess) return e;
  debug_selftest_kernel<<<1, 32>>>(d);
  e = cudaGetLastError();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e == cudaSuccess && h != 7) e = cudaErrorUnknown;
  return e;
}
#endif

cudaError_t configure_rollout_batch() {
  const int bytes = (int)(sizeof(DevScene) * kMaxBatchWarps);
  cudaError_t e =
      cudaFuncSetAttribute(rollout_persistent_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rollout_persistent_kernel<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rollout_persistent_kernel<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rollout_persistent_kernel<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

int rollout_batch_max_ctas_per_sm(int warps, int tpr, bool astar) {
  int n = 0;
  cudaError_t e;
  const size_t smem = sizeof(DevScene) * (size_t)warps;
  if (tpr == 8)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_persistent_kernel<8, true>, warps * 32, smem);
  else if (tpr == 32)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_persistent_kernel<32, true>, warps * 32, smem);
  else if (astar)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_persistent_kernel<1, true>, warps * 32, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_persistent_kernel<1, false>, warps * 32, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_order_batch(const DevScene* scenes_d, const BatchProblem* probs_d, int n_problems,
                               const float* theta, int32_t* perm, cudaStream_t st) {
  if (n_problems <= 0) return cudaSuccess;
  order_batch_kernel<<<n_problems, kOrderThreads, 0, st>>>(scenes_d, probs_d, theta, perm);
  return cudaGetLastError();
}

// The dispatch order of a batch's work items (a schedule, not arithmetic):
// longest first by a duration forecast, so that the items the persistent
// kernel starts last are the short ones and its warps finish together.
// The forecast of an item is the larger of its own recorded duration (a
// running average over CE iterations, or a static estimate before the
// first) and its problem's mean item duration (steadier: an item's samples
// are redrawn every iteration); erring long costs nothing, since only an
// item that runs longer than forecast and starts late lengthens the launch.  One CTA, a counting sort over 1024 bins of
// 16.4 us (the last bin holds everything longer), longest bin first; the
// order inside a bin may differ from run to run.
constexpr int kDispatchBins = 1024;
constexpr int kDispatchProblems = 256;  // problems per batch the mean is kept for (more share slots)

__global__ void __launch_bounds__(1024) dispatch_order_kernel(const uint32_t* __restrict__ idur,
                                                              const BatchItem* __restrict__ items, int n_items,
                                                              int32_t* __restrict__ dorder) {
  __shared__ int count[kDispatchBins];
  // per problem: summed durations in 2.05 us units and the item count.  A
  // slot holds at most 1024 / 256 problems of 2^20 / 32 items each, 2^17
  // items, so capping each item's share at 2^15 - 1 units (67 ms) keeps the
  // 32-bit sum from wrapping; only the problem mean sees the cap, and an item
  // that runs longer (many lanes or environments per sample) still sorts by
  // its own duration.
  constexpr uint32_t kShareCap = (1u << 15) - 1u;
  static_assert((uint64_t)kShareCap * (CEM_MAX_BATCH / kDispatchProblems) * (CEM_MAX_N / 32) < (1ull << 32),
                "problem duration sums must fit 32 bits");
  __shared__ uint32_t psum[kDispatchProblems];
  __shared__ int pcnt[kDispatchProblems];
  for (int b = threadIdx.x; b < kDispatchProblems; b += blockDim.x) {
    psum[b] = 0u;
    pcnt[b] = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_items; i += blockDim.x) {
    const int pr = items[i].problem % kDispatchProblems;
    atomicAdd(&psum[pr], min(idur[i] >> 4, kShareCap));
    atomicAdd(&pcnt[pr], 1);
  }
  __syncthreads();
  auto bin_of = [&](int i) {
    const int pr = items[i].problem % kDispatchProblems;
    const uint32_t mean = (psum[pr] / (uint32_t)max(pcnt[pr], 1)) << 4;
    const uint32_t key = max(mean, idur[i]);
    return kDispatchBins - 1 - (int)min(key >> 7, (uint32_t)(kDispatchBins - 1));
  };
  for (int b = threadIdx.x; b < kDispatchBins; b += blockDim.x) count[b] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_items; i += blockDim.x) atomicAdd(&count[bin_of(i)], 1);
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive prefix sum: each lane 32 consecutive bins
    const int lane = threadIdx.x;
    int v[kDispatchBins / 32], sum = 0;
#pragma unroll
    for (int i = 0; i < kDispatchBins / 32; ++i) {
      v[i] = sum;
      sum += count[lane * (kDispatchBins / 32) + i];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int base = incl - sum;
#pragma unroll
    for (int i = 0; i < kDispatchBins / 32; ++i) count[lane * (kDispatchBins / 32) + i] = base + v[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_items; i += blockDim.x)
    dorder[CEM_DIDX(atomicAdd(&count[CEM_DIDX(bin_of(i), kDispatchBins, 4)], 1), n_items, 5)] = i;
}

cudaError_t launch_dispatch_order(const uint32_t* idur, const BatchItem* items, int n_items, int32_t* dorder,
                                  cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  dispatch_order_kernel<<<1, 1024, 0, st>>>(idur, items, n_items, dorder);
  return cudaGetLastError();
}

cudaError_t launch_rollout_batch_persistent(const DevScene* scenes_d, const BatchProblem* probs_d,
                                            const BatchItem* items_d, int n_items, int* counter_d,
                                            const float* theta, float* J, uint8_t* cls, int grid, int warps,
                                            int tpr, const Track* tracks, const DrArgs* dr_in, cudaStream_t st,
                                            const int32_t* perm, const int32_t* dorder, uint32_t* idur,
                                            bool astar) {
  if (n_items <= 0) return cudaSuccess;
  if (warps < 1 || warps > kMaxBatchWarps || grid < 1) return cudaErrorInvalidValue;
  DrArgs dr{};  // M = 0: off
  if (dr_in) {
    if (dr_in->M < 1 || dr_in->M > 32 || (dr_in->M & (dr_in->M - 1)) || !tracks) return cudaErrorInvalidValue;
    dr = *dr_in;
  }
  if (tpr == 8)
    rollout_persistent_kernel<8, true><<<grid, warps * 32, sizeof(DevScene) * warps, st>>>(scenes_d, probs_d, items_d, n_items, counter_d, theta,
                                                             J, cls, tracks, dr, perm, dorder, idur);
  else if (tpr == 32)
    rollout_persistent_kernel<32, true><<<grid, warps * 32, sizeof(DevScene) * warps, st>>>(scenes_d, probs_d, items_d, n_items, counter_d, theta,
                                                              J, cls, tracks, dr, perm, dorder, idur);
  else if (tpr == 1 && astar)
    rollout_persistent_kernel<1, true><<<grid, warps * 32, sizeof(DevScene) * warps, st>>>(scenes_d, probs_d, items_d, n_items, counter_d, theta,
                                                             J, cls, tracks, dr, perm, dorder, idur);
  else if (tpr == 1)
    rollout_persistent_kernel<1, false><<<grid, warps * 32, sizeof(DevScene) * warps, st>>>(scenes_d, probs_d, items_d, n_items, counter_d, theta,
                                                             J, cls, tracks, dr, perm, dorder, idur);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_rollout(const DevScene* s_d, int kind, const float* theta, int N, float* J, uint8_t* cls,
                           int block, int tpr, const DrArgs* dr, cudaStream_t st, bool astar) {
  if (!dr || kind == CEM_SCENE_QUADRATIC)
    return dispatch<false>(s_d, kind, theta, N, 0, J, cls, nullptr, block, tpr, st, astar);
  if (N <= 0) return cudaSuccess;
  if (dr->M < 1 || dr->M > 32 || (dr->M & (dr->M - 1))) return cudaErrorInvalidValue;
  const int bt = block < 32 ? 32 : block;  // whole warps, so environment groups stay aligned
  const long long threads = (long long)N * dr->M;
  const int grid = (int)((threads + bt - 1) / bt);
  switch (kind) {
    case CEM_SCENE_REACH:
      rollout_dr_kernel<CEM_SCENE_REACH><<<grid, bt, 0, st>>>(s_d, theta, N, J, cls, *dr);
      break;
    case CEM_SCENE_PUSH:
      rollout_dr_kernel<CEM_SCENE_PUSH><<<grid, bt, 0, st>>>(s_d, theta, N, J, cls, *dr);
      break;
    case CEM_SCENE_PICKPLACE:
      rollout_dr_kernel<CEM_SCENE_PICKPLACE><<<grid, bt, 0, st>>>(s_d, theta, N, J, cls, *dr);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_trace(const DevScene* s_d, int kind, const float* theta, int N, int steps, float* states,
                         cudaStream_t st, bool astar) {
  return dispatch<true>(s_d, kind, theta, N, steps, nullptr, nullptr, states, 64, 1, st, astar);
}

}  // namespace cem
