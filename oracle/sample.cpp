// Oracle: Philox4x32-10 and the Gaussian sampling step of Algorithm 1
// ("Sample n_env(j) times Z_pi ~ phi(theta^j)", Sec. III-B).  Test
// infrastructure only.
//
// Philox4x32-10 follows Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3" (SC'11): a 4-word counter and 2-word key; each of the
// 10 rounds multiplies words 0 and 2 by the two Philox constants, swaps and
// xors the high halves with words 1, 3 and the round key; the key is bumped
// by the two Weyl constants between rounds.
//
// Counter layout (the paper names no RNG; this is the library's choice):
//   ctr = (sample n, call c, iteration j, problem p), key = seed (lo, hi).
// Uniform u = (r + 1) / 2^32 in (0, 1]; Box-Muller on consecutive pairs.
#include "oracle.h"
#include <cmath>
#include <cstring>
#include <vector>

static const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
static const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;

extern "C" void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)kMul0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)kMul1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (round < 9) { k0 += kWeyl0; k1 += kWeyl1; }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static int n_calls(int D) { return (D + 3) / 4; }

extern "C" void or_philox_words(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D,
                                uint32_t* words) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const int nc = n_calls(D);
  for (int n = 0; n < N; ++n)
    for (int c = 0; c < nc; ++c) {
      const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)c, iter, problem};
      or_philox4x32_10(ctr, key, words + ((size_t)n * nc + c) * 4);
    }
}

static double uniform_open0(uint32_t r) { return ((double)r + 1.0) * 0x1p-32; }

extern "C" void or_normals(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D, double* z) {
  const int nc = n_calls(D);
  std::vector<uint32_t> w((size_t)N * nc * 4);
  or_philox_words(seed, iter, problem, N, D, w.data());
  const double two_pi = 2.0 * M_PI;
  for (int n = 0; n < N; ++n) {
    const uint32_t* r = w.data() + (size_t)n * nc * 4;
    for (int d = 0; d < D; d += 2) {
      // pair (r[d], r[d+1]) -> (z_d, z_{d+1})
      double u1 = uniform_open0(r[d]);
      double u2 = uniform_open0(r[d + 1]);
      double rad = std::sqrt(-2.0 * std::log(u1));
      z[(size_t)n * D + d] = rad * std::cos(two_pi * u2);
      if (d + 1 < D) z[(size_t)n * D + d + 1] = rad * std::sin(two_pi * u2);
    }
  }
}

extern "C" void or_sample(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D,
                          const double* mean, const double* chol, double* theta) {
  std::vector<double> z((size_t)N * D);
  or_normals(seed, iter, problem, N, D, z.data());
  for (int n = 0; n < N; ++n)
    for (int i = 0; i < D; ++i) {
      double acc = mean[i];
      for (int j = 0; j <= i; ++j) acc += chol[i * D + j] * z[(size_t)n * D + j];
      theta[(size_t)n * D + i] = acc;
    }
}

// Iteration-0 rule of Sec. III-B / IV-A: uniform inside each parameter's
// region.  Uses the raw Philox words of iteration 0xFFFFFFFF so it never
// collides with a Gaussian iteration; word d serves parameter d.
//  * box: theta_d = lo_d + u_d (hi_d - lo_d);
//  * annulus r <= |p - c| <= R for a move goal p = nominal + (dx, dy):
//    uniform in area means P(|p - c| <= rho) = (rho^2 - r^2) / (R^2 - r^2), so
//    rho = sqrt(r^2 + u_d (R^2 - r^2)) and the angle is 2 pi u_{d+1}.
extern "C" void or_sample_uniform(const or_scene* s, uint64_t seed, uint32_t problem, int N,
                                  double* theta) {
  const int D = s->D, nc = n_calls(D);
  std::vector<uint32_t> w((size_t)N * nc * 4);
  or_philox_words(seed, 0xFFFFFFFFu, problem, N, D, w.data());
  for (int n = 0; n < N; ++n) {
    const uint32_t* r = w.data() + (size_t)n * nc * 4;
    double* th = theta + (size_t)n * D;
    for (int d = 0; d < D; ++d) th[d] = s->lo[d] + uniform_open0(r[d]) * (s->hi[d] - s->lo[d]);
    for (int a = 0; a < s->n_act; ++a) {
      if (s->act_region[a] != 1) continue;
      const int o = s->act_off[a];
      const double cx = s->act_ring[a][0], cy = s->act_ring[a][1];
      const double ri = s->act_ring[a][2], ro = s->act_ring[a][3];
      const double rho = std::sqrt(ri * ri + uniform_open0(r[o]) * (ro * ro - ri * ri));
      const double phi = 2.0 * M_PI * uniform_open0(r[o + 1]);
      th[o] = cx + rho * std::cos(phi) - s->act_nom[a][0];
      th[o + 1] = cy + rho * std::sin(phi) - s->act_nom[a][1];
    }
  }
}
