// Oracle: elite selection, distribution refit and the cross-entropy loop of
// Algorithm 1 (Sec. III-B).  FP64, plain loops.  Test infrastructure only.
//
// Readings of the paper used here (the paper is silent on each):
//  * ranking key (class, J, index) ascending; class 0 = every action
//    succeeded and psi_g(x_T) holds, 1 = every action succeeded but psi_g
//    fails (the fallback set of Sec. III-B), 2 = otherwise, 3 = non-finite J;
//  * elites come from the best class present among {0, 1}, at most N_e of
//    them ("if n_feasible < N_e only the n_feasible samples are used"); if
//    neither class occurs the N_e lowest-cost class-2 samples are used;
//  * update = maximum-likelihood Gaussian of the elites (the KL-minimising
//    CE update of Botev et al.): mean, covariance with 1/K_eff, plus a ridge
//    (1e-4 * range)^2 on the diagonal;
//  * a single elite ("add artificial noise"): covariance
//    diag((0.05 * range)^2) around it;
//  * the independent-normal model of Sec. IV-A is the diagonal mode;
//  * the returned best sample is the lowest key over all iterations.
#include "oracle.h"
#include <algorithm>
#include <cmath>
#include <vector>

namespace {
struct Key {
  int cls;
  float J;
  int idx;
};

bool key_less(const Key& a, const Key& b) {
  if (a.cls != b.cls) return a.cls < b.cls;
  if (a.J != b.J) return a.J < b.J;
  return a.idx < b.idx;
}

Key make_key(const float* J, const uint8_t* cls, int i) {
  Key k{cls[i], J[i], i};
  if (!std::isfinite(k.J)) { k.cls = 3; k.J = INFINITY; }
  if (k.cls > 3) k.cls = 3;
  return k;
}

// Lower Cholesky factor; false if a pivot is not positive.
bool cholesky(const double* A, int D, double* Lo) {
  for (int i = 0; i < D * D; ++i) Lo[i] = 0.0;
  for (int j = 0; j < D; ++j) {
    double s = A[j * D + j];
    for (int k = 0; k < j; ++k) s -= Lo[j * D + k] * Lo[j * D + k];
    if (!(s > 0.0)) return false;
    Lo[j * D + j] = std::sqrt(s);
    for (int i = j + 1; i < D; ++i) {
      double t = A[i * D + j];
      for (int k = 0; k < j; ++k) t -= Lo[i * D + k] * Lo[j * D + k];
      Lo[i * D + j] = t / Lo[j * D + j];
    }
  }
  return true;
}
}  // namespace

extern "C" int or_select(const float* J, const uint8_t* cls, int N, int K, int32_t* idx) {
  std::vector<Key> keys(N);
  int count[4] = {0, 0, 0, 0};
  for (int i = 0; i < N; ++i) {
    keys[i] = make_key(J, cls, i);
    ++count[keys[i].cls];
  }
  std::sort(keys.begin(), keys.end(), key_less);
  int c_star = count[0] > 0 ? 0 : count[1] > 0 ? 1 : count[2] > 0 ? 2 : -1;
  if (c_star < 0) return 0;
  int k_eff = std::min(K, count[c_star]);
  for (int i = 0; i < k_eff; ++i) idx[i] = keys[i].idx;
  return k_eff;
}

extern "C" int or_refit(const double* theta, int N, int D, const int32_t* idx, int k_eff, const double* lo,
                        const double* hi, int diag, double* mean, double* cov, double* chol) {
  (void)N;
  if (k_eff <= 0) return 0;  // nothing to learn from: keep the distribution
  std::vector<double> m(D, 0.0), C((size_t)D * D, 0.0);
  if (k_eff == 1) {
    for (int d = 0; d < D; ++d) {
      m[d] = theta[(size_t)idx[0] * D + d];
      double r = 0.05 * (hi[d] - lo[d]);
      C[d * D + d] = r * r;
    }
  } else {
    for (int e = 0; e < k_eff; ++e)
      for (int d = 0; d < D; ++d) m[d] += theta[(size_t)idx[e] * D + d];
    for (int d = 0; d < D; ++d) m[d] /= k_eff;
    for (int e = 0; e < k_eff; ++e) {
      const double* t = theta + (size_t)idx[e] * D;
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) C[i * D + j] += (t[i] - m[i]) * (t[j] - m[j]);
    }
    for (int i = 0; i < D * D; ++i) C[i] /= k_eff;
    for (int d = 0; d < D; ++d) {
      double r = 1e-4 * (hi[d] - lo[d]);
      C[d * D + d] += r * r;
    }
  }
  if (diag)
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j)
        if (i != j) C[i * D + j] = 0.0;
  std::vector<double> Lo((size_t)D * D);
  if (!cholesky(C.data(), D, Lo.data())) {
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j)
        if (i != j) C[i * D + j] = 0.0;
    if (!cholesky(C.data(), D, Lo.data())) return -4;
  }
  for (int d = 0; d < D; ++d) mean[d] = m[d];
  for (int i = 0; i < D * D; ++i) { cov[i] = C[i]; chol[i] = Lo[i]; }
  return 0;
}

extern "C" int or_cem(const or_scene* s, uint64_t seed, uint32_t problem, int N, int K, int iters, int diag,
                      int nthreads, double* best_theta, double* best_J, int* best_cls, double* mean,
                      double* cov, double* history, double* keff_hist) {
  const int D = s->D;
  std::vector<double> mu(D), C((size_t)D * D, 0.0), Lo((size_t)D * D, 0.0);
  for (int d = 0; d < D; ++d) {
    mu[d] = 0.5 * (s->lo[d] + s->hi[d]);
    double sd = 0.25 * (s->hi[d] - s->lo[d]);
    C[d * D + d] = sd * sd;
    Lo[d * D + d] = sd;
  }
  std::vector<double> th((size_t)N * D), J(N);
  std::vector<uint8_t> cl(N);
  std::vector<float> Jf(N);
  std::vector<int32_t> idx(std::max(K, 1));
  int bcls = 4;
  float bJf = INFINITY;
  double bJ = INFINITY;
  std::vector<double> bth(D, 0.0);
  for (int j = 0; j < iters; ++j) {
    or_sample(seed, (uint32_t)j, problem, N, D, mu.data(), Lo.data(), th.data());
    or_rollout(s, th.data(), N, J.data(), cl.data(), nthreads);
    for (int n = 0; n < N; ++n) Jf[n] = (float)J[n];
    int k_eff = or_select(Jf.data(), cl.data(), N, K, idx.data());
    if (k_eff > 0) {
      int b = idx[0];
      if (cl[b] < bcls || (cl[b] == bcls && Jf[b] < bJf)) {
        bcls = cl[b]; bJf = Jf[b]; bJ = J[b];
        for (int d = 0; d < D; ++d) bth[d] = th[(size_t)b * D + d];
      }
      int rc = or_refit(th.data(), N, D, idx.data(), k_eff, s->lo, s->hi, diag, mu.data(), C.data(), Lo.data());
      if (rc != 0) return rc;
    }
    if (history) history[j] = bJ;
    if (keff_hist) keff_hist[j] = k_eff;
  }
  for (int d = 0; d < D; ++d) { best_theta[d] = bth[d]; mean[d] = mu[d]; }
  for (int i = 0; i < D * D; ++i) cov[i] = C[i];
  *best_J = bJ;
  *best_cls = bcls;
  return 0;
}

// Linear sample-count schedule of Sec. IV-A, rounded to the nearest integer
// (halves up).
extern "C" int or_n_env(int n0, int n1, int j1, int j) {
  if (j1 <= 0 || j >= j1) return j1 <= 0 && j == 0 ? n0 : n1;
  const double v = (double)n0 + (double)(n1 - n0) * (double)j / (double)j1;
  return (int)std::floor(v + 0.5);
}

// The paper's variant of Algorithm 1 (Sec. III-B, IV-A): the initial
// distribution is uniform inside the parameter regions (iteration 0), the
// sampled batch shrinks by the schedule, and each later iteration samples
// the normal model refit from the previous elites.
extern "C" int or_cem_paper(const or_scene* s, uint64_t seed, uint32_t problem, int n0, int n1, int j1, int K,
                            int iters, int diag, int nthreads, double* best_theta, double* best_J, int* best_cls,
                            double* mean, double* cov, double* history, int* class_hist, int* n_hist) {
  const int D = s->D;
  const int nmax = std::max(n0, n1);
  std::vector<double> mu(D, 0.0), C((size_t)D * D, 0.0), Lo((size_t)D * D, 0.0);
  std::vector<double> th((size_t)nmax * D), J(nmax);
  std::vector<uint8_t> cl(nmax);
  std::vector<float> Jf(nmax);
  std::vector<int32_t> idx(std::max(K, 1));
  int bcls = 4;
  float bJf = INFINITY;
  double bJ = INFINITY;
  std::vector<double> bth(D, 0.0);
  for (int j = 0; j < iters; ++j) {
    const int N = or_n_env(n0, n1, j1, j);
    if (j == 0) or_sample_uniform(s, seed, problem, N, th.data());
    else or_sample(seed, (uint32_t)j, problem, N, D, mu.data(), Lo.data(), th.data());
    or_rollout(s, th.data(), N, J.data(), cl.data(), nthreads);
    for (int n = 0; n < N; ++n) Jf[n] = (float)J[n];
    const int k_eff = or_select(Jf.data(), cl.data(), N, K, idx.data());
    if (k_eff > 0) {
      const int b = idx[0];
      if (cl[b] < bcls || (cl[b] == bcls && Jf[b] < bJf)) {
        bcls = cl[b]; bJf = Jf[b]; bJ = J[b];
        for (int d = 0; d < D; ++d) bth[d] = th[(size_t)b * D + d];
      }
      const int rc = or_refit(th.data(), N, D, idx.data(), k_eff, s->lo, s->hi, diag, mu.data(), C.data(), Lo.data());
      if (rc != 0) return rc;
    } else if (j == 0) {
      return -4;  // no sample to start the normal model from
    }
    if (history) history[j] = bJ;
    if (n_hist) n_hist[j] = N;
    if (class_hist) {
      for (int c = 0; c < 4; ++c) class_hist[4 * j + c] = 0;
      for (int n = 0; n < N; ++n) class_hist[4 * j + cl[n]] += 1;
    }
  }
  for (int d = 0; d < D; ++d) { best_theta[d] = bth[d]; mean[d] = mu[d]; }
  for (int i = 0; i < D * D; ++i) cov[i] = C[i];
  *best_J = bJ;
  *best_cls = bcls;
  return 0;
}

// Algorithm 1 with domain-randomised evaluation: iteration j scores every
// sample by its mean cost (and worst class) over the M environments of
// iteration j; sampling, selection and refit are those of or_cem.
extern "C" int or_cem_dr(const or_scene* s, uint64_t seed, uint32_t problem, int N, int K, int iters, int diag,
                         int M, double dmu, double dm, uint64_t dr_seed, int nthreads, double* best_theta,
                         double* best_J, int* best_cls, double* mean, double* cov, double* history) {
  const int D = s->D;
  std::vector<double> mu(D), C((size_t)D * D, 0.0), Lo((size_t)D * D, 0.0);
  for (int d = 0; d < D; ++d) {
    mu[d] = 0.5 * (s->lo[d] + s->hi[d]);
    const double sd = 0.25 * (s->hi[d] - s->lo[d]);
    C[d * D + d] = sd * sd;
    Lo[d * D + d] = sd;
  }
  std::vector<double> th((size_t)N * D), J(N);
  std::vector<uint8_t> cl(N);
  std::vector<float> Jf(N);
  std::vector<int32_t> idx(std::max(K, 1));
  int bcls = 4;
  float bJf = INFINITY;
  double bJ = INFINITY;
  std::vector<double> bth(D, 0.0);
  for (int j = 0; j < iters; ++j) {
    or_sample(seed, (uint32_t)j, problem, N, D, mu.data(), Lo.data(), th.data());
    or_rollout_dr(s, th.data(), N, M, dmu, dm, dr_seed, (uint32_t)j, problem, J.data(), cl.data(), nthreads);
    for (int n = 0; n < N; ++n) Jf[n] = (float)J[n];
    const int k_eff = or_select(Jf.data(), cl.data(), N, K, idx.data());
    if (k_eff > 0) {
      const int b = idx[0];
      if (cl[b] < bcls || (cl[b] == bcls && Jf[b] < bJf)) {
        bcls = cl[b]; bJf = Jf[b]; bJ = J[b];
        for (int d = 0; d < D; ++d) bth[d] = th[(size_t)b * D + d];
      }
      const int rc = or_refit(th.data(), N, D, idx.data(), k_eff, s->lo, s->hi, diag, mu.data(), C.data(), Lo.data());
      if (rc != 0) return rc;
    }
    if (history) history[j] = bJ;
  }
  for (int d = 0; d < D; ++d) { best_theta[d] = bth[d]; mean[d] = mu[d]; }
  for (int i = 0; i < D * D; ++i) cov[i] = C[i];
  *best_J = bJ;
  *best_cls = bcls;
  return 0;
}
