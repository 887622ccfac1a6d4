// cem_solve_static: the device CE loop of cem_solve without any device
// allocation.
//
// Some callers cannot allocate device memory at the moment they want a plan:
// a controller running in a hard real-time loop, where cudaMalloc can block
// on the device or fail at an arbitrary moment; a plugin inside a host
// program that owns every byte of device memory through its own pool and
// forbids third-party allocations; or a process that has to run under a
// fixed memory cap decided at start-up.  This entry point serves them: it
// takes the scene and plan skeleton as host descriptors (no handle, whose
// creation allocates) and keeps every intermediate -- the prepared scene,
// the sampled parameters, costs, classes, the distribution and the loop
// state -- in one file-scope device array of fixed size.
//
// Properties callers must know:
//   - The array (kScratchBytes, 2 MiB) is part of the library image: every
//     GPU that loads the library holds it until the process exits.
//   - Every call looks up the array's device address for the current device
//     and opts the refit kernel into its shared memory (both are cheap host
//     calls after the first, and neither allocates), so a device reset,
//     which reloads the module at a possibly different address, needs no
//     special handling.  The first call on a device also loads the module;
//     make that first call before any stream capture on that device.
//   - If a launch fails after the call has started writing the array, the
//     call waits for the work it already queued before it returns the error,
//     so no kernel of a failed call still uses the array afterwards.
//   - All calls share the array and it keeps the previous call's contents;
//     the loop state is fully rewritten at the start of every call.  Calls
//     that overlap on the GPU (different streams or threads at once) race on
//     the array: serialise them.
//   - Limits: N * D <= 262144 parameters per batch (for example N = 16384 at
//     D = 16), iters <= 4096; larger requests fail with CEM_ERR_UNSUPPORTED.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

using namespace cem;

namespace {

constexpr size_t kScratchBytes = 2u << 20;
constexpr int kMaxParams = 262144;  // N * D
constexpr int kMaxIters = 4096;
constexpr int kMaxDevices = 64;

// the scratch memory of cem_solve_static (see the limits above)
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// byte offsets of the regions inside g_scratch
struct Layout {
  size_t scene, track, status, keff, mean, cov, chol, hist_J, hist_keff, hist_cnt, J, cls, theta, end;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(int N, int D) {
  Layout L;
  size_t o = 0;
  L.scene = o;
  o = up256(o + sizeof(DevScene));
  L.track = o;
  o = up256(o + sizeof(Track));
  L.status = o;
  o = up256(o + sizeof(int32_t));
  L.keff = o;
  o = up256(o + sizeof(int32_t));
  L.mean = o;
  o = up256(o + sizeof(float) * CEM_MAX_D);
  L.cov = o;
  o = up256(o + sizeof(float) * CEM_MAX_D * CEM_MAX_D);
  L.chol = o;
  o = up256(o + sizeof(float) * CEM_MAX_D * CEM_MAX_D);
  L.hist_J = o;
  o = up256(o + sizeof(float) * kMaxIters);
  L.hist_keff = o;
  o = up256(o + sizeof(int32_t) * kMaxIters);
  L.hist_cnt = o;
  o = up256(o + sizeof(int32_t) * 4 * kMaxIters);
  L.J = o;
  o = up256(o + sizeof(float) * (size_t)N);
  L.cls = o;
  o = up256(o + (size_t)N);
  L.theta = o;
  o = up256(o + sizeof(float) * (size_t)N * D);
  L.end = o;
  return L;
}

std::mutex g_setup_mu;

int fail(int code, const std::string& m) { return set_last_error(code, m); }

// Device address of g_scratch on the current device, looked up on every call
// together with the refit kernel's shared-memory attribute: after a device
// reset the module is loaded again (possibly at another address, and without
// the attribute), and a fresh lookup is right in every case.
int scratch_ptr(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(CEM_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || !p)
    return fail(CEM_ERR_CUDA, std::string("cudaGetSymbolAddress(g_scratch): ") + cudaGetErrorString(e));
  e = configure_refit();
  if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("refit kernel set-up: ") + cudaGetErrorString(e));
  *out = static_cast<unsigned char*>(p);
  return CEM_OK;
}

// Failure of a call that has already queued work on the array: wait for that
// work (its own result ignored) before reporting, so that nothing of this
// call still reads or writes the array when the caller moves on.
#define STATIC_CUDA(call)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      cudaStreamSynchronize(st);                                                          \
      return fail(CEM_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_));        \
    }                                                                                     \
  } while (0)

}  // namespace

extern "C" int cem_solve_static(const cem_scene_desc* scene, const cem_skeleton_desc* skel,
                                const cem_solve_params* p, cem_result* out, void* stream) {
  set_last_error(CEM_OK, "");
  if (!scene || !skel || !p || !out) return fail(CEM_ERR_INVALID_ARG, "null argument");
  int rc = validate_descriptors(scene, skel);
  if (rc != CEM_OK) return fail(rc, std::string("descriptor: ") + cem_last_error());
  const int D = skel->D;
  if (p->N < 1 || (long long)p->N * D > kMaxParams)
    return fail(CEM_ERR_UNSUPPORTED, "cem_solve_static holds at most N * D = 262144 parameters (N >= 1)");
  if (p->iters < 1 || p->iters > kMaxIters) return fail(CEM_ERR_UNSUPPORTED, "cem_solve_static runs 1..4096 iterations");
  if (p->K < 1 || p->K > CEM_MAX_K) return fail(CEM_ERR_UNSUPPORTED, "K must be in 1..4096");
  if (p->cov_mode != CEM_COV_FULL && p->cov_mode != CEM_COV_DIAG) return fail(CEM_ERR_INVALID_ARG, "unknown cov mode");
  const Layout L = layout(p->N, D);
  if (L.end > kScratchBytes) return fail(CEM_ERR_UNSUPPORTED, "request does not fit the 2 MiB scratch array");
  unsigned char* base = nullptr;
  rc = scratch_ptr(&base);
  if (rc != CEM_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;

  DevScene* scene_d = reinterpret_cast<DevScene*>(base + L.scene);
  Track* track_d = reinterpret_cast<Track*>(base + L.track);
  int32_t* status_d = reinterpret_cast<int32_t*>(base + L.status);
  int32_t* keff_d = reinterpret_cast<int32_t*>(base + L.keff);
  float* mean_d = reinterpret_cast<float*>(base + L.mean);
  float* cov_d = reinterpret_cast<float*>(base + L.cov);
  float* chol_d = reinterpret_cast<float*>(base + L.chol);
  float* hist_J_d = reinterpret_cast<float*>(base + L.hist_J);
  int32_t* hist_keff_d = reinterpret_cast<int32_t*>(base + L.hist_keff);
  int32_t* hist_cnt_d = reinterpret_cast<int32_t*>(base + L.hist_cnt);
  float* J_d = reinterpret_cast<float*>(base + L.J);
  uint8_t* cls_d = reinterpret_cast<uint8_t*>(base + L.cls);
  float* theta_d = reinterpret_cast<float*>(base + L.theta);

  // initial distribution and its Cholesky factor, on the host in FP64
  const DevScene host = prepare_scene(*scene, *skel);
  float mean[CEM_MAX_D], cov[CEM_MAX_D * CEM_MAX_D], chol[CEM_MAX_D * CEM_MAX_D];
  std::memset(cov, 0, sizeof(cov));
  std::memset(chol, 0, sizeof(chol));
  for (int d = 0; d < D; ++d) {
    mean[d] = p->init_mean_h ? p->init_mean_h[d] : 0.5f * (skel->lo[d] + skel->hi[d]);
    if (!p->init_cov_h) cov[d * D + d] = std::pow(0.25f * (skel->hi[d] - skel->lo[d]), 2.0f);
  }
  if (p->init_cov_h)
    for (int i = 0; i < D * D; ++i) cov[i] = p->init_cov_h[i];
  if (p->init_chol_h) {
    for (int i = 0; i < D * D; ++i) chol[i] = p->init_chol_h[i];
  } else {
    double Lf[CEM_MAX_D * CEM_MAX_D] = {0.0};
    for (int j = 0; j < D; ++j) {
      double s = cov[j * D + j];
      for (int k = 0; k < j; ++k) s -= Lf[j * D + k] * Lf[j * D + k];
      if (!(s > 0.0)) return fail(CEM_ERR_NOT_PD, "initial covariance is not positive definite");
      Lf[j * D + j] = std::sqrt(s);
      for (int i = j + 1; i < D; ++i) {
        double t = cov[i * D + j];
        for (int k = 0; k < j; ++k) t -= Lf[i * D + k] * Lf[j * D + k];
        Lf[i * D + j] = t / Lf[j * D + j];
      }
    }
    for (int i = 0; i < D * D; ++i) chol[i] = (float)Lf[i];
  }
  Track tr;
  std::memset(&tr, 0, sizeof(tr));
  tr.iter = p->start_iter;
  tr.base_iter = p->start_iter;
  tr.best_cls = 4;
  tr.best_J = INFINITY;
  tr.hist_len = p->iters;
  const int32_t zero = 0;
  // everything the loop reads is rewritten here, so no earlier call leaks in
  STATIC_CUDA(cudaMemcpyAsync(scene_d, &host, sizeof(DevScene), cudaMemcpyHostToDevice, st));
  STATIC_CUDA(cudaMemcpyAsync(mean_d, mean, sizeof(float) * D, cudaMemcpyHostToDevice, st));
  STATIC_CUDA(cudaMemcpyAsync(cov_d, cov, sizeof(float) * D * D, cudaMemcpyHostToDevice, st));
  STATIC_CUDA(cudaMemcpyAsync(chol_d, chol, sizeof(float) * D * D, cudaMemcpyHostToDevice, st));
  STATIC_CUDA(cudaMemcpyAsync(track_d, &tr, sizeof(Track), cudaMemcpyHostToDevice, st));
  STATIC_CUDA(cudaMemcpyAsync(status_d, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, st));

  RefitArgs a;
  std::memset(&a, 0, sizeof(a));
  a.theta = theta_d;
  a.J = J_d;
  a.cls = cls_d;
  a.N = p->N;
  a.D = D;
  a.K = p->K;
  a.cov_mode = p->cov_mode;
  for (int d = 0; d < D; ++d) {
    a.lo[d] = skel->lo[d];
    a.hi[d] = skel->hi[d];
  }
  a.mean = mean_d;
  a.cov = cov_d;
  a.chol = chol_d;
  a.k_eff = keff_d;
  a.track = track_d;
  a.hist_J = hist_J_d;
  a.hist_keff = hist_keff_d;
  a.hist_cnt = hist_cnt_d;
  a.status = status_d;
  const int block = default_rollout_block(p->N, host.kind, 1);
  for (int j = 0; j < p->iters; ++j) {
    STATIC_CUDA(launch_sample(mean_d, chol_d, p->seed, &track_d->iter, 0, p->problem, p->N, D, theta_d, st));
    STATIC_CUDA(launch_rollout(scene_d, host.kind, theta_d, p->N, J_d, cls_d, block, 1, nullptr, st, host.base_ctrl != 0));
    STATIC_CUDA(launch_refit(a, st));
  }
  int32_t status = 0;
  STATIC_CUDA(cudaMemcpyAsync(&tr, track_d, sizeof(Track), cudaMemcpyDeviceToHost, st));
  STATIC_CUDA(cudaMemcpyAsync(out->mean, mean_d, sizeof(float) * D, cudaMemcpyDeviceToHost, st));
  STATIC_CUDA(cudaMemcpyAsync(out->cov, cov_d, sizeof(float) * D * D, cudaMemcpyDeviceToHost, st));
  STATIC_CUDA(cudaMemcpyAsync(out->chol, chol_d, sizeof(float) * D * D, cudaMemcpyDeviceToHost, st));
  STATIC_CUDA(cudaMemcpyAsync(&status, status_d, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (p->best_J_hist_h)
    STATIC_CUDA(cudaMemcpyAsync(p->best_J_hist_h, hist_J_d, sizeof(float) * p->iters, cudaMemcpyDeviceToHost, st));
  if (p->k_eff_hist_h)
    STATIC_CUDA(cudaMemcpyAsync(p->k_eff_hist_h, hist_keff_d, sizeof(int32_t) * p->iters, cudaMemcpyDeviceToHost, st));
  if (p->class_count_hist_h)
    STATIC_CUDA(cudaMemcpyAsync(p->class_count_hist_h, hist_cnt_d, sizeof(int32_t) * 4 * p->iters,
                                cudaMemcpyDeviceToHost, st));
  STATIC_CUDA(cudaStreamSynchronize(st));
  out->elapsed_ms = 0.0f;
  out->D = D;
  out->iters_done = (int32_t)(tr.iter - tr.base_iter);
  out->best_J = tr.best_J;
  out->best_class = tr.best_cls;
  for (int d = 0; d < CEM_MAX_D; ++d) out->best_theta[d] = d < D ? tr.best_theta[d] : 0.0f;
  if (status != 0) return fail(CEM_ERR_NOT_PD, "covariance not positive definite after the diagonal fallback");
  return CEM_OK;
}
