// Batched CE: many independent plan-realization problems (different scenes,
// skeletons of 1..6 actions, uneven N, T and D) advance together, one CE
// iteration of Algorithm 1 (Sec. III-B) for all of them per step:
//   batched sample (one launch, blockIdx.y = problem)
//   -> persistent rollout (one launch draining a queue of (problem, chunk)
//      items, longest horizon first)
//   -> segmented select + refit (one CTA per problem),
// the three captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

using namespace cem;

namespace {

int fail(int code, const std::string& m) { return set_last_error(code, m); }

#define BATCH_CUDA(call)                                                                                     \
  do {                                                                                                       \
    cudaError_t e_ = (call);                                                                                 \
    if (e_ != cudaSuccess)                                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? CEM_ERR_NO_MEMORY : CEM_ERR_CUDA,                        \
                  std::string(#call ": ") + cudaGetErrorString(e_));                                         \
  } while (0)

constexpr int kMS = CEM_MAX_D, kMC = CEM_MAX_D * CEM_MAX_D;

}  // namespace

struct cem_batch_ctx {
  int P = 0, maxN = 0, maxK = 0, maxD = 0, n_items = 0, total_samples = 0, total_theta = 0;
  std::vector<BatchProblem> probs;
  std::vector<cem_skeleton_desc> skels;
  DevScene* scenes_d = nullptr;
  BatchProblem* probs_d = nullptr;
  BatchItem* items_d = nullptr;
  int* counter_d = nullptr;
  float* theta_d = nullptr;
  float* J_d = nullptr;
  uint8_t* cls_d = nullptr;
  float* mean_d = nullptr;  // [P][18]
  float* cov_d = nullptr;   // [P][18*18]
  float* chol_d = nullptr;  // [P][18*18]
  int32_t* keff_d = nullptr;
  int32_t* status_d = nullptr;
  int32_t* perm_d = nullptr;  // rollout order of every problem's samples (launch_order_batch)
  int32_t* dorder_d = nullptr;  // dispatch order of the work items (launch_dispatch_order)
  uint32_t* idur_d = nullptr;   // each work item's running-average duration (128 ns units), or its estimate
  Track* track_d = nullptr;
  RefitArgs* args_d = nullptr;
  int warps = 4, ctas_per_sm = 0;  // persistent launch shape (0 = occupancy)
  int tpr = 1;                     // lanes per pick-and-place rollout (1, 8 or 32)
  std::vector<int> order;          // problems by descending work (the queue order)
  std::vector<uint32_t> weight;    // per problem: the work estimate behind that order
  bool has_pickplace = false;
  bool has_astar = false;  // some pick-place problem has the A* base: the persistent kernel with the A* rollout
  bool dr_on = false;  // domain randomisation of every problem's rollouts
  DrArgs dr{};
  cudaGraphExec_t graph = nullptr;
  long long steps_per_iter = 0;
  // stage timing (cem_batch_set_timing): events before the sample, before
  // and after the persistent rollout, after the refit of each iteration
  bool timing = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // surrogate screening (cem_batch_set_screening): per problem the bounds
  // and scene values the features take, [P][2 * 18 + 16]
  cem_surrogate_handle sur = nullptr;
  float* screen_tab_d = nullptr;
  int n_pool = 0, n_explore = 0;
};

namespace {

void batch_free(cem_batch_ctx* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  for (cudaEvent_t& e : h->ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  void* ptrs[] = {h->scenes_d, h->probs_d, h->items_d, h->counter_d, h->theta_d, h->J_d, h->cls_d,
                  h->mean_d,   h->cov_d,   h->chol_d,  h->keff_d,    h->status_d, h->track_d, h->args_d,
                  h->screen_tab_d, h->perm_d, h->dorder_d, h->idur_d};
  for (void* p : ptrs) cudaFree(p);
}

int grid_size(const cem_batch_ctx* h) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = h->ctas_per_sm > 0 ? h->ctas_per_sm : rollout_batch_max_ctas_per_sm(h->warps, h->tpr, h->has_astar);
  return sms * per_sm;
}

// Before any duration is recorded, a work item is estimated by its problem's
// horizon (four times as heavy for pick-and-place), which gives the
// heavier-first dispatch order; the persistent kernel then keeps a running
// average of real durations for the next iterations' order.
cudaError_t upload_item_estimates(cem_batch_ctx* h, const std::vector<BatchItem>& items) {
  std::vector<uint32_t> est(items.size());
  for (size_t i = 0; i < items.size(); ++i) est[i] = h->weight[items[i].problem];
  if (items.empty()) return cudaSuccess;
  return cudaMemcpy(h->idur_d, est.data(), sizeof(uint32_t) * est.size(), cudaMemcpyHostToDevice);
}

// Which problems take part in the next iterations: flags on the device
// problem table and refit arguments, and a work queue of the active
// problems' chunks only (same order).  A captured graph holds the old queue
// length, so it is dropped.
int set_active(cem_batch_ctx* h, const std::vector<int>& active) {
  std::vector<BatchItem> items;
  for (int p : h->order) {
    h->probs[p].active = active[p] ? 1 : 0;
    if (active[p])
      for (int f = 0; f < h->probs[p].N; f += 32) items.push_back(BatchItem{p, f});
  }
  BATCH_CUDA(cudaMemcpy(h->probs_d, h->probs.data(), sizeof(BatchProblem) * h->P, cudaMemcpyHostToDevice));
  for (int p = 0; p < h->P; ++p) {
    const int32_t skip = active[p] ? 0 : 1;
    BATCH_CUDA(cudaMemcpy(reinterpret_cast<char*>(h->args_d + p) + offsetof(RefitArgs, skip), &skip, sizeof(skip),
                          cudaMemcpyHostToDevice));
  }
  if (!items.empty())
    BATCH_CUDA(cudaMemcpy(h->items_d, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
  BATCH_CUDA(upload_item_estimates(h, items));
  h->n_items = (int)items.size();
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return CEM_OK;
}

// With timing on, an event is recorded at each stage boundary (as event
// record nodes when the iteration is captured into a graph).
cudaError_t mark(cem_batch_ctx* h, int i, cudaStream_t st) {
  if (!h->timing) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  // an external event node inside a captured graph, a plain record otherwise
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(h->ev[i], st, cudaEventRecordExternal)
                                             : cudaEventRecord(h->ev[i], st);
}

constexpr int kTab = 2 * CEM_MAX_D + 16;  // per problem: lo, hi, scene values

// The candidates of one screened iteration: for every active problem, a pool
// of n_pool draws from its distribution scored by the surrogate, of which
// the first n_explore and the best-scored N_p - n_explore of the rest become
// its theta rows (as in the single-problem screened loop).
cudaError_t enqueue_screen(cem_batch_ctx* h, cudaStream_t st) {
  for (int p = 0; p < h->P; ++p) {
    const BatchProblem& b = h->probs[p];
    if (!b.active) continue;
    cudaError_t e = surrogate_screen_into(h->sur, h->mean_d + (size_t)p * kMS, h->chol_d + (size_t)p * kMC, b.seed,
                                          &h->track_d[p].iter, b.problem, h->n_pool, b.N, h->n_explore, b.D,
                                          h->screen_tab_d + (size_t)p * kTab,
                                          h->screen_tab_d + (size_t)p * kTab + 2 * CEM_MAX_D,
                                          h->theta_d + b.theta_off, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t enqueue(cem_batch_ctx* h, cudaStream_t st, bool screened = false) {
  cudaError_t e = mark(h, 0, st);
  if (e != cudaSuccess) return e;
  e = screened ? enqueue_screen(h, st)
               : launch_sample_batch(h->probs_d, h->P, h->maxN, h->mean_d, h->chol_d, h->track_d, h->theta_d, st);
  if (e != cudaSuccess) return e;
  const bool order = !h->dr_on;  // the randomised path keeps the identity order
  if (order) e = launch_order_batch(h->scenes_d, h->probs_d, h->P, h->theta_d, h->perm_d, st);
  if (e != cudaSuccess) return e;
  e = launch_dispatch_order(h->idur_d, h->items_d, h->n_items, h->dorder_d, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(h->counter_d, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = mark(h, 1, st);
  if (e != cudaSuccess) return e;
  e = launch_rollout_batch_persistent(h->scenes_d, h->probs_d, h->items_d, h->n_items, h->counter_d, h->theta_d,
                                      h->J_d, h->cls_d, grid_size(h), h->warps, h->tpr, h->track_d,
                                      h->dr_on ? &h->dr : nullptr, st, order ? h->perm_d : nullptr, h->dorder_d,
                                      h->idur_d, h->has_astar);
  if (e != cudaSuccess) return e;
  e = mark(h, 2, st);
  if (e != cudaSuccess) return e;
  e = launch_refit_batch(h->args_d, h->P, h->maxK, h->maxD, st);
  if (e != cudaSuccess) return e;
  return mark(h, 3, st);
}

}  // namespace

extern "C" {

int cem_batch_create(const cem_scene_desc* scenes, const cem_skeleton_desc* skels, const cem_problem_params* params,
                     int n_problems, cem_batch_handle* out) {
  set_last_error(CEM_OK, "");
  if (!out) return fail(CEM_ERR_INVALID_ARG, "out handle pointer is NULL");
  *out = nullptr;
  if (!scenes || !skels || !params) return fail(CEM_ERR_INVALID_ARG, "null descriptor array");
  if (n_problems < 1 || n_problems > CEM_MAX_BATCH) return fail(CEM_ERR_UNSUPPORTED, "1..1024 problems per batch");
  cem_batch_ctx* h = new cem_batch_ctx();
  h->P = n_problems;
  std::vector<DevScene> host(n_problems);
  long long theta_total = 0, sample_total = 0;
  for (int p = 0; p < n_problems; ++p) {
    int rc = validate_descriptors(&scenes[p], &skels[p]);
    if (rc != CEM_OK) {
      delete h;
      return fail(rc, "problem " + std::to_string(p) + ": " + cem_last_error());
    }
    const cem_problem_params& q = params[p];
    if (q.N < 1 || q.N > CEM_MAX_N || q.K < 1 || q.K > CEM_MAX_K ||
        (q.cov_mode != CEM_COV_FULL && q.cov_mode != CEM_COV_DIAG)) {
      delete h;
      return fail(CEM_ERR_UNSUPPORTED, "problem " + std::to_string(p) + ": N in 1..2^20, K in 1..4096, known cov mode");
    }
    host[p] = prepare_scene(scenes[p], skels[p]);
    if (host[p].kind == CEM_SCENE_PICKPLACE) h->has_pickplace = true;
    if (host[p].kind == CEM_SCENE_PICKPLACE && host[p].base_ctrl) h->has_astar = true;
    BatchProblem b;
    std::memset(&b, 0, sizeof(b));
    b.N = q.N;
    b.D = skels[p].D;
    b.K = q.K;
    b.kind = scenes[p].kind;
    b.theta_off = (int32_t)theta_total;
    b.sample_off = (int32_t)sample_total;
    b.problem = q.problem;
    b.seed = q.seed;
    b.active = 1;
    theta_total += (long long)q.N * b.D;
    sample_total += q.N;
    h->maxN = std::max(h->maxN, q.N);
    h->maxK = std::max(h->maxK, q.K);
    h->maxD = std::max(h->maxD, b.D);
    h->steps_per_iter += (long long)q.N * (scenes[p].kind == CEM_SCENE_QUADRATIC ? 1 : scenes[p].T);
    h->probs.push_back(b);
    h->skels.push_back(skels[p]);
  }
  if (theta_total > (1ll << 31) - 1 || sample_total > (1ll << 31) - 1) {
    delete h;
    return fail(CEM_ERR_UNSUPPORTED, "batch too large");
  }
  h->total_samples = (int)sample_total;
  h->total_theta = (int)theta_total;
  // work queue: problems by descending horizon (then by index), 32-sample chunks
  std::vector<int> order(n_problems);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const long long wa = host[a].kind == CEM_SCENE_QUADRATIC ? 1 : (long long)host[a].T * (host[a].kind == CEM_SCENE_PICKPLACE ? 4 : 1);
    const long long wb = host[b].kind == CEM_SCENE_QUADRATIC ? 1 : (long long)host[b].T * (host[b].kind == CEM_SCENE_PICKPLACE ? 4 : 1);
    return wa > wb;
  });
  h->order = order;
  h->weight.resize(n_problems);
  for (int p = 0; p < n_problems; ++p)
    h->weight[p] = host[p].kind == CEM_SCENE_QUADRATIC ? 1u : (uint32_t)host[p].T * (host[p].kind == CEM_SCENE_PICKPLACE ? 4u : 1u);
  std::vector<BatchItem> items;
  for (int p : order)
    for (int f = 0; f < h->probs[p].N; f += 32) items.push_back(BatchItem{p, f});
  h->n_items = (int)items.size();
  const size_t P = n_problems;
  cudaError_t e = configure_refit();
  if (e == cudaSuccess) e = configure_rollout_batch();
  auto M = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = dev_malloc(ptr, bytes);
  };
  M((void**)&h->scenes_d, sizeof(DevScene) * P);
  M((void**)&h->probs_d, sizeof(BatchProblem) * P);
  M((void**)&h->items_d, sizeof(BatchItem) * items.size());
  M((void**)&h->counter_d, sizeof(int));
  M((void**)&h->theta_d, sizeof(float) * (size_t)theta_total);
  M((void**)&h->J_d, sizeof(float) * (size_t)sample_total);
  M((void**)&h->cls_d, (size_t)sample_total);
  M((void**)&h->perm_d, sizeof(int32_t) * (size_t)sample_total);
  M((void**)&h->dorder_d, sizeof(int32_t) * items.size());
  M((void**)&h->idur_d, sizeof(uint32_t) * items.size());
  M((void**)&h->mean_d, sizeof(float) * P * kMS);
  M((void**)&h->cov_d, sizeof(float) * P * kMC);
  M((void**)&h->chol_d, sizeof(float) * P * kMC);
  M((void**)&h->keff_d, sizeof(int32_t) * P);
  M((void**)&h->status_d, sizeof(int32_t) * P);
  M((void**)&h->track_d, sizeof(Track) * P);
  M((void**)&h->args_d, sizeof(RefitArgs) * P);
  if (e == cudaSuccess) e = cudaMemcpy(h->scenes_d, host.data(), sizeof(DevScene) * P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->probs_d, h->probs.data(), sizeof(BatchProblem) * P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->items_d, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = upload_item_estimates(h, items);
  if (e == cudaSuccess) {
    std::vector<RefitArgs> args(P);
    for (size_t p = 0; p < P; ++p) {
      RefitArgs& a = args[p];
      std::memset(&a, 0, sizeof(a));
      const BatchProblem& b = h->probs[p];
      a.theta = h->theta_d + b.theta_off;
      a.J = h->J_d + b.sample_off;
      a.cls = h->cls_d + b.sample_off;
      a.N = b.N;
      a.D = b.D;
      a.K = b.K;
      a.cov_mode = params[p].cov_mode;
      for (int d = 0; d < b.D; ++d) {
        a.lo[d] = skels[p].lo[d];
        a.hi[d] = skels[p].hi[d];
      }
      a.mean = h->mean_d + p * kMS;
      a.cov = h->cov_d + p * kMC;
      a.chol = h->chol_d + p * kMC;
      a.k_eff = h->keff_d + p;
      a.track = h->track_d + p;
      a.status = h->status_d + p;
    }
    e = cudaMemcpy(h->args_d, args.data(), sizeof(RefitArgs) * P, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(h);
    delete h;
    return fail(e == cudaErrorMemoryAllocation ? CEM_ERR_NO_MEMORY : CEM_ERR_CUDA,
                std::string("cem_batch_create: ") + cudaGetErrorString(e));
  }
  *out = h;
  return cem_batch_reset(h, nullptr);
}

int cem_batch_destroy(cem_batch_handle h) {
  if (!h) return CEM_OK;
  cudaDeviceSynchronize();
  batch_free(h);
  delete h;
  return CEM_OK;
}

int cem_batch_reset(cem_batch_handle h, void* stream) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  bool all = true;
  for (const BatchProblem& b : h->probs) all = all && b.active;
  if (!all) {  // every problem takes part again (which also resets the dispatch estimates)
    const int rc = set_active(h, std::vector<int>(h->P, 1));
    if (rc != CEM_OK) return rc;
  } else {  // the first iteration's dispatch order comes from the estimates again
    std::vector<BatchItem> items;
    for (int p : h->order)
      for (int f = 0; f < h->probs[p].N; f += 32) items.push_back(BatchItem{p, f});
    BATCH_CUDA(upload_item_estimates(h, items));
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = h->P;
  std::vector<float> mean(P * kMS, 0.0f), cov(P * kMC, 0.0f), chol(P * kMC, 0.0f);
  std::vector<Track> tr(P);
  for (size_t p = 0; p < P; ++p) {
    const cem_skeleton_desc& k = h->skels[p];
    const int D = k.D;
    for (int d = 0; d < D; ++d) {
      const float sd = 0.25f * (k.hi[d] - k.lo[d]);
      mean[p * kMS + d] = 0.5f * (k.lo[d] + k.hi[d]);
      cov[p * kMC + d * D + d] = std::pow(sd, 2.0f);
      chol[p * kMC + d * D + d] = (float)std::sqrt((double)std::pow(sd, 2.0f));
    }
    std::memset(&tr[p], 0, sizeof(Track));
    tr[p].best_cls = 4;
    tr[p].best_J = INFINITY;
  }
  std::vector<int32_t> zeros(P, 0);
  BATCH_CUDA(cudaMemcpyAsync(h->mean_d, mean.data(), sizeof(float) * P * kMS, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->cov_d, cov.data(), sizeof(float) * P * kMC, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->chol_d, chol.data(), sizeof(float) * P * kMC, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->track_d, tr.data(), sizeof(Track) * P, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->status_d, zeros.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaStreamSynchronize(st));  // the host vectors die at return
  return CEM_OK;
}

int cem_batch_iterate(cem_batch_handle h, int iters, int use_graph, void* stream) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (iters < 0 || iters > 100000) return fail(CEM_ERR_UNSUPPORTED, "iters must be in 0..1e5");
  cudaStream_t st = (cudaStream_t)stream;
  if (use_graph && !h->graph) {
    cudaStream_t cap;
    BATCH_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = enqueue(h, cap);
      e = cudaStreamEndCapture(cap, &g);
      if (e1 != cudaSuccess) e = e1;
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
      }
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
  }
  for (int j = 0; j < iters; ++j) {
    if (use_graph) {
      BATCH_CUDA(cudaGraphLaunch(h->graph, st));
    } else {
      cudaError_t e = enqueue(h, st);
      if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("batch iteration: ") + cudaGetErrorString(e));
    }
  }
  return CEM_OK;
}

int cem_batch_read(cem_batch_handle h, cem_result* out, void* stream) {
  if (!h || !out) return fail(CEM_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = h->P;
  std::vector<Track> tr(P);
  std::vector<float> mean(P * kMS), cov(P * kMC), chol(P * kMC);
  std::vector<int32_t> status(P);
  BATCH_CUDA(cudaMemcpyAsync(tr.data(), h->track_d, sizeof(Track) * P, cudaMemcpyDeviceToHost, st));
  BATCH_CUDA(cudaMemcpyAsync(mean.data(), h->mean_d, sizeof(float) * P * kMS, cudaMemcpyDeviceToHost, st));
  BATCH_CUDA(cudaMemcpyAsync(cov.data(), h->cov_d, sizeof(float) * P * kMC, cudaMemcpyDeviceToHost, st));
  BATCH_CUDA(cudaMemcpyAsync(chol.data(), h->chol_d, sizeof(float) * P * kMC, cudaMemcpyDeviceToHost, st));
  BATCH_CUDA(cudaMemcpyAsync(status.data(), h->status_d, sizeof(int32_t) * P, cudaMemcpyDeviceToHost, st));
  BATCH_CUDA(cudaStreamSynchronize(st));
  int bad = 0;
  for (size_t p = 0; p < P; ++p) {
    const int D = h->probs[p].D;
    cem_result& r = out[p];
    std::memset(&r, 0, sizeof(r));
    r.D = D;
    r.best_J = tr[p].best_J;
    r.best_class = tr[p].best_cls;
    r.iters_done = (int32_t)(tr[p].iter - tr[p].base_iter);
    for (int d = 0; d < D; ++d) {
      r.best_theta[d] = tr[p].best_theta[d];
      r.mean[d] = mean[p * kMS + d];
    }
    for (int i = 0; i < D * D; ++i) {
      r.cov[i] = cov[p * kMC + i];
      r.chol[i] = chol[p * kMC + i];
    }
    if (status[p] != 0) ++bad;
  }
  if (bad) return fail(CEM_ERR_NOT_PD, std::to_string(bad) + " problem(s) kept an indefinite covariance");
  return CEM_OK;
}

int cem_batch_set_launch(cem_batch_handle h, int warps_per_cta, int ctas_per_sm) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (warps_per_cta < 1 || warps_per_cta > 8 || ctas_per_sm < 0 || ctas_per_sm > 64)
    return fail(CEM_ERR_INVALID_ARG, "warps per CTA in 1..8, CTAs per SM in 0..64 (0 = occupancy)");
  if (ctas_per_sm > rollout_batch_max_ctas_per_sm(warps_per_cta, h->tpr, h->has_astar))
    return fail(CEM_ERR_INVALID_ARG, "more CTAs per SM than can be resident: the persistent grid must fit");
  h->warps = warps_per_cta;
  h->ctas_per_sm = ctas_per_sm;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return CEM_OK;
}

int cem_batch_autotune(cem_batch_handle h, int* warps_out, int* ctas_out, float* best_ms_out) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  cudaEvent_t a, b;
  BATCH_CUDA(cudaEventCreate(&a));
  BATCH_CUDA(cudaEventCreate(&b));
  // theta from the initial distributions, then time the persistent rollout
  cudaError_t e = launch_sample_batch(h->probs_d, h->P, h->maxN, h->mean_d, h->chol_d, h->track_d, h->theta_d, 0);
  float best = INFINITY;
  int bw = h->warps, bc = h->ctas_per_sm, bt = h->tpr;
  const int cand_w[] = {1, 2, 4, 8};
  // lanes per pick-and-place rollout, then warps per CTA and CTAs per SM; a
  // lane width whose first shape is over twice the best so far is dropped
  for (int t : {1, 8, 32}) {
    if (t > 1 && !h->has_pickplace) break;
    bool first = true, drop = false;
    for (int w : cand_w) {
      const int maxc = rollout_batch_max_ctas_per_sm(w, t, h->has_astar);
      for (int c = 1; c <= maxc && e == cudaSuccess && !drop; c *= 2) {
        h->warps = w;
        h->ctas_per_sm = c;
        h->tpr = t;
        float tot = 0.0f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
          e = cudaMemsetAsync(h->counter_d, 0, sizeof(int), 0);
          if (e == cudaSuccess) e = cudaEventRecord(a, 0);
          if (e == cudaSuccess)
            e = launch_rollout_batch_persistent(h->scenes_d, h->probs_d, h->items_d, h->n_items, h->counter_d,
                                                h->theta_d, h->J_d, h->cls_d, grid_size(h), w, t, h->track_d,
                                                h->dr_on ? &h->dr : nullptr, 0, nullptr, nullptr, nullptr, h->has_astar);
          if (e == cudaSuccess) e = cudaEventRecord(b, 0);
          if (e == cudaSuccess) e = cudaEventSynchronize(b);
          float ms = 0.0f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
          if (rep > 0) tot += ms;
        }
        if (e == cudaSuccess && tot < best) {
          best = tot;
          bw = w;
          bc = c;
          bt = t;
        } else if (first && t > 1 && tot > 2.0f * best) {
          drop = true;
        }
        first = false;
      }
      if (drop) break;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->warps = bw;
  h->ctas_per_sm = bc;
  h->tpr = bt;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("batch autotune: ") + cudaGetErrorString(e));
  if (warps_out) *warps_out = bw;
  if (ctas_out) *ctas_out = bc;
  if (best_ms_out) *best_ms_out = best;
  return CEM_OK;
}

long long cem_batch_steps_per_iteration(cem_batch_handle h) { return h ? h->steps_per_iter : 0; }

int cem_batch_set_screening(cem_batch_handle h, cem_surrogate_handle s, const float* scene16_h, int n_pool,
                            int n_explore) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (!s) {
    h->sur = nullptr;
    return CEM_OK;
  }
  if (!scene16_h) return fail(CEM_ERR_INVALID_ARG, "null scene values");
  if (n_pool < h->maxN || n_pool > CEM_MAX_N)
    return fail(CEM_ERR_UNSUPPORTED, "n_pool must hold every problem's N and be at most 2^20");
  for (const BatchProblem& b : h->probs)
    if (n_explore < 0 || n_explore > b.N) return fail(CEM_ERR_INVALID_ARG, "0 <= n_explore <= N of every problem");
  int rc = surrogate_reserve_pool(s, n_pool, h->maxN, h->maxD);
  if (rc != CEM_OK) return rc;
  if (!h->screen_tab_d) BATCH_CUDA(dev_malloc(&h->screen_tab_d, sizeof(float) * kTab * (size_t)h->P));
  std::vector<float> tab((size_t)kTab * h->P, 0.0f);
  for (int p = 0; p < h->P; ++p) {
    float* t = tab.data() + (size_t)p * kTab;
    for (int d = 0; d < h->probs[p].D; ++d) {
      t[d] = h->skels[p].lo[d];
      t[CEM_MAX_D + d] = h->skels[p].hi[d];
    }
    for (int i = 0; i < 16; ++i) t[2 * CEM_MAX_D + i] = scene16_h[(size_t)p * 16 + i];
  }
  BATCH_CUDA(cudaMemcpy(h->screen_tab_d, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
  h->sur = s;
  h->n_pool = n_pool;
  h->n_explore = n_explore;
  return CEM_OK;
}

int cem_batch_iterate_screened(cem_batch_handle h, int iters, void* stream) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (!h->sur) return fail(CEM_ERR_INVALID_ARG, "no surrogate set (cem_batch_set_screening)");
  if (iters < 0 || iters > 100000) return fail(CEM_ERR_UNSUPPORTED, "iters must be in 0..1e5");
  cudaStream_t st = (cudaStream_t)stream;
  for (int j = 0; j < iters; ++j) {
    cudaError_t e = enqueue(h, st, true);
    if (e != cudaSuccess) return fail(CEM_ERR_CUDA, std::string("screened batch iteration: ") + cudaGetErrorString(e));
  }
  return CEM_OK;
}

int cem_batch_set_state(cem_batch_handle h, const cem_result* in, void* stream) {
  if (!h || !in) return fail(CEM_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = h->P;
  std::vector<float> mean(P * kMS, 0.0f), cov(P * kMC, 0.0f), chol(P * kMC, 0.0f);
  std::vector<Track> tr(P);
  for (size_t p = 0; p < P; ++p) {
    const cem_result& r = in[p];
    const int D = h->probs[p].D;
    if (r.D != D) return fail(CEM_ERR_INVALID_ARG, "problem " + std::to_string(p) + ": D differs from the batch's");
    if (r.iters_done < 0) return fail(CEM_ERR_INVALID_ARG, "problem " + std::to_string(p) + ": iters_done < 0");
    if (r.best_class < 0 || r.best_class > 4)
      return fail(CEM_ERR_INVALID_ARG, "problem " + std::to_string(p) + ": best_class outside 0..4");
    for (int d = 0; d < D; ++d) mean[p * kMS + d] = r.mean[d];
    for (int i = 0; i < D * D; ++i) {
      cov[p * kMC + i] = r.cov[i];
      chol[p * kMC + i] = r.chol[i];
    }
    std::memset(&tr[p], 0, sizeof(Track));
    tr[p].iter = (uint32_t)r.iters_done;
    tr[p].base_iter = 0;
    tr[p].best_cls = r.best_class;
    tr[p].best_J = r.best_class == 4 ? INFINITY : r.best_J;
    for (int d = 0; d < D; ++d) tr[p].best_theta[d] = r.best_theta[d];
  }
  std::vector<int32_t> zeros(P, 0);
  BATCH_CUDA(cudaMemcpyAsync(h->mean_d, mean.data(), sizeof(float) * P * kMS, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->cov_d, cov.data(), sizeof(float) * P * kMC, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->chol_d, chol.data(), sizeof(float) * P * kMC, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->track_d, tr.data(), sizeof(Track) * P, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaMemcpyAsync(h->status_d, zeros.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
  BATCH_CUDA(cudaStreamSynchronize(st));  // the host vectors die at return
  return CEM_OK;
}

size_t cem_batch_state_bytes(cem_batch_handle h) {
  if (!h) return 0;
  const size_t P = h->P;
  return P * (sizeof(float) * (kMS + 2 * kMC) + sizeof(Track) + sizeof(int32_t));
}

int cem_batch_set_timing(cem_batch_handle h, int on) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (on && !h->ev[0])
    for (cudaEvent_t& e : h->ev) BATCH_CUDA(cudaEventCreate(&e));
  if ((on != 0) != h->timing && h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  h->timing = on != 0;
  return CEM_OK;
}

int cem_batch_stage_ms(cem_batch_handle h, float* ms_out) {
  if (!h || !ms_out) return fail(CEM_ERR_INVALID_ARG, "null argument");
  if (!h->timing) return fail(CEM_ERR_INVALID_ARG, "stage timing is off (cem_batch_set_timing)");
  BATCH_CUDA(cudaEventSynchronize(h->ev[3]));
  for (int i = 0; i < 3; ++i) BATCH_CUDA(cudaEventElapsedTime(&ms_out[i], h->ev[i], h->ev[i + 1]));
  return CEM_OK;
}

int cem_batch_set_randomization(cem_batch_handle h, int M, float delta_mu, float delta_mass, uint64_t seed) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (M < 1 || M > 32 || (M & (M - 1))) return fail(CEM_ERR_INVALID_ARG, "M must be 1, 2, 4, 8, 16 or 32");
  if (!(delta_mu >= 0.0f && delta_mu < 1.0f) || !(delta_mass >= 0.0f && delta_mass < 1.0f))
    return fail(CEM_ERR_INVALID_ARG, "spreads must lie in [0, 1)");
  h->dr_on = !(M == 1 && delta_mu == 0.0f && delta_mass == 0.0f);
  h->dr = DrArgs{};
  h->dr.M = M;
  h->dr.dmu = delta_mu;
  h->dr.dm = delta_mass;
  h->dr.seed = seed;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return CEM_OK;
}

int cem_batch_set_active(cem_batch_handle h, const int32_t* active_h) {
  if (!h || !active_h) return fail(CEM_ERR_INVALID_ARG, "null argument");
  std::vector<int> a(h->P);
  for (int p = 0; p < h->P; ++p) a[p] = active_h[p] ? 1 : 0;
  return set_active(h, a);
}

int cem_multiplan_solve(const cem_scene_desc* scene, const cem_skeleton_desc* plans, int n_plans,
                        const cem_multiplan_params* p, cem_result* per_plan_out, int32_t* iters_out,
                        int32_t* best_plan_out) {
  set_last_error(CEM_OK, "");
  if (!scene || !plans || !p || !per_plan_out) return fail(CEM_ERR_INVALID_ARG, "null argument");
  if (n_plans < 1 || n_plans > CEM_MAX_BATCH) return fail(CEM_ERR_UNSUPPORTED, "1..1024 plans");
  if (p->iters < 1 || p->iters > 100000 || p->halving_iters < 0 || p->keep < 0)
    return fail(CEM_ERR_UNSUPPORTED, "iters in 1..1e5, halving_iters >= 0, keep >= 0");
  std::vector<cem_scene_desc> scenes(n_plans, *scene);
  std::vector<cem_problem_params> pp(n_plans);
  for (int i = 0; i < n_plans; ++i) {
    std::memset(&pp[i], 0, sizeof(pp[i]));
    pp[i].seed = p->seed;
    pp[i].N = p->N;
    pp[i].K = p->K;
    pp[i].cov_mode = p->cov_mode;
    pp[i].problem = (uint32_t)i;
  }
  cem_batch_handle h = nullptr;
  int rc = cem_batch_create(scenes.data(), plans, pp.data(), n_plans, &h);
  if (rc != CEM_OK) return rc;
  std::vector<int> active(n_plans, 1), ran(n_plans, 0);
  std::vector<cem_result> res(n_plans);
  const int keep = p->keep > 0 ? p->keep : 1;
  auto key_less = [&](int a, int b) {  // (class, best cost, plan index) ascending
    if (res[a].best_class != res[b].best_class) return res[a].best_class < res[b].best_class;
    if (res[a].best_J != res[b].best_J) return res[a].best_J < res[b].best_J;
    return a < b;
  };
  int done = 0;
  while (rc == CEM_OK && done < p->iters) {
    const int step = p->halving_iters > 0 ? std::min(p->halving_iters, p->iters - done) : p->iters - done;
    rc = cem_batch_iterate(h, step, 1, nullptr);
    if (rc != CEM_OK) break;
    done += step;
    for (int i = 0; i < n_plans; ++i) ran[i] += active[i] ? step : 0;
    int n_active = 0;
    for (int a : active) n_active += a;
    if (p->halving_iters > 0 && done < p->iters && n_active > keep) {
      rc = cem_batch_read(h, res.data(), nullptr);
      if (rc != CEM_OK) break;
      std::vector<int> alive;
      for (int i = 0; i < n_plans; ++i)
        if (active[i]) alive.push_back(i);
      std::sort(alive.begin(), alive.end(), key_less);
      const int survivors = std::max(keep, (n_active + 1) / 2);
      for (size_t r = (size_t)survivors; r < alive.size(); ++r) active[alive[r]] = 0;
      rc = set_active(h, active);
    }
  }
  if (rc == CEM_OK) rc = cem_batch_read(h, res.data(), nullptr);
  cem_batch_destroy(h);
  if (rc != CEM_OK) return rc;
  int best = 0;
  for (int i = 1; i < n_plans; ++i)
    if (key_less(i, best)) best = i;
  for (int i = 0; i < n_plans; ++i) {
    per_plan_out[i] = res[i];
    if (iters_out) iters_out[i] = ran[i];
  }
  if (best_plan_out) *best_plan_out = best;
  return CEM_OK;
}

int cem_batch_set_threads_per_rollout(cem_batch_handle h, int tpr) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (tpr != 1 && tpr != 8 && tpr != 32) return fail(CEM_ERR_INVALID_ARG, "threads per rollout must be 1, 8 or 32");
  if (h->ctas_per_sm > rollout_batch_max_ctas_per_sm(h->warps, tpr, h->has_astar)) h->ctas_per_sm = 0;
  h->tpr = tpr;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return CEM_OK;
}

int cem_batch_get_launch(cem_batch_handle h, int* warps_out, int* ctas_out, int* tpr_out) {
  if (!h) return fail(CEM_ERR_INVALID_ARG, "null handle");
  if (warps_out) *warps_out = h->warps;
  if (ctas_out) *ctas_out = h->ctas_per_sm > 0 ? h->ctas_per_sm : rollout_batch_max_ctas_per_sm(h->warps, h->tpr, h->has_astar);
  if (tpr_out) *tpr_out = h->tpr;
  return CEM_OK;
}

}  // extern "C"
