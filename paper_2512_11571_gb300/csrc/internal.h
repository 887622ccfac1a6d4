// Internal declarations of the cemtamp CUDA library (device scene layout,
// kernel launchers, error helpers).  Not part of the public ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/cemtamp.h"

namespace cem {

// Scene prepared for the device: the descriptor's values plus derived
// constants (inertias, friction capacities per step, 1/m), all FP32.  One
// copy lives in global memory per handle; kernels stage it in shared memory.
struct DevScene {
  int32_t kind, T, cost_step, D;
  int32_t n_act, n_geoms, goal_obj_region, goal_obj_held;
  int32_t goal_base_region, pad0, pad1, pad2;
  float dt, g, eps, k_contact;
  float c_contact, contact_mu, force_limit, w_time;
  float w_goal, w_viol, w_obj, w_base;
  // planar base
  float bhx, bhy, mb, Ib;
  float dt_mb, dt_Ib, base_cap, base_wcap;  // dt/m, dt/I, mu g dt, mu m g rbar dt / I
  float yaw_kp, yaw_kd, base_start[3], base_v0[3];
  // block
  float khx, khy, mk, Ik;
  float dt_mk, dt_Ik, block_cap, block_wcap;
  float block_start[3], block_v0[3];
  float goal_center[3], goal_half[3];
  // pick-place
  float oh, mo, obj_mu, dt_mo;
  float obj_start[3], obj_v0[3];
  float arm_l1, arm_l2, arm_z, arm_kp, arm_kd, arm_home[2];
  float grasp_reach, grasp_kp, grip_tol;
  float obj_region_c[3], obj_region_h[3], base_region_c[3], base_region_h[3];
  float obj_cap;  // mu dt (per unit normal force)
  // skeleton
  int32_t act_kind[CEM_MAX_ACTIONS], act_off[CEM_MAX_ACTIONS], act_ref[CEM_MAX_ACTIONS];
  int32_t act_region[CEM_MAX_ACTIONS];  // initial sampling region: 0 box, 1 annulus
  float act_nom[CEM_MAX_ACTIONS][3], act_yaw[CEM_MAX_ACTIONS];
  float act_ring[CEM_MAX_ACTIONS][4];   // annulus centre x, y, inner, outer radius
  float lo[CEM_MAX_D], hi[CEM_MAX_D];
  // geometry
  int32_t geom_nslab[CEM_MAX_GEOMS], geom_flags[CEM_MAX_GEOMS];  // bit0 base, bit1 object
  float slab[CEM_MAX_GEOMS][CEM_MAX_SLABS][5];
  // the same slabs with a pick-and-place mover's support folded in, laid
  // out for 16-byte loads: oslab = (n_x, n_y, n_z, lo - r | hi + r, unused)
  // with r = h (|n_x| + |n_y| + |n_z|) for the object cube; bslab = (n_x,
  // n_y, lo - r, hi + r) with r = bhx |n_x| + bhy |n_y| for the base
  // footprint, its slabs with n_z == 0 only (bslab_n of them, in their
  // original order)
  alignas(16) float oslab[CEM_MAX_GEOMS][CEM_MAX_SLABS][8];
  alignas(16) float bslab[CEM_MAX_GEOMS][CEM_MAX_SLABS][4];
  int32_t bslab_n[CEM_MAX_GEOMS];
  // quadratic
  float theta_star[CEM_MAX_D];
  float A[CEM_MAX_D * CEM_MAX_D];
  // A* base controller (pick-place): grown-footprint corners and their
  // mutual visibility (bit j of corner_vis[i]), built on the host
  int32_t base_ctrl, n_corners;
  float base_infl, wp_switch, pid_ki, pid_irad, pid_imax, pad3;
  float corner[CEM_MAX_CORNERS][2];
  uint64_t corner_vis[CEM_MAX_CORNERS];
};

static_assert(offsetof(DevScene, oslab) % 16 == 0 && offsetof(DevScene, bslab) % 16 == 0,
              "mover slabs are read with 16-byte loads");

// Best-ever sample and iteration counter of a device-resident CE loop.
struct Track {
  uint32_t iter;       // Philox iteration of the next sample
  uint32_t base_iter;  // iteration of the first sample (history index 0)
  int32_t best_cls;    // 4 = none yet
  float best_J;
  float best_theta[CEM_MAX_D];
  int32_t hist_len;
  int32_t pad;
};

// One problem of a batch, as the batched kernels see it.
struct BatchProblem {
  int32_t N, D, K, kind;
  int32_t theta_off;   // float offset of the problem's theta rows in the batch buffer
  int32_t sample_off;  // offset of its J / class entries
  uint32_t problem;    // Philox problem id
  int32_t active;      // 0: the problem is left out of sampling, rollouts and refits
  uint64_t seed;
};

// A unit of work of the persistent rollout kernel: 32 consecutive samples
// (one warp) of one problem.
struct BatchItem {
  int32_t problem, first;
};

struct RefitArgs {
  const float* theta;
  const float* J;
  const uint8_t* cls;
  int N, D, K, cov_mode;
  float lo[CEM_MAX_D], hi[CEM_MAX_D];
  float* mean;
  float* cov;
  float* chol;
  int32_t* elite_idx;
  int32_t* k_eff;
  Track* track;
  float* hist_J;
  int32_t* hist_keff;
  int32_t* hist_cnt;  // [hist_len][4] samples per class and iteration (may be null)
  int32_t* status;    // set to CEM_ERR_NOT_PD when the covariance stays indefinite
  int32_t skip;       // batched refit: 1 leaves this problem untouched (eliminated plan)
};

// kernel launchers (stream-ordered, no synchronisation)
cudaError_t launch_sample(const float* mean, const float* chol, uint64_t seed, const uint32_t* iter_ptr,
                          uint32_t iter, uint32_t problem, int N, int D, float* theta, cudaStream_t st);
cudaError_t launch_philox_words(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D, uint32_t* words,
                                cudaStream_t st);
// uniform initial sampling inside the regions of the scene's skeleton
cudaError_t launch_sample_uniform(const DevScene* s_d, uint64_t seed, uint32_t problem, int N, int D, float* theta,
                                  cudaStream_t st);
// Domain randomisation of a rollout launch: M environments per sample (a
// power of two <= 32) scaling friction by 1 + dmu (2u - 1) and the
// manipulated body's mass by 1 + dm (2u' - 1), u, u' from the Philox block
// (m, 256, iteration, problem) under `seed`; the iteration is *iter_ptr when
// set (a device loop), else `iter`.
struct DrArgs {
  int M;
  float dmu, dm;
  uint32_t problem, iter;
  uint64_t seed;
  const uint32_t* iter_ptr;
};

// block = threads per CTA; tpr = lanes per rollout (1, 8 or 32; used for
// pick-and-place scenes, the other kinds always run one lane per rollout);
// dr = domain randomisation or null (then tpr applies; with dr, one lane per
// environment); astar = the scene has the A* base controller (false takes
// the kernel without the A* rollout for a pick-and-place scene with the PD
// base: the same compiled rollout as the batched kernel's)
cudaError_t launch_rollout(const DevScene* s_d, int kind, const float* theta, int N, float* J, uint8_t* cls,
                           int block, int tpr, const DrArgs* dr, cudaStream_t st, bool astar = true);
cudaError_t launch_trace(const DevScene* s_d, int kind, const float* theta, int N, int steps, float* states,
                         cudaStream_t st, bool astar = true);
cudaError_t launch_refit(const RefitArgs& a, cudaStream_t st);
// opts the refit kernel into its dynamic shared memory (once per device, before any capture)
cudaError_t configure_refit();
size_t refit_smem_bytes(int K, int D);
cudaError_t launch_refit_batch(const RefitArgs* args_d, int n_problems, int maxK, int maxD, cudaStream_t st);
// batched sampling: problem p draws N_p rows from means[p*18..], chols[p*324..]
// (D_p x D_p row-major) at Philox iteration tracks[p].iter
cudaError_t launch_sample_batch(const BatchProblem* probs_d, int n_problems, int maxN, const float* means,
                                const float* chols, const Track* tracks, float* theta, cudaStream_t st);
// persistent rollout over a work queue of (problem, 32-sample chunk) items;
// *counter must be zero at launch
// perm (may be null = identity): lane position k of a problem rolls out
// sample perm[sample_off + k] (the randomised path keeps the identity);
// dorder (may be null = identity): the k-th item taken is items[dorder[k]];
// idur (may be null): a running average of each item's duration is kept there
// astar: whether any problem of the batch has the A* base controller (false
// launches the kernel without the A* rollout; it must then be true of none)
cudaError_t launch_rollout_batch_persistent(const DevScene* scenes_d, const BatchProblem* probs_d,
                                            const BatchItem* items_d, int n_items, int* counter_d,
                                            const float* theta, float* J, uint8_t* cls, int grid, int warps,
                                            int tpr, const Track* tracks, const DrArgs* dr, cudaStream_t st,
                                            const int32_t* perm = nullptr, const int32_t* dorder = nullptr,
                                            uint32_t* idur = nullptr, bool astar = true);
// the dispatch order of the work items, longest forecast duration first
// (idur: per item, 128 ns units, a running average the persistent kernel
// keeps; blended with the item's problem mean)
cudaError_t launch_dispatch_order(const uint32_t* idur, const BatchItem* items, int n_items, int32_t* dorder,
                                  cudaStream_t st);
// the rollout order of every problem of a batch (see order_batch_kernel):
// perm[sample_off + k] for k < N, from the theta just sampled
cudaError_t launch_order_batch(const DevScene* scenes_d, const BatchProblem* probs_d, int n_problems,
                               const float* theta, int32_t* perm, cudaStream_t st);
// (astar selects the kernel instantiation whose occupancy is asked)
int rollout_batch_max_ctas_per_sm(int warps, int tpr, bool astar = true);
// opts the persistent kernel into its dynamic shared memory (one DevScene
// per warp; before any capture)
cudaError_t configure_rollout_batch();

// host helpers shared by the C entry points (capi.cu)
int validate_descriptors(const cem_scene_desc* s, const cem_skeleton_desc* k);
DevScene prepare_scene(const cem_scene_desc& s, const cem_skeleton_desc& k);
// rollout threads per CTA when none is set (kind: CEM_SCENE_*, tpr: lanes per rollout)
int default_rollout_block(int N, int kind = -1, int tpr = 1);
// records the thread-local message returned by cem_last_error; returns code
int set_last_error(int code, const std::string& msg);

// The device workspace of a handle's CE loop (cem_solve and the screened
// loop share it).
struct SolveBuffers {
  float* theta;
  float* J;
  uint8_t* cls;
  float* mean;
  float* cov;
  float* chol;
  int32_t* keff;
  int32_t* status;
  Track* track;
  float* hist_J;
  int32_t* hist_keff;
  int32_t* hist_cnt;
  cudaStream_t stream;
  cudaEvent_t ev0, ev1;
  const DevScene* scene;
  int kind, block, tpr;
  bool astar;        // the scene has the A* base controller
  const DrArgs* dr;  // the handle's domain randomisation (null when off)
};
const cem_skeleton_desc& handle_skeleton(cem_handle h);
int handle_solve_buffers(cem_handle h, int N, int iters, SolveBuffers* b);
// initial distribution of cem_solve_params (or the default) and a fresh loop state
int handle_init_distribution(cem_handle h, const cem_solve_params* p, SolveBuffers* b);
// copies the loop's results to the host, synchronises and fills *out
int handle_read_result(cem_handle h, const cem_solve_params* p, SolveBuffers* b, cem_result* out);

// ---- screening of the batched CE (surrogate.cu)
// reserves the surrogate's pool workspace for n_pool candidates
int surrogate_reserve_pool(cem_surrogate_handle s, int n_pool, int n_keep, int D);
// draws n_pool candidates of one problem from (mean, chol) at Philox
// iteration *iter_ptr, scores them (features from the device tables lohi[2 x
// 18] and scene16[16]), keeps the first n_explore draws and the best-scored
// n_keep - n_explore of the rest, in ascending pool order, into theta_keep
cudaError_t surrogate_screen_into(cem_surrogate_handle s, const float* mean, const float* chol, uint64_t seed,
                                  const uint32_t* iter_ptr, uint32_t problem, int n_pool, int n_keep, int n_explore,
                                  int D, const float* lohi, const float* scene16, float* theta_keep, cudaStream_t st);
// reads and clears the tcgen05 forward's status word (-1 on a copy error)
int surrogate_status_word(cem_surrogate_handle s);

// ---- fused tcgen05 surrogate forward (48 -> 4 x 256 GELU -> 1)
struct MlpTcOffsets {
  int w[4];  // element offsets of W0..W3 in the flat BF16 parameter vector
};
struct MlpTcArgs {
  const void* x;         // BF16 [M x 48] features (used when xf is null)
  const float* xf;       // FP32 [M x 48] features, rounded to BF16 in the kernel (16-byte aligned), or null
  int M;
  const void* wpack;     // canonical weight image from mlp_tc_pack
  const float* bias[4];  // FP32 biases of the hidden layers
  const void* w_out;     // BF16 [256] output weights
  const float* b_out;    // FP32 output bias
  const float* norm;     // [mu, sigma]
  float* y;              // [M] scores
  int* status;           // set non-zero if a bounded wait expired
  int expire_test;       // failure-detection test: skip the first weight copy so its wait runs out
};
bool mlp_tc_supported(int in_dim, int width, int depth);
size_t mlp_tc_pack_bytes();
cudaError_t mlp_tc_pack(const void* pb, const MlpTcOffsets& off, void* pack, cudaStream_t st);
cudaError_t mlp_tc_forward(const MlpTcArgs& a, cudaStream_t st);

// ---- dense layers of the surrogate (csrc/surrogate.cu tiled path,
// csrc/gemm_tc.cu tcgen05 path)
// C[M x N] = op(A)[M x K] * op(B)[K x N], BF16 operands, FP32 accumulation,
// op(A)(m, k) = a_kmajor ? A[m * lda + k] : A[k * lda + m],
// op(B)(k, n) = b_kmajor ? B[n * ldb + k] : B[k * ldb + n], and a fused
// epilogue: EPI_F32 stores C (or split-K partials), EPI_BIAS_GELU stores
// z = C + bias (FP32, optional) and GELU(z) (BF16), EPI_GELU_BWD stores
// C * GELU'(zsave) (BF16).
enum { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_GELU_BWD = 2 };

struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;
  int lda, a_kmajor;
  const __nv_bfloat16* B;
  int ldb, b_kmajor;
  float* C;  // EPI_F32: output; EPI_BIAS_GELU: pre-activation z (may be null)
  int ldc;
  __nv_bfloat16* Cb;  // EPI_BIAS_GELU: activation; EPI_GELU_BWD: dz
  int ldcb;
  const float* bias;   // EPI_BIAS_GELU
  const float* zsave;  // EPI_GELU_BWD
  int ldz;
  // EPI_F32 split-K: blockIdx.z takes rows [z kchunk, (z + 1) kchunk) of the
  // reduction and writes its partial tile to part + z M N (row-major); the
  // partials are then summed in z order (deterministic)
  int kchunk;
  float* part;
  // EPI_F32, tcgen05 path only: n_real > 0 appends a row of ones to op(B)
  // (MN-major B with n_real real rows, N = n_real + 16), so column n_real of
  // C is the row sum of op(A) (a bias gradient); it goes to cbias[m], the
  // columns < n_real to C
  int n_real;
  float* cbias;
};
// tcgen05 path: shapes it takes (operand rows and leading dimensions in
// whole 16-byte units, N a multiple of 16, 16-byte aligned bases)
bool gemm_tc_supported(const GemmArgs& g);
// the same product and epilogue on the 5th-generation tensor cores; a
// pipeline wait that runs out sets *status (device int) non-zero
cudaError_t gemm_tc(int epi, const GemmArgs& g, int* status, cudaStream_t st);

// Every device allocation of the library goes through dev_malloc: a plain
// cudaMalloc, except that the test hook cem_test_fail_allocation can make
// the k-th next one report cudaErrorMemoryAllocation without allocating
// (host-side fault injection: the out-of-memory paths run on a GPU without
// exhausting its memory).
cudaError_t dev_malloc_bytes(void** p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_bytes(reinterpret_cast<void**>(p), bytes);
}

// Bounds checks of the debug build (compiled with -DCEM_DEBUG into
// libcemtamp_debug.so by build.build(debug=True)).  CEM_DIDX(i, n, code)
// is i when 0 <= i < n; otherwise it records `code` in the translation
// unit's status word (the first code stays) and returns the nearest index
// in range, so the access stays inside its buffer and no thread takes
// another path (the warp-collective code around the sites is unchanged).
// The release build compiles it to i.  Check sites guarantee n >= 1.
#ifdef CEM_DEBUG
static __device__ int g_cem_dbg_status;  // one word per translation unit
__device__ __forceinline__ int cem_didx(int i, int n, int code) {
  if (i >= 0 && i < n) return i;
  atomicCAS(&g_cem_dbg_status, 0, code);
  return i < 0 ? 0 : n - 1;
}
#define CEM_DIDX(i, n, code) ::cem::cem_didx((i), (n), (code))
// the host side of one translation unit's status word: read it (and zero it)
#define CEM_DEBUG_STATUS_ACCESSOR(name)                                                    \
  cudaError_t name(int* code, bool reset) {                                                \
    cudaError_t e = cudaMemcpyFromSymbol(code, g_cem_dbg_status, sizeof(int));             \
    if (e == cudaSuccess && reset) {                                                       \
      const int zero = 0;                                                                  \
      e = cudaMemcpyToSymbol(g_cem_dbg_status, &zero, sizeof(int));                        \
    }                                                                                      \
    return e;                                                                              \
  }
cudaError_t debug_status_rollout(int* code, bool reset);
cudaError_t debug_status_refit(int* code, bool reset);
cudaError_t debug_status_surrogate(int* code, bool reset);
// one thread indexes a 3-element shared array at 5 through CEM_DIDX (code
// 99): the access lands on element 2 and rollout.cu's word records 99
cudaError_t debug_selftest_rollout();
#else
#define CEM_DIDX(i, n, code) (i)
#endif

}  // namespace cem
