/*
 * cemtamp -- C ABI of the GB300 (sm_103a) cross-entropy plan-realization
 * library.
 *
 * The library implements the data-parallel hot path of "Cross-Entropy
 * Optimization of Physically Grounded Task and Motion Plans" (arXiv
 * 2512.11571): Algorithm 1 (Sec. III-B) iterates
 *     sample n_env parameter vectors theta ~ N(mean, cov)      -> cem_sample
 *     roll every sample out through the plan's controllers and a
 *     contact-rich rigid-body simulation, score it with the plan
 *     cost of Problem 2                                        -> cem_rollout_batch
 *     refit mean and covariance from the top-N_e elites        -> cem_refit
 * until the iteration budget is spent (cem_solve runs the whole loop).
 *
 * Conventions for every entry point:
 *   - Pointers with a `_d` suffix are DEVICE memory owned by the caller
 *     (for example torch tensors).  They are checked with
 *     cudaPointerGetAttributes; a host pointer yields CEM_ERR_INVALID_ARG.
 *     Pointers with an `_h` suffix are host memory.
 *   - Arrays are dense row-major FP32 unless stated: theta[N][D],
 *     mean[D], cov[D][D], chol[D][D] (lower triangular, zeros above).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream.  Calls are stream-ordered and asynchronous; only
 *     cem_solve, cem_solve_static, cem_batch_reset/read/autotune,
 *     cem_surrogate_* and cem_autotune synchronise, when they return host
 *     results.
 *   - The library owns only the memory behind a handle; it is freed by
 *     cem_scene_destroy / cem_batch_destroy.
 *   - Return value 0 is success; negative values are the cem_status codes
 *     below, with a message in cem_last_error() (thread-local).
 *   - Limits: D <= CEM_MAX_D, N <= 2^20, K <= 4096, T <= 1,000,000.
 *
 * A handle may be used from one host thread at a time; calls on different
 * handles are independent.
 */
#ifndef CEMTAMP_H
#define CEMTAMP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CEM_MAX_D 18
#define CEM_MAX_ACTIONS 6
#define CEM_MAX_GEOMS 16
#define CEM_MAX_SLABS 6
#define CEM_MAX_K 4096
#define CEM_MAX_N (1 << 20)
#define CEM_TRACE_W 20
#define CEM_MAX_BATCH 1024
#define CEM_MAX_CORNERS 48 /* corners of the base planner's visibility graph */

typedef enum {
  CEM_OK = 0,
  CEM_ERR_INVALID_ARG = -1,
  CEM_ERR_CUDA = -2,
  CEM_ERR_TIMEOUT = -3,
  CEM_ERR_NOT_PD = -4,
  CEM_ERR_UNSUPPORTED = -5,
  CEM_ERR_NO_MEMORY = -6
} cem_status;

/* Scene kinds: which dynamics and cost the rollout runs. */
typedef enum {
  CEM_SCENE_QUADRATIC = 0, /* J = (theta - theta*)^T A (theta - theta*), no dynamics */
  CEM_SCENE_REACH = 1,     /* planar box base, one moveTo action */
  CEM_SCENE_PUSH = 2,      /* planar base + free block: moveTo, push */
  CEM_SCENE_PICKPLACE = 3  /* base + 2-link arm + object: move/grasp/move/place/move */
} cem_scene_kind;

/* Action kinds of a plan skeleton (the action schemas of Eq. 2 / Eq. 8-10).
 * theta slice per action: MOVE and PUSH (dx, dy, kp); GRASP (approach
 * azimuth, grip-height offset); PLACE (dx, dy, dz of the release point). */
typedef enum { CEM_ACT_MOVE = 0, CEM_ACT_PUSH = 1, CEM_ACT_GRASP = 2, CEM_ACT_PLACE = 3 } cem_action_kind;

typedef enum { CEM_COST_INTERP = 0, CEM_COST_STEP = 1 } cem_cost_mode;
typedef enum { CEM_COV_FULL = 0, CEM_COV_DIAG = 1 } cem_cov_mode;

/* A convex static body is the intersection of slabs lo <= n . x <= hi,
 * where each slab is the body's exact projection interval on the unit axis
 * n.  Finite bodies list the world x, y, z axes first (their bounding box)
 * and then their own face normals; half-spaces use one slab with a large
 * lo or hi. */
typedef struct {
  float n[3];
  float lo, hi;
} cem_slab;

typedef struct {
  int32_t n_slabs;
  int32_t collide_base;   /* base footprint collides (slabs with n_z == 0) */
  int32_t collide_object; /* object cube collides (all slabs) */
  int32_t reserved;
  cem_slab slab[CEM_MAX_SLABS];
} cem_geom;

/* Scene: physical constants, geometry and goal regions (SI units).  Fields a
 * scene kind does not use are ignored. */
typedef struct {
  int32_t kind;      /* cem_scene_kind */
  int32_t T;         /* horizon in steps */
  int32_t cost_mode; /* cem_cost_mode */
  int32_t reserved0;
  float dt, g, eps; /* step, gravity, success tolerance */
  /* planar base: half extents, mass, ground friction, start pose (x,y,yaw)
   * and velocity (vx,vy,wz), yaw PD gains */
  float base_half[2], base_mass, base_mu, base_start[3], base_v0[3], yaw_kp, yaw_kd;
  /* free block of the push task */
  float block_half[2], block_mass, block_mu, block_start[3], block_v0[3];
  /* penalty contact stiffness, damping, contact friction, force limit */
  float k_contact, c_contact, contact_mu, force_limit;
  /* cost weights */
  float w_time, w_goal, w_viol, w_obj, w_base;
  /* goal point (reach) or region centre/half size (push) */
  float goal_center[3], goal_half[3];
  /* pick-place object (cube half size, mass, friction, start, velocity) */
  float obj_half, obj_mass, obj_mu, obj_start[3], obj_v0[3];
  /* 2-link arm: link lengths, shoulder height, joint PD gains, home pose */
  float arm_l1, arm_l2, arm_z, arm_kp, arm_kd, arm_home[2];
  /* grasp: base stand-off distance, base gain, grip height tolerance */
  float grasp_reach, grasp_kp, grip_tol;
  float obj_region_c[3], obj_region_h[3], base_region_c[3], base_region_h[3];
  int32_t goal_obj_region, goal_obj_held, goal_base_region, n_geoms;
  cem_geom geom[CEM_MAX_GEOMS];
  float theta_star[CEM_MAX_D];
  float A[CEM_MAX_D * CEM_MAX_D];
  /* moveTo controller of the pick-place base (Sec. IV-A: A* paths tracked by
   * a PID controller).  0: PD straight at the goal.  1: A* over the
   * visibility graph of the base footprints (slabs with n_z == 0 of bodies
   * with collide_base) grown by base_inflate along their normals (corners
   * pushed 1 mm out, at most CEM_MAX_CORNERS; a footprint holding an
   * endpoint is used ungrown, or skipped, for that endpoint's edges),
   * planned when the action starts; waypoints tracked by PD, advancing
   * within wp_switch of one, the goal by PID with integral gain
   * pid_ki * kp, integrating only within pid_irad of the goal, |I| <=
   * pid_imax per axis. */
  int32_t base_controller;
  float base_inflate, wp_switch, pid_ki, pid_irad, pid_imax;
} cem_scene_desc;

typedef struct {
  int32_t kind;         /* cem_action_kind */
  int32_t theta_offset; /* first index of the action's theta slice */
  int32_t success_ref;  /* moveTo success measured from 0: nominal, 1: nominal + offset */
  int32_t init_region;  /* initial sampling region (Sec. III-B): 0 the box of the action's
                           bounds, 1 (moveTo only) an annulus for the goal (dx, dy) */
  float nominal[3]; /* nominal target (region centre) */
  float yaw;        /* base yaw target (planar tasks) */
  float region[4];  /* init_region 1: annulus centre x, y (world), inner and outer radius */
} cem_action_desc;

/* Plan skeleton pi = (a_1..a_k) and the box bounds of its parameters. */
typedef struct {
  int32_t n_actions, D;
  cem_action_desc action[CEM_MAX_ACTIONS];
  float lo[CEM_MAX_D], hi[CEM_MAX_D];
} cem_skeleton_desc;

typedef struct cem_ctx* cem_handle;

/* Problem 2 (Sec. III-B): a scene with its dynamics f, the symbolic plan pi
 * and the goal psi_g.  Validates and copies both descriptors to the device.
 * Errors: CEM_ERR_INVALID_ARG (bad descriptor), CEM_ERR_UNSUPPORTED
 * (D > 18, more than 6 actions or 16 geometries), CEM_ERR_CUDA. */
int cem_scene_create(const cem_scene_desc* scene, const cem_skeleton_desc* skel, cem_handle* out);
int cem_scene_destroy(cem_handle h);

/* Sample step of Algorithm 1: theta_d[n] = mean_d + chol_d z_n, z_n the
 * standard normals of Philox4x32-10 (Salmon et al., SC'11) with counter
 * (n, c, iter, problem) and key = seed, Box-Muller on word pairs.  N = 0 is
 * a no-op. */
int cem_sample(cem_handle h, const float* mean_d, const float* chol_d, uint64_t seed, uint32_t iter,
               uint32_t problem, int N, float* theta_d, void* stream);

/* The initial distribution of Sec. III-B: N vectors uniform inside each
 * parameter's region -- the box [lo, hi], or for a moveTo goal with
 * init_region 1 the annulus r <= |p - c| <= R, area-uniform (radius
 * sqrt(r^2 + u (R^2 - r^2)), angle 2 pi u').  Parameter d uses word d of the
 * Philox block (n, d / 4, 0xFFFFFFFF, problem) with u = (word + 1) 2^-32;
 * theta_d[N][D] is not clamped. */
int cem_sample_uniform(cem_handle h, uint64_t seed, uint32_t problem, int N, float* theta_d, void* stream);

/* The same Philox words the sampler draws: words_d[N][4*ceil(D/4)] (u32). */
int cem_philox_words(cem_handle h, uint64_t seed, uint32_t iter, uint32_t problem, int N, uint32_t* words_d,
                     void* stream);

/* Evaluate step of Algorithm 1 (Sec. III-B, Problem 2): roll out each row
 * of theta_d (clamped to the bounds) for T steps; J_d[n] = plan cost,
 * cls_d[n] = 0 (every action succeeded and psi_g(x_T)), 1 (every action
 * succeeded, psi_g false), 2 (otherwise), 3 (non-finite cost). */
int cem_rollout_batch(cem_handle h, const float* theta_d, int N, float* J_d, uint8_t* cls_d, void* stream);

/* Per-step state of each rollout for `steps` steps: states_d[N][steps][20],
 * the state after each step.  Planar scenes: base x, y, yaw, vx, vy, w, then
 * the block's six values, then the index of the active action, zeros after.
 * Pick-place: base x, y, vx, vy, joints q1, q2, dq1, dq2, arm azimuth,
 * object x, y, z, vx, vy, vz, attached (0/1), action index, end-effector
 * x, y, z. */
int cem_rollout_trace(cem_handle h, const float* theta_d, int N, int steps, float* states_d, void* stream);

/* Update step of Algorithm 1 with the elite rules of Sec. III-B: rank by
 * (class, J, index); elites are the K lowest of the best class present in
 * {0, 1} (fewer if fewer exist), else of class 2; mean/cov (1/K_eff, ridge
 * (1e-4 range)^2) and its Cholesky factor; one elite -> cov =
 * diag((0.05 range)^2).  mean_d/cov_d/chol_d are read-write and kept when
 * no elite exists.  elite_idx_d (K entries, ascending key) and k_eff_d may
 * be NULL.  Errors: CEM_ERR_UNSUPPORTED if K > 4096. */
int cem_refit(cem_handle h, const float* theta_d, const float* J_d, const uint8_t* cls_d, int N, int K,
              int cov_mode, float* mean_d, float* cov_d, float* chol_d, int32_t* elite_idx_d, int32_t* k_eff_d,
              void* stream);

typedef struct {
  uint64_t seed;
  int32_t N, K, iters, cov_mode;
  uint32_t problem;
  uint32_t start_iter;    /* Philox iteration of the first sample (resume) */
  int32_t use_graph;      /* capture one CE iteration in a CUDA graph and replay it */
  int32_t reserved;
  const float* init_mean_h; /* D values or NULL -> midpoint of the bounds */
  const float* init_cov_h;  /* D x D or NULL -> diag((range / 4)^2) */
  float* best_J_hist_h;     /* iters values or NULL: best cost so far per iteration */
  int32_t* k_eff_hist_h;    /* iters values or NULL */
  /* D x D lower Cholesky factor of init_cov_h, or NULL -> factorised on the
   * host.  Passing the chol of a previous cem_result with its mean, cov and
   * start_iter = iterations done resumes a run exactly. */
  const float* init_chol_h;
  /* iters x 4 values or NULL: samples of class 0..3 in each iteration
   * (class 0 / n_env is the success rate of Fig. 5) */
  int32_t* class_count_hist_h;
} cem_solve_params;

typedef struct {
  float best_theta[CEM_MAX_D];
  float best_J;
  int32_t best_class;
  int32_t D;
  int32_t iters_done;
  float mean[CEM_MAX_D];
  float cov[CEM_MAX_D * CEM_MAX_D];
  float elapsed_ms; /* device time of the loop (CUDA events) */
  float chol[CEM_MAX_D * CEM_MAX_D]; /* Cholesky factor of cov (the sampler's state) */
} cem_result;

/* Algorithm 1 end to end on the device: the distribution starts on the host
 * (params), every iteration runs sample -> rollout -> refit, and the best
 * sample over all iterations plus the final mean/cov come back to the host.
 * Synchronous. */
int cem_solve(cem_handle h, const cem_solve_params* p, cem_result* out);

/* The paper's CE variant (Sec. III-B, IV-A): iteration 0 draws n0 samples
 * with cem_sample_uniform, iteration j >= 1 draws n_env(j) samples from the
 * normal model refit at j - 1 (Philox iteration j), where n_env falls
 * linearly from n0 at j = 0 to n1 at j = j1 (rounded to nearest, halves up)
 * and stays at n1; K = N_e elites per refit; cov_mode CEM_COV_DIAG is the
 * paper's independent normal.  Histories as in cem_solve_params, plus the
 * samples drawn per iteration.  Not graph-captured (the batch size
 * changes).  Synchronous. */
typedef struct {
  uint64_t seed;
  int32_t n0, n1, j1; /* the schedule; n0, n1 in 1..2^20, j1 >= 0 */
  int32_t K, iters, cov_mode;
  uint32_t problem;
  int32_t reserved;
  float* best_J_hist_h;         /* iters values or NULL */
  int32_t* k_eff_hist_h;        /* iters values or NULL */
  int32_t* class_count_hist_h;  /* iters x 4 values or NULL */
  int32_t* n_env_hist_h;        /* iters values or NULL */
} cem_paper_params;
int cem_solve_paper(cem_handle h, const cem_paper_params* p, cem_result* out);
/* The A* path the pick-place base follows from (sx, sy) to (gx, gy) in a
 * scene with base_controller 1 (the rollout's planner, run on the device):
 * *n_out waypoints after the start, ending with the goal, the first `cap`
 * written to xy_h[2 i], xy_h[2 i + 1].  CEM_ERR_UNSUPPORTED without the A*
 * controller.  Synchronous. */
int cem_base_path(cem_handle h, float sx, float sy, float gx, float gy, float* xy_h, int cap, int* n_out);
/* Bounds checks of the debug build (libcemtamp_debug.so, built with
 * CEM_DEBUG): every kernel index checked there that left its buffer was
 * clamped into range and its code recorded (the first per source file).
 * Synchronises the device, writes the first recorded code to *code_out (0:
 * none; 1 dispatch-order entry, 2 rollout-order entry, 3 rollout-order
 * position, 4 order bin, 5 dispatch-order position, 6 geometry index,
 * 7 parameter index, 8 elite index, 9 screened row index) and, if reset,
 * clears the record.  A release build writes 0 and returns
 * CEM_ERR_UNSUPPORTED. */
int cem_debug_status(int* code_out, int reset);
/* Test hook (host-side fault injection): the k-th device allocation the
 * library makes from now on reports cudaErrorMemoryAllocation without
 * allocating, as if the device were full, so every call's out-of-memory
 * path can be exercised (it returns CEM_ERR_NO_MEMORY and releases what it
 * had allocated).  k = 0 switches the hook off; it also goes off once the
 * failure has happened.  CEM_ERR_INVALID_ARG for k < 0.  Host only. */
int cem_test_fail_allocation(int k);
/* Debug build only: one in-bounds kernel indexes a 3-element array at 5
 * through the checks, which clamp it to element 2 and record code 99 for
 * cem_debug_status (shows that the checks are compiled in and fire).
 * Synchronous.  A release build returns CEM_ERR_UNSUPPORTED. */
int cem_debug_selftest(void);
/* n_env of iteration j under the schedule (n0, n1, j1) (host function). */
int cem_n_env(int n0, int n1, int j1, int j);

/* cem_solve for callers that cannot allocate device memory (no paper
 * counterpart).  Hard real-time control loops, plugins whose host owns all
 * device memory through its own pool, and processes under a fixed memory cap
 * cannot call cudaMalloc while planning; this entry point allocates nothing.
 * It takes the descriptors directly (a handle would allocate) and runs the
 * same sample -> rollout -> refit loop on `stream`, keeping every
 * intermediate in one 2 MiB file-scope device array that every GPU loading
 * the library holds until the process exits.  Limits: N * D <= 262144,
 * iters <= 4096, otherwise CEM_ERR_UNSUPPORTED.  Every call looks up the
 * array's address on the current device (so a device reset needs nothing
 * special); the first call on a device also loads the module, so make it
 * before any stream capture.  All calls share the array (the loop state is
 * rewritten at the start of each call), so calls that overlap on the GPU
 * race: serialise them.  A call that fails after queuing work waits for that
 * work before it returns.  p->use_graph is ignored.  Synchronous; results as
 * cem_solve (elapsed_ms = 0). */
int cem_solve_static(const cem_scene_desc* scene, const cem_skeleton_desc* skel, const cem_solve_params* p,
                     cem_result* out, void* stream);

/* ---- Batched CE: many independent problems advance together ------------
 * One iteration of Algorithm 1 for every problem of the batch per step: a
 * batched sampler, ONE persistent rollout launch whose warps drain a queue
 * of (problem, 32-sample chunk) items (longest horizon first), and a
 * segmented select + refit (one CTA per problem).  Problems may differ in
 * scene kind, skeleton length, N, K, D and T.  Results per problem are
 * identical to cem_solve with the same seed, problem id and start_iter = 0.
 * There is no device-side wait between warps or CTAs. */
typedef struct {
  uint64_t seed;
  int32_t N, K, cov_mode;
  uint32_t problem; /* Philox problem id */
} cem_problem_params;

typedef struct cem_batch_ctx* cem_batch_handle;

/* Copies n_problems scenes/skeletons/params (arrays) to the device and resets
 * every distribution.  Errors as cem_scene_create, per problem. */
int cem_batch_create(const cem_scene_desc* scenes, const cem_skeleton_desc* skels, const cem_problem_params* params,
                     int n_problems, cem_batch_handle* out);
int cem_batch_destroy(cem_batch_handle h);
/* Initial distributions (mid-bounds, diag((range/4)^2)), iteration 0,
 * no best sample yet.  Synchronous. */
int cem_batch_reset(cem_batch_handle h, void* stream);
/* `iters` CE iterations of every problem on `stream` (asynchronous); with
 * use_graph the iteration is captured once and replayed. */
int cem_batch_iterate(cem_batch_handle h, int iters, int use_graph, void* stream);
/* Best sample so far, current mean/cov per problem: out[n_problems].  Synchronous. */
int cem_batch_read(cem_batch_handle h, cem_result* out, void* stream);
/* Persistent launch shape: warps per CTA (1..8) and CTAs per SM (0 = as
 * many as can be resident). */
int cem_batch_set_launch(cem_batch_handle h, int warps_per_cta, int ctas_per_sm);
/* Times the persistent rollout over warps per CTA and CTAs per SM on the
 * current device and keeps the fastest shape.  Synchronous. */
int cem_batch_autotune(cem_batch_handle h, int* warps_out, int* ctas_out, float* best_ms_out);
/* Simulated steps of one batch iteration: sum over problems of N * T. */
long long cem_batch_steps_per_iteration(cem_batch_handle h);
/* Restores every problem's CE state from in[n_problems] as cem_batch_read
 * wrote it: mean, cov, chol, the best sample (best_class 4 = none yet) and
 * iters_done, taken as the Philox iteration of the next sample (a batch
 * counts iterations from 0 after cem_batch_reset).  Reading after an
 * iteration and restoring before the next continues the run exactly (the
 * checkpoint/resume of a batch).  Errors: CEM_ERR_INVALID_ARG if a
 * problem's D differs or a class is outside 0..4.  Synchronous. */
int cem_batch_set_state(cem_batch_handle h, const cem_result* in, void* stream);
/* Bytes of device state that cem_batch_set_state writes and cem_batch_read
 * reads (per-problem distribution slots of the 18-parameter maximum, the
 * best-sample track and the status word). */
size_t cem_batch_state_bytes(cem_batch_handle h);
/* Stage timing of batch iterations: with on != 0 every iteration records
 * CUDA events on its stream at the stage boundaries (event record nodes in
 * a captured graph, so the graph is re-captured when this changes);
 * cem_batch_stage_ms waits for the last iteration and writes its sample,
 * persistent rollout and refit times in ms to ms_out[3] (the rollout time
 * is the persistent kernel alone).  Errors: CEM_ERR_INVALID_ARG while
 * timing is off. */
int cem_batch_set_timing(cem_batch_handle h, int on);
int cem_batch_stage_ms(cem_batch_handle h, float* ms_out);
/* Domain randomisation of every problem of the batch, as
 * cem_set_randomization for a single problem (environments of each problem's
 * own iteration and Philox problem id, under `seed`): a batched problem
 * equals cem_solve of that problem with the same randomisation.  The
 * randomised samples take one lane per environment (lanes per rollout 1). */
int cem_batch_set_randomization(cem_batch_handle h, int M, float delta_mu, float delta_mass, uint64_t seed);
/* Which problems take part in the next iterations (active_h[n_problems],
 * non-zero = active).  An inactive problem is not sampled, rolled out or
 * refit: its distribution, best sample and iteration count stay as they
 * are.  cem_batch_reset makes every problem active again. */
int cem_batch_set_active(cem_batch_handle h, const int32_t* active_h);
/* Lanes per pick-and-place rollout in the persistent launch: 1, 8 or 32
 * (other scene kinds always take one lane per rollout).  With 8 or 32, a
 * lane group holds one rollout's state, splits its per-geometry contact
 * queries and neighbour-list rebuilds, and sums the contact forces with warp
 * shuffles in ascending geometry order: the results are bit-identical for
 * every width.  cem_batch_autotune also searches this width. */
int cem_batch_set_threads_per_rollout(cem_batch_handle h, int tpr);
/* The current persistent launch shape (CTAs per SM resolved when automatic). */
int cem_batch_get_launch(cem_batch_handle h, int* warps_out, int* ctas_out, int* tpr_out);
/* ---- Multi-plan search (Sec. III: the optimiser could search several
 * candidate plans at once; Sec. V: evaluating many plans is expensive) ----
 * One scene, n_plans candidate skeletons, each realised by Algorithm 1 as a
 * problem of one batch (problem id = plan index, common seed, N, K).  With
 * halving_iters > 0 the budget is spent by successive halving: every
 * halving_iters iterations the active plans are ranked by their best
 * (class, cost, plan index) and the better half (at least `keep`) stays
 * active; eliminated plans stop where they are.  per_plan_out[n_plans] gets
 * every plan's result (each identical to cem_solve of that plan for the
 * iterations it ran), iters_out[n_plans] (may be NULL) those iteration
 * counts, *best_plan_out the plan with the lowest (class, cost, index).
 * Synchronous. */
typedef struct {
  uint64_t seed;
  int32_t N, K, iters, cov_mode;
  int32_t halving_iters; /* 0: every plan runs all iterations */
  int32_t keep;          /* plans kept at least (0 -> 1) */
} cem_multiplan_params;
int cem_multiplan_solve(const cem_scene_desc* scene, const cem_skeleton_desc* plans, int n_plans,
                        const cem_multiplan_params* p, cem_result* per_plan_out, int32_t* iters_out,
                        int32_t* best_plan_out);

/* ---- Learned cost surrogate (not in the paper) ---------------------------
 * An MLP score(x), x = [theta normalised to [-1, 1] by the bounds (clamped)
 * and zero-padded to 32 | 16 scene features], `depth` hidden layers
 * Linear + GELU of width `width`, a scalar output, then score = mu + sigma *
 * out.  BF16 weights and activations, FP32 accumulation on the tensor cores,
 * FP32 master weights.  Parameters are one FP32 vector: for each layer its
 * weights (out x in, row-major) then its biases. */
typedef struct cem_surrogate_ctx* cem_surrogate_handle;

/* in_dim must be 48; width 8..1024 (multiple of 8); depth 1..8.  Weights
 * start uniform in +-1/sqrt(fan_in) from `seed`; mu = 0, sigma = 1. */
int cem_surrogate_create(int in_dim, int width, int depth, uint64_t seed, cem_surrogate_handle* out);
int cem_surrogate_destroy(cem_surrogate_handle s);
int cem_surrogate_num_params(cem_surrogate_handle s);
/* Host copies of the FP32 parameters and of (mu, sigma); norm_h may be NULL.
 * set_params also clears the optimiser state. */
int cem_surrogate_set_params(cem_surrogate_handle s, const float* params_h, const float* norm_h);
int cem_surrogate_get_params(cem_surrogate_handle s, float* params_h, float* norm_h);
/* x_d[M][48] FP32 -> y_d[M] scores (stream-ordered).  Features are rounded
 * to BF16 (nearest even) before the first layer.  With width 256 and depth 4
 * this (and screening) runs one persistent fused tcgen05 kernel (128-row
 * tiles, two per SM in flight); when x_d is 16-byte aligned that kernel
 * reads and rounds the FP32 rows itself, otherwise a conversion pass runs
 * first (same scores, bit for bit).  If one of its bounded pipeline waits
 * expires, that CTA's scores are NaN and cem_surrogate_status reports the
 * code. */
int cem_surrogate_forward(cem_surrogate_handle s, const float* x_d, int M, float* y_d, void* stream);
/* Forward path for inference: 0 automatic (tcgen05 where the shape allows),
 * 1 the tiled mma.sync GEMM, 2 tcgen05 (CEM_ERR_UNSUPPORTED unless width 256
 * and depth 4).  Training follows cem_surrogate_set_gemm_path. */
int cem_surrogate_set_forward_path(cem_surrogate_handle s, int path);
/* Failure-detection test hook: while on != 0, tcgen05 forwards leave their
 * first weight-copy barrier without its arrival, so every CTA's first
 * pipeline wait runs out after 1 s with nothing in flight; the CTA then
 * frees its TMEM, writes NaN scores and sets status 1.  The context stays
 * usable; switch it off (0) for normal forwards. */
int cem_surrogate_test_expire_wait(cem_surrogate_handle s, int on);
/* The path inference takes now: 1 tiled GEMM, 2 tcgen05; -1 for NULL. */
int cem_surrogate_forward_path(cem_surrogate_handle s);
/* Dense layers of training (cem_surrogate_gradient, cem_surrogate_train)
 * and of the layer-by-layer inference forward: 0 automatic or 2 = the
 * tcgen05 GEMM (128 x 64 tiles, both operand majors read straight
 * by the tensor core, fused bias + GELU / GELU' / split-K epilogues; a layer
 * whose shape it does not take runs on the tiled kernel), 1 = the tiled
 * mma.sync GEMM.  Same products, FP32 accumulation order differs.  3 = an
 * FP32 debug path for cem_surrogate_gradient only: FP32 inputs, the FP32
 * master weights, FP32 activations and gradients, FP32 SIMT products summed
 * in ascending index order (no BF16 rounding anywhere; slow); training and
 * inference then take the automatic path.  Errors: CEM_ERR_INVALID_ARG for
 * another value.  A tcgen05 GEMM whose bounded wait expires sets status
 * 1 / 2 (read by cem_surrogate_status). */
int cem_surrogate_set_gemm_path(cem_surrogate_handle s, int path);
/* The path training GEMMs take now: 1 tiled, 2 tcgen05, 3 the FP32 debug
 * gradient; -1 for NULL. */
int cem_surrogate_gemm_path(cem_surrogate_handle s);
/* One AdamW step of the training loop's optimiser with a given gradient
 * grad_h (num_params floats, host): the same kernel and state (FP32 master
 * weights, FP32 moments, the step counter that sets the bias correction,
 * beta 0.9 / 0.999, eps 1e-8, decoupled decay on weights only) as
 * cem_surrogate_train; the BF16 copy is refreshed.  set_params clears the
 * moments and the counter.  Synchronous. */
int cem_surrogate_adamw_step(cem_surrogate_handle s, const float* grad_h, float lr, float weight_decay);
/* The optimiser's state: first and second moments (num_params floats each,
 * host) and the AdamW steps taken so far (the next step's bias correction
 * uses steps_taken + 1).  Set it to check or resume one step from a known
 * state; get it to checkpoint.  get synchronises. */
int cem_surrogate_set_adam_state(cem_surrogate_handle s, const float* m1_h, const float* m2_h, long long steps_taken);
int cem_surrogate_get_adam_state(cem_surrogate_handle s, float* m1_h, float* m2_h, long long* steps_taken);
/* Synchronises, writes and clears the tcgen05 forward's status word: 0, or
 * 1 / 2 if a wait for the weight copy / the MMAs expired.  A non-zero code
 * also makes cem_solve_screened return CEM_ERR_TIMEOUT. */
int cem_surrogate_status(cem_surrogate_handle s, int* status_h);
/* Full-batch gradient of mean((out - (t - mu)/sigma)^2) over M rows into
 * grad_h (num_params floats) and the loss into *loss_h.  Synchronous. */
int cem_surrogate_gradient(cem_surrogate_handle s, const float* x_d, const float* t_d, int M, float* grad_h,
                           float* loss_h);
/* `steps` AdamW steps (beta 0.9/0.999, eps 1e-8, decoupled decay on
 * weights) on minibatches of `batch` rows drawn with replacement by Philox
 * from (x_d[M][48], t_d[M]); normalize != 0 first sets (mu, sigma) to the
 * targets' mean and standard deviation.  loss_hist_h (steps floats) may be
 * NULL.  Synchronous. */
int cem_surrogate_train(cem_surrogate_handle s, const float* x_d, const float* t_d, int M, int batch, int steps,
                        float lr, float weight_decay, uint64_t seed, int normalize, float* loss_hist_h);
/* Training target of simulated samples: t_d[n] = log(1 + max(J_d[n], 0) +
 * 10 * cls_d[n]); a non-finite cost maps to log(1 + 1e6).  For costs below
 * 10 it is ordered like the CE key (class first, then J). */
int cem_surrogate_targets(const float* J_d, const uint8_t* cls_d, int N, float* t_d, void* stream);
/* The surrogate's input features of N parameter vectors (FP32 x_d[N][48]). */
int cem_surrogate_features(cem_surrogate_handle s, const float* theta_d, int N, int D, const float* lo_h,
                           const float* hi_h, const float* scene16_h, float* x_d, void* stream);
/* Screening: draw n_pool candidates from N(mean_d, chol_d chol_d^T) exactly
 * as cem_sample does, score them, keep the n_keep lowest scores (ties by
 * index) in ascending pool-index order: theta_keep_d[n_keep][D] and, if not
 * NULL, their pool indices keep_idx_d[n_keep]. */
int cem_surrogate_screen(cem_handle h, cem_surrogate_handle s, const float* mean_d, const float* chol_d, uint64_t seed,
                         uint32_t iter, uint32_t problem, int n_pool, int n_keep, const float* scene16_h,
                         float* theta_keep_d, int32_t* keep_idx_d, void* stream);
/* Screened CE loop: as cem_solve, but each iteration samples n_pool
 * candidates and rolls out p->N of them: the first n_explore draws
 * unscreened (exploration from the current distribution) and the
 * p->N - n_explore best-scored of the rest; the refit uses their simulated
 * costs only (elites never come from the surrogate).  Synchronous. */
int cem_solve_screened(cem_handle h, cem_surrogate_handle s, const float* scene16_h, const cem_solve_params* p,
                       int n_pool, int n_explore, cem_result* out);
/* Online fine-tuning of the surrogate during a screened run (not in the
 * paper, which has no surrogate): the features and score targets of every
 * simulated sample go into a device ring of `capacity` rows (a multiple of
 * p->N, at most 2^22; the most recent samples win), and after every `every`
 * iterations (0 = never, not after the last) the surrogate takes `steps`
 * AdamW steps of `batch` rows drawn from the filled part of the ring, with
 * the target normalisation of its earlier training kept.  seed + iteration
 * draws the batches. */
typedef struct {
  int32_t every, steps, batch, capacity;
  float lr, weight_decay;
  uint64_t seed;
} cem_finetune_params;
/* cem_solve_screened with the fine-tuning above; the surrogate's weights
 * change.  With every = 0 the result equals cem_solve_screened's.  Errors:
 * CEM_ERR_INVALID_ARG for bad fine-tune parameters, CEM_ERR_NO_MEMORY if the
 * ring does not fit, CEM_ERR_UNSUPPORTED unless the surrogate takes the 48
 * standard features.  Synchronous. */
int cem_solve_screened_ft(cem_handle h, cem_surrogate_handle s, const float* scene16_h, const cem_solve_params* p,
                          int n_pool, int n_explore, const cem_finetune_params* ft, cem_result* out);

/* Surrogate screening of every problem of the batch (not in the paper):
 * each screened iteration draws n_pool candidates per problem from its
 * distribution exactly as the single-problem screened loop does, scores
 * them with the surrogate s (features from the problem's bounds and its 16
 * scene values scene16_h[p * 16 ...]), and rolls out N_p of them: the first
 * n_explore draws and the N_p - n_explore best-scored of the rest; elites
 * come from simulated costs only.  A problem's screened batch iterations
 * equal cem_solve_screened of that problem bit for bit.  The batch keeps the
 * pointer s (keep the surrogate alive); s = NULL switches screening off.
 * Errors: CEM_ERR_UNSUPPORTED unless every N_p <= n_pool <= 2^20 and the
 * surrogate takes the 48 standard features, CEM_ERR_INVALID_ARG unless
 * 0 <= n_explore <= every N_p.  Synchronous (copies the tables once). */
int cem_batch_set_screening(cem_batch_handle h, cem_surrogate_handle s, const float* scene16_h, int n_pool,
                            int n_explore);
/* `iters` screened CE iterations of every active problem on `stream`
 * (asynchronous, not graph-captured).  A tcgen05 forward whose bounded wait
 * expired leaves NaN scores and its status word set (cem_surrogate_status).
 * Errors: CEM_ERR_INVALID_ARG without cem_batch_set_screening. */
int cem_batch_iterate_screened(cem_batch_handle h, int iters, void* stream);

/* Threads per block of the rollout kernel: 0 (automatic), 2, 4, 8, 16 or a
 * multiple of 32 up to 256. */
int cem_set_launch(cem_handle h, int block_threads);
/* Domain randomisation (Sec. IV-C: plans robust to bounded uncertainty in
 * friction or mass).  Every sample is rolled out in M environments (M = 1,
 * 2, 4, 8, 16 or 32): environment m scales every friction coefficient by
 * 1 + delta_mu (2u - 1) and the manipulated body's (block, object) mass by
 * 1 + delta_mass (2u' - 1), with u, u' = (word + 1) 2^-32 from the first two
 * words of the Philox block (m, 256, iteration, problem) under `seed`.  All
 * samples of an iteration share the M environments; the CE loops (cem_solve,
 * cem_solve_paper, cem_solve_screened) draw fresh ones each iteration (their
 * iteration and problem id), cem_rollout_batch uses iteration 0 and
 * problem 0.  A sample's cost is its mean over the environments and its class
 * the worst one (feasible only if feasible everywhere).  The M environments
 * of a sample run on M adjacent lanes (one lane each, whatever the lanes per
 * rollout setting) and are combined by warp shuffles.  M = 1 with both
 * spreads 0 switches it off.  Spreads in [0, 1).  Batches take it from
 * cem_batch_set_randomization; traces, the autotuner and cem_solve_static
 * run without it. */
int cem_set_randomization(cem_handle h, int M, float delta_mu, float delta_mass, uint64_t seed);
/* Lanes per rollout for pick-and-place scenes: 1, 8 or 32 (other scene
 * kinds always take one lane; the trace always one).  A group of G lanes
 * holds one rollout's state, splits the per-geometry contact queries and
 * neighbour-list rebuilds, and sums the contact forces with warp shuffles in
 * ascending geometry order: J and the class are bit-identical for every G.
 * With G > 1 a CTA of max(block, 32) threads carries block / G rollouts. */
int cem_set_threads_per_rollout(cem_handle h, int tpr);
/* The launch shape cem_rollout_batch uses for N samples: threads per block
 * and lanes per rollout. */
int cem_get_launch(cem_handle h, int N, int* block_out, int* tpr_out);
/* Times candidate block sizes (and, for pick-and-place scenes, 1, 8 or 32
 * lanes per rollout) for this scene and N on the current device and keeps
 * the fastest; results are cached in a text file ("<key>|<block>|<lanes>")
 * when cache_path is not NULL.  Writes the chosen block size; cem_get_launch
 * reports both. */
int cem_autotune(cem_handle h, int N, const char* cache_path, int* block_out);

/* Thread-local message of the last failing call ("" if none). */
const char* cem_last_error(void);
/* Library version string. */
const char* cem_version(void);

#ifdef __cplusplus
}
#endif
#endif
