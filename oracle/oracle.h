/*
 * FP64 CPU oracle for cross-entropy plan realization -- TEST INFRASTRUCTURE.
 *
 * This is the plain, slow, obviously-correct restatement of the method that
 * the CUDA library is checked against.  Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, constant or helper with the CUDA path; the two only consume the
 * same scene dictionaries produced by the seeded workload generator.
 *
 * What it restates (the paper is arXiv 2512.11571):
 *   - Algorithm 1 (Plan Parameter Cross-Entropy Optimization): sample,
 *     evaluate, update from the top N_e, loop (Sec. III-B).
 *   - The elite rules of Sec. III-B: fewer feasible than N_e -> use only the
 *     feasible ones; a single feasible -> add artificial noise; no sample
 *     reaching psi_g -> rank those whose actions all succeeded.
 *   - Problem 2 (Sec. III-B): cost = sum of per-step action costs (1 per
 *     step while the action is unfinished, Sec. IV-A) + end cost; the next
 *     action starts at the step after success (Problem 1, t_{0,i+1}=T_i+1).
 *   - The rigid-body dynamics x_{t+1} = f(x_t, a_i) (Eq. 1b) are not given
 *     by the paper (it uses IsaacGym); the model here is the documented
 *     reading: semi-implicit Euler, penalty contact, Coulomb friction.
 *   - Philox4x32-10 from Salmon et al., SC'11, "Parallel random numbers: as
 *     easy as 1, 2, 3", and the Box-Muller transform.
 *
 * Parity status (tests/test_oracle_*.py): Philox (published known-answer
 * vectors), Box-Muller statistics, selection, refit, the CE loop on a
 * quadratic; in the rollouts, ground friction, the position and heading PD
 * responses, the time-to-reach cost, body-contact momentum and energy, the
 * contact point, the force-limit penalty, free flight, resting penetration,
 * ramp statics and sliding, IK/FK, the pick-and-place action sequencing
 * (attach, grip tolerance, release velocity, settling) and the goal tests
 * and costs of every task are pinned by closed forms, invariants and
 * hand-built special cases.  The paper prints no worked example, so no
 * whole-task cost is pinned to a printed value; the whole-task costs are
 * pinned through those parts.
 */
#ifndef CEM_ORACLE_H
#define CEM_ORACLE_H
#include <stdint.h>

#define OR_MAX_D 18
#define OR_MAX_ACT 6
#define OR_MAX_GEOM 16
#define OR_MAX_SLAB 6
#define OR_TRACE_W 20
#define OR_MAX_CORNERS 48

enum { OR_QUAD = 0, OR_REACH = 1, OR_PUSH = 2, OR_PICKPLACE = 3 };
enum { OR_MOVE = 0, OR_PUSH_ACT = 1, OR_GRASP = 2, OR_PLACE = 3 };

/* One problem: scene + plan skeleton, all in SI units.  Field meaning is the
 * workload generator's dictionary keys. */
typedef struct {
  int32_t kind, T, cost_step, D;
  double dt, g, eps;
  /* planar base */
  double base_half[2], base_mass, base_mu, base_start[3], base_v0[3], yaw_kp, yaw_kd;
  /* free block (push) */
  double block_half[2], block_mass, block_mu, block_start[3], block_v0[3];
  double k_contact, c_contact, contact_mu, force_limit;
  double w_time, w_goal, w_viol, w_obj, w_base;
  double goal_center[3], goal_half[3];
  /* pick-place object and arm */
  double obj_half, obj_mass, obj_mu, obj_start[3], obj_v0[3];
  double arm_l1, arm_l2, arm_z, arm_kp, arm_kd, arm_home[2];
  double grasp_reach, grasp_kp, grip_tol;
  double obj_region_c[3], obj_region_h[3], base_region_c[3], base_region_h[3];
  int32_t goal_obj_region, goal_obj_held, goal_base_region, n_geoms;
  int32_t geom_nslab[OR_MAX_GEOM], geom_base[OR_MAX_GEOM], geom_obj[OR_MAX_GEOM];
  double slab[OR_MAX_GEOM][OR_MAX_SLAB][5]; /* nx, ny, nz, lo, hi */
  /* quadratic */
  double theta_star[OR_MAX_D], A[OR_MAX_D * OR_MAX_D];
  /* skeleton */
  int32_t n_act, act_kind[OR_MAX_ACT], act_off[OR_MAX_ACT], act_ref_target[OR_MAX_ACT];
  double act_nom[OR_MAX_ACT][3], act_yaw[OR_MAX_ACT];
  double lo[OR_MAX_D], hi[OR_MAX_D];
  /* initial sampling region of each action (Sec. III-B, IV-A): 0 = the box
   * [lo, hi] of its parameters, 1 = an annulus for a move goal's (dx, dy):
   * act_ring = (centre x, centre y, inner radius, outer radius) */
  int32_t act_region[OR_MAX_ACT];
  double act_ring[OR_MAX_ACT][4];
  /* moveTo controller of the pick-place base (Sec. IV-A): 0 = PD to the
   * goal; 1 = A* waypoints (base_infl = footprint growth) tracked by PD,
   * advancing within wp_switch of a waypoint, with an integral term
   * (gain pid_ki * kp, active within pid_irad of the goal, |I| <= pid_imax
   * per axis) on the final one */
  int32_t base_ctrl;
  double base_infl, wp_switch, pid_ki, pid_irad, pid_imax;
} or_scene;

typedef struct {
  uint64_t add, mul, div, sqrt, transc;
} or_ops;

#ifdef __cplusplus
extern "C" {
/* Test switch: when on, the push base-block contact test runs on every step
 * instead of only where the block's bounding circle reaches the base (the
 * skip is exact; results must be identical either way). */
void or_set_exhaustive_contacts(int on);
#endif
/* Philox4x32-10 block: out = philox(ctr, key). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Raw Philox words for N samples: words[n*4*ncall + 4*c + i]. */
void or_philox_words(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D, uint32_t* words);
/* Standard normals z[N*D] and theta = mean + chol z (chol lower, row-major). */
void or_normals(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D, double* z);
void or_sample(uint64_t seed, uint32_t iter, uint32_t problem, int N, int D, const double* mean,
               const double* chol, double* theta);
/* Uniform initial sampling inside each parameter's region (paper's
 * iteration-0 rule): the box [lo, hi], or area-uniform in an annulus for a
 * move goal flagged act_region = 1. */
void or_sample_uniform(const or_scene* s, uint64_t seed, uint32_t problem, int N, double* theta);
/* Samples of CE iteration j under the linear schedule: n0 at j = 0 to n1 at
 * j = j1, constant after (Sec. IV-A: 3000 -> 300 by iteration 10). */
int or_n_env(int n0, int n1, int j1, int j);
/* Roll out N parameter vectors; nthreads <= 0 -> hardware concurrency. */
void or_rollout(const or_scene* s, const double* theta, int N, double* J, uint8_t* cls, int nthreads);
/* Domain randomisation factors of CE iteration iter: friction scale smu[M]
 * and manipulated-body mass scale sm[M] (Philox block (m, 256, iter, problem)). */
void or_dr_factors(uint64_t seed, uint32_t iter, uint32_t problem, int M, double dmu, double dm, double* smu,
                   double* sm);
/* Rollouts under M randomised environments: J = mean, class = worst. */
void or_rollout_dr(const or_scene* s, const double* theta, int N, int M, double dmu, double dm, uint64_t seed,
                   uint32_t iter, uint32_t problem, double* J, uint8_t* cls, int nthreads);
/* Per-step state trace of one rollout: states[(steps) * OR_TRACE_W]. */
void or_rollout_trace(const or_scene* s, const double* theta, int steps, double* states);
/* The end of a pick-place rollout on a given final state (trace layout:
 * base x, y at 0, 1, object x, y, z at 9, 10, 11, attached at 15): the goal
 * test psi_g, the plan cost J = w_time t_done + w_obj d_obj + w_base d_base
 * and the class (complete = every action succeeded). */
void or_pickplace_final(const or_scene* s, const double* state, int complete, double t_done, double* J, int* cls);
/* Flop tally of one rollout (added into *ops); returns the step count. */
int or_rollout_count(const or_scene* s, const double* theta, or_ops* ops);
/* Elite selection on FP32 costs: ascending (class, J, index); writes the
 * K_eff elite indices and returns K_eff. */
int or_select(const float* J, const uint8_t* cls, int N, int K, int32_t* idx);
/* Refit mean/cov/chol (FP64) from elites; returns 0, or -4 if not PD. */
int or_refit(const double* theta, int N, int D, const int32_t* idx, int k_eff, const double* lo,
             const double* hi, int diag, double* mean, double* cov, double* chol);
/* Corners of the base planner's visibility graph: xy[2 i], xy[2 i + 1];
 * returns their number (the first `cap` are written). */
int or_base_corners(const or_scene* s, double* xy, int cap);
/* A* waypoints of the base from (sx, sy) to (gx, gy), ending with the goal;
 * returns their number (the first `cap` are written). */
int or_plan_path(const or_scene* s, double sx, double sy, double gx, double gy, double* xy, int cap);
/* Mean distance from the centre over a (2a x 2b) rectangle (numerical). */
double or_mean_radius(double a, double b);
/* Full CE loop (Algorithm 1), FP64.  history[iters] = best J so far. */
int or_cem(const or_scene* s, uint64_t seed, uint32_t problem, int N, int K, int iters, int diag,
           int nthreads, double* best_theta, double* best_J, int* best_cls, double* mean,
           double* cov, double* history, double* keff_hist);
/* or_cem with every iteration's rollouts domain-randomised (or_rollout_dr
 * with the loop's iteration index). */
int or_cem_dr(const or_scene* s, uint64_t seed, uint32_t problem, int N, int K, int iters, int diag, int M,
              double dmu, double dm, uint64_t dr_seed, int nthreads, double* best_theta, double* best_J,
              int* best_cls, double* mean, double* cov, double* history);
/* The paper's CE variant (Sec. III-B, IV-A): iteration 0 draws n0 samples
 * uniformly in the parameter regions, iteration j >= 1 draws or_n_env(j)
 * Gaussian samples (Philox iteration j) from the refit; class_hist[4 j + c]
 * = samples of class c in iteration j, n_hist[j] = samples drawn. */
int or_cem_paper(const or_scene* s, uint64_t seed, uint32_t problem, int n0, int n1, int j1, int K, int iters,
                 int diag, int nthreads, double* best_theta, double* best_J, int* best_cls, double* mean,
                 double* cov, double* history, int* class_hist, int* n_hist);
#ifdef __cplusplus
}
#endif
#endif
