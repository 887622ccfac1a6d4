"""FP64 CPU oracle for the CEM plan-realization path -- TEST INFRASTRUCTURE.

Plain, slow restatement of the method (Algorithm 1 of arXiv 2512.11571 and
the library's documented dynamics reading) that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference legs may import this package.  It shares no code
with the CUDA path; both consume the dictionaries of the ``workload``
package, each with its own marshalling.

Parity status: see ``oracle.h``.  The paper prints no worked example, so no
whole-task rollout cost is pinned to a printed value; every part of each
rollout (controllers, contacts, friction, integration, action switching,
goal tests and costs) is pinned by closed forms, invariants and hand-built
special cases in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = ["sample.cpp", "rollout.cpp", "cem.cpp", "plan2d.cpp"]

MAX_D, MAX_ACT, MAX_GEOM, MAX_SLAB, TRACE_W = 18, 6, 16, 6, 20
KIND = {"quadratic": 0, "reach": 1, "push": 2, "pickplace": 3}
ACT = {"move": 0, "push": 1, "grasp": 2, "place": 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (portable flags: x86 and Arm)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(HERE, "oracle.h"), os.path.join(HERE, "plan2d.h")])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Scene(C.Structure):
    D3 = C.c_double * 3
    _fields_ = [
        ("kind", C.c_int32), ("T", C.c_int32), ("cost_step", C.c_int32), ("D", C.c_int32),
        ("dt", C.c_double), ("g", C.c_double), ("eps", C.c_double),
        ("base_half", C.c_double * 2), ("base_mass", C.c_double), ("base_mu", C.c_double),
        ("base_start", C.c_double * 3), ("base_v0", C.c_double * 3), ("yaw_kp", C.c_double),
        ("yaw_kd", C.c_double),
        ("block_half", C.c_double * 2), ("block_mass", C.c_double), ("block_mu", C.c_double),
        ("block_start", C.c_double * 3), ("block_v0", C.c_double * 3),
        ("k_contact", C.c_double), ("c_contact", C.c_double), ("contact_mu", C.c_double),
        ("force_limit", C.c_double),
        ("w_time", C.c_double), ("w_goal", C.c_double), ("w_viol", C.c_double),
        ("w_obj", C.c_double), ("w_base", C.c_double),
        ("goal_center", C.c_double * 3), ("goal_half", C.c_double * 3),
        ("obj_half", C.c_double), ("obj_mass", C.c_double), ("obj_mu", C.c_double),
        ("obj_start", C.c_double * 3), ("obj_v0", C.c_double * 3),
        ("arm_l1", C.c_double), ("arm_l2", C.c_double), ("arm_z", C.c_double),
        ("arm_kp", C.c_double), ("arm_kd", C.c_double), ("arm_home", C.c_double * 2),
        ("grasp_reach", C.c_double), ("grasp_kp", C.c_double), ("grip_tol", C.c_double),
        ("obj_region_c", C.c_double * 3), ("obj_region_h", C.c_double * 3),
        ("base_region_c", C.c_double * 3), ("base_region_h", C.c_double * 3),
        ("goal_obj_region", C.c_int32), ("goal_obj_held", C.c_int32),
        ("goal_base_region", C.c_int32), ("n_geoms", C.c_int32),
        ("geom_nslab", C.c_int32 * MAX_GEOM), ("geom_base", C.c_int32 * MAX_GEOM),
        ("geom_obj", C.c_int32 * MAX_GEOM),
        ("slab", ((C.c_double * 5) * MAX_SLAB) * MAX_GEOM),
        ("theta_star", C.c_double * MAX_D), ("A", C.c_double * (MAX_D * MAX_D)),
        ("n_act", C.c_int32), ("act_kind", C.c_int32 * MAX_ACT), ("act_off", C.c_int32 * MAX_ACT),
        ("act_ref_target", C.c_int32 * MAX_ACT),
        ("act_nom", (C.c_double * 3) * MAX_ACT), ("act_yaw", C.c_double * MAX_ACT),
        ("lo", C.c_double * MAX_D), ("hi", C.c_double * MAX_D),
        ("act_region", C.c_int32 * MAX_ACT), ("act_ring", (C.c_double * 4) * MAX_ACT),
        ("base_ctrl", C.c_int32), ("base_infl", C.c_double), ("wp_switch", C.c_double), ("pid_ki", C.c_double),
        ("pid_irad", C.c_double), ("pid_imax", C.c_double),
    ]


class _Ops(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("add", "mul", "div", "sqrt", "transc")]


def _set(arr, vals):
    for i, v in enumerate(vals):
        arr[i] = v


def pack(scene: dict, skel: dict, T: int | None = None) -> _Scene:
    """Marshal a workload (scene, skeleton) pair into the oracle's struct."""
    s = _Scene()
    s.kind = KIND[scene["kind"]]
    s.T = int(scene["T"] if T is None else T)
    s.cost_step = 1 if scene.get("cost_mode", "interp") == "step" else 0
    s.D = len(skel["lo"])
    if s.D > MAX_D:
        raise ValueError("D > 18")
    s.dt, s.g, s.eps = scene["dt"], scene["g"], scene.get("eps", 0.0)
    for key in ("base_mass", "base_mu", "yaw_kp", "yaw_kd", "block_mass", "block_mu", "k_contact",
                "c_contact", "contact_mu", "force_limit", "w_time", "w_goal", "w_viol", "w_obj",
                "w_base", "obj_half", "obj_mass", "obj_mu", "arm_l1", "arm_l2", "arm_z", "arm_kp",
                "arm_kd", "grasp_reach", "grasp_kp", "grip_tol"):
        if key in scene:
            setattr(s, key, float(scene[key]))
    for key in ("base_half", "base_start", "block_half", "block_start", "goal_center", "goal_half",
                "obj_start", "arm_home", "base_v0", "block_v0", "obj_v0"):
        if key in scene:
            _set(getattr(s, key), scene[key])
    for key, name in (("obj_region_center", "obj_region_c"), ("obj_region_half", "obj_region_h"),
                      ("base_region_center", "base_region_c"), ("base_region_half", "base_region_h")):
        if key in scene:
            _set(getattr(s, name), scene[key])
    for key in ("goal_obj_region", "goal_obj_held", "goal_base_region"):
        setattr(s, key, int(bool(scene.get(key, False))))
    if scene.get("base_controller", "pd") == "astar":  # A* waypoints + PID (Sec. IV-A)
        s.base_ctrl = 1
        s.base_infl, s.wp_switch = scene["base_inflate"], scene["wp_switch"]
        s.pid_ki, s.pid_irad, s.pid_imax = scene["pid_ki"], scene["pid_irad"], scene["pid_imax"]
    geoms = scene.get("geoms", [])
    if len(geoms) > MAX_GEOM:
        raise ValueError("too many geometries")
    s.n_geoms = len(geoms)
    for gi, gm in enumerate(geoms):
        s.geom_nslab[gi] = len(gm["slabs"])
        s.geom_base[gi] = int(gm["base"])
        s.geom_obj[gi] = int(gm["obj"])
        for si, sl in enumerate(gm["slabs"]):
            _set(s.slab[gi][si], sl)
    if scene["kind"] == "quadratic":
        _set(s.theta_star, scene["theta_star"])
        D = s.D
        for i in range(D):
            for j in range(D):
                s.A[i * D + j] = scene["A"][i * D + j]
    acts = skel["actions"]
    s.n_act = len(acts)
    off = 0
    width = {"move": 3, "push": 3, "grasp": 2, "place": 3}
    for i, a in enumerate(acts):
        s.act_kind[i] = ACT[a["kind"]]
        s.act_off[i] = off
        s.act_ref_target[i] = 1 if a.get("success_ref", "nominal") == "target" else 0
        _set(s.act_nom[i], a["nominal"])
        s.act_yaw[i] = a.get("yaw", 0.0)
        reg = a.get("region")
        if reg is not None:  # annulus of a move goal: centre (x, y), radii (inner, outer)
            if reg["kind"] != "ring" or a["kind"] != "move":
                raise ValueError("only move goals take an annulus region")
            s.act_region[i] = 1
            _set(s.act_ring[i], [reg["center"][0], reg["center"][1], reg["radii"][0], reg["radii"][1]])
        off += width[a["kind"]]
    if acts and off != s.D:
        raise ValueError("skeleton width does not match bounds")
    _set(s.lo, skel["lo"])
    _set(s.hi, skel["hi"])
    return s


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp, fp = C.POINTER(C.c_double), C.POINTER(C.c_float)
            u8p, i32p, u32p = C.POINTER(C.c_uint8), C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
            sp = C.POINTER(_Scene)
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_set_exhaustive_contacts.argtypes = [C.c_int]
            L.or_philox_words.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, u32p]
            L.or_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, dp]
            L.or_sample.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, dp, dp, dp]
            L.or_sample_uniform.argtypes = [sp, C.c_uint64, C.c_uint32, C.c_int, dp]
            L.or_rollout.argtypes = [sp, dp, C.c_int, dp, u8p, C.c_int]
            L.or_rollout_trace.argtypes = [sp, dp, C.c_int, dp]
            L.or_pickplace_final.argtypes = [sp, dp, C.c_int, C.c_double, dp, C.POINTER(C.c_int)]
            L.or_rollout_count.argtypes = [sp, dp, C.POINTER(_Ops)]
            L.or_rollout_count.restype = C.c_int
            L.or_select.argtypes = [fp, u8p, C.c_int, C.c_int, i32p]
            L.or_select.restype = C.c_int
            L.or_refit.argtypes = [dp, C.c_int, C.c_int, i32p, C.c_int, dp, dp, C.c_int, dp, dp, dp]
            L.or_refit.restype = C.c_int
            L.or_mean_radius.argtypes = [C.c_double, C.c_double]
            L.or_mean_radius.restype = C.c_double
            L.or_cem.argtypes = [sp, C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 dp, dp, C.POINTER(C.c_int), dp, dp, dp, dp]
            L.or_cem.restype = C.c_int
            L.or_dr_factors.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_double, C.c_double,
                                        dp, dp]
            L.or_rollout_dr.argtypes = [sp, dp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint64,
                                        C.c_uint32, C.c_uint32, dp, u8p, C.c_int]
            L.or_cem_dr.argtypes = [sp, C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_double, C.c_double, C.c_uint64, C.c_int, dp, dp, C.POINTER(C.c_int),
                                    dp, dp, dp]
            L.or_cem_dr.restype = C.c_int
            L.or_n_env.argtypes = [C.c_int] * 4
            L.or_base_corners.argtypes = [sp, dp, C.c_int]
            L.or_base_corners.restype = C.c_int
            L.or_plan_path.argtypes = [sp, C.c_double, C.c_double, C.c_double, C.c_double, dp, C.c_int]
            L.or_plan_path.restype = C.c_int
            L.or_n_env.restype = C.c_int
            L.or_cem_paper.argtypes = [sp, C.c_uint64, C.c_uint32] + [C.c_int] * 7 + [
                dp, dp, C.POINTER(C.c_int), dp, dp, dp, i32p, i32p]
            L.or_cem_paper.restype = C.c_int
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def philox_words(seed, it, problem, N, D):
    nc = (D + 3) // 4
    w = np.zeros((N, nc * 4), np.uint32)
    lib().or_philox_words(seed, it, problem, N, D, _p(w, C.c_uint32))
    return w


def normals(seed, it, problem, N, D):
    z = np.zeros((N, D), np.float64)
    lib().or_normals(seed, it, problem, N, D, _p(z, C.c_double))
    return z


def sample(seed, it, problem, N, mean, chol):
    mean = np.ascontiguousarray(mean, np.float64)
    chol = np.ascontiguousarray(chol, np.float64)
    D = mean.shape[0]
    th = np.zeros((N, D), np.float64)
    lib().or_sample(seed, it, problem, N, D, _p(mean, C.c_double), _p(chol, C.c_double), _p(th, C.c_double))
    return th


def sample_uniform(scene, skel, seed, problem, N):
    s = pack(scene, skel)
    th = np.zeros((N, s.D), np.float64)
    lib().or_sample_uniform(C.byref(s), seed, problem, N, _p(th, C.c_double))
    return th


def rollout(scene, skel, theta, T=None, nthreads=0):
    s = pack(scene, skel, T)
    th = np.ascontiguousarray(theta, np.float64).reshape(-1, s.D)
    N = th.shape[0]
    J = np.zeros(N, np.float64)
    cls = np.zeros(N, np.uint8)
    lib().or_rollout(C.byref(s), _p(th, C.c_double), N, _p(J, C.c_double), _p(cls, C.c_uint8), nthreads)
    return J, cls


def trace(scene, skel, theta, steps):
    s = pack(scene, skel, steps)
    th = np.ascontiguousarray(theta, np.float64).reshape(-1)
    out = np.zeros((steps, TRACE_W), np.float64)
    lib().or_rollout_trace(C.byref(s), _p(th, C.c_double), steps, _p(out, C.c_double))
    return out


def pickplace_final(scene, skel, state, complete, t_done):
    """(J, class) that a pick-place rollout ending in `state` (one row of the
    trace layout) with every action done (complete) by t_done gets."""
    s = pack(scene, skel)
    st = np.zeros(TRACE_W, np.float64)
    st[:len(state)] = state
    J = C.c_double()
    c = C.c_int()
    lib().or_pickplace_final(C.byref(s), _p(st, C.c_double), int(bool(complete)), float(t_done), C.byref(J),
                             C.byref(c))
    return J.value, c.value


def count_ops(scene, skel, theta, T=None):
    """Summed op tally over the given parameter vectors, and the step count."""
    s = pack(scene, skel, T)
    th = np.ascontiguousarray(theta, np.float64).reshape(-1, s.D)
    ops = _Ops()
    steps = 0
    for n in range(th.shape[0]):
        row = np.ascontiguousarray(th[n])
        steps += lib().or_rollout_count(C.byref(s), _p(row, C.c_double), C.byref(ops))
    return dict(add=ops.add, mul=ops.mul, div=ops.div, sqrt=ops.sqrt, transc=ops.transc, steps=steps)


def select(J, cls, K):
    J = np.ascontiguousarray(J, np.float32)
    cls = np.ascontiguousarray(cls, np.uint8)
    N = J.shape[0]
    idx = np.zeros(max(K, 1), np.int32)
    k = lib().or_select(_p(J, C.c_float), _p(cls, C.c_uint8), N, K, _p(idx, C.c_int32))
    return idx[:k]


def refit(theta, idx, lo, hi, diag=False, mean=None, cov=None, chol=None):
    theta = np.ascontiguousarray(theta, np.float64)
    N, D = theta.shape
    idx = np.ascontiguousarray(idx, np.int32)
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    mean = np.zeros(D) if mean is None else np.array(mean, np.float64)
    cov = np.zeros((D, D)) if cov is None else np.array(cov, np.float64)
    chol = np.zeros((D, D)) if chol is None else np.array(chol, np.float64)
    rc = lib().or_refit(_p(theta, C.c_double), N, D, _p(idx, C.c_int32), len(idx), _p(lo, C.c_double),
                        _p(hi, C.c_double), int(diag), _p(mean, C.c_double), _p(cov, C.c_double),
                        _p(chol, C.c_double))
    return rc, mean, cov, chol


def mean_radius(a, b):
    return lib().or_mean_radius(a, b)


def cem(scene, skel, seed, N, K, iters, problem=0, diag=False, nthreads=0):
    s = pack(scene, skel)
    D = s.D
    bt = np.zeros(D)
    bJ = C.c_double()
    bc = C.c_int()
    mean = np.zeros(D)
    cov = np.zeros((D, D))
    hist = np.zeros(iters)
    keff = np.zeros(iters)
    rc = lib().or_cem(C.byref(s), seed, problem, N, K, iters, int(diag), nthreads, _p(bt, C.c_double),
                      C.byref(bJ), C.byref(bc), _p(mean, C.c_double), _p(cov, C.c_double),
                      _p(hist, C.c_double), _p(keff, C.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle CE loop failed: {rc}")
    return dict(best_theta=bt, best_J=bJ.value, best_cls=bc.value, mean=mean, cov=cov, history=hist,
                k_eff=keff)


def n_env(n0, n1, j1, j):
    """Samples of CE iteration j under the linear schedule (Sec. IV-A)."""
    return lib().or_n_env(n0, n1, j1, j)


def cem_paper(scene, skel, seed, n0=3000, n1=300, j1=10, K=50, iters=20, problem=0, diag=True, nthreads=0):
    """The paper's CE variant: uniform initial sampling in the parameter
    regions, the n_env schedule, the independent-normal model (diag)."""
    s = pack(scene, skel)
    D = s.D
    bt = np.zeros(D)
    bJ = C.c_double()
    bc = C.c_int()
    mean = np.zeros(D)
    cov = np.zeros((D, D))
    hist = np.zeros(iters)
    counts = np.zeros((iters, 4), np.int32)
    ns = np.zeros(iters, np.int32)
    rc = lib().or_cem_paper(C.byref(s), seed, problem, n0, n1, j1, K, iters, int(diag), nthreads,
                            _p(bt, C.c_double), C.byref(bJ), C.byref(bc), _p(mean, C.c_double),
                            _p(cov, C.c_double), _p(hist, C.c_double), _p(counts, C.c_int32),
                            _p(ns, C.c_int32))
    if rc != 0:
        raise RuntimeError(f"oracle CE loop failed: {rc}")
    return dict(best_theta=bt, best_J=bJ.value, best_cls=bc.value, mean=mean, cov=cov, history=hist,
                class_counts=counts, n_env=ns)


def set_exhaustive_contacts(on):
    """Test switch: run the push base-block contact test on every step instead
    of only where the block's bounding circle reaches the base."""
    lib().or_set_exhaustive_contacts(int(bool(on)))


def dr_factors(seed, it, problem, M, dmu, dm):
    """Friction and mass scales of the M randomised environments of iteration it."""
    smu, sm = np.zeros(M), np.zeros(M)
    lib().or_dr_factors(seed, it, problem, M, dmu, dm, _p(smu, C.c_double), _p(sm, C.c_double))
    return smu, sm


def rollout_dr(scene, skel, theta, M, dmu, dm, seed, it=0, problem=0, T=None, nthreads=0):
    """Mean cost and worst class of each sample over M randomised environments."""
    s = pack(scene, skel, T)
    th = np.ascontiguousarray(theta, np.float64).reshape(-1, s.D)
    N = th.shape[0]
    J = np.zeros(N, np.float64)
    cls = np.zeros(N, np.uint8)
    lib().or_rollout_dr(C.byref(s), _p(th, C.c_double), N, M, dmu, dm, seed, it, problem, _p(J, C.c_double),
                        _p(cls, C.c_uint8), nthreads)
    return J, cls


def cem_dr(scene, skel, seed, N, K, iters, M, dmu, dm, dr_seed, problem=0, diag=False, nthreads=0):
    s = pack(scene, skel)
    D = s.D
    bt = np.zeros(D)
    bJ = C.c_double()
    bc = C.c_int()
    mean = np.zeros(D)
    cov = np.zeros((D, D))
    hist = np.zeros(iters)
    rc = lib().or_cem_dr(C.byref(s), seed, problem, N, K, iters, int(diag), M, dmu, dm, dr_seed, nthreads,
                         _p(bt, C.c_double), C.byref(bJ), C.byref(bc), _p(mean, C.c_double),
                         _p(cov, C.c_double), _p(hist, C.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle CE loop failed: {rc}")
    return dict(best_theta=bt, best_J=bJ.value, best_cls=bc.value, mean=mean, cov=cov, history=hist)


def base_corners(scene, skel):
    """Corners of the base planner's visibility graph, shape (n, 2)."""
    s = pack(scene, skel)
    xy = np.zeros(2 * 64)
    n = lib().or_base_corners(C.byref(s), _p(xy, C.c_double), 64)
    return xy[:2 * min(n, 64)].reshape(-1, 2)


def plan_path(scene, skel, start, goal):
    """A* waypoints of the base from start to goal (ending with the goal)."""
    s = pack(scene, skel)
    xy = np.zeros(2 * 64)
    n = lib().or_plan_path(C.byref(s), float(start[0]), float(start[1]), float(goal[0]), float(goal[1]),
                           _p(xy, C.c_double), 64)
    return xy[:2 * min(n, 64)].reshape(-1, 2)
