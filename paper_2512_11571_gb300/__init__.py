"""Python binding of libcemtamp, the GB300 cross-entropy plan-realization library.

Argument marshalling only: every step of the path (Philox sampling, the
fused rollout, elite selection and refit, the device-resident CE loop) runs
in the library's CUDA kernels.  PyTorch is used for device memory and
streams.  The functions keep the C names of ``include/cemtamp.h``; ``Scene``
wraps a handle.  There is no CPU fallback: importing works without a GPU,
but every call needs the compiled library and a CUDA device and raises
otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcemtamp.so")
# the same library with the kernels' bounds checks compiled in (build.build(debug=True))
DEBUG_LIB_PATH = os.path.join(HERE, "libcemtamp_debug.so")

MAX_D, MAX_ACTIONS, MAX_GEOMS, MAX_SLABS, MAX_K, TRACE_W = 18, 6, 16, 6, 4096, 20
SCENE_KIND = {"quadratic": 0, "reach": 1, "push": 2, "pickplace": 3}
ACTION_KIND = {"move": 0, "push": 1, "grasp": 2, "place": 3}
ACTION_WIDTH = {"move": 3, "push": 3, "grasp": 2, "place": 3}
COV = {"full": 0, "diag": 1}
STATUS = {0: "CEM_OK", -1: "CEM_ERR_INVALID_ARG", -2: "CEM_ERR_CUDA", -3: "CEM_ERR_TIMEOUT",
          -4: "CEM_ERR_NOT_PD", -5: "CEM_ERR_UNSUPPORTED", -6: "CEM_ERR_NO_MEMORY"}

EXPORTS = [
    "cem_scene_create", "cem_scene_destroy", "cem_sample", "cem_philox_words", "cem_rollout_batch",
    "cem_rollout_trace", "cem_refit", "cem_solve", "cem_solve_static", "cem_set_launch", "cem_autotune",
    "cem_batch_create", "cem_batch_destroy", "cem_batch_reset", "cem_batch_iterate", "cem_batch_read",
    "cem_batch_set_launch", "cem_batch_autotune", "cem_batch_steps_per_iteration",
    "cem_batch_set_threads_per_rollout", "cem_batch_get_launch", "cem_set_threads_per_rollout", "cem_get_launch",
    "cem_solve_paper", "cem_sample_uniform", "cem_n_env", "cem_debug_status", "cem_debug_selftest", "cem_test_fail_allocation", "cem_surrogate_test_expire_wait",
    "cem_set_randomization",
    "cem_batch_set_active", "cem_multiplan_solve", "cem_base_path",
    "cem_batch_set_randomization", "cem_batch_set_state", "cem_batch_state_bytes", "cem_batch_set_timing",
    "cem_batch_stage_ms", "cem_batch_set_screening", "cem_batch_iterate_screened",
    "cem_surrogate_create", "cem_surrogate_destroy", "cem_surrogate_num_params", "cem_surrogate_set_params",
    "cem_surrogate_get_params", "cem_surrogate_forward", "cem_surrogate_gradient", "cem_surrogate_train",
    "cem_surrogate_features", "cem_surrogate_screen", "cem_solve_screened", "cem_surrogate_targets",
    "cem_solve_screened_ft",
    "cem_surrogate_set_forward_path", "cem_surrogate_forward_path", "cem_surrogate_status",
    "cem_surrogate_set_gemm_path", "cem_surrogate_gemm_path", "cem_surrogate_adamw_step",
    "cem_surrogate_set_adam_state", "cem_surrogate_get_adam_state",
    "cem_last_error", "cem_version",
]


class CemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


# ----------------------------------------------------------- C structures
class cem_slab(C.Structure):
    _fields_ = [("n", C.c_float * 3), ("lo", C.c_float), ("hi", C.c_float)]


class cem_geom(C.Structure):
    _fields_ = [("n_slabs", C.c_int32), ("collide_base", C.c_int32), ("collide_object", C.c_int32),
                ("reserved", C.c_int32), ("slab", cem_slab * MAX_SLABS)]


F3 = C.c_float * 3
F2 = C.c_float * 2


class cem_scene_desc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("T", C.c_int32), ("cost_mode", C.c_int32), ("reserved0", C.c_int32),
        ("dt", C.c_float), ("g", C.c_float), ("eps", C.c_float),
        ("base_half", F2), ("base_mass", C.c_float), ("base_mu", C.c_float), ("base_start", F3),
        ("base_v0", F3), ("yaw_kp", C.c_float), ("yaw_kd", C.c_float),
        ("block_half", F2), ("block_mass", C.c_float), ("block_mu", C.c_float), ("block_start", F3),
        ("block_v0", F3),
        ("k_contact", C.c_float), ("c_contact", C.c_float), ("contact_mu", C.c_float),
        ("force_limit", C.c_float),
        ("w_time", C.c_float), ("w_goal", C.c_float), ("w_viol", C.c_float), ("w_obj", C.c_float),
        ("w_base", C.c_float),
        ("goal_center", F3), ("goal_half", F3),
        ("obj_half", C.c_float), ("obj_mass", C.c_float), ("obj_mu", C.c_float), ("obj_start", F3),
        ("obj_v0", F3),
        ("arm_l1", C.c_float), ("arm_l2", C.c_float), ("arm_z", C.c_float), ("arm_kp", C.c_float),
        ("arm_kd", C.c_float), ("arm_home", F2),
        ("grasp_reach", C.c_float), ("grasp_kp", C.c_float), ("grip_tol", C.c_float),
        ("obj_region_c", F3), ("obj_region_h", F3), ("base_region_c", F3), ("base_region_h", F3),
        ("goal_obj_region", C.c_int32), ("goal_obj_held", C.c_int32), ("goal_base_region", C.c_int32),
        ("n_geoms", C.c_int32),
        ("geom", cem_geom * MAX_GEOMS),
        ("theta_star", C.c_float * MAX_D), ("A", C.c_float * (MAX_D * MAX_D)),
        ("base_controller", C.c_int32), ("base_inflate", C.c_float), ("wp_switch", C.c_float),
        ("pid_ki", C.c_float), ("pid_irad", C.c_float), ("pid_imax", C.c_float),
    ]


class cem_action_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("theta_offset", C.c_int32), ("success_ref", C.c_int32),
                ("init_region", C.c_int32), ("nominal", F3), ("yaw", C.c_float), ("region", C.c_float * 4)]


class cem_skeleton_desc(C.Structure):
    _fields_ = [("n_actions", C.c_int32), ("D", C.c_int32), ("action", cem_action_desc * MAX_ACTIONS),
                ("lo", C.c_float * MAX_D), ("hi", C.c_float * MAX_D)]


class cem_solve_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("N", C.c_int32), ("K", C.c_int32), ("iters", C.c_int32),
                ("cov_mode", C.c_int32), ("problem", C.c_uint32), ("start_iter", C.c_uint32),
                ("use_graph", C.c_int32), ("reserved", C.c_int32),
                ("init_mean_h", C.POINTER(C.c_float)), ("init_cov_h", C.POINTER(C.c_float)),
                ("best_J_hist_h", C.POINTER(C.c_float)), ("k_eff_hist_h", C.POINTER(C.c_int32)),
                ("init_chol_h", C.POINTER(C.c_float)), ("class_count_hist_h", C.POINTER(C.c_int32))]


class cem_paper_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("n0", C.c_int32), ("n1", C.c_int32), ("j1", C.c_int32),
                ("K", C.c_int32), ("iters", C.c_int32), ("cov_mode", C.c_int32), ("problem", C.c_uint32),
                ("reserved", C.c_int32),
                ("best_J_hist_h", C.POINTER(C.c_float)), ("k_eff_hist_h", C.POINTER(C.c_int32)),
                ("class_count_hist_h", C.POINTER(C.c_int32)), ("n_env_hist_h", C.POINTER(C.c_int32))]


class cem_problem_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("N", C.c_int32), ("K", C.c_int32), ("cov_mode", C.c_int32),
                ("problem", C.c_uint32)]


class cem_multiplan_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("N", C.c_int32), ("K", C.c_int32), ("iters", C.c_int32),
                ("cov_mode", C.c_int32), ("halving_iters", C.c_int32), ("keep", C.c_int32)]


class cem_finetune_params(C.Structure):
    _fields_ = [("every", C.c_int32), ("steps", C.c_int32), ("batch", C.c_int32), ("capacity", C.c_int32),
                ("lr", C.c_float), ("weight_decay", C.c_float), ("seed", C.c_uint64)]


class cem_result(C.Structure):
    _fields_ = [("best_theta", C.c_float * MAX_D), ("best_J", C.c_float), ("best_class", C.c_int32),
                ("D", C.c_int32), ("iters_done", C.c_int32), ("mean", C.c_float * MAX_D),
                ("cov", C.c_float * (MAX_D * MAX_D)), ("elapsed_ms", C.c_float),
                ("chol", C.c_float * (MAX_D * MAX_D))]


# ------------------------------------------------------------- marshalling
def _set(arr, vals):
    for i, v in enumerate(vals):
        arr[i] = float(v)


def pack_scene(scene: dict, skel: dict, T: int | None = None):
    """Workload dictionaries -> (cem_scene_desc, cem_skeleton_desc)."""
    s = cem_scene_desc()
    s.kind = SCENE_KIND[scene["kind"]]
    s.T = int(scene["T"] if T is None else T)
    s.cost_mode = 1 if scene.get("cost_mode", "interp") == "step" else 0
    s.dt, s.g, s.eps = scene["dt"], scene["g"], scene.get("eps", 0.0)
    for key in ("base_mass", "base_mu", "yaw_kp", "yaw_kd", "block_mass", "block_mu", "k_contact",
                "c_contact", "contact_mu", "force_limit", "w_time", "w_goal", "w_viol", "w_obj", "w_base",
                "obj_half", "obj_mass", "obj_mu", "arm_l1", "arm_l2", "arm_z", "arm_kp", "arm_kd",
                "grasp_reach", "grasp_kp", "grip_tol"):
        if key in scene:
            setattr(s, key, float(scene[key]))
    for key in ("base_half", "base_start", "base_v0", "block_half", "block_start", "block_v0",
                "goal_center", "goal_half", "obj_start", "obj_v0", "arm_home"):
        if key in scene:
            _set(getattr(s, key), scene[key])
    for key, name in (("obj_region_center", "obj_region_c"), ("obj_region_half", "obj_region_h"),
                      ("base_region_center", "base_region_c"), ("base_region_half", "base_region_h")):
        if key in scene:
            _set(getattr(s, name), scene[key])
    for key in ("goal_obj_region", "goal_obj_held", "goal_base_region"):
        setattr(s, key, int(bool(scene.get(key, False))))
    geoms = scene.get("geoms", [])
    if len(geoms) > MAX_GEOMS:
        raise ValueError("at most 16 geometries")
    s.n_geoms = len(geoms)
    for gi, gm in enumerate(geoms):
        g = s.geom[gi]
        if len(gm["slabs"]) > MAX_SLABS:
            raise ValueError("at most 6 slabs per geometry")
        g.n_slabs = len(gm["slabs"])
        g.collide_base = int(gm["base"])
        g.collide_object = int(gm["obj"])
        for si, (nx, ny, nz, lo, hi) in enumerate(gm["slabs"]):
            _set(g.slab[si].n, (nx, ny, nz))
            g.slab[si].lo = lo
            g.slab[si].hi = hi
    D = len(skel["lo"])
    if D > MAX_D:
        raise ValueError("D > 18")
    if scene.get("base_controller", "pd") == "astar":  # A* waypoints + PID (Sec. IV-A)
        s.base_controller = 1
        s.base_inflate, s.wp_switch = scene["base_inflate"], scene["wp_switch"]
        s.pid_ki, s.pid_irad, s.pid_imax = scene["pid_ki"], scene["pid_irad"], scene["pid_imax"]
    if scene["kind"] == "quadratic":
        _set(s.theta_star, scene["theta_star"])
        for i in range(D * D):
            s.A[i] = scene["A"][i]
    k = cem_skeleton_desc()
    k.D = D
    acts = skel["actions"]
    if len(acts) > MAX_ACTIONS:
        raise ValueError("at most 6 actions")
    k.n_actions = len(acts)
    off = 0
    for i, a in enumerate(acts):
        k.action[i].kind = ACTION_KIND[a["kind"]]
        k.action[i].theta_offset = off
        k.action[i].success_ref = 1 if a.get("success_ref", "nominal") == "target" else 0
        _set(k.action[i].nominal, a["nominal"])
        k.action[i].yaw = a.get("yaw", 0.0)
        reg = a.get("region")
        if reg is not None:  # annulus of a moveTo goal for the initial sampling
            k.action[i].init_region = 1 if reg["kind"] == "ring" else -1
            _set(k.action[i].region, [reg["center"][0], reg["center"][1], reg["radii"][0], reg["radii"][1]])
        off += ACTION_WIDTH[a["kind"]]
    _set(k.lo, skel["lo"])
    _set(k.hi, skel["hi"])
    return s, k


# ------------------------------------------------------------------ loading
_lib = None


def load(path: str | None = None):
    """Load libcemtamp.so once per process (DEBUG_LIB_PATH, the bounds-checked
    build, when path says so or when the environment sets CEMTAMP_DEBUG=1);
    raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = DEBUG_LIB_PATH if os.environ.get("CEMTAMP_DEBUG") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} is not built ({path}); run paper_2512_11571_gb300/build.py")
    L = C.CDLL(path)
    vp, fp, u8p, i32p, u32p = C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p
    H = C.c_void_p
    L.cem_scene_create.argtypes = [C.POINTER(cem_scene_desc), C.POINTER(cem_skeleton_desc), C.POINTER(H)]
    L.cem_scene_destroy.argtypes = [H]
    L.cem_sample.argtypes = [H, fp, fp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, fp, vp]
    L.cem_philox_words.argtypes = [H, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, u32p, vp]
    L.cem_rollout_batch.argtypes = [H, fp, C.c_int, fp, u8p, vp]
    L.cem_rollout_trace.argtypes = [H, fp, C.c_int, C.c_int, fp, vp]
    L.cem_refit.argtypes = [H, fp, fp, u8p, C.c_int, C.c_int, C.c_int, fp, fp, fp, i32p, i32p, vp]
    L.cem_solve.argtypes = [H, C.POINTER(cem_solve_params), C.POINTER(cem_result)]
    L.cem_solve_paper.argtypes = [H, C.POINTER(cem_paper_params), C.POINTER(cem_result)]
    L.cem_sample_uniform.argtypes = [H, C.c_uint64, C.c_uint32, C.c_int, vp, vp]
    L.cem_n_env.argtypes = [C.c_int] * 4
    L.cem_debug_status.argtypes = [C.POINTER(C.c_int), C.c_int]
    L.cem_debug_selftest.argtypes = []
    L.cem_test_fail_allocation.argtypes = [C.c_int]
    L.cem_set_randomization.argtypes = [H, C.c_int, C.c_float, C.c_float, C.c_uint64]
    L.cem_batch_set_active.argtypes = [H, C.POINTER(C.c_int32)]
    L.cem_batch_set_randomization.argtypes = [H, C.c_int, C.c_float, C.c_float, C.c_uint64]
    L.cem_base_path.argtypes = [H, C.c_float, C.c_float, C.c_float, C.c_float, C.POINTER(C.c_float), C.c_int,
                                C.POINTER(C.c_int)]
    L.cem_multiplan_solve.argtypes = [C.POINTER(cem_scene_desc), C.POINTER(cem_skeleton_desc), C.c_int,
                                      C.POINTER(cem_multiplan_params), C.POINTER(cem_result),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.cem_solve_static.argtypes = [C.POINTER(cem_scene_desc), C.POINTER(cem_skeleton_desc),
                                   C.POINTER(cem_solve_params), C.POINTER(cem_result), vp]
    L.cem_set_launch.argtypes = [H, C.c_int]
    L.cem_batch_create.argtypes = [C.POINTER(cem_scene_desc), C.POINTER(cem_skeleton_desc),
                                   C.POINTER(cem_problem_params), C.c_int, C.POINTER(H)]
    L.cem_batch_destroy.argtypes = [H]
    L.cem_batch_reset.argtypes = [H, vp]
    L.cem_batch_iterate.argtypes = [H, C.c_int, C.c_int, vp]
    L.cem_batch_read.argtypes = [H, C.POINTER(cem_result), vp]
    L.cem_batch_set_launch.argtypes = [H, C.c_int, C.c_int]
    L.cem_batch_autotune.argtypes = [H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float)]
    L.cem_batch_steps_per_iteration.argtypes = [H]
    L.cem_batch_set_state.argtypes = [H, C.POINTER(cem_result), vp]
    L.cem_batch_state_bytes.argtypes = [H]
    L.cem_batch_set_timing.argtypes = [H, C.c_int]
    L.cem_batch_stage_ms.argtypes = [H, C.POINTER(C.c_float)]
    L.cem_batch_set_screening.argtypes = [H, H, C.POINTER(C.c_float), C.c_int, C.c_int]
    L.cem_batch_iterate_screened.argtypes = [H, C.c_int, vp]
    ip = C.POINTER(C.c_int)
    L.cem_batch_set_threads_per_rollout.argtypes = [H, C.c_int]
    L.cem_batch_get_launch.argtypes = [H, ip, ip, ip]
    L.cem_set_threads_per_rollout.argtypes = [H, C.c_int]
    L.cem_get_launch.argtypes = [H, C.c_int, ip, ip]
    fptr, i32ptr = C.POINTER(C.c_float), C.POINTER(C.c_int32)
    L.cem_surrogate_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(H)]
    L.cem_surrogate_destroy.argtypes = [H]
    L.cem_surrogate_num_params.argtypes = [H]
    L.cem_surrogate_set_params.argtypes = [H, fptr, fptr]
    L.cem_surrogate_get_params.argtypes = [H, fptr, fptr]
    L.cem_surrogate_forward.argtypes = [H, vp, C.c_int, vp, vp]
    L.cem_surrogate_set_forward_path.argtypes = [H, C.c_int]
    L.cem_surrogate_forward_path.argtypes = [H]
    L.cem_surrogate_set_gemm_path.argtypes = [H, C.c_int]
    L.cem_surrogate_gemm_path.argtypes = [H]
    L.cem_surrogate_adamw_step.argtypes = [H, fptr, C.c_float, C.c_float]
    L.cem_surrogate_set_adam_state.argtypes = [H, fptr, fptr, C.c_longlong]
    L.cem_surrogate_get_adam_state.argtypes = [H, fptr, fptr, C.POINTER(C.c_longlong)]
    L.cem_surrogate_test_expire_wait.argtypes = [H, C.c_int]
    L.cem_surrogate_status.argtypes = [H, C.POINTER(C.c_int)]
    L.cem_surrogate_gradient.argtypes = [H, vp, vp, C.c_int, fptr, fptr]
    L.cem_surrogate_train.argtypes = [H, vp, vp, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64,
                                      C.c_int, fptr]
    L.cem_surrogate_features.argtypes = [H, vp, C.c_int, C.c_int, fptr, fptr, fptr, vp, vp]
    L.cem_surrogate_targets.argtypes = [vp, vp, C.c_int, vp, vp]
    L.cem_surrogate_screen.argtypes = [H, H, vp, vp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, fptr,
                                       vp, vp, vp]
    L.cem_solve_screened.argtypes = [H, H, fptr, C.POINTER(cem_solve_params), C.c_int, C.c_int,
                                     C.POINTER(cem_result)]
    L.cem_solve_screened_ft.argtypes = [H, H, fptr, C.POINTER(cem_solve_params), C.c_int, C.c_int,
                                        C.POINTER(cem_finetune_params), C.POINTER(cem_result)]
    L.cem_autotune.argtypes = [H, C.c_int, C.c_char_p, C.POINTER(C.c_int)]
    L.cem_last_error.restype = C.c_char_p
    L.cem_version.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("cem_last_error", "cem_version"):
            getattr(L, name).restype = C.c_int
    L.cem_batch_steps_per_iteration.restype = C.c_longlong
    L.cem_batch_state_bytes.restype = C.c_size_t
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise CemError(rc, load().cem_last_error().decode())


# The library takes plain device pointers and cannot see a buffer's size or
# type, so the wrappers check both before the call: a short or mistyped
# tensor would otherwise be read or written out of bounds on the device.
# Parameters per sample of each live scene handle, input width of each
# surrogate handle (sizes that the C calls take from the handle):
_SCENE_D: dict[int, int] = {}
_SUR_IN: dict[int, int] = {}
_BATCH_N: dict[int, int] = {}  # problems of each live batch handle
FEATURES = 48  # cem_surrogate_features writes x[N][48]


def _ptr(t, dtype=None, n=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor of `dtype` (a torch dtype
    or a tuple of them) holding at least `n` elements."""
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name}: expected dtype {dtype}, got {t.dtype}")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name}: needs at least {n} elements, has {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _f32t():
    import torch

    return torch.float32


def _u8t():
    import torch

    return torch.uint8


def _i32t():
    import torch

    return (torch.int32, getattr(torch, "uint32", torch.int32))


def _dim(h):
    """Parameters per sample of scene handle h (None if not created here)."""
    return _SCENE_D.get(getattr(h, "value", h))


def _mul(*a):
    """Product of sizes, None if one is unknown."""
    r = 1
    for x in a:
        if x is None:
            return None
        r *= int(x)
    return r


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# --------------------------------------------------------- C-named wrappers
def cem_scene_create(scene: dict, skel: dict, T: int | None = None):
    s, k = pack_scene(scene, skel, T)
    h = C.c_void_p()
    _check(load().cem_scene_create(C.byref(s), C.byref(k), C.byref(h)))
    _SCENE_D[h.value] = len(skel["lo"])
    return h


def cem_scene_destroy(h):
    _check(load().cem_scene_destroy(h))
    _SCENE_D.pop(getattr(h, "value", h), None)


def cem_sample(h, mean, chol, seed, it, problem, N, theta, stream=None):
    D = _dim(h)
    _check(load().cem_sample(h, _ptr(mean, _f32t(), D, "mean"), _ptr(chol, _f32t(), _mul(D, D), "chol"), seed, it,
                             problem, N, _ptr(theta, _f32t(), _mul(N, D), "theta"), _stream(stream)))


def cem_philox_words(h, seed, it, problem, N, words, stream=None):
    D = _dim(h)
    nw = None if D is None else 4 * ((D + 3) // 4)
    _check(load().cem_philox_words(h, seed, it, problem, N, _ptr(words, _i32t(), _mul(N, nw), "words"),
                                   _stream(stream)))


def cem_rollout_batch(h, theta, N, J, cls, stream=None):
    _check(load().cem_rollout_batch(h, _ptr(theta, _f32t(), _mul(N, _dim(h)), "theta"), N,
                                    _ptr(J, _f32t(), N, "J"), _ptr(cls, _u8t(), N, "cls"), _stream(stream)))


def cem_rollout_trace(h, theta, N, steps, states, stream=None):
    _check(load().cem_rollout_trace(h, _ptr(theta, _f32t(), _mul(N, _dim(h)), "theta"), N, steps,
                                    _ptr(states, _f32t(), _mul(N, steps, TRACE_W), "states"), _stream(stream)))


def cem_refit(h, theta, J, cls, N, K, cov_mode, mean, cov, chol, elite_idx=None, k_eff=None, stream=None):
    D = _dim(h)
    f = _f32t()
    _check(load().cem_refit(h, _ptr(theta, f, _mul(N, D), "theta"), _ptr(J, f, N, "J"), _ptr(cls, _u8t(), N, "cls"),
                            N, K, cov_mode, _ptr(mean, f, D, "mean"), _ptr(cov, f, _mul(D, D), "cov"),
                            _ptr(chol, f, _mul(D, D), "chol"), _ptr(elite_idx, _i32t(), K, "elite_idx"),
                            _ptr(k_eff, _i32t(), 1, "k_eff"), _stream(stream)))


def cem_solve(h, params: cem_solve_params):
    out = cem_result()
    _check(load().cem_solve(h, C.byref(params), C.byref(out)))
    return out


def cem_solve_paper(h, params: cem_paper_params):
    out = cem_result()
    _check(load().cem_solve_paper(h, C.byref(params), C.byref(out)))
    return out


def cem_sample_uniform(h, seed, problem, N, theta, stream=None):
    _check(load().cem_sample_uniform(h, seed, problem, N, _ptr(theta, _f32t(), _mul(N, _dim(h)), "theta"),
                                     _stream(stream)))


def cem_set_randomization(h, M, delta_mu, delta_mass, seed):
    _check(load().cem_set_randomization(h, int(M), float(delta_mu), float(delta_mass), int(seed)))


def cem_base_path(h, start, goal):
    """Waypoints (n, 2) of the A* path of the pick-place base, ending with the goal."""
    xy = np.zeros(2 * 64, np.float32)
    n = C.c_int(0)
    _check(load().cem_base_path(h, float(start[0]), float(start[1]), float(goal[0]), float(goal[1]),
                                xy.ctypes.data_as(C.POINTER(C.c_float)), 64, C.byref(n)))
    return xy[:2 * min(n.value, 64)].reshape(-1, 2)


def cem_n_env(n0, n1, j1, j):
    return int(load().cem_n_env(n0, n1, j1, j))


def cem_debug_status(reset=False):
    """First bounds-check code the debug library recorded (0: none); raises
    CemError (CEM_ERR_UNSUPPORTED) on the release library."""
    code = C.c_int(0)
    _check(load().cem_debug_status(C.byref(code), int(bool(reset))))
    return code.value


def cem_debug_selftest():
    """Debug library only: makes one clamped check fire (code 99)."""
    _check(load().cem_debug_selftest())


def cem_test_fail_allocation(k):
    """Test hook: the k-th next device allocation fails (0: off)."""
    _check(load().cem_test_fail_allocation(int(k)))


def cem_solve_static(scene: dict, skel: dict, params: cem_solve_params, stream=None):
    """cem_solve without device allocation (see include/cemtamp.h)."""
    s, k = pack_scene(scene, skel)
    out = cem_result()
    _check(load().cem_solve_static(C.byref(s), C.byref(k), C.byref(params), C.byref(out), _stream(stream)))
    return out


def cem_set_launch(h, block):
    _check(load().cem_set_launch(h, block))


def cem_autotune(h, N, cache_path=None):
    b = C.c_int()
    _check(load().cem_autotune(h, N, cache_path.encode() if cache_path else None, C.byref(b)))
    return b.value


def cem_set_threads_per_rollout(h, tpr):
    _check(load().cem_set_threads_per_rollout(h, int(tpr)))


def cem_get_launch(h, N):
    b, t = C.c_int(0), C.c_int(0)
    _check(load().cem_get_launch(h, int(N), C.byref(b), C.byref(t)))
    return b.value, t.value


def cem_batch_set_threads_per_rollout(h, tpr):
    _check(load().cem_batch_set_threads_per_rollout(h, int(tpr)))


def cem_batch_get_launch(h):
    w, c, t = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(load().cem_batch_get_launch(h, C.byref(w), C.byref(c), C.byref(t)))
    return w.value, c.value, t.value


def cem_batch_create(problems):
    """problems: list of dicts with scene, skel, N, K and optional seed,
    problem, cov ('full' | 'diag')."""
    n = len(problems)
    scenes = (cem_scene_desc * n)()
    skels = (cem_skeleton_desc * n)()
    params = (cem_problem_params * n)()
    for i, pr in enumerate(problems):
        s, k = pack_scene(pr["scene"], pr["skel"])
        scenes[i], skels[i] = s, k
        params[i].seed = pr.get("seed", 0)
        params[i].N, params[i].K = pr["N"], pr["K"]
        params[i].cov_mode = COV[pr.get("cov", "full")]
        params[i].problem = pr.get("problem", i)
    h = C.c_void_p()
    _check(load().cem_batch_create(scenes, skels, params, n, C.byref(h)))
    _BATCH_N[h.value] = n
    return h


def cem_batch_set_randomization(h, M, delta_mu, delta_mass, seed):
    _check(load().cem_batch_set_randomization(h, int(M), float(delta_mu), float(delta_mass), int(seed)))


def cem_batch_set_active(h, active):
    a = np.ascontiguousarray(np.asarray(active, np.int32)).reshape(-1)
    n = _BATCH_N.get(getattr(h, "value", h))
    if n is not None and a.size != n:
        raise ValueError(f"active: expected one flag per problem ({n}), got {a.size}")
    _check(load().cem_batch_set_active(h, a.ctypes.data_as(C.POINTER(C.c_int32))))


def cem_multiplan_solve(scene: dict, plans: list, seed, N, K, iters, halving_iters=0, keep=1, cov_mode="full"):
    """Realise every candidate plan (skeleton) of one scene in one batch, with
    optional successive halving; returns (per-plan result dicts, best plan)."""
    n = len(plans)
    skels = (cem_skeleton_desc * n)()
    s0 = None
    for i, sk in enumerate(plans):
        s, k = pack_scene(scene, sk)
        s0 = s if s0 is None else s0
        skels[i] = k
    p = cem_multiplan_params()
    p.seed, p.N, p.K, p.iters, p.cov_mode = seed, N, K, iters, COV[cov_mode]
    p.halving_iters, p.keep = halving_iters, keep
    out = (cem_result * n)()
    its = np.zeros(n, np.int32)
    best = C.c_int32(-1)
    _check(load().cem_multiplan_solve(C.byref(s0), skels, n, C.byref(p), out,
                                      its.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(best)))
    res = []
    for i in range(n):
        r, D = out[i], out[i].D
        res.append(dict(best_theta=np.array(r.best_theta[:D]), best_J=r.best_J, best_cls=r.best_class,
                        mean=np.array(r.mean[:D]), cov=np.array(r.cov[:D * D]).reshape(D, D),
                        chol=np.array(r.chol[:D * D]).reshape(D, D),
                        iters_done=r.iters_done, iters_run=int(its[i])))
    return res, best.value


def cem_batch_destroy(h):
    _check(load().cem_batch_destroy(h))
    _BATCH_N.pop(getattr(h, "value", h), None)


def cem_batch_reset(h, stream=None):
    _check(load().cem_batch_reset(h, _stream(stream)))


def cem_batch_iterate(h, iters, use_graph=True, stream=None):
    _check(load().cem_batch_iterate(h, iters, int(use_graph), _stream(stream)))


def cem_batch_read(h, n_problems, stream=None):
    n = _BATCH_N.get(getattr(h, "value", h))
    if n is not None and n_problems != n:
        raise ValueError(f"n_problems: the batch holds {n} problems, got {n_problems}")
    out = (cem_result * n_problems)()
    _check(load().cem_batch_read(h, out, _stream(stream)))
    return out


def cem_batch_set_state(h, results, stream=None):
    """Restore every problem's state from a cem_result array of
    cem_batch_read (the same object, or one built field by field)."""
    n = _BATCH_N.get(getattr(h, "value", h))
    if n is not None and len(results) != n:
        raise ValueError(f"results: the batch holds {n} problems, got {len(results)}")
    if not isinstance(results, C.Array) or results._type_ is not cem_result:
        raise TypeError("results must be a ctypes array of cem_result (as cem_batch_read returns)")
    _check(load().cem_batch_set_state(h, results, _stream(stream)))


def cem_batch_state_bytes(h):
    return int(load().cem_batch_state_bytes(h))


def cem_batch_set_timing(h, on):
    _check(load().cem_batch_set_timing(h, int(bool(on))))


def cem_batch_stage_ms(h):
    ms = (C.c_float * 3)()
    _check(load().cem_batch_stage_ms(h, ms))
    return float(ms[0]), float(ms[1]), float(ms[2])


def cem_batch_set_screening(h, s, scene16, n_pool, n_explore):
    """scene16: [n_problems x 16] scene values (s = None switches screening off)."""
    n = _BATCH_N.get(getattr(h, "value", h))
    if s is None:
        _check(load().cem_batch_set_screening(h, None, None, 0, 0))
        return
    t, tp = _f32(scene16, None if n is None else 16 * n, "scene16")
    _check(load().cem_batch_set_screening(h, s, tp, int(n_pool), int(n_explore)))


def cem_batch_iterate_screened(h, iters, stream=None):
    _check(load().cem_batch_iterate_screened(h, int(iters), _stream(stream)))


def cem_batch_set_launch(h, warps_per_cta, ctas_per_sm=0):
    _check(load().cem_batch_set_launch(h, warps_per_cta, ctas_per_sm))


def cem_batch_autotune(h):
    w, c, ms = C.c_int(), C.c_int(), C.c_float()
    _check(load().cem_batch_autotune(h, C.byref(w), C.byref(c), C.byref(ms)))
    return w.value, c.value, ms.value


def cem_batch_steps_per_iteration(h):
    return int(load().cem_batch_steps_per_iteration(h))


class Batch:
    """Many independent CE problems advanced together (one library handle)."""

    def __init__(self, problems):
        self.problems = problems
        self.n = len(problems)
        self.h = cem_batch_create(problems)

    def close(self):
        if self.h is not None and _lib is not None:
            cem_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        cem_batch_reset(self.h, stream)

    def iterate(self, iters, use_graph=True, stream=None):
        cem_batch_iterate(self.h, iters, use_graph, stream)

    def read_raw(self, stream=None):
        """The cem_result array of cem_batch_read, as the C call wrote it."""
        return cem_batch_read(self.h, self.n, stream)

    def set_state(self, results, stream=None):
        """Restore the state that read_raw returned (exact resume)."""
        cem_batch_set_state(self.h, results, stream)

    @property
    def state_bytes(self):
        return cem_batch_state_bytes(self.h)

    def set_screening(self, surrogate, scene16, n_pool, n_explore=0):
        """Screen every problem's candidates with `surrogate` (a Surrogate, or
        None to switch off); scene16: [n_problems x 16]."""
        self._surrogate = surrogate
        cem_batch_set_screening(self.h, None if surrogate is None else surrogate.h, scene16, n_pool, n_explore)

    def iterate_screened(self, iters, stream=None):
        cem_batch_iterate_screened(self.h, iters, stream)

    def set_timing(self, on=True):
        cem_batch_set_timing(self.h, on)

    def stage_ms(self):
        """(sample, persistent rollout, refit) ms of the last iteration."""
        return cem_batch_stage_ms(self.h)

    def read(self, stream=None):
        out = cem_batch_read(self.h, self.n, stream)
        res = []
        for r in out:
            D = r.D
            res.append(dict(best_theta=np.array(r.best_theta[:D]), best_J=r.best_J, best_cls=r.best_class,
                            mean=np.array(r.mean[:D]), cov=np.array(r.cov[:D * D]).reshape(D, D),
                            chol=np.array(r.chol[:D * D]).reshape(D, D), iters_done=r.iters_done))
        return res

    def autotune(self):
        return cem_batch_autotune(self.h)

    def set_threads_per_rollout(self, tpr):
        cem_batch_set_threads_per_rollout(self.h, tpr)

    def set_randomization(self, M=1, delta_mu=0.0, delta_mass=0.0, seed=0):
        """Domain randomisation of every problem (off: M=1, 0, 0)."""
        cem_batch_set_randomization(self.h, M, delta_mu, delta_mass, seed)

    def set_active(self, active):
        """Which problems take part in the next iterations (reset: all)."""
        cem_batch_set_active(self.h, active)

    def launch(self):
        """(warps per CTA, CTAs per SM, lanes per pick-and-place rollout)."""
        return cem_batch_get_launch(self.h)

    def set_launch(self, warps_per_cta, ctas_per_sm=0):
        cem_batch_set_launch(self.h, warps_per_cta, ctas_per_sm)

    @property
    def steps_per_iteration(self):
        return cem_batch_steps_per_iteration(self.h)


def _f32(a, n=None, name="array"):
    """FP32 host copy of `a` and its pointer; `n`: the element count the call reads."""
    a = np.ascontiguousarray(a, np.float32)
    if n is not None and a.size != n:
        raise ValueError(f"{name}: expected {n} elements, got {a.size}")
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def cem_surrogate_create(in_dim=48, width=256, depth=4, seed=0):
    h = C.c_void_p()
    _check(load().cem_surrogate_create(in_dim, width, depth, seed, C.byref(h)))
    _SUR_IN[h.value] = int(in_dim)
    return h


def cem_surrogate_destroy(s):
    _check(load().cem_surrogate_destroy(s))
    _SUR_IN.pop(getattr(s, "value", s), None)


def _in_dim(s):
    return _SUR_IN.get(getattr(s, "value", s))


def cem_surrogate_num_params(s):
    return int(load().cem_surrogate_num_params(s))


def cem_surrogate_set_params(s, params, norm=None):
    p, pp = _f32(params, cem_surrogate_num_params(s), "params")
    if norm is not None:
        n, pn = _f32(norm, 2, "norm")
    _check(load().cem_surrogate_set_params(s, pp, pn if norm is not None else None))


def cem_surrogate_get_params(s):
    p = np.zeros(cem_surrogate_num_params(s), np.float32)
    n = np.zeros(2, np.float32)
    _check(load().cem_surrogate_get_params(s, p.ctypes.data_as(C.POINTER(C.c_float)),
                                           n.ctypes.data_as(C.POINTER(C.c_float))))
    return p, n


def cem_surrogate_forward(s, x, y, stream=None):
    M = x.shape[0]
    _check(load().cem_surrogate_forward(s, _ptr(x, _f32t(), _mul(M, _in_dim(s)), "x"), M, _ptr(y, _f32t(), M, "y"),
                                        _stream(stream)))


def cem_surrogate_set_forward_path(s, path):
    _check(load().cem_surrogate_set_forward_path(s, int(path)))


def cem_surrogate_test_expire_wait(s, on):
    _check(load().cem_surrogate_test_expire_wait(s, int(bool(on))))


def cem_surrogate_forward_path(s):
    return int(load().cem_surrogate_forward_path(s))


def cem_surrogate_set_gemm_path(s, path):
    _check(load().cem_surrogate_set_gemm_path(s, int(path)))


def cem_surrogate_gemm_path(s):
    return int(load().cem_surrogate_gemm_path(s))


def cem_surrogate_adamw_step(s, grad, lr=1e-3, weight_decay=1e-4):
    g, gp = _f32(grad, cem_surrogate_num_params(s), "grad")
    _check(load().cem_surrogate_adamw_step(s, gp, float(lr), float(weight_decay)))


def cem_surrogate_set_adam_state(s, m1, m2, steps_taken):
    n = cem_surrogate_num_params(s)
    a, ap = _f32(m1, n, "m1")
    b, bp = _f32(m2, n, "m2")
    _check(load().cem_surrogate_set_adam_state(s, ap, bp, int(steps_taken)))


def cem_surrogate_get_adam_state(s):
    n = cem_surrogate_num_params(s)
    m1, m2 = np.zeros(n, np.float32), np.zeros(n, np.float32)
    t = C.c_longlong()
    _check(load().cem_surrogate_get_adam_state(s, m1.ctypes.data_as(C.POINTER(C.c_float)),
                                               m2.ctypes.data_as(C.POINTER(C.c_float)), C.byref(t)))
    return m1, m2, t.value


def cem_surrogate_status(s):
    code = C.c_int(0)
    _check(load().cem_surrogate_status(s, C.byref(code)))
    return code.value


def cem_surrogate_gradient(s, x, t):
    g = np.zeros(cem_surrogate_num_params(s), np.float32)
    loss = C.c_float()
    M = x.shape[0]
    _check(load().cem_surrogate_gradient(s, _ptr(x, _f32t(), _mul(M, _in_dim(s)), "x"), _ptr(t, _f32t(), M, "t"), M,
                                         g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
    return g, loss.value


def cem_surrogate_train(s, x, t, batch, steps, lr=1e-3, weight_decay=1e-4, seed=0, normalize=True):
    hist = np.zeros(max(steps, 1), np.float32)
    M = x.shape[0]
    _check(load().cem_surrogate_train(s, _ptr(x, _f32t(), _mul(M, _in_dim(s)), "x"), _ptr(t, _f32t(), M, "t"), M, batch,
                                      steps, lr, weight_decay, seed, int(normalize),
                                      hist.ctypes.data_as(C.POINTER(C.c_float))))
    return hist[:steps]


def cem_surrogate_features(s, theta, lo, hi, scene16, x, stream=None):
    N, D = theta.shape[0], theta.shape[1]
    lo_, plo = _f32(lo, D, "lo")
    hi_, phi = _f32(hi, D, "hi")
    sc_, psc = _f32(scene16, 16, "scene16")
    _check(load().cem_surrogate_features(s, _ptr(theta, _f32t(), N * D, "theta"), N, D, plo, phi, psc,
                                         _ptr(x, _f32t(), N * FEATURES, "x"), _stream(stream)))


def cem_surrogate_targets(J, cls, t, stream=None):
    N = J.shape[0]
    _check(load().cem_surrogate_targets(_ptr(J, _f32t(), N, "J"), _ptr(cls, _u8t(), N, "cls"), N,
                                        _ptr(t, _f32t(), N, "t"), _stream(stream)))


def cem_surrogate_screen(h, s, mean, chol, seed, it, problem, n_pool, n_keep, scene16, theta_keep, keep_idx=None,
                         stream=None):
    sc_, psc = _f32(scene16, 16, "scene16")
    D = _dim(h)
    f = _f32t()
    _check(load().cem_surrogate_screen(h, s, _ptr(mean, f, D, "mean"), _ptr(chol, f, _mul(D, D), "chol"), seed, it,
                                       problem, n_pool, n_keep, psc, _ptr(theta_keep, f, _mul(n_keep, D), "theta_keep"),
                                       _ptr(keep_idx, _i32t(), n_keep, "keep_idx"), _stream(stream)))


def cem_solve_screened(h, s, scene16, params: cem_solve_params, n_pool, n_explore=0):
    sc_, psc = _f32(scene16, 16, "scene16")
    out = cem_result()
    _check(load().cem_solve_screened(h, s, psc, C.byref(params), n_pool, n_explore, C.byref(out)))
    return out


def cem_solve_screened_ft(h, s, scene16, params: cem_solve_params, n_pool, n_explore, ft: cem_finetune_params):
    sc_, psc = _f32(scene16, 16, "scene16")
    out = cem_result()
    _check(load().cem_solve_screened_ft(h, s, psc, C.byref(params), n_pool, n_explore, C.byref(ft), C.byref(out)))
    return out


class Surrogate:
    """The cost surrogate MLP (one library handle)."""

    def __init__(self, width=256, depth=4, seed=0):
        self.h = cem_surrogate_create(48, width, depth, seed)

    def close(self):
        if self.h is not None and _lib is not None:
            cem_surrogate_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, x, stream=None):
        import torch

        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        cem_surrogate_forward(self.h, x, y, stream)
        return y

    def set_forward_path(self, path):
        """0 automatic, 1 tiled mma.sync GEMM, 2 fused tcgen05 kernel."""
        cem_surrogate_set_forward_path(self.h, path)

    @property
    def forward_path(self):
        return cem_surrogate_forward_path(self.h)

    def set_gemm_path(self, path):
        """Training GEMMs: 0 automatic, 1 tiled mma.sync, 2 tcgen05, 3 the FP32 debug gradient."""
        cem_surrogate_set_gemm_path(self.h, path)

    @property
    def gemm_path(self):
        return cem_surrogate_gemm_path(self.h)

    def test_expire_wait(self, on):
        """Failure-detection hook: make the tcgen05 forward's first wait run out."""
        cem_surrogate_test_expire_wait(self.h, on)

    def adamw_step(self, grad, lr=1e-3, weight_decay=1e-4):
        """One optimiser step of the training loop with the given gradient."""
        cem_surrogate_adamw_step(self.h, grad, lr, weight_decay)

    def set_adam_state(self, m1, m2, steps_taken):
        cem_surrogate_set_adam_state(self.h, m1, m2, steps_taken)

    def adam_state(self):
        """(first moments, second moments, steps taken)."""
        return cem_surrogate_get_adam_state(self.h)

    def status(self):
        """Reads and clears the fused kernel's status word (0 = no wait expired)."""
        return cem_surrogate_status(self.h)

    def train(self, x, t, batch=4096, steps=1000, lr=1e-3, weight_decay=1e-4, seed=0, normalize=True):
        return cem_surrogate_train(self.h, x, t, batch, steps, lr, weight_decay, seed, normalize)

    def features(self, theta, lo, hi, scene16, stream=None):
        import torch

        x = torch.empty((theta.shape[0], 48), dtype=torch.float32, device=theta.device)
        cem_surrogate_features(self.h, theta, lo, hi, scene16, x, stream)
        return x

    def params(self):
        return cem_surrogate_get_params(self.h)

    def set_params(self, params, norm=None):
        cem_surrogate_set_params(self.h, params, norm)

    def gradient(self, x, t):
        return cem_surrogate_gradient(self.h, x, t)


# ----------------------------------------------------------- convenience
class Scene:
    """A scene + plan skeleton on the device (one library handle)."""

    def __init__(self, scene: dict, skel: dict, T: int | None = None):
        self.scene, self.skel = scene, skel
        self.D = len(skel["lo"])
        self.T = int(scene["T"] if T is None else T)
        self.lo = np.asarray(skel["lo"], np.float32)
        self.hi = np.asarray(skel["hi"], np.float32)
        self.h = cem_scene_create(scene, skel, T)

    def close(self):
        if self.h is not None and _lib is not None:
            cem_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # device tensors in, device tensors out
    def sample(self, mean, chol, seed, it, N, problem=0, stream=None):
        import torch

        theta = torch.empty((N, self.D), dtype=torch.float32, device=mean.device)
        cem_sample(self.h, mean, chol, seed, it, problem, N, theta, stream)
        return theta

    def philox_words(self, seed, it, N, problem=0, stream=None):
        import torch

        nc = (self.D + 3) // 4
        w = torch.empty((N, 4 * nc), dtype=torch.int32, device="cuda")
        cem_philox_words(self.h, seed, it, problem, N, w, stream)
        return w

    def rollout(self, theta, stream=None):
        import torch

        N = theta.shape[0]
        J = torch.empty(N, dtype=torch.float32, device=theta.device)
        cls = torch.empty(N, dtype=torch.uint8, device=theta.device)
        cem_rollout_batch(self.h, theta, N, J, cls, stream)
        return J, cls

    def trace(self, theta, steps, stream=None):
        import torch

        N = theta.shape[0]
        st = torch.empty((N, steps, TRACE_W), dtype=torch.float32, device=theta.device)
        cem_rollout_trace(self.h, theta, N, steps, st, stream)
        return st

    def refit(self, theta, J, cls, K, mean, cov, chol, cov_mode="full", stream=None):
        import torch

        idx = torch.full((K,), -1, dtype=torch.int32, device=J.device)
        keff = torch.zeros(1, dtype=torch.int32, device=J.device)
        cem_refit(self.h, theta, J, cls, J.shape[0], K, COV[cov_mode], mean, cov, chol, idx, keff, stream)
        return idx, keff

    def solve(self, seed, N, K, iters, cov_mode="full", problem=0, start_iter=0, use_graph=True,
              init_mean=None, init_cov=None, init_chol=None):
        p = cem_solve_params()
        p.seed, p.N, p.K, p.iters, p.cov_mode = seed, N, K, iters, COV[cov_mode]
        p.problem, p.start_iter, p.use_graph = problem, start_iter, int(use_graph)
        keep = []
        if init_mean is not None:
            m = np.ascontiguousarray(init_mean, np.float32)
            keep.append(m)
            p.init_mean_h = m.ctypes.data_as(C.POINTER(C.c_float))
        if init_cov is not None:
            c = np.ascontiguousarray(init_cov, np.float32)
            keep.append(c)
            p.init_cov_h = c.ctypes.data_as(C.POINTER(C.c_float))
        if init_chol is not None:
            L = np.ascontiguousarray(init_chol, np.float32)
            keep.append(L)
            p.init_chol_h = L.ctypes.data_as(C.POINTER(C.c_float))
        hist = np.zeros(iters, np.float32)
        keff = np.zeros(iters, np.int32)
        counts = np.zeros((iters, 4), np.int32)
        p.best_J_hist_h = hist.ctypes.data_as(C.POINTER(C.c_float))
        p.k_eff_hist_h = keff.ctypes.data_as(C.POINTER(C.c_int32))
        p.class_count_hist_h = counts.ctypes.data_as(C.POINTER(C.c_int32))
        r = cem_solve(self.h, p)
        D = self.D
        return dict(best_theta=np.array(r.best_theta[:D]), best_J=r.best_J, best_cls=r.best_class,
                    mean=np.array(r.mean[:D]), cov=np.array(r.cov[:D * D]).reshape(D, D),
                    chol=np.array(r.chol[:D * D]).reshape(D, D),
                    iters_done=r.iters_done, elapsed_ms=r.elapsed_ms, history=hist, k_eff=keff,
                    class_counts=counts)

    def solve_paper(self, seed, n0=3000, n1=300, j1=10, K=50, iters=20, cov_mode="diag", problem=0):
        """The paper's CE variant (Sec. III-B, IV-A): uniform initial samples in
        the parameter regions, n_env falling linearly n0 -> n1 by iteration j1,
        the independent-normal model."""
        p = cem_paper_params()
        p.seed, p.n0, p.n1, p.j1, p.K, p.iters = seed, n0, n1, j1, K, iters
        p.cov_mode, p.problem = COV[cov_mode], problem
        hist = np.zeros(iters, np.float32)
        keff = np.zeros(iters, np.int32)
        counts = np.zeros((iters, 4), np.int32)
        ns = np.zeros(iters, np.int32)
        p.best_J_hist_h = hist.ctypes.data_as(C.POINTER(C.c_float))
        p.k_eff_hist_h = keff.ctypes.data_as(C.POINTER(C.c_int32))
        p.class_count_hist_h = counts.ctypes.data_as(C.POINTER(C.c_int32))
        p.n_env_hist_h = ns.ctypes.data_as(C.POINTER(C.c_int32))
        r = cem_solve_paper(self.h, p)
        D = self.D
        return dict(best_theta=np.array(r.best_theta[:D]), best_J=r.best_J, best_cls=r.best_class,
                    mean=np.array(r.mean[:D]), cov=np.array(r.cov[:D * D]).reshape(D, D),
                    iters_done=r.iters_done, elapsed_ms=r.elapsed_ms, history=hist, k_eff=keff,
                    class_counts=counts, n_env=ns)

    def base_path(self, start, goal):
        """The A* waypoints the base would follow (A* controller scenes)."""
        return cem_base_path(self.h, start, goal)

    def sample_uniform(self, seed, N, problem=0, stream=None):
        import torch

        theta = torch.empty((N, self.D), dtype=torch.float32, device="cuda")
        cem_sample_uniform(self.h, seed, problem, N, theta, stream)
        return theta

    def set_launch(self, block):
        cem_set_launch(self.h, block)

    def set_randomization(self, M=1, delta_mu=0.0, delta_mass=0.0, seed=0):
        """Domain randomisation: mean cost / worst class over M environments with
        friction and manipulated-body mass scaled within +-delta (off: M=1, 0, 0)."""
        cem_set_randomization(self.h, M, delta_mu, delta_mass, seed)

    def set_threads_per_rollout(self, tpr):
        """Lanes per pick-and-place rollout: 1, 8 or 32 (bit-identical results)."""
        cem_set_threads_per_rollout(self.h, tpr)

    def launch(self, N):
        """(threads per block, lanes per rollout) that a rollout of N samples uses."""
        return cem_get_launch(self.h, N)

    def solve_screened(self, surrogate, scene16, seed, N, K, iters, n_pool, n_explore=0, cov_mode="full",
                       problem=0, finetune=None):
        """Screened CE loop; finetune = dict(every, steps, batch, capacity, lr,
        weight_decay, seed) fine-tunes the surrogate on the run's own samples."""
        p = cem_solve_params()
        p.seed, p.N, p.K, p.iters, p.cov_mode, p.problem = seed, N, K, iters, COV[cov_mode], problem
        hist = np.zeros(iters, np.float32)
        keff = np.zeros(iters, np.int32)
        p.best_J_hist_h = hist.ctypes.data_as(C.POINTER(C.c_float))
        p.k_eff_hist_h = keff.ctypes.data_as(C.POINTER(C.c_int32))
        if finetune is None:
            r = cem_solve_screened(self.h, surrogate.h, scene16, p, n_pool, n_explore)
        else:
            f = dict(every=5, steps=100, batch=4096, capacity=4 * N, lr=5e-4, weight_decay=1e-4, seed=0)
            f.update(finetune)
            ft = cem_finetune_params(int(f["every"]), int(f["steps"]), int(f["batch"]), int(f["capacity"]),
                                     float(f["lr"]), float(f["weight_decay"]), int(f["seed"]))
            r = cem_solve_screened_ft(self.h, surrogate.h, scene16, p, n_pool, n_explore, ft)
        D = self.D
        return dict(best_theta=np.array(r.best_theta[:D]), best_J=r.best_J, best_cls=r.best_class,
                    mean=np.array(r.mean[:D]), cov=np.array(r.cov[:D * D]).reshape(D, D),
                    chol=np.array(r.chol[:D * D]).reshape(D, D),
                    iters_done=r.iters_done, elapsed_ms=r.elapsed_ms, history=hist, k_eff=keff)

    def autotune(self, N, cache_path=None):
        return cem_autotune(self.h, N, cache_path)
