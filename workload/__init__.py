"""Seeded synthetic workloads for the CEM plan-realization path.

This module only *describes* problems: scene geometry, physical constants,
the plan skeleton (actions, nominal targets, parameter bounds) and the CEM
settings.  It holds none of the method's arithmetic (no dynamics, no
controller law, no sampling, no elite selection).  Both the FP64 oracle and
the CUDA library consume the dictionaries it returns, each through its own
marshalling code.

Scenes stand in for the paper's IsaacGym scenes (Sec. IV-A), which are not
available; the shapes follow the paper's two tasks:

* ``reach``     -- one moveTo action of a planar box base (a 1-action plan).
* ``push``      -- moveTo + push of a free block into a target region
                   (the move-and-push task, Sec. IV-A, plan pi_m&p).
* ``pickplace`` -- moveTo, grasp, moveTo, place, moveTo-exit with a ramp
                   obstacle between two tables (the pick-and-place task,
                   Sec. IV-A, plan pi_p&p, Eq. 7-10).
* ``quadratic`` -- J = (theta - theta*)^T A (theta - theta*), no dynamics,
                   used to test the CE loop against a known minimiser.

Randomness here is numpy's PCG64 seeded per problem; it only draws scene
properties (friction, slope, obstacle poses), never CEM samples.
"""
from __future__ import annotations

import math

import numpy as np

G = 9.81
BIG = 1.0e3  # extent used for half-spaces (walls, ground) in slab form

# ---------------------------------------------------------------- geometry


def _box_slabs(cx, cy, z0, z1, hx, hy, yaw=0.0):
    """Slabs (unit axis n, lo, hi) of a prism with a rectangular footprint.

    A convex static body is stored as the list of its projection intervals
    on a set of axes that includes the world x, y, z axes (so that the
    axis-aligned movers' own axes are covered) plus its own face normals.
    """
    c, s = math.cos(yaw), math.sin(yaw)
    ex = abs(c) * hx + abs(s) * hy
    ey = abs(s) * hx + abs(c) * hy
    slabs = [
        (1.0, 0.0, 0.0, cx - ex, cx + ex),
        (0.0, 1.0, 0.0, cy - ey, cy + ey),
        (0.0, 0.0, 1.0, z0, z1),
    ]
    if abs(s) > 1e-12 and abs(c) > 1e-12:
        pu = c * cx + s * cy
        pw = -s * cx + c * cy
        slabs.append((c, s, 0.0, pu - hx, pu + hx))
        slabs.append((-s, c, 0.0, pw - hy, pw + hy))
    return slabs


def _ramp_slabs(x0, x1, y0, y1, z_low, slope):
    """Wedge: footprint [x0,x1]x[y0,y1], top surface falling from x0 to x1.

    Height at x is z_low + (x1 - x) tan(slope); the low edge (x = x1) meets
    the neighbouring table top at z_low.
    """
    t = math.tan(slope)
    z_hi = z_low + (x1 - x0) * t
    n = (math.sin(slope), 0.0, math.cos(slope))
    hi = n[0] * x1 + n[2] * z_low
    lo = n[0] * x0  # vertex (x0, *, 0) has the lowest projection
    return [
        (1.0, 0.0, 0.0, x0, x1),
        (0.0, 1.0, 0.0, y0, y1),
        (0.0, 0.0, 1.0, 0.0, z_hi),
        (n[0], n[1], n[2], lo, hi),
    ], z_hi


def _halfspace(nx, ny, nz, lo, hi):
    return [(nx, ny, nz, lo, hi)]


# ---------------------------------------------------------------- configs

ARENA = (-3.0, 3.0, -2.0, 2.0)
TABLE1 = (-1.6, 0.9, 0.3, 0.3, 0.5)   # cx, cy, hx, hy, top z
TABLE2 = (1.4, 0.9, 0.3, 0.3, 0.5)
RAMP_FOOT = (0.3, 1.1, 0.5, 1.3)      # x0, x1, y0, y1 (x1 abuts table 2)
START_PP = (-2.4, -1.4)
EXIT = (-0.6, -1.4, 0.5, 0.5)         # cx, cy, hx, hy


def reach_scene(seed: int = 0, T: int = 400, dt: float = 0.005, cost_mode: str = "interp"):
    """One-action plan: planar box base moves to (2.0, 1.0) under a PD law.

    theta = (dx, dy, kp): target offset and PD gain.  Fixed scene; the seed
    is accepted for a uniform interface but draws nothing.
    """
    del seed
    scene = dict(
        kind="reach", T=T, dt=dt, g=G, cost_mode=cost_mode, eps=0.05,
        base_half=(0.25, 0.20), base_mass=10.0, base_mu=0.6,
        base_start=(0.0, 0.0, 0.0), yaw_kp=25.0, yaw_kd=10.0,
        w_time=1.0, w_goal=10.0, w_viol=0.0,
        goal_center=(2.0, 1.0, 0.0), goal_half=(0.0, 0.0, 0.0),
    )
    skel = dict(
        actions=[dict(kind="move", nominal=(2.0, 1.0, 0.0), yaw=0.0, success_ref="nominal")],
        lo=[-0.2, -0.2, 5.0], hi=[0.2, 0.2, 50.0],
    )
    return scene, skel


def push_scene(seed: int = 0, T: int = 1000, dt: float = 0.002, cost_mode: str = "interp",
               start_in_contact: bool = False):
    """Move-and-push: base moves behind a block, then pushes it into a region.

    Per scene: block friction mu ~ U[0.4, 0.6]; region bearing
    phi ~ U[-pi/4, pi/4]; region centre 1.5 m from the block along phi.
    ``start_in_contact`` starts the base pressed against the block, both
    aligned with the push direction (a contact-heavy variant for
    short-horizon parity tests).
    """
    rng = np.random.default_rng(seed)
    mu = float(rng.uniform(0.4, 0.6))
    phi = float(rng.uniform(-math.pi / 4, math.pi / 4))
    b0 = (1.0, 0.0)
    u = (math.cos(phi), math.sin(phi))
    region = (b0[0] + 1.5 * u[0], b0[1] + 1.5 * u[1])
    approach = (b0[0] - 0.35 * u[0], b0[1] - 0.35 * u[1])
    push_goal = (region[0] - 0.3 * u[0], region[1] - 0.3 * u[1])
    base_start = (0.0, 0.0, 0.0)
    block_yaw = 0.0
    if start_in_contact:  # base face pressed 2 mm into the aligned block's back face
        base_start = (b0[0] - 0.298 * u[0], b0[1] - 0.298 * u[1], phi)
        block_yaw = phi
    scene = dict(
        kind="push", T=T, dt=dt, g=G, cost_mode=cost_mode, eps=0.05,
        base_half=(0.25, 0.20), base_mass=10.0, base_mu=0.6,
        base_start=base_start, yaw_kp=400.0, yaw_kd=40.0,
        block_half=(0.05, 0.05), block_mass=0.5, block_mu=mu,
        block_start=(b0[0], b0[1], block_yaw),
        k_contact=2.0e4, c_contact=50.0, contact_mu=mu, force_limit=20.0,
        w_time=1.0, w_goal=20.0, w_viol=5.0,
        goal_center=(region[0], region[1], 0.0), goal_half=(0.15, 0.15, 0.0),
    )
    skel = dict(
        actions=[
            dict(kind="move", nominal=(approach[0], approach[1], 0.0), yaw=phi, success_ref="nominal"),
            dict(kind="push", nominal=(push_goal[0], push_goal[1], 0.0), yaw=phi, success_ref="nominal"),
        ],
        lo=[-0.2, -0.2, 5.0, -0.3, -0.3, 5.0], hi=[0.2, 0.2, 50.0, 0.3, 0.3, 50.0],
    )
    return scene, skel


def _pp_boxes(rng, n=3, half=0.2, height=0.4):
    """Obstacle boxes at uniform, non-overlapping positions in the arena."""
    keep_out = [  # (cx, cy, hx, hy) regions the boxes must stay clear of
        (TABLE1[0], TABLE1[1], 0.9, 0.9),
        (TABLE2[0], TABLE2[1], 0.9, 0.9),
        ((RAMP_FOOT[0] + RAMP_FOOT[1]) / 2, (RAMP_FOOT[2] + RAMP_FOOT[3]) / 2, 1.0, 0.9),
        (START_PP[0], START_PP[1], 0.6, 0.6),
        (EXIT[0], EXIT[1], 0.8, 0.8),
    ]
    r = half * math.sqrt(2.0)
    boxes = []
    for _ in range(10000):
        if len(boxes) == n:
            break
        x = float(rng.uniform(ARENA[0] + r + 0.1, ARENA[1] - r - 0.1))
        y = float(rng.uniform(ARENA[2] + r + 0.1, ARENA[3] - r - 0.1))
        yaw = float(rng.uniform(0.0, math.pi / 2))
        ok = all(abs(x - cx) > hx + r or abs(y - cy) > hy + r for cx, cy, hx, hy in keep_out)
        ok = ok and all(math.hypot(x - bx, y - by) > 2 * r + 0.6 for bx, by, _ in boxes)
        if ok:
            boxes.append((x, y, yaw))
    if len(boxes) != n:
        raise RuntimeError("box placement failed")
    return boxes, half, height


def pickplace_scene(seed: int = 0, n_actions: int = 5, T: int = 3000, dt: float = 0.002,
                    cost_mode: str = "interp", obstacle: str = "ramp", regions: str = "box",
                    controller: str = "pd"):
    """Pick-and-place with a ramp (or box) obstacle between two tables.

    Per scene: ramp slope ~ U[15, 30] deg, object friction mu ~ U[0.2, 0.4],
    three 0.4 m obstacle boxes at seeded non-overlapping poses in the
    6 x 4 m arena.  ``n_actions`` in 3..6 truncates or extends the 5-action
    skeleton (used by the 64-problem batch).

    ``regions="paper"`` gives the two table approaches annulus regions around
    their tables for uniform initial sampling (the paper's Table_1 / Table_2
    rings, radii scaled to these 0.6 m tables and the 4 m arena: 0.65..0.9 m),
    with the move bounds widened to contain them; the other parameters keep
    their boxes (the Exit box is the paper's 1 x 1 m rectangle).

    ``controller="astar"`` drives every moveTo of the base along A* waypoints
    (footprints grown by the base's half-diagonal) tracked by PD, switching
    within 0.25 m, with an integral term (gain 2 kp, active within 0.3 m of
    the goal, |I| <= 0.5 m s) on the final one, as in the paper's experiments;
    the default "pd" drives straight at the goal.
    """
    if regions not in ("box", "paper"):
        raise ValueError("regions is 'box' or 'paper'")
    if controller not in ("pd", "astar"):
        raise ValueError("controller is 'pd' or 'astar'")
    if not 3 <= n_actions <= 6:
        raise ValueError("pick-place skeletons have 3..6 actions")
    rng = np.random.default_rng(seed)
    slope = math.radians(float(rng.uniform(15.0, 30.0)))
    mu = float(rng.uniform(0.2, 0.4))
    boxes, bh, bz = _pp_boxes(rng)

    geoms = []
    geoms.append(dict(slabs=_halfspace(0, 0, 1, -BIG, 0.0), base=False, obj=True))      # ground
    geoms.append(dict(slabs=_halfspace(1, 0, 0, ARENA[1], BIG), base=True, obj=True))   # walls
    geoms.append(dict(slabs=_halfspace(1, 0, 0, -BIG, ARENA[0]), base=True, obj=True))
    geoms.append(dict(slabs=_halfspace(0, 1, 0, ARENA[3], BIG), base=True, obj=True))
    geoms.append(dict(slabs=_halfspace(0, 1, 0, -BIG, ARENA[2]), base=True, obj=True))
    for t in (TABLE1, TABLE2):
        geoms.append(dict(slabs=_box_slabs(t[0], t[1], 0.0, t[4], t[2], t[3]), base=True, obj=True))
    if obstacle == "ramp":
        slabs, z_hi = _ramp_slabs(*RAMP_FOOT, TABLE2[4], slope)
    else:  # the paper's second setup: the obstacle without a slanted side
        z_hi = TABLE2[4] + (RAMP_FOOT[1] - RAMP_FOOT[0]) * math.tan(slope)
        slabs = _box_slabs((RAMP_FOOT[0] + RAMP_FOOT[1]) / 2, (RAMP_FOOT[2] + RAMP_FOOT[3]) / 2,
                           0.0, z_hi, (RAMP_FOOT[1] - RAMP_FOOT[0]) / 2, (RAMP_FOOT[3] - RAMP_FOOT[2]) / 2)
    geoms.append(dict(slabs=slabs, base=True, obj=True))
    for (x, y, yaw) in boxes:
        geoms.append(dict(slabs=_box_slabs(x, y, 0.0, bz, bh, bh, yaw), base=True, obj=True))

    oh = 0.05
    t2 = TABLE2
    scene = dict(
        kind="pickplace", T=T, dt=dt, g=G, cost_mode=cost_mode, eps=0.05,
        base_half=(0.25, 0.20), base_mass=10.0, base_mu=0.1,
        base_start=(START_PP[0], START_PP[1], 0.0), yaw_kp=0.0, yaw_kd=0.0,
        k_contact=2.0e4, c_contact=50.0, contact_mu=mu, force_limit=0.0,
        obj_half=oh, obj_mass=0.5, obj_mu=mu,
        obj_start=(TABLE1[0], TABLE1[1], TABLE1[4] + oh),
        arm_l1=0.45, arm_l2=0.45, arm_z=0.45, arm_kp=64.0, arm_kd=16.0,
        arm_home=(1.2, -2.0),
        grasp_reach=0.55, grasp_kp=20.0, grip_tol=0.04,
        w_time=1.0, w_obj=10.0, w_base=10.0,
        obj_region_center=(t2[0], t2[1], t2[4] + oh), obj_region_half=(t2[2], t2[3], 0.01),
        base_region_center=(EXIT[0], EXIT[1], 0.0), base_region_half=(EXIT[2], EXIT[3], 0.0),
        goal_obj_region=False, goal_obj_held=False, goal_base_region=False,
        geoms=geoms,
        slope=slope, ramp_top=z_hi, boxes=boxes,
    )
    if controller == "astar":
        scene.update(base_controller="astar", base_inflate=math.hypot(0.25, 0.20), wp_switch=0.25,
                     pid_ki=2.0, pid_irad=0.3, pid_imax=0.5)
    mv = lambda nom: dict(kind="move", nominal=(nom[0], nom[1], 0.0), yaw=0.0, success_ref="target")
    acts, lo, hi = [], [], []
    ring = lambda t: dict(kind="ring", center=(t[0], t[1]), radii=(0.65, 0.9))
    # moveTo(Start, Table1)
    acts.append(mv((TABLE1[0], TABLE1[1] - 0.7)))
    if regions == "paper":
        acts[-1]["region"] = ring(TABLE1)
        lo += [-0.9, -0.6, 5.0]; hi += [0.9, 1.6, 50.0]
    else:
        lo += [-0.6, -0.6, 5.0]; hi += [0.6, 0.6, 50.0]
    # grasp(Cube): approach azimuth and grip-height offset
    acts.append(dict(kind="grasp", nominal=scene["obj_start"], yaw=0.0, success_ref="target"))
    lo += [-math.pi, -0.06]; hi += [math.pi, 0.06]
    # moveTo(Table1, Table2)
    acts.append(mv((0.9, 0.9)))
    if regions == "paper":
        acts[-1]["region"] = ring(TABLE2)
        lo += [-1.3, -1.0, 5.0]; hi += [1.4, 1.0, 50.0]
    else:
        lo += [-1.3, -1.0, 5.0]; hi += [1.3, 1.0, 50.0]
    if n_actions >= 4:  # place(Target)
        acts.append(dict(kind="place", nominal=(t2[0], t2[1], t2[4] + oh), yaw=0.0, success_ref="target"))
        lo += [-1.1, -0.3, 0.0]; hi += [0.3, 0.3, 0.5]
    if n_actions == 6:  # an extra waypoint move before the exit
        acts.append(mv((0.0, -0.6)))
        lo += [-0.8, -0.6, 5.0]; hi += [0.8, 0.6, 50.0]
    if n_actions >= 5:  # moveTo(Table2, Exit)
        acts.append(mv((EXIT[0], EXIT[1])))
        lo += [-0.5, -0.5, 5.0]; hi += [0.5, 0.5, 50.0]
    if n_actions == 3:
        scene["goal_obj_held"] = True
        scene["goal_base_region"] = True
        scene["base_region_center"] = (0.5, 0.1, 0.0)
        scene["base_region_half"] = (1.0, 0.35, 0.0)
    elif n_actions == 4:
        scene["goal_obj_region"] = True
    else:
        scene["goal_obj_region"] = True
        scene["goal_base_region"] = True
    skel = dict(actions=acts, lo=lo, hi=hi)
    return scene, skel


def pickplace_plans(seed: int = 0, T: int = 3000, obstacle: str = "ramp"):
    """One pick-place scene and four candidate plans (skeletons) for it: the
    direct 5-action plan, and 6-action plans through a waypoint south of the
    tables, in the far north-west corner, and in the far south-east corner
    (the last two are long detours).  All four share the scene's goals."""
    scene, direct = pickplace_scene(seed, n_actions=5, T=T, obstacle=obstacle)
    plans = [direct]
    for wp in ((0.0, -0.6), (-2.4, 1.6), (2.4, -1.5)):
        _, sk = pickplace_scene(seed, n_actions=6, T=T, obstacle=obstacle)
        sk["actions"][4] = dict(sk["actions"][4], nominal=(wp[0], wp[1], 0.0))
        plans.append(sk)
    return scene, plans


def quadratic_scene(seed: int = 0, D: int = 6):
    """J = (theta - theta*)^T A (theta - theta*) with a seeded SPD A.

    Bounds are [-1, 1]^D; theta* is drawn inside [-0.5, 0.5]^D.
    """
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
    ev = np.exp(rng.uniform(math.log(0.5), math.log(5.0), D))
    A = (Q * ev) @ Q.T
    A = 0.5 * (A + A.T)
    ts = rng.uniform(-0.5, 0.5, D)
    scene = dict(kind="quadratic", T=1, dt=1.0, g=G, cost_mode="interp", eps=0.0,
                 theta_star=ts.tolist(), A=A.reshape(-1).tolist())
    skel = dict(actions=[], lo=[-1.0] * D, hi=[1.0] * D)
    return scene, skel


CONFIGS = {
    0: dict(name="reach-1action", N=256, K=25, iters=10),
    1: dict(name="move-push-2action", N=4096, K=200, iters=20),
    2: dict(name="pickplace-ramp-5action", N=16384, K=512, iters=25),
}


def config(i: int, seed: int = 0, **kw):
    """(scene, skeleton, cem settings) for single-problem workloads 0-2."""
    if i == 0:
        s, k = reach_scene(seed, **kw)
    elif i == 1:
        s, k = push_scene(seed, **kw)
    elif i == 2:
        s, k = pickplace_scene(seed, **kw)
    else:
        raise ValueError("single-problem workloads are 0, 1, 2")
    return s, k, dict(CONFIGS[i])


def batch_problems(seed: int = 0, n_problems: int = 64):
    """64 independent problems with skeletons of 1..6 actions.

    L ~ U{1..6}; N ~ log-uniform [512, 8192] (rounded to a multiple of 32);
    T = 400 (L = 1), 1000 (L = 2), 3000 (L >= 3).  Problem p's scene uses
    seed 1000 + p.  K = max(8, N // 20).
    """
    rng = np.random.default_rng(seed)
    probs = []
    for p in range(n_problems):
        L = int(rng.integers(1, 7))
        N = int(round(math.exp(rng.uniform(math.log(512), math.log(8192))) / 32.0)) * 32
        if L == 1:
            s, k = reach_scene(1000 + p)
        elif L == 2:
            s, k = push_scene(1000 + p)
        else:
            s, k = pickplace_scene(1000 + p, n_actions=L)
        probs.append(dict(scene=s, skel=k, N=N, K=max(8, N // 20), L=L))
    return probs


def scene_features(scene) -> np.ndarray:
    """16-d scene descriptor for the surrogate: slope, mu, ramp pose,
    three box poses (x, y, yaw), two zero pads."""
    f = np.zeros(16, np.float32)
    if scene["kind"] != "pickplace":
        return f
    f[0] = scene["slope"]
    f[1] = scene["obj_mu"]
    f[2] = 0.5 * (RAMP_FOOT[0] + RAMP_FOOT[1])
    f[3] = 0.5 * (RAMP_FOOT[2] + RAMP_FOOT[3])
    f[4] = 0.0
    for i, (x, y, yaw) in enumerate(scene["boxes"]):
        f[5 + 3 * i: 8 + 3 * i] = (x, y, yaw)
    return f
