"""Pins of the oracle's pick-and-place sequencing (Sec. IV-A: moveTo, grasp,
moveTo, place, moveTo-exit; the grasp is a rigid attachment and the place a
release, Sec. IV-A and Problem 2), CPU only.

The rollouts that exercise grasp, carry, place and release come from a
converged distribution: the oracle's own CE (N = 512, K = 50, 10
iterations) on pick-place scenes 0, 1 and 5, after which most samples
finish all five actions.  Each test checks a property that a plausible slip
would break: an attachment offset with the wrong sign or recomputed every
step, a grasp that ignores the grip-height tolerance, a release with zero
velocity, the velocity of the wrong step or a throw, explicit instead of
semi-implicit Euler in free flight, a penetration that is not mg/k at rest,
a goal test that accepts a held object or ignores the base.
"""
import functools
import math

import numpy as np
import pytest

import workload
from pickplace_common import (ACT, ATT, BX, BY, EX, EY, EZ, GRIP, OVX, OVY, OVZ, OX, OY, OZ, SEEDS, converged,
                              events)


@functools.lru_cache(maxsize=None)
def traces(seed, n=6):
    import oracle

    sc, sk, mean, L = converged(seed)
    th = oracle.sample(1234, 0, 0, n, mean, L)
    return th, [oracle.trace(sc, sk, th[i], sc["T"]) for i in range(n)]


def finished(seed):
    th, trs = traces(seed)
    return [(th[i], tr) for i, tr in enumerate(trs) if tr[-1, ACT] == 5]


def test_converged_rollouts_reach_the_last_action(orc):
    for seed in SEEDS:
        assert len(finished(seed)) >= 3, f"scene {seed}: too few samples finish all five actions"


@pytest.mark.parametrize("seed", SEEDS)
def test_grasp_attaches_with_a_constant_offset(orc, seed):
    """From the grasp on, the object keeps a fixed offset from the end
    effector while base and arm move (1e-12 m), it moves exactly as the end
    effector does, and at the attaching step the end effector is within the
    success tolerance of the grasp point (object + grip-height offset)."""
    sc, sk, _, _ = converged(seed)
    for th, tr in finished(seed):
        ka, kr = events(tr)
        assert ka is not None and kr is not None and ka < kr
        held = slice(ka, kr)  # steps after which the object is attached
        off = tr[held, OX:OZ + 1] - tr[held, EX:EZ + 1]
        assert np.abs(off - off[0]).max() < 1e-12
        d_ee = np.diff(tr[ka:kr, EX:EZ + 1], axis=0)
        d_obj = np.diff(tr[ka:kr, OX:OZ + 1], axis=0)
        assert np.abs(d_ee - d_obj).max() < 1e-12
        assert np.abs(d_ee).max() > 1e-4  # it is carried somewhere, not at rest
        grasp_pt = tr[ka - 1, OX:OZ + 1] + np.array([0.0, 0.0, np.clip(th[GRIP], sk["lo"][GRIP], sk["hi"][GRIP])])
        assert np.linalg.norm(tr[ka, EX:EZ + 1] - grasp_pt) <= sc["eps"] + 1e-12
        # the action index advances exactly at the attaching step
        assert tr[ka - 1, ACT] == 1 and tr[ka, ACT] == 2


@pytest.mark.parametrize("seed", SEEDS)
def test_grip_height_beyond_tolerance_never_attaches(orc, seed):
    """The same parameter vectors with the grip-height offset just beyond
    the tolerance (either sign) never grasp: the object stays free, the plan
    stays at the grasp action, and the sample ends in class 2."""
    sc, sk, _, _ = converged(seed)
    tol = sc["grip_tol"]
    for th, _ in finished(seed)[:2]:
        for h in (tol + 0.004, -(tol + 0.004)):
            t2 = th.copy()
            t2[GRIP] = h
            tr = orc.trace(sc, sk, t2, sc["T"])
            assert tr[:, ATT].max() == 0.0
            assert tr[:, ACT].max() <= 1
            _, cls = orc.rollout(sc, sk, t2[None, :])
            assert cls[0] == 2


def ee_velocity(sc, row):
    """End-effector velocity from one trace row: base velocity plus the
    arm's, the forward kinematics differentiated at fixed azimuth."""
    bvx, bvy, q1, q2, dq1, dq2, beta = row[2], row[3], row[4], row[5], row[6], row[7], row[8]
    l1, l2 = sc["arm_l1"], sc["arm_l2"]
    w12 = dq1 + dq2
    dr = -(l1 * math.sin(q1) * dq1 + l2 * math.sin(q1 + q2) * w12)
    dz = l1 * math.cos(q1) * dq1 + l2 * math.cos(q1 + q2) * w12
    return np.array([bvx + dr * math.cos(beta), bvy + dr * math.sin(beta), dz])


def test_place_releases_with_the_end_effector_velocity(orc):
    """At the releasing step the object leaves the gripper with the end
    effector's velocity of that step (base velocity plus the arm's joint
    rates through the forward kinematics at fixed azimuth, 1e-12); where
    the arm's azimuth did not jump in that step this plus the azimuth's
    turn r dbeta / dt agrees with the end effector's finite difference to
    the second-order bound dt (l1 + l2) w^2 (w the summed angular rates); no
    release is a throw (below 2 m/s).  From the next step on,
    while the object is clear of every body (its bottom 5 mm above the
    Table-2 top and its footprint past the ramp's end), it flies freely
    under semi-implicit Euler (v += -g dt, then x += v dt, exactly)."""
    n_checked, n_fd = 0, 0
    for seed in SEEDS:
        sc, sk, _, _ = converged(seed)
        dt, g, h = sc["dt"], sc["g"], sc["obj_half"]
        top, ramp_end = workload.TABLE2[4], workload.RAMP_FOOT[1]
        l12 = sc["arm_l1"] + sc["arm_l2"]

        def clear(row):
            return row[OZ] - h > top + 5e-3 and row[OX] - h > ramp_end + 5e-3

        for _, tr in finished(seed):
            _, kr = events(tr)
            v = ee_velocity(sc, tr[kr])
            assert np.allclose(tr[kr, OVX:OVZ + 1], v, rtol=0, atol=1e-12)
            assert np.linalg.norm(v) < 2.0
            dbeta = (tr[kr, 8] - tr[kr - 1, 8] + math.pi) % (2 * math.pi) - math.pi
            if abs(dbeta) < 1e-2:  # no azimuth jump in this step
                # the finite difference also holds the azimuth's turn as the
                # base moves: r dbeta / dt along the arm plane's normal
                q1, q2, beta = tr[kr, 4], tr[kr, 5], tr[kr, 8]
                r = sc["arm_l1"] * math.cos(q1) + sc["arm_l2"] * math.cos(q1 + q2)
                v_az = r * dbeta / dt * np.array([-math.sin(beta), math.cos(beta), 0.0])
                v_fd = (tr[kr, EX:EZ + 1] - tr[kr - 1, EX:EZ + 1]) / dt
                w = abs(tr[kr, 6]) + abs(tr[kr, 6] + tr[kr, 7]) + abs(dbeta) / dt
                assert np.abs(v_fd - v - v_az).max() <= dt * l12 * w * w + 1e-9
                n_fd += 1
            assert tr[kr, ACT] == 4 and tr[kr - 1, ACT] == 3
            k = kr
            while clear(tr[k]) and clear(tr[k + 1]):
                v_next = tr[k, OVX:OVZ + 1] + np.array([0.0, 0.0, -g * dt])
                assert np.allclose(tr[k + 1, OVX:OVZ + 1], v_next, rtol=0, atol=1e-12)
                assert np.allclose(tr[k + 1, OX:OZ + 1], tr[k, OX:OZ + 1] + v_next * dt, rtol=0, atol=1e-12)
                k += 1
            n_checked += k > kr
    assert n_checked >= 5 and n_fd >= 5


def test_held_object_moves_with_the_end_effector_velocity(orc):
    """While the object is held its velocity state is the end effector's
    (1e-12) at every step of the carry."""
    for seed in SEEDS:
        sc, sk, _, _ = converged(seed)
        for _, tr in finished(seed)[:3]:
            ka, kr = events(tr)
            for k in range(ka + 1, kr, 37):  # the attaching step still moved it as a free body
                assert np.allclose(tr[k, OVX:OVZ + 1], ee_velocity(sc, tr[k]), rtol=0, atol=1e-12)


def test_released_object_settles_at_mg_over_k(orc):
    """An object released over the Table-2 top (directly, or sliding down
    the ramp onto it) comes to rest pressed into it by the resting
    penetration mg/k of the penalty contact (1e-7 m), with no residual
    velocity, and the sample ends with every action done (class 0 or 1)."""
    n = 0
    for seed in SEEDS:
        sc, sk, _, _ = converged(seed)
        h, top = sc["obj_half"], workload.TABLE2[4]
        delta = sc["obj_mass"] * sc["g"] / sc["k_contact"]
        for th, tr in finished(seed):
            _, kr = events(tr)
            end = tr[-1]
            on_table = abs(end[OX] - workload.TABLE2[0]) < 0.3 and abs(end[OY] - workload.TABLE2[1]) < 0.3
            if not on_table or kr > sc["T"] - 500:
                continue
            n += 1
            assert abs(end[OZ] - (top + h - delta)) < 1e-7
            assert np.abs(end[OVX:OVZ + 1]).max() < 1e-6
            J, cls = orc.rollout(sc, sk, th[None, :])
            assert cls[0] in (0, 1)
    assert n >= 10


def test_dropped_object_falls_by_the_closed_form_and_settles(orc):
    """Hand-built: the object starts 0.3 m above the Table-2 top and is never
    grasped (grip-height beyond tolerance).  Semi-implicit Euler gives
    v_k = -k g dt and z_k = z_0 - g dt^2 k (k + 1) / 2 exactly until the
    contact, and the object comes to rest at top + h - mg/k."""
    sc, sk, _ = workload.config(2, seed=0, T=1500)
    x0, y0, top, h = workload.TABLE2[0], workload.TABLE2[1], workload.TABLE2[4], sc["obj_half"]
    z0 = top + h + 0.3
    sc = dict(sc, obj_start=(x0, y0, z0))
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    th = (lo + hi) / 2
    th[GRIP] = hi[GRIP]
    tr = orc.trace(sc, sk, th, sc["T"])
    dt, g = sc["dt"], sc["g"]
    k = np.arange(1, 200)
    z = z0 - g * dt * dt * k * (k + 1) / 2
    free = z - h > top  # no penetration yet
    assert free.sum() > 100
    assert np.allclose(tr[k - 1, OZ][free], z[free], rtol=0, atol=1e-12)
    assert np.allclose(tr[k - 1, OVZ][free], (-k * g * dt)[free], rtol=0, atol=1e-12)
    assert np.abs(tr[:, OX] - x0).max() < 1e-12 and np.abs(tr[:, OY] - y0).max() < 1e-12
    delta = sc["obj_mass"] * g / sc["k_contact"]
    assert abs(tr[-1, OZ] - (top + h - delta)) < 1e-9
    assert tr[:, ATT].max() == 0.0


def _state(bx, by, ox, oy, oz, attached):
    s = np.zeros(20)
    s[BX], s[BY], s[OX], s[OY], s[OZ], s[ATT] = bx, by, ox, oy, oz, attached
    return s


def test_final_goal_and_class_on_hand_built_states(orc):
    """psi_g and the plan cost from hand-built final states of the 5-action
    plan: object resting in the Table-2 region and base in Exit -> class 0
    with J = t; the object still held -> not class 0; the base 0.3 m beyond
    the Exit box -> class 1 with J = t + 10 * 0.3; the object off the region
    by (0.2, 0, 0.1) -> J = t + 10 * sqrt(0.05); an unfinished plan -> class
    2; a non-finite cost -> class 3."""
    sc, sk, _ = workload.config(2, seed=0)
    oc, ohw = sc["obj_region_center"], sc["obj_region_half"]
    bc, bhw = sc["base_region_center"], sc["base_region_half"]
    t = 3.25
    good = _state(bc[0], bc[1], oc[0], oc[1], oc[2], 0)
    J, c = orc.pickplace_final(sc, sk, good, True, t)
    assert c == 0 and J == pytest.approx(t, abs=1e-15)
    J, c = orc.pickplace_final(sc, sk, _state(bc[0], bc[1], oc[0], oc[1], oc[2], 1), True, t)
    assert c == 1
    J, c = orc.pickplace_final(sc, sk, _state(bc[0] + bhw[0] + 0.3, bc[1], oc[0], oc[1], oc[2], 0), True, t)
    assert c == 1 and J == pytest.approx(t + 10 * 0.3, abs=1e-12)
    J, c = orc.pickplace_final(sc, sk, _state(bc[0], bc[1], oc[0] + ohw[0] + 0.2, oc[1], oc[2] + ohw[2] + 0.1, 0),
                               True, t)
    assert c == 1 and J == pytest.approx(t + 10 * math.sqrt(0.2 ** 2 + 0.1 ** 2), abs=1e-12)
    # just inside the boxes' corners still counts
    e = 1e-9
    J, c = orc.pickplace_final(sc, sk, _state(bc[0] + bhw[0] - e, bc[1] - bhw[1] + e, oc[0] - ohw[0] + e,
                                              oc[1] + ohw[1] - e, oc[2] + ohw[2] - e, 0), True, t)
    assert c == 0 and J == pytest.approx(t, abs=1e-15)
    J, c = orc.pickplace_final(sc, sk, good, False, t)
    assert c == 2
    J, c = orc.pickplace_final(sc, sk, good, True, float("nan"))
    assert c == 3 and math.isnan(J)


def test_final_goal_of_the_held_object_plan(orc):
    """The 3-action skeleton (move, grasp, move) asks for the object held
    and the base in its region: held -> class 0 with J = t; dropped -> class
    1 with J = t + w_obj * 1."""
    sc, sk = workload.pickplace_scene(0, n_actions=3)
    bc = sc["base_region_center"]
    J, c = orc.pickplace_final(sc, sk, _state(bc[0], bc[1], 0.0, 0.0, 0.0, 1), True, 2.0)
    assert c == 0 and J == pytest.approx(2.0, abs=1e-15)
    J, c = orc.pickplace_final(sc, sk, _state(bc[0], bc[1], 0.0, 0.0, 0.0, 0), True, 2.0)
    assert c == 1 and J == pytest.approx(2.0 + sc["w_obj"], abs=1e-12)
