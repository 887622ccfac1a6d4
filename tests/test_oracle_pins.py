"""Pins of the FP64 oracle against closed forms, invariants and library routines.

Each test checks one building block of the method against something other
than the oracle itself, chosen so that a plausible slip (a dropped term, a
wrong sign, a transposed index, explicit instead of semi-implicit Euler)
fails.  CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- sampling
def test_philox_known_answers(orc):
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_philox_counter_layout(orc):
    # word (n, c) of the sample table is philox((n, c, iter, problem), seed)
    seed, it, prob = 0x1234_5678_9ABC_DEF0, 7, 3
    w = orc.philox_words(seed, it, prob, 5, 7)
    assert w.shape == (5, 8)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for n in range(5):
        for c in range(2):
            assert w[n, 4 * c:4 * c + 4].tolist() == orc.philox([n, c, it, prob], key).tolist()


def test_uniform_words_chi2(orc):
    w = orc.philox_words(42, 0, 0, 1 << 16, 16).reshape(-1)  # 2^20 words
    hist = np.bincount((w >> 24).astype(np.int64), minlength=256)
    chi2, p = stats.chisquare(hist)
    assert 1e-4 < p < 1 - 1e-4


def test_box_muller_normals(orc):
    z = orc.normals(7, 3, 1, 50000, 6)
    flat = z.reshape(-1)
    assert abs(flat.mean()) < 0.01
    assert abs(flat.var() - 1.0) < 0.01
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # the cos/sin halves of a Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.02


def test_sample_covariance(orc):
    rng = np.random.default_rng(0)
    D = 5
    B = rng.standard_normal((D, D))
    cov = B @ B.T + 0.5 * np.eye(D)
    L = np.linalg.cholesky(cov)
    mean = rng.standard_normal(D)
    th = orc.sample(3, 0, 0, 200000, mean, L)
    assert np.allclose(th.mean(0), mean, atol=0.02)
    assert np.allclose(np.cov(th.T), cov, atol=0.05 * np.abs(cov).max())


# ---------------------------------------------------------------- dynamics
def _reach(T, dt=0.002, **over):
    sc, sk = workload.reach_scene(T=T, dt=dt)
    sc.update(over)
    sk["lo"][2] = 0.0
    return sc, sk


def test_sliding_block_decelerates_at_mu_g(orc):
    # no controller force (kp = 0): the base slides on the ground from v0 = 1 m/s
    v0, mu, dt = 1.0, 0.5, 0.002
    sc, sk = _reach(200, dt, base_mu=mu, base_v0=(v0, 0.0, 0.0), yaw_kp=0.0, yaw_kd=0.0)
    tr = orc.trace(sc, sk, np.zeros(3), 200)
    step = mu * 9.81 * dt
    v, x = v0, 0.0
    vs, xs = [], []
    for _ in range(200):  # exact discrete closed form of the implicit clamp
        v = 0.0 if v <= step else v - step
        x += dt * v
        vs.append(v)
        xs.append(x)
    np.testing.assert_allclose(tr[:, 3], vs, rtol=0, atol=1e-12)
    np.testing.assert_allclose(tr[:, 0], xs, rtol=0, atol=1e-12)
    assert np.count_nonzero(tr[:, 3]) == math.ceil(v0 / step) - 1
    # continuous limit: stopping distance v0^2 / (2 mu g) within O(v0 dt)
    assert abs(tr[-1, 0] - v0 ** 2 / (2 * mu * 9.81)) < 2 * v0 * dt
    assert np.all(tr[:, 1] == 0.0)


def test_spin_friction_uses_mean_radius(orc):
    # a spinning footprint loses mu m g rbar dt / I of angular velocity per step
    w0, mu, dt = 2.0, 0.5, 0.002
    a, b = 0.25, 0.20
    d = math.hypot(a, b)
    rbar = (a * b * d / 3 + a ** 3 / 6 * math.log((b + d) / a) + b ** 3 / 6 * math.log((a + d) / b)) / (a * b)
    assert abs(orc.mean_radius(a, b) - rbar) < 1e-7
    sc, sk = _reach(100, dt, base_mu=mu, base_v0=(0.0, 0.0, w0), yaw_kp=0.0, yaw_kd=0.0)
    tr = orc.trace(sc, sk, np.zeros(3), 100)
    I = 10.0 * ((2 * a) ** 2 + (2 * b) ** 2) / 12
    dw = mu * 10.0 * 9.81 * rbar * dt / I
    expect = np.maximum(w0 - dw * np.arange(1, 101), 0.0)
    expect[expect <= 0] = 0.0
    np.testing.assert_allclose(tr[:, 5], expect, atol=1e-6)


def test_pd_step_response(orc):
    # friction off: semi-implicit Euler of a unit-mass PD law, kd = 2 sqrt(kp)
    kp, dt, T = 16.0, 0.002, 1500
    sc, sk = _reach(T, dt, base_mu=0.0, yaw_kp=0.0, yaw_kd=0.0)
    tr = orc.trace(sc, sk, np.array([0.0, 0.0, kp]), T)
    kd = 2 * math.sqrt(kp)
    M = np.array([[1 - dt * dt * kp, dt * (1 - dt * kd)], [-dt * kp, 1 - dt * kd]])
    for axis, g in ((0, 2.0), (1, 1.0)):
        e0 = np.array([0.0 - g, 0.0])
        E = np.array([np.linalg.matrix_power(M, k + 1) @ e0 for k in range(T)])
        np.testing.assert_allclose(tr[:, axis] - g, E[:, 0], atol=1e-12)
        np.testing.assert_allclose(tr[:, 3 + axis], E[:, 1], atol=1e-11)
        # continuous critically damped response e0 (1 + w t) exp(-w t)
        w = math.sqrt(kp)
        t = dt * np.arange(1, T + 1)
        cont = e0[0] * (1 + w * t) * np.exp(-w * t)
        assert np.max(np.abs(tr[:, axis] - g - cont)) < 2 * w * dt * abs(e0[0])


def test_time_to_reach_cost(orc):
    # J = t_reach + 10 |p_T - goal| with the crossing interpolated (or step-counted)
    kp, dt, T = 16.0, 0.002, 1500
    for mode in ("interp", "step"):
        sc, sk = _reach(T, dt, base_mu=0.0, yaw_kp=0.0, yaw_kd=0.0, cost_mode=mode)
        kd = 2 * math.sqrt(kp)
        M = np.array([[1 - dt * dt * kp, dt * (1 - dt * kd)], [-dt * kp, 1 - dt * kd]])
        ex, ey = np.array([-2.0, 0.0]), np.array([-1.0, 0.0])
        dist = [math.hypot(ex[0], ey[0])]
        for _ in range(T):
            ex, ey = M @ ex, M @ ey
            dist.append(math.hypot(ex[0], ey[0]))
        k = next(i for i in range(1, T + 1) if dist[i] <= 0.05) - 1  # step index that crossed
        if mode == "interp":
            t = (k + (dist[k] - 0.05) / (dist[k] - dist[k + 1])) * dt
        else:
            t = (k + 1) * dt
        J, cls = orc.rollout(sc, sk, np.array([[0.0, 0.0, kp]]))
        assert cls[0] == 0
        assert abs(J[0] - (t + 10 * dist[T])) < 1e-12


def _push_free(T=400, mu_c=0.5, c=50.0):
    sc, sk = workload.push_scene(0, T=T)
    sc.update(base_mu=0.0, block_mu=0.0, yaw_kp=0.0, yaw_kd=0.0, contact_mu=mu_c, c_contact=c,
              base_start=(0.3, -0.12, 0.1), base_v0=(1.2, 0.25, 0.6), block_start=(1.0, 0.0, 0.35))
    sk["lo"][2] = 0.0
    sk["lo"][5] = 0.0
    return sc, sk


def _momenta(tr, sc):
    mb, mk = sc["base_mass"], sc["block_mass"]
    Ib = mb * (4 * sc["base_half"][0] ** 2 + 4 * sc["base_half"][1] ** 2) / 12
    Ik = mk * (4 * sc["block_half"][0] ** 2 + 4 * sc["block_half"][1] ** 2) / 12
    P = mb * tr[:, 3:5] + mk * tr[:, 9:11]
    L = (mb * (tr[:, 0] * tr[:, 4] - tr[:, 1] * tr[:, 3]) + Ib * tr[:, 5]
         + mk * (tr[:, 6] * tr[:, 10] - tr[:, 7] * tr[:, 9]) + Ik * tr[:, 11])
    E = 0.5 * mb * (tr[:, 3] ** 2 + tr[:, 4] ** 2) + 0.5 * Ib * tr[:, 5] ** 2 \
        + 0.5 * mk * (tr[:, 9] ** 2 + tr[:, 10] ** 2) + 0.5 * Ik * tr[:, 11] ** 2
    return P, L, E


def test_body_contact_conserves_momentum(orc):
    # equal and opposite normal and friction impulses at one contact point:
    # linear and angular momentum are conserved exactly; energy only drops
    sc, sk = _push_free()
    tr = orc.trace(sc, sk, np.zeros(6), 400)
    P, L, E = _momenta(tr, sc)
    assert np.abs(tr[-1, 9:12]).max() > 0.1  # the block was hit and moves/spins
    np.testing.assert_allclose(P - P[0], 0.0, atol=1e-11)
    np.testing.assert_allclose(L - L[0], 0.0, atol=1e-11)
    assert E.max() <= E[0] + 1e-9  # kinetic energy never exceeds the initial total
    assert E[-1] < E[0]


def test_push_broad_phase_skip_is_exact(orc):
    # the push rollout tests base-block contact only where the block's
    # bounding circle reaches the base; running the exact test on every step
    # instead must give the same trajectories, costs and classes bit for bit
    # (initial distribution and converged-style samples, contact-heavy),
    # while the op tally shows the skipped work
    results = []
    for seed in (0, 3):
        sc, sk = workload.push_scene(seed, T=600)
        lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
        th = np.random.default_rng(seed).uniform(lo, hi, (48, len(lo)))
        for exhaustive in (False, True):
            orc.set_exhaustive_contacts(exhaustive)
            try:
                J, c = orc.rollout(sc, sk, th)
                tr = orc.trace(sc, sk, th[0], 600)
                ops = orc.count_ops(sc, sk, th[:8])
            finally:
                orc.set_exhaustive_contacts(False)
            results.append((J, c, tr, ops))
        (J0, c0, t0, o0), (J1, c1, t1, o1) = results[-2:]
        assert np.array_equal(J0, J1) and np.array_equal(c0, c1) and np.array_equal(t0, t1)
        assert o1["add"] + o1["mul"] > o0["add"] + o0["mul"]  # the exact test ran more often
    sc, sk = _push_free()
    tr0 = orc.trace(sc, sk, np.zeros(6), 400)
    orc.set_exhaustive_contacts(True)
    try:
        tr1 = orc.trace(sc, sk, np.zeros(6), 400)
    finally:
        orc.set_exhaustive_contacts(False)
    assert np.array_equal(tr0, tr1) and np.abs(tr0[-1, 9:12]).max() > 0.1  # a real collision, unchanged


def _push_head_on(T, force_limit, weights=(0.0, 0.0, 1.0)):
    """A base sliding at 1.2 m/s along +x into a block at rest, both at yaw 0
    and centred on y = 0, nothing rubbing (ground, contact and controllers
    off, kp = 0): the contact normal stays +x and the contact point on the x
    axis, so the block only translates and every normal impulse goes into its
    x momentum.  weights = (w_time, w_goal, w_viol)."""
    sc, sk = workload.push_scene(0, T=T)
    sc.update(base_mu=0.0, block_mu=0.0, contact_mu=0.0, yaw_kp=0.0, yaw_kd=0.0,
              base_start=(0.3, 0.0, 0.0), base_v0=(1.2, 0.0, 0.0), block_start=(1.0, 0.0, 0.0),
              force_limit=force_limit, w_time=weights[0], w_goal=weights[1], w_viol=weights[2])
    sk["lo"][2] = 0.0
    sk["lo"][5] = 0.0
    return sc, sk


def test_force_limit_penalty_is_the_impulse_above_the_limit(orc):
    """With only the violation weight on, J = sum_t max(F_n,t - F_lim, 0) dt.
    F_n,t is read back from the block's x momentum (m dv = F_n dt each step,
    nothing else acts on it): at F_lim = 0 the penalty is the whole normal
    impulse m v_T; a wrong threshold sign, a missing dt or a penalty on
    |F_n| fails here."""
    T = 400
    sc, sk = _push_head_on(T, 0.0)
    tr = orc.trace(sc, sk, np.zeros(6), T)
    vx = np.concatenate([[0.0], tr[:, 9]])
    mk, dt = sc["block_mass"], sc["dt"]
    Fn = mk * np.diff(vx) / dt
    assert vx[-1] > 1.0 and np.all(Fn >= -1e-9) and (Fn > 1.0).sum() >= 5  # a real collision
    np.testing.assert_allclose(tr[:, 10:12], 0.0, atol=0.0)  # the block never turns or drifts in y
    J0, cls0 = orc.rollout(sc, sk, np.zeros((1, 6)))
    assert abs(J0[0] - mk * vx[-1]) <= 1e-12 * mk * vx[-1]
    for flim in (0.3 * Fn.max(), 0.8 * Fn.max(), 2.0 * Fn.max()):
        sc, sk = _push_head_on(T, flim)
        J, _ = orc.rollout(sc, sk, np.zeros((1, 6)))
        expect = np.sum(np.maximum(Fn - flim, 0.0)) * dt
        assert abs(J[0] - expect) <= 1e-9 * max(expect, 1.0), (flim, J[0], expect)
    assert J[0] == 0.0  # below the limit throughout


def _at_rest_on_targets(kind, base_xy, block_xy=None):
    """Every action's success target (its nominal point) put where the base
    rests with kp = 0, so action i succeeds at step i with the base inside
    eps from the start (crossing fraction 0): t_done = (L - 1) dt."""
    if kind == "reach":
        sc, sk = workload.reach_scene(T=3)
        sk["lo"][2] = 0.0
    else:
        sc, sk = workload.push_scene(0, T=3)
        sk["lo"][2] = sk["lo"][5] = 0.0
        sc.update(block_start=(block_xy[0], block_xy[1], 0.0), block_mu=0.0)
    sc.update(base_start=(base_xy[0], base_xy[1], 0.0), base_mu=0.0, yaw_kp=0.0, yaw_kd=0.0)
    for a in sk["actions"]:
        a["nominal"] = (base_xy[0], base_xy[1], 0.0)
    return sc, sk


def test_push_goal_test_and_region_distance(orc):
    """Both actions done at steps 0 and 1 (t_done = dt) with the block at rest
    far from the base: class 0 exactly when the block centre is inside the
    goal rectangle (a hair inside a corner included), else class 1 (a micron
    outside included), and J = w_time dt + w_goal * (distance from the block
    centre to the rectangle)."""
    sc0, _ = workload.push_scene(0)
    (cx, cy, _), (hx, hy, _) = sc0["goal_center"], sc0["goal_half"]
    cases = [((0.0, 0.0), 0, 0.0), ((hx - 1e-9, -(hy - 1e-9)), 0, 0.0), ((hx + 1e-6, 0.0), 1, 1e-6),
             ((hx + 0.3, 0.1), 1, 0.3), ((-(hx + 0.3), hy + 0.4), 1, 0.5), ((0.05, -(hy + 0.25)), 1, 0.25)]
    for (dx, dy), cls_expect, dist in cases:
        sc, sk = _at_rest_on_targets("push", (cx - 3.0, cy - 3.0), (cx + dx, cy + dy))
        J, cls = orc.rollout(sc, sk, np.zeros((1, 6)))
        assert cls[0] == cls_expect, (dx, dy)
        assert abs(J[0] - (sc["w_time"] * sc["dt"] + sc["w_goal"] * dist)) < 1e-12, (dx, dy, J[0])


def test_reach_goal_test_and_distance(orc):
    """A one-action reach done at step 0 (t_done = 0) with the base at rest:
    class 0 at the goal centre, class 1 when the action's target lies 0.5 m
    from it (the action succeeds, the task does not), J = 10 * distance."""
    for off, cls_expect in ((0.0, 0), (0.04, 0), (0.5, 1)):
        sc, sk = _at_rest_on_targets("reach", (2.0 + off, 1.0))
        J, cls = orc.rollout(sc, sk, np.zeros((1, 3)))
        assert cls[0] == cls_expect and abs(J[0] - sc["w_goal"] * off) < 1e-12, (off, J[0], cls[0])


def test_yaw_pd_step_response(orc):
    """Heading control alone (no translation, no ground friction): the yaw
    follows semi-implicit Euler of the unit-inertia PD law toward the
    action's heading, exactly the matrix recurrence of the position test."""
    ykp, ykd, dt, T, yaw_t = 25.0, 10.0, 0.002, 800, 0.6
    sc, sk = _reach(T, dt, base_mu=0.0, yaw_kp=ykp, yaw_kd=ykd)
    sk["actions"][0]["yaw"] = yaw_t
    tr = orc.trace(sc, sk, np.zeros(3), T)
    M = np.array([[1 - dt * dt * ykp, dt * (1 - dt * ykd)], [-dt * ykp, 1 - dt * ykd]])
    e0 = np.array([0.0 - yaw_t, 0.0])
    E = np.array([np.linalg.matrix_power(M, k + 1) @ e0 for k in range(T)])
    np.testing.assert_allclose(tr[:, 2] - yaw_t, E[:, 0], atol=1e-12)
    np.testing.assert_allclose(tr[:, 5], E[:, 1], atol=1e-11)
    np.testing.assert_allclose(tr[:, 0:2], 0.0, atol=0.0)  # the base turns in place


def test_body_contact_elastic_without_damping(orc):
    # no damping, no friction: the penalty spring returns the energy
    sc, sk = _push_free(T=600, mu_c=0.0, c=0.0)
    tr = orc.trace(sc, sk, np.zeros(6), 600)
    P, L, E = _momenta(tr, sc)
    assert np.abs(tr[-1, 9:11]).max() > 0.1
    assert abs(E[-1] - E[0]) / E[0] < 0.02


def _corner_contact(block_yaw, depth_fn):
    """A base at rest at the origin (yaw 0) and a block at rest rotated by
    block_yaw, placed so that its corners left of the base's front face
    (x = 0.25) penetrate it as depth_fn(corners) says; no friction anywhere,
    no controller force on the block.  Returns the scene, the skeleton, the
    block centre and its corners."""
    sc, sk = workload.push_scene(0, T=2)
    sc.update(base_mu=0.0, block_mu=0.0, contact_mu=0.0, c_contact=50.0, yaw_kp=0.0, yaw_kd=0.0,
              base_start=(0.0, 0.0, 0.0), base_v0=(0.0, 0.0, 0.0), block_v0=(0.0, 0.0, 0.0))
    h = sc["block_half"][0]
    c, s = math.cos(block_yaw), math.sin(block_yaw)
    local = np.array([(-h, -h), (h, -h), (-h, h), (h, h)])
    rot = local @ np.array([[c, s], [-s, c]])  # corner offsets in the world frame
    cx = 0.25 - rot[:, 0].min() - depth_fn(rot)
    cy = 0.05
    sc["block_start"] = (cx, cy, block_yaw)
    return sc, sk, np.array([cx, cy]), rot + np.array([cx, cy])


def _block_first_step(orc, sc, sk):
    th = np.array([0.0, 0.0, 5.0, 0.0, 0.0, 5.0])
    tr = orc.trace(sc, sk, th, 1)
    return tr[0, 9:12]  # block vx, vy, w after one step from rest


def test_single_corner_contact_point_is_that_corner(orc):
    """One corner of a block rotated by 0.5 rad penetrates the base's front
    face by 1 mm: the minimum-overlap axis is the face normal +x, the depth
    1 mm, and the contact point is that corner, so after one step from rest
    the block has v = dt k d / m along +x and spin w = dt (r x F) / I with r
    from its centre to the corner (the centres' midpoint, or any other
    point, gives another spin)."""
    d = 1e-3
    sc, sk, ctr, corners = _corner_contact(0.5, lambda rot: d)
    inside = corners[:, 0] < 0.25
    assert inside.sum() == 1
    q = corners[inside][0]
    dt, k, m = sc["dt"], sc["k_contact"], sc["block_mass"]
    I = m * (4 * sc["block_half"][0] ** 2 + 4 * sc["block_half"][1] ** 2) / 12
    F = np.array([k * d, 0.0])
    r = q - ctr
    v, w = _block_first_step(orc, sc, sk)[:2], _block_first_step(orc, sc, sk)[2]
    np.testing.assert_allclose(v, dt * F / m, rtol=0, atol=1e-12)
    assert abs(w - dt * (r[0] * F[1] - r[1] * F[0]) / I) < 1e-9
    assert abs(w) > 1e-3  # the corner's lever arm is what spins the block


def test_two_corner_contact_point_is_penetration_weighted(orc):
    """A block rotated by 0.03 rad with both left corners 0.4 mm and about
    3.4 mm inside the base's front face: depth = the deeper corner's, and
    the contact point is the corners' mean weighted by their penetrations
    below the face (not their plain mean), which fixes the block's first
    spin."""
    sc, sk, ctr, corners = _corner_contact(0.03, lambda rot: 3.4e-3)
    inside = corners[:, 0] < 0.25
    assert inside.sum() == 2
    pen = 0.25 - corners[inside, 0]
    q = (pen[:, None] * corners[inside]).sum(0) / pen.sum()
    q_plain = corners[inside].mean(0)
    dt, k, m = sc["dt"], sc["k_contact"], sc["block_mass"]
    I = m * (4 * sc["block_half"][0] ** 2 + 4 * sc["block_half"][1] ** 2) / 12
    F = np.array([k * pen.max(), 0.0])
    out = _block_first_step(orc, sc, sk)
    np.testing.assert_allclose(out[:2], dt * F / m, rtol=0, atol=1e-12)
    w_weighted = dt * ((q - ctr)[0] * F[1] - (q - ctr)[1] * F[0]) / I
    w_plain = dt * ((q_plain - ctr)[0] * F[1] - (q_plain - ctr)[1] * F[0]) / I
    assert abs(out[2] - w_weighted) < 1e-9
    assert abs(w_weighted - w_plain) > 1e-3  # the two rules are told apart


def _object_scene(T, geoms, obj_start, obj_v0=(0, 0, 0), mu=0.3, c=50.0):
    # the object alone: the robot only runs a moveTo far away from it
    sc, _ = workload.pickplace_scene(0, T=T)
    sc.update(geoms=geoms, obj_start=obj_start, obj_v0=obj_v0, obj_mu=mu, contact_mu=mu, c_contact=c)
    sk = dict(actions=[dict(kind="move", nominal=(-2.4, -1.4, 0.0), yaw=0.0, success_ref="target")],
              lo=[-0.1, -0.1, 5.0], hi=[0.1, 0.1, 50.0])
    return sc, sk


GROUND = dict(slabs=[(0.0, 0.0, 1.0, -1e3, 0.0)], base=False, obj=True)


def test_free_flight_is_exact(orc):
    dt, T = 0.002, 300
    sc, sk = _object_scene(T, [GROUND], (0.0, 0.0, 3.0), (0.5, -0.2, 2.0))
    th = 0.5 * (np.array(sk["lo"]) + np.array(sk["hi"]))
    tr = orc.trace(sc, sk, th, T)
    k = np.arange(1, T + 1)
    vz = 2.0 - 9.81 * dt * k
    z = 3.0 + dt * np.cumsum(vz)
    np.testing.assert_allclose(tr[:, 14], vz, atol=1e-12)
    np.testing.assert_allclose(tr[:, 11], z, atol=1e-12)
    np.testing.assert_allclose(tr[:, 9], 0.5 * dt * k, atol=1e-12)


def test_resting_penetration_is_mg_over_k(orc):
    sc, sk = _object_scene(4000, [GROUND], (0.0, 0.0, 0.05))
    th = 0.5 * (np.array(sk["lo"]) + np.array(sk["hi"]))
    tr = orc.trace(sc, sk, th, 4000)
    delta = 0.05 - tr[-1, 11]
    assert abs(delta - 0.5 * 9.81 / 2.0e4) < 1e-9
    assert abs(tr[-1, 14]) < 1e-9


def test_bounce_energy_bounded_no_drift(orc):
    # no damping, no friction: symplectic Euler keeps the energy oscillation
    # bounded (O(w dt)) with no secular drift over 1e5 steps
    T = 100000
    sc, sk = _object_scene(T, [GROUND], (0.0, 0.0, 0.3), mu=0.0, c=0.0)
    th = 0.5 * (np.array(sk["lo"]) + np.array(sk["hi"]))
    tr = orc.trace(sc, sk, th, T)
    m, k, g = 0.5, 2.0e4, 9.81
    z, vz = tr[:, 11], tr[:, 14]
    pen = np.maximum(0.05 - z, 0.0)
    E = 0.5 * m * vz ** 2 + m * g * z + 0.5 * k * pen ** 2
    E0 = m * g * 0.3
    w = math.sqrt(k / m)
    assert np.max(np.abs(E - E0)) / E0 < 2 * w * 0.002
    # each bounce moves the flight energy by a bounded, phase-dependent amount;
    # a non-symplectic (explicit) step would instead gain ~(w dt)^2 per contact step
    last = E[-T // 10:].mean()
    assert abs(last - E0) / E0 < 0.05


def _ramp_scene(slope_deg, mu, T):
    s = math.radians(slope_deg)
    slabs, z_hi = workload._ramp_slabs(0.0, 2.0, -0.5, 0.5, 0.2, s)
    n = slabs[3]
    cx = 0.6
    h = 0.05
    cz = (n[4] + h * (abs(n[0]) + abs(n[2])) - n[0] * cx) / n[2]
    geoms = [GROUND, dict(slabs=slabs, base=False, obj=True)]
    return _object_scene(T, geoms, (cx, 0.0, cz), mu=mu), s


def test_ramp_static_when_friction_suffices(orc):
    (sc, sk), s = _ramp_scene(15.0, 0.4, 1500)  # tan 15 deg = 0.27 < 0.4
    th = 0.5 * (np.array(sk["lo"]) + np.array(sk["hi"]))
    tr = orc.trace(sc, sk, th, 1500)
    assert abs(tr[-1, 9] - 0.6) < 2e-3
    assert np.abs(tr[-500:, 12]).max() < 1e-3


def test_ramp_slides_at_g_sin_minus_mu_cos(orc):
    (sc, sk), s = _ramp_scene(30.0, 0.2, 400)  # tan 30 deg = 0.58 > 0.2
    th = 0.5 * (np.array(sk["lo"]) + np.array(sk["hi"]))
    tr = orc.trace(sc, sk, th, 400)
    v_along = tr[:, 12] * math.cos(s) - tr[:, 14] * math.sin(s)  # down-slope speed
    acc = (v_along[350] - v_along[150]) / (200 * 0.002)
    expect = 9.81 * (math.sin(s) - 0.2 * math.cos(s))
    assert abs(acc - expect) / expect < 0.02


def test_arm_ik_fk_consistent(orc):
    # a place-only skeleton: the arm's joint PD drives the end effector onto
    # any reachable target (IK and FK are inverse of each other)
    sc, sk = workload.pickplace_scene(0, T=3000)
    sc.update(geoms=[GROUND], base_start=(0.0, 0.0, 0.0))
    sk = dict(actions=[dict(kind="place", nominal=(0.0, 0.0, 0.0), yaw=0.0, success_ref="target")],
              lo=[-2.0, -2.0, -1.0], hi=[2.0, 2.0, 2.0])
    for tgt in ((0.5, 0.3, 0.7), (-0.4, 0.2, 0.2), (0.1, -0.6, 0.9)):
        tr = orc.trace(sc, sk, np.array(tgt), 3000)
        np.testing.assert_allclose(tr[-1, 17:20], tgt, atol=1e-6)
        assert tr[-1, 16] == 1  # the place action succeeded
    # out of reach: the arm stretches along the bearing to the target
    tr = orc.trace(sc, sk, np.array((1.9, 0.0, 0.45)), 3000)
    np.testing.assert_allclose(tr[-1, 17:20], (0.899, 0.0, 0.45), atol=1e-6)


# ------------------------------------------------------ selection and refit
def test_select_matches_lexsort(orc):
    rng = np.random.default_rng(1)
    for trial in range(50):
        N = int(rng.integers(1, 65))
        J = rng.choice(np.array([0.5, 1.0, 1.5, 2.0, 7.25], np.float32), N)  # many ties
        cls = rng.choice(np.arange(4), N, p=[0.2, 0.3, 0.4, 0.1]).astype(np.uint8)
        J[cls == 3] = np.nan if trial % 2 else np.inf
        K = int(rng.integers(1, 20))
        idx = orc.select(J, cls, K)
        Jk = np.where(cls == 3, np.inf, J)
        order = np.lexsort((np.arange(N), Jk, cls))
        present = [c for c in (0, 1) if np.any(cls == c)]
        if present:
            cstar = present[0]
        elif np.any(cls == 2):
            cstar = 2
        else:
            assert len(idx) == 0
            continue
        expect = [i for i in order if cls[i] == cstar][:K]
        assert idx.tolist() == expect


def test_refit_matches_numpy(orc):
    rng = np.random.default_rng(2)
    N, D = 300, 7
    th = rng.standard_normal((N, D)) * rng.uniform(0.1, 2, D)
    lo, hi = -np.ones(D) * 3, np.ones(D) * 5
    idx = rng.choice(N, 40, replace=False).astype(np.int32)
    rc, mean, cov, chol = orc.refit(th, idx, lo, hi)
    e = th[idx]
    ref_cov = np.cov(e.T, bias=True) + np.diag((1e-4 * (hi - lo)) ** 2)
    assert rc == 0
    np.testing.assert_allclose(mean, e.mean(0), atol=1e-13)
    np.testing.assert_allclose(cov, ref_cov, atol=1e-13)
    np.testing.assert_allclose(chol, np.linalg.cholesky(ref_cov), atol=1e-12)
    rc, mean, cov, chol = orc.refit(th, idx, lo, hi, diag=True)
    np.testing.assert_allclose(cov, np.diag(np.diag(ref_cov)), atol=1e-13)
    # a single elite: the sample itself with artificial noise 0.05 * range
    rc, mean, cov, chol = orc.refit(th, idx[:1], lo, hi)
    np.testing.assert_allclose(mean, th[idx[0]])
    np.testing.assert_allclose(cov, np.diag((0.05 * (hi - lo)) ** 2))
    # no elites: the distribution is kept
    m0, c0 = np.arange(D, dtype=float), np.eye(D) * 2.0
    rc, mean, cov, chol = orc.refit(th, idx[:0], lo, hi, mean=m0, cov=c0, chol=np.sqrt(c0))
    np.testing.assert_allclose(mean, m0)
    np.testing.assert_allclose(cov, c0)


def test_refit_rank_deficient_stays_pd(orc):
    # K_eff <= D: the ridge keeps the covariance positive definite
    rng = np.random.default_rng(3)
    th = rng.standard_normal((10, 8))
    rc, mean, cov, chol = orc.refit(th, np.arange(3, dtype=np.int32), -np.ones(8), np.ones(8))
    assert rc == 0
    assert np.all(np.linalg.eigvalsh(cov) > 0)
    np.testing.assert_allclose(chol @ chol.T, cov, atol=1e-14)


def test_cem_quadratic_converges_to_minimiser(orc):
    for seed in range(3):
        sc, sk = workload.quadratic_scene(seed, D=6)
        r = orc.cem(sc, sk, seed, N=512, K=50, iters=30)
        assert np.linalg.norm(r["mean"] - np.array(sc["theta_star"])) < 1e-3 * 2.0
        assert r["best_J"] < 1e-4
        assert r["best_cls"] == 0


def test_op_counter_on_quadratic(orc):
    sc, sk = workload.quadratic_scene(0, D=5)
    ops = orc.count_ops(sc, sk, np.zeros((1, 5)))
    D = 5
    assert ops["add"] == D * (2 * D + 2)
    assert ops["mul"] == D * (D + 1)
    assert ops["div"] == 0 and ops["sqrt"] == 0 and ops["transc"] == 0
