"""Pins of the oracle's base planner and waypoint tracking (Sec. IV-A: A*
paths for the mobile base, tracked by a PID controller).

The planner is checked against a closed-form detour around one square, the
straight line when nothing is in the way, path validity (no segment enters
a grown footprint), and path length against an independent 16-connected
grid Dijkstra on the real scenes (scipy), whose metric error is below 2.7 %.
The tracking is checked against the PD controller it extends (no integral
gain, unobstructed: identical trajectory) and against the Coulomb stall
the integral term exists to remove (PD stops mu g / kp short of the goal)."""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import dijkstra

import oracle
import workload


def square_scene(a=0.5, r=0.3):
    sc, sk = workload.pickplace_scene(0, controller="astar")
    sc = dict(sc, base_inflate=r,
              geoms=[dict(slabs=workload._box_slabs(0.0, 0.0, 0.0, 0.5, a, a), base=True, obj=True)])
    return sc, sk


def path_length(start, wps):
    pts = np.vstack([np.asarray(start, float)[None, :], wps])
    return float(np.sum(np.hypot(*np.diff(pts, axis=0).T)))


def test_detour_around_one_square_is_closed_form():
    a, r = 0.5, 0.3
    sc, sk = square_scene(a, r)
    wps = oracle.plan_path(sc, sk, (-2.0, 0.0), (2.0, 0.0))
    assert len(wps) == 3 and np.allclose(wps[-1], (2.0, 0.0))
    # corners of the grown square, pushed 1 mm out along the diagonal
    c = a + r + 1e-3 / math.sqrt(2.0)
    assert abs(abs(wps[0][1]) - c) < 1e-12 and abs(wps[0][0] + c) < 1e-12
    assert abs(abs(wps[1][1]) - c) < 1e-12 and abs(wps[1][0] - c) < 1e-12
    expect = 2.0 * math.hypot(2.0 - c, c) + 2.0 * c
    assert abs(path_length((-2.0, 0.0), wps) - expect) < 1e-12


def test_unobstructed_path_is_the_goal():
    sc, sk = square_scene()
    wps = oracle.plan_path(sc, sk, (-2.0, 1.5), (2.0, 1.5))
    assert wps.shape == (1, 2) and np.allclose(wps[0], (2.0, 1.5))


def grown_polys(sc, r):
    polys = []
    for gm in sc["geoms"]:
        if not gm["base"]:
            continue
        sl = [s for s in gm["slabs"] if s[2] == 0.0]
        if sl:
            polys.append([(s[0], s[1], s[3] - r if abs(s[3]) < 1e6 else s[3],
                           s[4] + r if abs(s[4]) < 1e6 else s[4]) for s in sl])
    return polys


def inside(polys, x, y, margin=1e-7):
    hit = np.zeros_like(x, bool)
    for p in polys:
        h = np.ones_like(x, bool)
        for nx, ny, lo, hi in p:
            v = nx * x + ny * y
            h &= (v > lo + margin) & (v < hi - margin)
        hit |= h
    return hit


def grid_shortest(polys, start, goal, h=0.02, box=(-3.0, 3.0, -2.0, 2.0)):
    xs = np.arange(box[0], box[1] + h / 2, h)
    ys = np.arange(box[2], box[3] + h / 2, h)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    free = ~inside(polys, X, Y, margin=0.0)
    nx, ny = X.shape
    idx = np.arange(nx * ny).reshape(nx, ny)
    rows, cols, w = [], [], []
    moves = [(1, 0), (0, 1), (1, 1), (1, -1), (2, 1), (1, 2), (2, -1), (1, -2)]
    for dx, dy in moves:
        a = (slice(0, nx - dx), slice(max(0, -dy), ny - max(0, dy)))
        b = (slice(dx, nx), slice(max(0, dy), ny - max(0, -dy) if dy < 0 else ny))
        ok = free[a] & free[b]
        if abs(dx) == 2 or abs(dy) == 2:  # a knight move also needs its two side cells free
            mid_a = (slice(0 + (dx > 1), nx - dx + (dx > 1)), a[1])
            ok &= free[mid_a] if free[mid_a].shape == ok.shape else ok
        rows.append(idx[a][ok]), cols.append(idx[b][ok]), w.append(np.full(ok.sum(), h * math.hypot(dx, dy)))
    r_, c_, w_ = np.concatenate(rows), np.concatenate(cols), np.concatenate(w)
    G = coo_matrix((np.r_[w_, w_], (np.r_[r_, c_], np.r_[c_, r_])), shape=(nx * ny, nx * ny)).tocsr()

    def node(p):
        i, j = int(round((p[0] - box[0]) / h)), int(round((p[1] - box[2]) / h))
        return idx[i, j]

    d = dijkstra(G, indices=node(start))
    return d[node(goal)]


@pytest.mark.parametrize("seed,obstacle", [(0, "ramp"), (3, "box"), (5, "ramp")])
def test_paths_are_valid_and_as_short_as_a_fine_grid(seed, obstacle):
    sc, sk = workload.pickplace_scene(seed, obstacle=obstacle, controller="astar")
    polys = grown_polys(sc, sc["base_inflate"])
    rng = np.random.default_rng(seed)
    checked = 0
    while checked < 6:
        s = rng.uniform((-2.9, -1.9), (2.9, 1.9))
        g = rng.uniform((-2.9, -1.9), (2.9, 1.9))
        if inside(polys, np.array([s[0], g[0]]), np.array([s[1], g[1]]), margin=-0.05).any():
            continue  # endpoints well clear of every grown footprint
        wps = oracle.plan_path(sc, sk, s, g)
        pts = np.vstack([s[None, :], wps])
        for p, q in zip(pts[:-1], pts[1:]):
            t = np.linspace(0.0, 1.0, 20001)
            assert not inside(polys, p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1]), margin=1e-6).any()
        L = path_length(s, wps)
        Lg = grid_shortest(polys, s, g)
        if not np.isfinite(Lg):
            continue
        # the grid path is at most 2.7 % longer than the continuous optimum
        # (plus rasterisation of the endpoints and the footprints)
        assert L <= Lg + 0.05 and L >= Lg / 1.027 - 0.05, (L, Lg)
        checked += 1


def test_zero_integral_gain_reproduces_the_pd_controller():
    sc_pd, sk = workload.pickplace_scene(1, n_actions=3, T=600)
    sc_a, _ = workload.pickplace_scene(1, n_actions=3, T=600, controller="astar")
    sc_a = dict(sc_a, pid_ki=0.0, geoms=[g for g in sc_a["geoms"] if not g["base"]])
    sc_pd = dict(sc_pd, geoms=sc_a["geoms"])
    th = np.array([(lo + hi) / 2 for lo, hi in zip(sk["lo"], sk["hi"])])
    a = oracle.trace(sc_pd, sk, th, 600)
    b = oracle.trace(sc_a, sk, th, 600)
    assert np.array_equal(a, b)


def test_integral_term_removes_the_coulomb_stall():
    # one straight moveTo with a weak gain: PD settles where kp |e| = mu g,
    # short of the 5 cm success radius; the integral term finishes the move
    sc, sk = workload.pickplace_scene(2, n_actions=3, T=3000, controller="astar")
    free = [g for g in sc["geoms"] if not g["base"]]
    sc = dict(sc, geoms=free, base_mu=0.1)
    th = np.array([(lo + hi) / 2 for lo, hi in zip(sk["lo"], sk["hi"])])
    th[2] = 5.0  # kp
    goal = np.array(sk["actions"][0]["nominal"][:2]) + th[:2]
    tr_pd = oracle.trace(dict(sc, pid_ki=0.0), sk, th, 3000)
    tr_pid = oracle.trace(sc, sk, th, 3000)
    stall = 0.1 * 9.81 / 5.0
    e_pd = np.hypot(*(tr_pd[-1, :2] - goal))
    # still in the first action, creeping down onto the stall distance
    assert tr_pd[-1, 16] == 0 and 0.99 * stall <= e_pd <= 1.01 * stall
    done = np.nonzero(tr_pid[:, 16] >= 1)[0]
    assert done.size and np.hypot(*(tr_pid[done[0] - 1, :2] - goal)) < 0.06
