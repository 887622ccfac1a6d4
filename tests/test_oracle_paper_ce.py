"""Pins of the oracle's paper-faithful CE variant (Sec. III-B, IV-A): the
n_env schedule, uniform initial sampling inside the parameter regions
(boxes and annuli), and the loop that starts from those samples.

Each pin checks the oracle against something it does not compute itself:
the schedule's closed form, the distribution of a uniform point in an
annulus (radial CDF (rho^2 - r^2) / (R^2 - r^2), uniform angle), box
marginals, the raw Philox words (pinned by the published KAT), and a
quadratic cost whose elites a test can rank with numpy."""
import math

import numpy as np
import pytest

import oracle
import workload


def ks_stat(x, cdf):
    """One-sample Kolmogorov-Smirnov statistic of x against cdf."""
    x = np.sort(np.asarray(x))
    n = len(x)
    F = cdf(x)
    return max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(n) / n))


KS99 = 1.63  # 99 % critical value of sqrt(n) * D_n


def test_schedule_closed_form():
    # 3000 -> 300 linearly by iteration 10, constant afterwards (Sec. IV-A)
    for j in range(25):
        assert oracle.n_env(3000, 300, 10, j) == 3000 - 270 * min(j, 10)
    # rounding to the nearest integer, and growing schedules
    assert [oracle.n_env(10, 0, 4, j) for j in range(6)] == [10, 8, 5, 3, 0, 0]  # 7.5 -> 8, 2.5 -> 3
    assert [oracle.n_env(100, 400, 3, j) for j in range(5)] == [100, 200, 300, 400, 400]
    assert oracle.n_env(500, 50, 0, 0) == 500 and oracle.n_env(500, 50, 0, 3) == 50


def paper_skeleton():
    sc, sk = workload.pickplace_scene(0, regions="paper")
    return sc, sk


def test_annulus_samples_are_area_uniform():
    sc, sk = paper_skeleton()
    N = 20000
    th = oracle.sample_uniform(sc, sk, 11, 3, N)
    off = 0
    width = {"move": 3, "grasp": 2, "place": 3}
    rings = 0
    for a in sk["actions"]:
        reg = a.get("region")
        if reg is not None:
            rings += 1
            px = a["nominal"][0] + th[:, off] - reg["center"][0]
            py = a["nominal"][1] + th[:, off + 1] - reg["center"][1]
            rho = np.hypot(px, py)
            ri, ro = reg["radii"]
            assert rho.min() >= ri - 1e-12 and rho.max() <= ro + 1e-12
            d = ks_stat(rho, lambda s: (s * s - ri * ri) / (ro * ro - ri * ri))
            assert d * math.sqrt(N) < KS99
            ang = np.arctan2(py, px)
            d = ks_stat(ang, lambda t: (t + math.pi) / (2 * math.pi))
            assert d * math.sqrt(N) < KS99
            # the annulus lies inside the bounds, so clamping never moves a draw
            assert np.all(th[:, off] >= sk["lo"][off]) and np.all(th[:, off] <= sk["hi"][off])
            assert np.all(th[:, off + 1] >= sk["lo"][off + 1]) and np.all(th[:, off + 1] <= sk["hi"][off + 1])
        off += width[a["kind"]]
    assert rings == 2


def test_box_parameters_are_uniform_and_use_their_philox_word():
    sc, sk = paper_skeleton()
    N = 5000
    th = oracle.sample_uniform(sc, sk, 5, 1, N)
    w = oracle.philox_words(5, 0xFFFFFFFF, 1, N, len(sk["lo"]))
    ring_dims = {0, 1, 5, 6}
    for d in range(len(sk["lo"])):
        if d in ring_dims:
            continue
        lo, hi = sk["lo"][d], sk["hi"][d]
        u = (w[:, d].astype(np.float64) + 1.0) * 2.0 ** -32
        np.testing.assert_allclose(th[:, d], lo + u * (hi - lo), rtol=0, atol=1e-12 * max(1.0, abs(hi)))
        d_ks = ks_stat(th[:, d], lambda x: (x - lo) / (hi - lo))
        assert d_ks * math.sqrt(N) < KS99


def test_disc_is_the_annulus_with_zero_inner_radius():
    sc, sk = workload.reach_scene(0)
    sk = dict(sk)
    a = dict(sk["actions"][0])
    a["region"] = dict(kind="ring", center=(a["nominal"][0], a["nominal"][1]), radii=(0.0, 0.2))
    sk["actions"] = [a]
    N = 20000
    th = oracle.sample_uniform(sc, sk, 2, 0, N)
    rho = np.hypot(th[:, 0], th[:, 1])
    assert rho.max() <= 0.2 + 1e-12
    # uniform in the disc: E[rho^2] = R^2 / 2, P(rho <= R / 2) = 1/4
    assert abs(np.mean(rho ** 2) - 0.02) < 4 * 0.2 ** 2 / math.sqrt(12 * N)
    assert ks_stat(rho, lambda s: (s / 0.2) ** 2) * math.sqrt(N) < KS99
    # a point read straight from the words: rho = R sqrt(u_0), angle 2 pi u_1
    w = oracle.philox_words(2, 0xFFFFFFFF, 0, 3, 3)
    u0 = (w[:, 0].astype(np.float64) + 1.0) * 2.0 ** -32
    u1 = (w[:, 1].astype(np.float64) + 1.0) * 2.0 ** -32
    np.testing.assert_allclose(th[:3, 0], 0.2 * np.sqrt(u0) * np.cos(2 * math.pi * u1), atol=1e-12)
    np.testing.assert_allclose(th[:3, 1], 0.2 * np.sqrt(u0) * np.sin(2 * math.pi * u1), atol=1e-12)


def test_first_iteration_refits_from_the_uniform_samples():
    sc, sk = workload.quadratic_scene(4, D=5)
    n0, K = 800, 40
    r = oracle.cem_paper(sc, sk, 9, n0=n0, n1=100, j1=3, K=K, iters=1, diag=True)
    th = oracle.sample_uniform(sc, sk, 9, 0, n0)
    D = len(sk["lo"])
    A = np.array(sc["A"]).reshape(D, D)
    e = th - np.array(sc["theta_star"])
    J = np.einsum("ni,ij,nj->n", e, A, e).astype(np.float32)
    elite = np.lexsort((np.arange(n0), J))[:K]
    np.testing.assert_allclose(r["mean"], th[elite].mean(0), rtol=0, atol=1e-12)
    assert r["n_env"][0] == n0 and r["class_counts"][0].tolist() == [n0, 0, 0, 0]
    assert r["best_J"] == pytest.approx(float(np.einsum("i,ij,j->", e[elite[0]], A, e[elite[0]])), rel=1e-9)
    # the normal model is independent per parameter (Sec. IV-A)
    assert np.count_nonzero(r["cov"] - np.diag(np.diag(r["cov"]))) == 0


def test_paper_loop_converges_on_a_quadratic():
    sc, sk = workload.quadratic_scene(1, D=8)
    r = oracle.cem_paper(sc, sk, 3, n0=2000, n1=300, j1=10, K=50, iters=20, diag=True)
    assert r["n_env"].tolist() == [oracle.n_env(2000, 300, 10, j) for j in range(20)]
    assert np.all(r["class_counts"].sum(1) == r["n_env"])
    assert np.all(np.diff(r["history"]) <= 0)
    assert np.abs(r["mean"] - np.array(sc["theta_star"])).max() < 5e-3


def test_paper_loop_counts_classes_on_pick_place():
    sc, sk = workload.pickplace_scene(1, regions="paper", T=300)
    r = oracle.cem_paper(sc, sk, 2, n0=96, n1=32, j1=2, K=8, iters=3)
    assert r["n_env"].tolist() == [96, 64, 32]
    assert np.all(r["class_counts"].sum(1) == r["n_env"])
    assert np.all(r["class_counts"] >= 0)
    assert r["best_cls"] <= 2 and np.isfinite(r["best_J"])
