"""Pins of the oracle's domain randomisation (Sec. IV-C: plans made robust
to bounded uncertainty in friction or mass).

The factors are checked against the raw Philox words (pinned by the
published known-answer vectors); a randomised rollout against plain
rollouts of scene dictionaries scaled here in Python (every friction
coefficient by s_mu, the manipulated body's mass by s_m), averaged and
worst-classed here; and the degenerate settings (no spread, one
environment) against the plain rollout and CE loop bit for bit."""
import numpy as np
import pytest

import oracle
import workload


def factors_from_words(seed, it, problem, M, dmu, dm):
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    smu, sm = [], []
    for m in range(M):
        r = oracle.philox(np.array([m, 256, it, problem], np.uint32), key)
        u0 = (float(r[0]) + 1.0) * 2.0 ** -32
        u1 = (float(r[1]) + 1.0) * 2.0 ** -32
        smu.append(1.0 + dmu * (2.0 * u0 - 1.0))
        sm.append(1.0 + dm * (2.0 * u1 - 1.0))
    return np.array(smu), np.array(sm)


@pytest.mark.parametrize("seed,it,problem", [(0, 0, 0), (12345678901234, 7, 3), (2 ** 64 - 1, 0xFFFF, 9)])
def test_factors_come_from_their_philox_block(seed, it, problem):
    smu, sm = oracle.dr_factors(seed, it, problem, 8, 0.3, 0.2)
    esmu, esm = factors_from_words(seed, it, problem, 8, 0.3, 0.2)
    np.testing.assert_allclose(smu, esmu, rtol=0, atol=1e-15)
    np.testing.assert_allclose(sm, esm, rtol=0, atol=1e-15)
    assert np.all(np.abs(smu - 1) <= 0.3) and np.all(np.abs(sm - 1) <= 0.2)
    z_mu, z_m = oracle.dr_factors(seed, it, problem, 8, 0.0, 0.0)
    assert np.all(z_mu == 1.0) and np.all(z_m == 1.0)


def scaled(scene, smu, sm):
    e = dict(scene)
    for k in ("base_mu", "block_mu", "contact_mu", "obj_mu"):
        if k in e:
            e[k] = e[k] * smu
    for k in ("block_mass", "obj_mass"):
        if k in e:
            e[k] = e[k] * sm
    return e


@pytest.mark.parametrize("task", ["push", "pickplace", "reach"])
def test_randomised_cost_is_the_mean_and_worst_class(task):
    if task == "push":
        sc, sk = workload.push_scene(3, T=600)
    elif task == "pickplace":
        sc, sk = workload.pickplace_scene(2, T=500)
    else:
        sc, sk = workload.reach_scene(1)
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    rng = np.random.default_rng(4)
    th = rng.uniform(lo, hi, (40, len(lo)))
    M, dmu, dm = 4, 0.9, 0.5
    J, cls = oracle.rollout_dr(sc, sk, th, M, dmu, dm, seed=11, it=2, problem=1)
    smu, sm = factors_from_words(11, 2, 1, M, dmu, dm)
    Js, cs = [], []
    for m in range(M):
        j, c = oracle.rollout(scaled(sc, smu[m], sm[m]), sk, th)
        Js.append(j)
        cs.append(c)
    Js, cs = np.array(Js), np.array(cs)
    np.testing.assert_allclose(J, Js.mean(0), rtol=1e-13, atol=1e-13)
    assert np.array_equal(cls, cs.max(0))
    if task == "push":  # friction spread this wide changes some samples' outcome
        assert np.any(cs.min(0) != cs.max(0)) or np.any(np.ptp(Js, 0) > 1e-6)


def test_no_spread_equals_the_plain_rollout():
    sc, sk = workload.push_scene(1, T=400)
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    th = np.random.default_rng(0).uniform(lo, hi, (25, len(lo)))
    J0, c0 = oracle.rollout(sc, sk, th)
    for M in (1, 4):
        J, c = oracle.rollout_dr(sc, sk, th, M, 0.0, 0.0, seed=5)
        assert np.array_equal(J, J0) and np.array_equal(c, c0)


def test_loop_without_spread_equals_plain_cem():
    sc, sk = workload.reach_scene(0)
    a = oracle.cem(sc, sk, 3, 128, 12, 4)
    b = oracle.cem_dr(sc, sk, 3, 128, 12, 4, M=2, dmu=0.0, dm=0.0, dr_seed=77)
    assert a["best_J"] == b["best_J"] and a["best_cls"] == b["best_cls"]
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["history"], b["history"])
