"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Bars: Philox words and elite indices bit-exact; per-step state within
1e-5 relative over 50 steps (denominator max(|x|, 1e-3)); rollout cost
within 1e-3 relative for the contact-free task at full horizon and for
the contact tasks at a 200-step horizon.  Samples whose FP64 cost moves by
more than 1e-3 relative when theta moves by 1e-6 of its range are
"borderline" (a discrete event sits within rounding of the sample): they
are excluded from the 1e-3 check and their rate must stay below 1%.
"""
import math

import numpy as np
import pytest

import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    return P


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def init_dist(skel):
    lo, hi = np.array(skel["lo"]), np.array(skel["hi"])
    return (lo + hi) / 2, np.diag((hi - lo) / 4)


def draw(P, sc, skel, N, seed=1, it=0, spread=1.0):
    """theta from the GPU sampler at the initial distribution (float32)."""
    mean, chol = init_dist(skel)
    with P.Scene(sc, skel) as S:
        th = S.sample(dev(mean), dev(chol * spread), seed, it, N)
    torch.cuda.synchronize()
    return th.cpu().numpy()


def rel(a, b, floor):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def borderline(orc, sc, skel, th, J0, T, idx, tol=1e-3, reps=8, seed=0):
    rng = np.random.default_rng(seed)
    rngs = (np.array(skel["hi"]) - np.array(skel["lo"]))
    out = []
    for i in idx:
        bl = False
        for _ in range(reps):
            u = rng.standard_normal(len(rngs))
            u /= np.linalg.norm(u)
            Jp, _ = orc.rollout(sc, skel, (th[i] + 1e-6 * rngs * u)[None], T=T)
            if abs(Jp[0] - J0[i]) / max(abs(J0[i]), 1e-3) > tol:
                bl = True
                break
        out.append(bl)
    return np.array(out, bool)


# ------------------------------------------------------------------ sampling
@pytest.mark.parametrize("D,N", [(3, 1), (6, 777), (14, 4096), (18, 65536)])
def test_philox_words_bit_exact(P, orc, D, N):
    sc, sk = workload.quadratic_scene(0, D=D)
    with P.Scene(sc, sk) as S:
        for seed, it, prob in ((0, 0, 0), (0xDEADBEEF12345678, 17, 63)):
            w = S.philox_words(seed, it, N, problem=prob)
            torch.cuda.synchronize()
            got = w.cpu().numpy().view(np.uint32)
            ref = orc.philox_words(seed, it, prob, N, D)
            assert np.array_equal(got, ref)


@pytest.mark.parametrize("D,N", [(3, 256), (14, 1000), (18, 4097)])
def test_sample_matches_oracle(P, orc, D, N):
    rng = np.random.default_rng(D)
    B = rng.standard_normal((D, D)) * 0.3
    cov = B @ B.T + 0.2 * np.eye(D)
    L = np.linalg.cholesky(cov).astype(np.float32)
    mean = rng.standard_normal(D).astype(np.float32)
    sc, sk = workload.quadratic_scene(0, D=D)
    with P.Scene(sc, sk) as S:
        th = S.sample(dev(mean), dev(L), 99, 5, N, problem=2)
    torch.cuda.synchronize()
    ref = orc.sample(99, 5, 2, N, mean.astype(np.float64), L.astype(np.float64))
    assert np.max(np.abs(th.cpu().numpy() - ref)) < 2e-5 * (1 + np.abs(ref).max())


def test_sample_empty_is_noop(P):
    sc, sk = workload.quadratic_scene(0, D=4)
    with P.Scene(sc, sk) as S:
        th = torch.full((1, 4), 7.0, device="cuda")
        P.cem_sample(S.h, dev(np.zeros(4)), dev(np.eye(4)), 1, 0, 0, 0, th)
        torch.cuda.synchronize()
        assert torch.all(th == 7.0)


def test_host_pointer_rejected(P):
    sc, sk = workload.quadratic_scene(0, D=4)
    import ctypes as C

    with P.Scene(sc, sk) as S:
        host = np.zeros(16, np.float32)
        rc = P.load().cem_sample(S.h, C.c_void_p(host.ctypes.data), C.c_void_p(host.ctypes.data), 1, 0, 0, 4,
                                 C.c_void_p(host.ctypes.data), None)
        assert rc == -1


# ---------------------------------------------------------- rollout: state
# Contact-free motion must hold 1e-5 relative per step.  A body in penalty
# contact feels k * depth with depth the difference of two O(1) FP32
# positions: one position quantum ulp(|x|) is a force error k ulp and a
# velocity error k ulp dt / m per step.  For those bodies the velocity
# columns (and the positions they integrate) are held to that bound,
# accumulated over the steps taken; everything else keeps the 1e-5 bar.
def quantum_bound(k_c, dt, m, xmax, lever, steps):
    ulp = np.spacing(np.float32(xmax)).astype(np.float64)
    dv = k_c * dt * ulp / m  # per step
    k = np.arange(1, steps + 1)[:, None]
    v = k * dv
    x = dt * k * (k + 1) / 2 * dv
    return v, x, v / lever


def state_tolerance(name, sc, ref, steps):
    tol = 1e-5 * np.maximum(np.abs(ref), 1e-3)
    if name == "push-contact":
        m = min(sc["base_mass"], sc["block_mass"])
        v, x, w = quantum_bound(sc["k_contact"], sc["dt"], m, 4.0, min(sc["block_half"]), steps)
        for cols, b in (((0, 1, 6, 7), x), ((3, 4, 9, 10), v), ((5, 11), w), ((2, 8), x / min(sc["block_half"]))):
            for c in cols:
                tol[:, c] = np.maximum(tol[:, c], b[:, 0])
    if name == "pickplace":  # the object rests on table 1 in penalty contact
        v, x, _ = quantum_bound(sc["k_contact"], sc["dt"], sc["obj_mass"], 2.0, 1.0, steps)
        for c in (9, 10, 11):
            tol[:, c] = np.maximum(tol[:, c], x[:, 0])
        for c in (12, 13, 14):
            tol[:, c] = np.maximum(tol[:, c], v[:, 0])
    return tol


TRACE_CASES = [
    ("reach", lambda: workload.reach_scene(0)),
    ("push", lambda: workload.push_scene(3)),
    ("push-contact", lambda: workload.push_scene(4, start_in_contact=True)),
    ("pickplace", lambda: workload.pickplace_scene(5)),
]


@pytest.mark.parametrize("name,make", TRACE_CASES, ids=[c[0] for c in TRACE_CASES])
def test_per_step_state_50_steps(P, orc, name, make):
    sc, sk = make()
    th = draw(P, sc, sk, 64, seed=11)
    with P.Scene(sc, sk) as S:
        st = S.trace(dev(th), 50)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    worst = 0.0
    for i in range(th.shape[0]):
        ref = orc.trace(sc, sk, th[i].astype(np.float64), 50)
        if name in ("reach", "push"):  # contact-free: the block never moves
            assert np.all(ref[:, 9:12] == 0.0)
        ratio = np.abs(st[i] - ref) / state_tolerance(name, sc, ref, 50)
        worst = max(worst, ratio.max())
    assert worst <= 1.0, worst


# ----------------------------------------------------------- rollout: cost
def cost_parity(P, orc, sc, sk, th, T, tol=1e-3):
    with P.Scene(sc, sk, T=T) as S:
        J, cls = S.rollout(dev(th))
    torch.cuda.synchronize()
    J, cls = J.cpu().numpy(), cls.cpu().numpy()
    Jr, cr = orc.rollout(sc, sk, th.astype(np.float64), T=T)
    r = rel(J, Jr, 1e-3)
    bad = np.where((r > tol) | (cls != cr))[0]
    bl = borderline(orc, sc, sk, th.astype(np.float64), Jr, T, bad)
    hard = bad[~bl]
    assert len(hard) == 0, (hard[:10], J[hard[:10]], Jr[hard[:10]], cls[hard[:10]], cr[hard[:10]])
    assert bl.sum() <= 0.01 * len(th), bl.sum()
    return J, cls, Jr, cr


def test_reach_cost_full_horizon(P, orc):
    sc, sk = workload.reach_scene(0)
    th = draw(P, sc, sk, 1000, seed=3)
    J, cls, Jr, cr = cost_parity(P, orc, sc, sk, th, sc["T"])
    assert (cls == 0).sum() > 0 and (cls == 2).sum() > 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_push_cost_200_steps(P, orc, seed):
    sc, sk = workload.push_scene(seed)
    th = draw(P, sc, sk, 1000, seed=seed)
    cost_parity(P, orc, sc, sk, th, 200)


def test_push_contact_start_cost_200_steps(P, orc):
    sc, sk = workload.push_scene(7, start_in_contact=True)
    th = draw(P, sc, sk, 1000, seed=7)
    cost_parity(P, orc, sc, sk, th, 200)


@pytest.mark.parametrize("seed", [0, 1])
def test_pickplace_cost_200_steps(P, orc, seed):
    sc, sk = workload.pickplace_scene(seed)
    th = draw(P, sc, sk, 512, seed=seed)
    cost_parity(P, orc, sc, sk, th, 200)


def test_quadratic_cost(P, orc):
    sc, sk = workload.quadratic_scene(2, D=9)
    th = draw(P, sc, sk, 3000, seed=2, spread=2.0)
    with P.Scene(sc, sk) as S:
        J, cls = S.rollout(dev(th))
    Jr, cr = orc.rollout(sc, sk, th.astype(np.float64))
    assert np.all(cls.cpu().numpy() == 0)
    assert np.max(rel(J.cpu().numpy(), Jr, 1e-3)) < 1e-5


@pytest.mark.parametrize("N", [1, 31, 33, 1000])
def test_ragged_batches(P, orc, N):
    sc, sk = workload.reach_scene(0)
    th = draw(P, sc, sk, N, seed=N)
    cost_parity(P, orc, sc, sk, th, sc["T"])


def test_full_size_push_sampled(P, orc):
    # the bench workload (N = 4096, T = 1000) in its launch shape; the first
    # 200 steps of 64 sampled rollouts are compared one by one
    sc, sk, cm = workload.config(1, seed=0)
    th = draw(P, sc, sk, cm["N"], seed=5)
    with P.Scene(sc, sk) as S:
        J, cls = S.rollout(dev(th))
    torch.cuda.synchronize()
    J, cls = J.cpu().numpy(), cls.cpu().numpy()
    assert np.all(np.isfinite(J)) and np.all(cls <= 2)
    pick = np.random.default_rng(0).choice(cm["N"], 64, replace=False)
    cost_parity(P, orc, sc, sk, th[pick], 200)
    # at full horizon the discrete events may legitimately diverge: most agree
    Jr, cr = orc.rollout(sc, sk, th[pick].astype(np.float64))
    agree = (rel(J[pick], Jr, 1e-3) <= 1e-3) & (cls[pick] == cr)
    assert agree.mean() >= 0.9


def test_full_size_pickplace_sampled(P, orc):
    sc, sk, cm = workload.config(2, seed=0)
    th = draw(P, sc, sk, cm["N"], seed=6)
    with P.Scene(sc, sk) as S:
        J, cls = S.rollout(dev(th))
    torch.cuda.synchronize()
    J, cls = J.cpu().numpy(), cls.cpu().numpy()
    assert np.all(np.isfinite(J)) and np.all(cls <= 2)
    pick = np.random.default_rng(1).choice(cm["N"], 32, replace=False)
    cost_parity(P, orc, sc, sk, th[pick], 200)


# ------------------------------------------------------- select and refit
def refit_case(P, orc, J, cls, theta, K, lo, hi, diag=False):
    N, D = theta.shape
    sc, sk = workload.quadratic_scene(0, D=D)
    sk = dict(sk, lo=list(lo), hi=list(hi))
    m0 = np.arange(D, dtype=np.float32)
    c0 = np.eye(D, dtype=np.float32) * 2
    mean, cov, chol = dev(m0), dev(c0), dev(np.sqrt(c0))
    with P.Scene(sc, sk) as S:
        idx, keff = S.refit(dev(theta), dev(J), dev(cls, torch.uint8), K, mean, cov, chol,
                            cov_mode="diag" if diag else "full")
    torch.cuda.synchronize()
    k = int(keff.item())
    ref_idx = orc.select(J, cls, K)
    assert k == len(ref_idx)
    assert np.array_equal(idx.cpu().numpy()[:k], ref_idx)
    rc, rm, rcov, rch = orc.refit(theta.astype(np.float64), ref_idx, lo, hi, diag=diag,
                                  mean=m0.astype(np.float64), cov=c0.astype(np.float64),
                                  chol=np.sqrt(c0).astype(np.float64))
    assert rc == 0
    for got, ref in ((mean, rm), (cov, rcov), (chol, rch)):
        g = got.cpu().numpy().reshape(ref.shape)
        assert np.max(np.abs(g - ref)) <= 1e-6 * max(1.0, np.abs(ref).max())
    return k


@pytest.mark.parametrize("N,K,D", [(64, 8, 3), (1000, 50, 6), (4096, 200, 6), (5003, 300, 7), (16384, 512, 14),
                                   (65536, 1024, 18), (100, 300, 5)])
def test_select_refit_matches_oracle(P, orc, N, K, D):
    rng = np.random.default_rng(N + K)
    theta = (rng.standard_normal((N, D)) * rng.uniform(0.2, 3, D)).astype(np.float32)
    J = rng.choice(np.linspace(0.5, 9, 37).astype(np.float32), N)  # heavy ties
    cls = rng.choice(4, N, p=[0.1, 0.2, 0.6, 0.1]).astype(np.uint8)
    J[cls == 3] = np.nan
    lo, hi = -np.ones(D) * 4, np.ones(D) * 6
    k = refit_case(P, orc, J, cls, theta, K, lo, hi)
    assert k == min(K, int((cls == 0).sum()))
    refit_case(P, orc, J, cls, theta, K, lo, hi, diag=True)


def test_refit_rules(P, orc):
    rng = np.random.default_rng(5)
    N, D = 500, 4
    theta = rng.standard_normal((N, D)).astype(np.float32)
    lo, hi = -np.ones(D), np.ones(D) * 3
    J = rng.uniform(0, 5, N).astype(np.float32)
    # only class 1 and 2 present: class 1 is ranked (the fallback set)
    cls = np.full(N, 2, np.uint8)
    cls[[7, 70, 300]] = 1
    assert refit_case(P, orc, J, cls, theta, 50, lo, hi) == 3
    # a single feasible sample: artificial noise around it
    cls = np.full(N, 2, np.uint8)
    cls[123] = 0
    assert refit_case(P, orc, J, cls, theta, 50, lo, hi) == 1
    # nothing but class 2: the K best class-2 samples
    cls = np.full(N, 2, np.uint8)
    assert refit_case(P, orc, J, cls, theta, 50, lo, hi) == 50
    # every cost non-finite: no elites, distribution kept
    Jn = np.full(N, np.inf, np.float32)
    assert refit_case(P, orc, Jn, cls, theta, 50, lo, hi) == 0
    # rank-deficient elites (K_eff <= D): the ridge keeps it PD
    cls = np.full(N, 2, np.uint8)
    cls[[1, 2, 3]] = 0
    assert refit_case(P, orc, J, cls, theta, 50, lo, hi) == 3
    # empty batch
    assert refit_case(P, orc, J[:0], cls[:0], theta[:0], 10, lo, hi) == 0


# ------------------------------------------------------------ the CE loop
def test_solve_graph_equals_eager(P):
    sc, sk, cm = workload.config(0, seed=0)
    with P.Scene(sc, sk) as S:
        a = S.solve(3, cm["N"], cm["K"], cm["iters"], use_graph=True)
        b = S.solve(3, cm["N"], cm["K"], cm["iters"], use_graph=False)
    assert a["best_J"] == b["best_J"]
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["history"], b["history"])


def test_solve_quadratic_reaches_minimiser(P):
    for seed in range(3):
        sc, sk = workload.quadratic_scene(seed, D=6)
        with P.Scene(sc, sk) as S:
            r = S.solve(seed, 512, 50, 30)
        assert np.linalg.norm(r["mean"] - np.array(sc["theta_star"])) < 2e-3
        assert r["best_cls"] == 0 and r["best_J"] < 1e-4


# Converged CE settings per workload: the full reach and move-and-push
# settings; pick-place at N = 2048, K = 128, 10 iterations (the full 16384
# samples x 25 iterations x 8 seeds would keep the FP64 oracle busy for
# minutes; the CE rules, the rollout and the refit are the same).
CE_CASES = {0: dict(N=256, K=25, iters=10), 1: dict(N=4096, K=200, iters=20), 2: dict(N=2048, K=128, iters=10)}


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_converged_cost_matches_oracle_cem(P, orc, cfg):
    """Converged CE cost against the FP64 oracle's CE over 8 seeds (each seed
    its own scene): the mean best cost over the 8 seeds within 2 % of the
    oracle's, and seed by seed at least 6 of 8 within 2 % with the same
    feasibility class.  CE on a multimodal cost can settle in another mode
    once FP32 rounding changes one early elite set (the paper reports such
    per-seed mode spread, Sec. IV-B), hence 6 of 8 per seed."""
    cm = CE_CASES[cfg]
    gpu, ref, cls_g, cls_r = [], [], [], []
    for seed in range(8):
        sc, sk, _ = workload.config(cfg, seed=seed)
        with P.Scene(sc, sk) as S:
            r = S.solve(seed, cm["N"], cm["K"], cm["iters"])
        o = orc.cem(sc, sk, seed, cm["N"], cm["K"], cm["iters"])
        gpu.append(r["best_J"])
        ref.append(o["best_J"])
        cls_g.append(r["best_cls"])
        cls_r.append(o["best_cls"])
    gpu, ref = np.array(gpu), np.array(ref)
    assert abs(gpu.mean() - ref.mean()) <= 0.02 * ref.mean(), (gpu, ref)
    close = np.abs(gpu - ref) / ref <= 0.02
    assert close.sum() >= 6, (gpu, ref)
    assert np.all(np.array(cls_g)[close] == np.array(cls_r)[close])


# ---------------------------------------------------------- robustness, state
@pytest.mark.parametrize("make", [lambda: workload.reach_scene(0), lambda: workload.push_scene(2),
                                  lambda: workload.pickplace_scene(1, T=400)])
def test_nan_parameters_give_class_3(P, orc, make):
    sc, sk = make()
    th = draw(P, sc, sk, 64, seed=4)
    D = th.shape[1]
    for i in range(0, 64, 4):
        th[i, i % D] = np.nan
    with P.Scene(sc, sk) as S:
        J, cls = S.rollout(dev(th))
    Jr, cr = orc.rollout(sc, sk, th.astype(np.float64))
    assert np.array_equal(cls.cpu().numpy(), cr)
    assert np.array_equal(np.isfinite(J.cpu().numpy()), np.isfinite(Jr))


def test_resume_reproduces_the_run(P):
    # the CE state is (mean, cov, chol, iteration): splitting a run at
    # iteration 4 and resuming from the returned state changes nothing
    sc, sk, cm = workload.config(1, seed=3)
    with P.Scene(sc, sk) as S:
        full = S.solve(9, cm["N"], cm["K"], 9)
        first = S.solve(9, cm["N"], cm["K"], 4)
        second = S.solve(9, cm["N"], cm["K"], 5, start_iter=4, init_mean=first["mean"], init_cov=first["cov"],
                         init_chol=first["chol"])
    assert np.array_equal(second["mean"], full["mean"])
    assert np.array_equal(second["cov"], full["cov"])
    assert np.array_equal(second["chol"], full["chol"])
    best = min((first["best_cls"], first["best_J"]), (second["best_cls"], second["best_J"]))
    assert best == (full["best_cls"], full["best_J"])
    assert np.array_equal(np.concatenate([first["history"], np.minimum(second["history"], first["best_J"])]),
                          full["history"]) or full["best_cls"] != 0


def test_autotune_and_cache(P, tmp_path):
    sc, sk, cm = workload.config(1, seed=0)
    cache = str(tmp_path / "tune.txt")
    with P.Scene(sc, sk) as S:
        b = S.autotune(cm["N"], cache)
        assert b in (2, 4, 8, 16, 32, 64, 128, 256)
        lines = open(cache).read().strip().splitlines()
        # "<key>|<block>|<lanes per rollout>"; push rollouts keep one lane
        assert len(lines) == 1 and lines[0].endswith("|%d|1" % b)
        assert S.autotune(cm["N"], cache) == b  # read back from the cache
        assert len(open(cache).read().strip().splitlines()) == 1
        r = S.solve(1, cm["N"], cm["K"], 2)
    assert np.isfinite(r["best_J"])


def test_binding_rejects_short_or_mistyped_buffers(P):
    """A buffer shorter than the call's sizes, or of another type, raises in
    the wrapper; no kernel sees it."""
    sc, sk, _ = workload.config(1)
    with P.Scene(sc, sk) as S:
        N, D = 64, S.D
        th = torch.zeros((N, D), device="cuda")
        J = torch.empty(N, device="cuda")
        cls = torch.empty(N, dtype=torch.uint8, device="cuda")
        mean, chol = torch.zeros(D, device="cuda"), torch.eye(D, device="cuda")
        with pytest.raises(ValueError, match="theta"):
            P.cem_rollout_batch(S.h, th[: N - 1], N, J, cls)
        with pytest.raises(ValueError, match="J"):
            P.cem_rollout_batch(S.h, th, N, J[: N - 1], cls)
        with pytest.raises(TypeError, match="cls"):
            P.cem_rollout_batch(S.h, th, N, J, cls.float())
        with pytest.raises(ValueError, match="chol"):
            P.cem_sample(S.h, mean, chol[:-1], 0, 0, 0, N, th)
        with pytest.raises(TypeError, match="mean"):
            P.cem_sample(S.h, mean.double(), chol, 0, 0, 0, N, th)
        with pytest.raises(ValueError, match="elite_idx"):
            P.cem_refit(S.h, th, J, cls, N, 8, 0, mean, chol @ chol.T, chol.clone(),
                        torch.empty(4, dtype=torch.int32, device="cuda"))
        # the same calls with the right buffers still run
        P.cem_sample(S.h, mean, chol, 0, 0, 0, N, th)
        P.cem_rollout_batch(S.h, th, N, J, cls)
        torch.cuda.synchronize()
        assert torch.isfinite(J).all()
