"""The A* base controller on the GPU (Sec. IV-A: A* paths tracked by a PID
controller) against the oracle.

The device planner (FP32 queries on a host-built FP64 corner graph) must
return the oracle's waypoints; rollouts that plan at every moveTo must match
the oracle per step and in cost at the plain parity tolerances, with the
same "borderline" exclusion (a discrete event within rounding of the
sample), both from the initial distribution (600 steps) and from a
converged one over the whole horizon (every action of the plan, each moveTo
planned from where the base stands), and lane groups must stay
bit-identical to one lane."""
import numpy as np
import pytest

import oracle
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def draw(P, sc, sk, N, seed):
    lo, hi = np.array(sk["lo"]), np.array(sk["hi"])
    with P.Scene(sc, sk) as S:
        th = S.sample(dev((lo + hi) / 2), dev(np.diag((hi - lo) / 4)), seed, 0, N)
    torch.cuda.synchronize()
    return th.cpu().numpy()


@pytest.mark.parametrize("seed,obstacle,regions", [(0, "ramp", "box"), (3, "box", "paper"), (6, "ramp", "paper")])
def test_device_planner_matches_oracle(P, seed, obstacle, regions):
    sc, sk = workload.pickplace_scene(seed, obstacle=obstacle, regions=regions, controller="astar")
    rng = np.random.default_rng(seed)
    same = 0
    n = 60
    with P.Scene(sc, sk) as S:
        for _ in range(n):
            s = rng.uniform((-2.9, -1.9), (2.9, 1.9))
            g = rng.uniform((-2.9, -1.9), (2.9, 1.9))
            a = S.base_path(s, g).astype(np.float64)
            b = oracle.plan_path(sc, sk, s.astype(np.float32).astype(np.float64),
                                 g.astype(np.float32).astype(np.float64))
            if a.shape == b.shape and np.abs(a - b).max() <= 1e-5:
                same += 1
    # equal-length alternatives and knife-edge visibility may differ in FP32
    assert same >= 0.95 * n, same


def test_per_step_base_and_arm_state(P):
    sc, sk = workload.pickplace_scene(5, controller="astar")
    th = draw(P, sc, sk, 64, seed=11)
    steps = 50
    with P.Scene(sc, sk) as S:
        st = S.trace(dev(th), steps).cpu().numpy()
    worst = 0.0
    for i in range(th.shape[0]):
        ref = oracle.trace(sc, sk, th[i].astype(np.float64), steps)
        cols = list(range(0, 9))  # base x, y, vx, vy, joints, joint rates, azimuth
        tol = 1e-5 * np.maximum(np.abs(ref[:, cols]), 1e-3)
        worst = max(worst, float((np.abs(st[i][:, cols] - ref[:, cols]) / tol).max()))
    assert worst <= 1.0, worst


def borderline(sc, sk, th, J0, T, idx, tol=1e-3, reps=8, seed=0):
    rng = np.random.default_rng(seed)
    rngs = np.array(sk["hi"]) - np.array(sk["lo"])
    out = []
    for i in idx:
        bl = False
        for _ in range(reps):
            u = rng.standard_normal(len(rngs))
            u /= np.linalg.norm(u)
            Jp, _ = oracle.rollout(sc, sk, (th[i] + 1e-6 * rngs * u)[None], T=T)
            if abs(Jp[0] - J0[i]) / max(abs(J0[i]), 1e-3) > tol:
                bl = True
                break
        out.append(bl)
    return np.array(out, bool)


@pytest.mark.parametrize("seed,regions", [(0, "box"), (2, "paper")])
def test_cost_parity_600_steps(P, seed, regions):
    sc, sk = workload.pickplace_scene(seed, regions=regions, controller="astar")
    th = draw(P, sc, sk, 256, seed=seed)
    T = 600
    with P.Scene(sc, sk, T=T) as S:
        J, cls = S.rollout(dev(th))
    J, cls = J.cpu().numpy(), cls.cpu().numpy()
    Jr, cr = oracle.rollout(sc, sk, th.astype(np.float64), T=T)
    r = np.abs(J - Jr) / np.maximum(np.abs(Jr), 1e-3)
    bad = np.where((r > 1e-3) | (cls != cr))[0]
    bl = borderline(sc, sk, th.astype(np.float64), Jr, T, bad)
    # a waypoint switch decided one step apart in FP32 and FP64 is a discrete
    # event the 1e-6 probe can miss; such a sample must still show an outcome
    # of the FP64 model close by (theta moved by 1e-6 or 1e-5 of its range)
    from pickplace_common import nearby_outcome

    rest = bad[~bl]
    near = nearby_outcome(lambda t: oracle.rollout(sc, sk, t, T=T), sk, th, rest, J, cls)
    hard = rest[~near]
    assert len(hard) == 0, (hard[:10], J[hard[:10]], Jr[hard[:10]])
    assert len(bad) - len(hard) <= 0.02 * len(th), len(bad)


def test_lane_groups_are_bit_identical_with_planning(P):
    sc, sk = workload.pickplace_scene(4, regions="paper", controller="astar")
    th = draw(P, sc, sk, 500, seed=4)
    out = []
    with P.Scene(sc, sk, T=1500) as S:
        for tpr in (1, 8, 32):
            S.set_threads_per_rollout(tpr)
            J, cls = S.rollout(dev(th))
            out.append((J.cpu().numpy(), cls.cpu().numpy()))
    for J, c in out[1:]:
        assert np.array_equal(J.view(np.uint32), out[0][0].view(np.uint32)) and np.array_equal(c, out[0][1])


def test_paper_loop_with_planner(P):
    sc, sk = workload.pickplace_scene(0, regions="paper", controller="astar")
    with P.Scene(sc, sk) as S:
        r = S.solve_paper(3, iters=12)
    assert np.all(r["class_counts"].sum(1) == r["n_env"])
    rate = r["class_counts"][:, 0] / r["n_env"]
    assert rate[-1] >= rate[0] and np.isfinite(r["best_J"])


def test_controller_validation(P):
    sc, sk = workload.push_scene(0)
    sc = dict(sc, base_controller="astar", base_inflate=0.3, wp_switch=0.25, pid_ki=2.0, pid_irad=0.3,
              pid_imax=0.5)
    with pytest.raises(P.CemError):
        P.Scene(sc, sk)
    sc2, sk2 = workload.pickplace_scene(0, controller="astar")
    with pytest.raises(P.CemError):
        P.Scene(dict(sc2, wp_switch=0.0), sk2)
    with P.Scene(*workload.pickplace_scene(0)) as S:  # no planner graph
        with pytest.raises(P.CemError):
            S.base_path((0, 0), (1, 1))


def converged_astar(seed, n, sample_seed):
    """The A* scene of a pick-and-place seed with n samples of the
    distribution the oracle's CE converged to on the same scene with the
    straight-line base controller (the plan's parameters mean the same
    under both controllers: the targets, gains, grasp and place offsets)."""
    from pickplace_common import converged

    _, _, mean, L = converged(seed)
    sc, sk = workload.pickplace_scene(seed, controller="astar")
    th = oracle.sample(sample_seed, 0, 0, n, mean, L).astype(np.float32)
    return sc, sk, th


def test_full_horizon_cost_and_class_through_every_action(P):
    """256 converged samples per scene over T = 3000 with A* planning at
    every moveTo: cost within 1e-3 and class exactly except for borderline
    samples (FP64 cost moves by more than 1e-3 when theta moves by 1e-6 of
    its range: a success test, contact onset or waypoint switch within
    rounding), which stay below 2 %; a third of the samples or more finish
    all five actions on every scene."""
    from pickplace_common import SEEDS, borderline

    n_bl = n_all = 0
    for seed in SEEDS:
        sc, sk, th = converged_astar(seed, 256, 4321)
        with P.Scene(sc, sk) as S:
            J, cls = S.rollout(dev(th))
        J, cls = J.cpu().numpy(), cls.cpu().numpy()
        Jr, cr = oracle.rollout(sc, sk, th.astype(np.float64))
        assert np.isin(cr, (0, 1)).mean() >= 1 / 3, (seed, np.bincount(cr, minlength=4))
        r = np.abs(J - Jr) / np.maximum(np.abs(Jr), 1e-3)
        bad = np.where((r > 1e-3) | (cls != cr))[0]
        bl = borderline(lambda t: oracle.rollout(sc, sk, t)[0], sk, th, Jr, bad)
        hard = bad[~bl]
        assert len(hard) == 0, (seed, hard[:8], J[hard[:8]], Jr[hard[:8]], cls[hard[:8]], cr[hard[:8]])
        n_bl += int(bl.sum())
        n_all += len(th)
    assert n_bl <= 0.02 * n_all, (n_bl, n_all)


def test_per_step_state_through_every_action(P):
    """8 converged samples per scene traced over the whole horizon with A*
    planning: every action's end on the oracle's step (or one step apart
    with the cost still within 1e-3: a crossing within FP32 rounding of eps,
    at most 2 of the 24), and the state from step 0 to 25 steps after the
    release within the shared pick-and-place bar (1e-4 m / rad, 1e-3 m/s,
    flags exactly)."""
    from pickplace_common import ACT, SEEDS, events, state_error, transitions

    n_cmp = n_shift = 0
    for seed in SEEDS:
        sc, sk, th = converged_astar(seed, 8, 99)
        T = sc["T"]
        with P.Scene(sc, sk) as S:
            st = S.trace(dev(th), T).cpu().numpy().astype(np.float64)
            J, cls = S.rollout(dev(th))
        J, cls = J.cpu().numpy(), cls.cpu().numpy()
        for i in range(th.shape[0]):
            ref = oracle.trace(sc, sk, th[i].astype(np.float64), T)
            tg, tr_ = transitions(st[i]), transitions(ref)
            if tg != tr_:
                assert tg.keys() == tr_.keys() and all(abs(tg[k] - tr_[k]) <= 1 for k in tg), (seed, i, tg, tr_)
                Jr, cr = oracle.rollout(sc, sk, th[i:i + 1].astype(np.float64))
                assert abs(J[i] - Jr[0]) <= 1e-3 * max(abs(Jr[0]), 1e-3) and cls[i] == cr[0], (seed, i)
                n_shift += 1
                continue
            ka, kr = events(ref)
            end = min(kr + 25, T) if kr is not None else T
            worst, where = state_error(st[i, :end], ref[:end])
            assert worst <= 1.0, (seed, i, where, worst, st[i, where[0]], ref[where[0]])
            n_cmp += ref[-1, ACT] == 5
    assert n_shift <= 2 and n_cmp >= 8, (n_shift, n_cmp)
