"""cem_solve_static: the CE loop for callers that cannot allocate device memory.

Real-time control loops, plugins whose host owns all device memory, and
processes under a fixed memory cap cannot call cudaMalloc while they plan.
cem_solve_static serves them from a fixed file-scope device array.  This
test checks, through the C ABI, that it returns what the handle-based
cem_solve returns for the same request (reach, push and pick-place), on two
calls in a row (the shared array keeps the previous call's contents, so the
second call checks that nothing leaks from the first); that a split run
resumed from its returned distribution ends where the unsplit run ends; and
that calls after the first leave the device's free memory unchanged.  It is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

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


def make_params(P, seed, N, K, iters):
    p = P.cem_solve_params()
    p.seed, p.N, p.K, p.iters, p.cov_mode, p.problem, p.start_iter, p.use_graph = seed, N, K, iters, 0, 0, 0, 0
    hist = np.zeros(iters, np.float32)
    keff = np.zeros(iters, np.int32)
    p.best_J_hist_h = hist.ctypes.data_as(C.POINTER(C.c_float))
    p.k_eff_hist_h = keff.ctypes.data_as(C.POINTER(C.c_int32))
    return p, hist, keff


def close(a, b, rel=1e-6):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.all(np.abs(a - b) <= rel * np.maximum(1.0, np.abs(b)))


# pick-place (D = 14) at N = 4096 keeps the test short; N * D stays far below the limit
CASES = [("reach", lambda: workload.config(0, seed=2)), ("push", lambda: workload.config(1, seed=1)),
         ("pickplace", lambda: (*workload.config(2, seed=3)[:2], dict(N=4096, K=128)))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_static_solve_matches_handle_solve(P, name, make):
    sc, sk, cm = make()
    N, K, iters = cm["N"], cm["K"], 6
    D = len(sk["lo"])
    L = P.load()
    ref_p, ref_hist, ref_keff = make_params(P, 5, N, K, iters)
    with P.Scene(sc, sk) as S:
        ref = P.cem_solve(S.h, ref_p)
    s, k = P.pack_scene(sc, sk)
    for call in range(2):
        p, hist, keff = make_params(P, 5, N, K, iters)
        out = P.cem_result()
        rc = L.cem_solve_static(C.byref(s), C.byref(k), C.byref(p), C.byref(out), None)
        assert rc == 0, L.cem_last_error().decode()
        assert out.iters_done == iters and out.best_class == ref.best_class
        assert close(out.best_J, ref.best_J)
        assert close(out.best_theta[:D], ref.best_theta[:D])
        assert close(out.mean[:D], ref.mean[:D])
        assert close(out.cov[:D * D], ref.cov[:D * D])
        assert close(hist, ref_hist) and np.array_equal(keff, ref_keff)


def static_solve(P, s, k, seed, N, K, iters, start_iter=0, init=None):
    p, hist, keff = make_params(P, seed, N, K, iters)
    p.start_iter = start_iter
    keep = []
    if init is not None:
        for name, field in (("mean", "init_mean_h"), ("cov", "init_cov_h"), ("chol", "init_chol_h")):
            a = np.ascontiguousarray(init[name], np.float32)
            keep.append(a)
            setattr(p, field, a.ctypes.data_as(C.POINTER(C.c_float)))
    out = P.cem_result()
    L = P.load()
    rc = L.cem_solve_static(C.byref(s), C.byref(k), C.byref(p), C.byref(out), None)
    assert rc == 0, L.cem_last_error().decode()
    return out, hist


def test_static_solve_resumes_exactly(P):
    """A run split after 3 iterations and resumed from the returned mean, cov
    and factor with start_iter = 3 ends in the same distribution as the
    unsplit 6-iteration run, and the better of the two halves' best samples
    is the unsplit run's best sample."""
    sc, sk, cm = workload.config(1, seed=4)
    D = len(sk["lo"])
    s, k = P.pack_scene(sc, sk)
    full, _ = static_solve(P, s, k, 9, 2048, 100, 6)
    a, _ = static_solve(P, s, k, 9, 2048, 100, 3)
    init = dict(mean=np.array(a.mean[:D]), cov=np.array(a.cov[:D * D]), chol=np.array(a.chol[:D * D]))
    b, _ = static_solve(P, s, k, 9, 2048, 100, 3, start_iter=3, init=init)
    for f in ("mean", "cov", "chol"):
        n = D if f == "mean" else D * D
        assert np.array_equal(np.array(getattr(b, f)[:n]), np.array(getattr(full, f)[:n])), f
    best = min((a, b), key=lambda r: (r.best_class, r.best_J))
    assert best.best_class == full.best_class and best.best_J == full.best_J
    assert np.array_equal(np.array(best.best_theta[:D]), np.array(full.best_theta[:D]))


def test_static_solve_allocates_nothing(P):
    """After a first call (which loads the module), further calls leave the
    device's free memory exactly where it was."""
    sc, sk, cm = workload.config(0, seed=2)
    s, k = P.pack_scene(sc, sk)
    static_solve(P, s, k, 3, cm["N"], cm["K"], 4)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        static_solve(P, s, k, 3, cm["N"], cm["K"], 4)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_solve_rejects_oversize(P):
    sc, sk, cm = workload.config(2, seed=0)  # D = 14: N = 20000 exceeds N * D <= 262144
    s, k = P.pack_scene(sc, sk)
    p, _, _ = make_params(P, 1, 20000, 64, 2)
    out = P.cem_result()
    L = P.load()
    assert L.cem_solve_static(C.byref(s), C.byref(k), C.byref(p), C.byref(out), None) == -5
    assert b"262144" in L.cem_last_error()
