"""The bounds-checked debug build (libcemtamp_debug.so, CEM_DEBUG) on the GPU.

compute-sanitizer is not available on the GB300 pool, so the kernels carry
their own checks in a debug build: every checked index (the dispatch and
rollout orders, their output positions and bins, geometry and parameter
indexes, elite indexes, screened row indexes) that leaves its buffer is
clamped into range and its code recorded.  A child process loads the debug
library and runs the bench's 64-problem batch, a mixed batch with ragged and
tiny problems, single solves of every task and a surrogate-screened solve;
the test asserts that no check fired and that every result equals the
release library's bit for bit (the checks change no arithmetic), then makes
one check fire on purpose through an in-bounds self-test (the clamp keeps
the access inside its array)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the workload both libraries run: (kind of run, results as plain lists)
WORK = r'''
import json, sys
import numpy as np
import workload
import paper_2512_11571_gb300 as P


def problems():
    big = workload.batch_problems(0)
    for i, p in enumerate(big):
        p["seed"] = 3
        p["problem"] = i
    mixed = []
    sc, sk = workload.reach_scene(0)
    mixed.append(dict(scene=sc, skel=sk, N=1, K=1, seed=11))
    sc, sk = workload.push_scene(1)
    mixed.append(dict(scene=sc, skel=sk, N=333, K=30, seed=12))
    for L in (3, 6):
        sc, sk = workload.pickplace_scene(2 + L, n_actions=L, T=600)
        mixed.append(dict(scene=sc, skel=sk, N=33 + 40 * L, K=16, seed=20 + L))
    sc, sk = workload.pickplace_scene(9, n_actions=5, T=400, obstacle="box")
    mixed.append(dict(scene=sc, skel=sk, N=8192 + 40, K=64, seed=29))
    for i, p in enumerate(mixed):
        p["problem"] = 100 + i
    singles = [workload.reach_scene(2), workload.push_scene(3, T=400), workload.pickplace_scene(4, T=600)]
    return big, mixed, singles


def run():
    big, mixed, singles = problems()
    out = {}
    for name, probs, iters in (("big", big, 2), ("mixed", mixed, 3)):
        with P.Batch(probs) as B:
            B.iterate(iters, use_graph=True)
            got = B.read()
        out[name] = [[float(g["best_J"]), int(g["best_cls"]), np.asarray(g["mean"]).tolist(),
                      np.asarray(g["best_theta"]).tolist()] for g in got]
    out["single"] = []
    for j, (sc, sk) in enumerate(singles):
        with P.Scene(sc, sk) as S:
            r = S.solve(50 + j, 512, 32, 3, problem=j, use_graph=False)
        out["single"].append([float(r["best_J"]), int(r["best_cls"]), np.asarray(r["mean"]).tolist(),
                              np.asarray(r["best_theta"]).tolist()])
    sc, sk, _ = workload.config(2, seed=3)  # surrogate-screened: the kept rows gathered from the pool
    with P.Scene(sc, sk, T=400) as Sc, P.Surrogate(256, 4, seed=4) as S:
        r = Sc.solve_screened(S, workload.scene_features(sc), seed=1, N=512, K=32, iters=3, n_pool=4096)
    out["screened"] = [[float(r["best_J"]), int(r["best_cls"]), np.asarray(r["mean"]).tolist(),
                        np.asarray(r["best_theta"]).tolist()]]
    return out
'''

CHILD = WORK + r'''
P.load(P.DEBUG_LIB_PATH)
res = run()
res["debug_status"] = P.cem_debug_status(reset=True)
P.cem_debug_selftest()  # one clamped access, recorded as code 99
res["selftest_status"] = [P.cem_debug_status(reset=True), P.cem_debug_status()]
print(json.dumps(res))
'''


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    build.build(debug=True)
    P.load()
    return P


def test_debug_build_fires_no_check_and_changes_no_result(P):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    dbg = json.loads(r.stdout.strip().splitlines()[-1])
    assert dbg.pop("debug_status") == 0
    assert dbg.pop("selftest_status") == [99, 0]  # the checks are compiled in, fire, and reset
    scope = {}
    exec(compile(WORK, "work", "exec"), scope)
    rel = scope["run"]()
    assert dbg.keys() == rel.keys()
    for k in rel:
        assert len(dbg[k]) == len(rel[k])
        for i, (a, b) in enumerate(zip(dbg[k], rel[k])):
            assert a[0] == b[0] and a[1] == b[1], (k, i, a[:2], b[:2])
            assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3]), (k, i)
