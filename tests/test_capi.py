"""C-ABI checks that need no GPU: the library builds, exports every entry
point that include/cemtamp.h declares, the ctypes mirrors of the public
structs have the C layout, and host-side argument validation rejects bad
descriptors before any CUDA call."""
import ctypes as C
import os
import re
import subprocess

import pytest

import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cemtamp.h")


@pytest.fixture(scope="module")
def pkg():
    import paper_2512_11571_gb300 as P
    from paper_2512_11571_gb300 import build

    build.build()
    P.load()
    return P


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:\w+\s+)*\w+\s*\*?\s*(cem_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cem_scene_create", "cem_scene_destroy", "cem_sample", "cem_rollout_batch", "cem_refit",
                 "cem_solve", "cem_last_error", "cem_autotune"):
        assert must in names


def test_library_exports_every_declared_symbol(pkg):
    lib = C.CDLL(pkg.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    for n in declared_functions():
        assert re.search(rf"\bT {n}\b", out), n


def test_debug_library_builds_with_the_same_exports(pkg):
    # the bounds-checked build (CEM_DEBUG) compiles from the same sources and
    # exports the same entry points as the release library
    from paper_2512_11571_gb300 import build

    path = build.build(debug=True)
    assert path == pkg.DEBUG_LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in declared_functions():
        assert re.search(rf"\bT {n}\b", out), n


def test_binding_names_match_header(pkg):
    assert sorted(pkg.EXPORTS) == sorted(n for n in declared_functions())
    for n in pkg.EXPORTS:
        if n not in ("cem_last_error", "cem_version"):
            assert callable(getattr(pkg, n))


def _c_offsets(struct_name, fields, tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    lines.append(f'printf("%zu\\n", sizeof({struct_name}));')
    for f in fields:
        lines.append(f'printf("%zu\\n", offsetof({struct_name}, {f}));')
    lines.append("return 0;}")
    c = tmp_path / f"{struct_name}.c"
    exe = tmp_path / f"{struct_name}.out"
    c.write_text("\n".join(lines))
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(c)], check=True)
    return [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]


@pytest.mark.parametrize("name", ["cem_slab", "cem_geom", "cem_scene_desc", "cem_action_desc",
                                  "cem_skeleton_desc", "cem_solve_params", "cem_result", "cem_problem_params",
                                  "cem_paper_params", "cem_finetune_params"])
def test_struct_layout_matches_header(pkg, name, tmp_path):
    cls = getattr(pkg, name)
    fields = [f[0] for f in cls._fields_]
    got = _c_offsets(name, fields, tmp_path)
    assert got[0] == C.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in fields]


def _create(pkg, scene, skel):
    s, k = pkg.pack_scene(scene, skel)
    h = C.c_void_p()
    return pkg.load().cem_scene_create(C.byref(s), C.byref(k), C.byref(h)), s, k


def test_validation_rejects_bad_descriptors(pkg):
    L = pkg.load()
    sc, sk = workload.reach_scene()
    s, k = pkg.pack_scene(sc, sk)
    h = C.c_void_p()
    # too many parameters
    k2 = pkg.cem_skeleton_desc.from_buffer_copy(k)
    k2.D = 19
    assert L.cem_scene_create(C.byref(s), C.byref(k2), C.byref(h)) == -5
    # theta slices not covering D
    k3 = pkg.cem_skeleton_desc.from_buffer_copy(k)
    k3.D = 4
    assert L.cem_scene_create(C.byref(s), C.byref(k3), C.byref(h)) == -1
    assert b"cover" in L.cem_last_error()
    # inverted bounds
    k4 = pkg.cem_skeleton_desc.from_buffer_copy(k)
    k4.lo[0], k4.hi[0] = 1.0, -1.0
    assert L.cem_scene_create(C.byref(s), C.byref(k4), C.byref(h)) == -1
    # grasp in a planar scene
    k5 = pkg.cem_skeleton_desc.from_buffer_copy(k)
    k5.action[0].kind = 2
    assert L.cem_scene_create(C.byref(s), C.byref(k5), C.byref(h)) == -1
    # non-positive step, unknown kind, horizon 0
    s2 = pkg.cem_scene_desc.from_buffer_copy(s)
    s2.dt = 0.0
    assert L.cem_scene_create(C.byref(s2), C.byref(k), C.byref(h)) == -1
    s3 = pkg.cem_scene_desc.from_buffer_copy(s)
    s3.kind = 9
    assert L.cem_scene_create(C.byref(s3), C.byref(k), C.byref(h)) == -1
    s4 = pkg.cem_scene_desc.from_buffer_copy(s)
    s4.T = 0
    assert L.cem_scene_create(C.byref(s4), C.byref(k), C.byref(h)) == -5
    # NULL descriptors and NULL out pointer
    assert L.cem_scene_create(None, C.byref(k), C.byref(h)) == -1
    assert L.cem_scene_create(C.byref(s), C.byref(k), None) == -1
    # calls on a NULL handle
    assert L.cem_rollout_batch(None, None, 1, None, None, None) == -1
    assert L.cem_refit(None, None, None, None, 1, 1, 0, None, None, None, None, None, None) == -1
    assert L.cem_scene_destroy(None) == 0
    assert L.cem_set_threads_per_rollout(None, 8) == -1
    assert L.cem_get_launch(None, 1, None, None) == -1
    assert L.cem_solve_paper(None, None, None) == -1
    assert L.cem_sample_uniform(None, 1, 0, 4, None, None) == -1
    # initial-sampling regions: an annulus only on a moveTo goal, 0 <= inner < outer
    k6 = pkg.cem_skeleton_desc.from_buffer_copy(k)
    k6.action[0].init_region = 2
    assert L.cem_scene_create(C.byref(s), C.byref(k6), C.byref(h)) == -1
    k7 = pkg.cem_skeleton_desc.from_buffer_copy(k)
    k7.action[0].init_region = 1
    k7.action[0].region[:] = [0.0, 0.0, 0.5, 0.5]
    assert L.cem_scene_create(C.byref(s), C.byref(k7), C.byref(h)) == -1
    assert b"annulus" in L.cem_last_error()


def test_release_build_has_no_bounds_checks(pkg):
    # the release library answers the debug-status query without touching the device
    if os.environ.get("CEMTAMP_DEBUG") == "1":
        pytest.skip("the session runs on the debug library")
    code = C.c_int(-1)
    rc = pkg.load().cem_debug_status(C.byref(code), 0)
    assert pkg.STATUS[rc] == "CEM_ERR_UNSUPPORTED" and code.value == 0
    assert "release build" in pkg.load().cem_last_error().decode()
    with pytest.raises(pkg.CemError) as e:
        pkg.cem_debug_status()
    assert pkg.STATUS[e.value.code] == "CEM_ERR_UNSUPPORTED"
    assert pkg.STATUS[pkg.load().cem_debug_selftest()] == "CEM_ERR_UNSUPPORTED"


def test_n_env_schedule_matches_oracle(pkg):
    """The library's integer schedule against the oracle's (Sec. IV-A)."""
    import oracle

    for n0, n1, j1 in ((3000, 300, 10), (10, 0 + 1, 4), (100, 400, 3), (777, 65, 7), (5, 5, 2), (500, 50, 0)):
        for j in range(14):
            assert pkg.cem_n_env(n0, n1, j1, j) == oracle.n_env(n0, n1, j1, j), (n0, n1, j1, j)


def test_paper_regions_pack(pkg):
    sc, sk = workload.pickplace_scene(0, regions="paper")
    s, k = pkg.pack_scene(sc, sk)
    assert [k.action[i].init_region for i in range(5)] == [1, 0, 1, 0, 0]
    assert list(k.action[0].region) == pytest.approx([-1.6, 0.9, 0.65, 0.9])


def test_pick_place_descriptor_packs(pkg):
    sc, sk = workload.pickplace_scene(3)
    s, k = pkg.pack_scene(sc, sk)
    assert k.D == 14 and k.n_actions == 5
    assert [k.action[i].theta_offset for i in range(5)] == [0, 3, 5, 8, 11]
    assert s.n_geoms == len(sc["geoms"])


def test_batch_validation_names_the_problem(pkg):
    L = pkg.load()
    n = 3
    scenes = (pkg.cem_scene_desc * n)()
    skels = (pkg.cem_skeleton_desc * n)()
    params = (pkg.cem_problem_params * n)()
    for i in range(n):
        sc, sk = workload.reach_scene()
        scenes[i], skels[i] = pkg.pack_scene(sc, sk)
        params[i].N, params[i].K = 64, 8
    skels[1].D = 4  # slices no longer cover D
    h = C.c_void_p()
    assert L.cem_batch_create(scenes, skels, params, n, C.byref(h)) == -1
    assert b"problem 1" in L.cem_last_error()
    skels[1].D = 3
    params[2].K = 5000
    assert L.cem_batch_create(scenes, skels, params, n, C.byref(h)) == -5
    assert L.cem_batch_create(scenes, skels, params, 0, C.byref(h)) == -5
    assert L.cem_batch_iterate(None, 1, 1, None) == -1
    assert L.cem_batch_set_threads_per_rollout(None, 8) == -1
    assert L.cem_batch_get_launch(None, None, None, None) == -1


def test_binding_checks_buffers_before_the_call(pkg):
    """The wrappers refuse host arrays of the wrong length and non-CUDA
    tensors before anything reaches the library (sizes the C call cannot
    see: it takes plain pointers)."""
    np = pytest.importorskip("numpy")
    torch = pytest.importorskip("torch")
    th = torch.zeros(4, 3)
    with pytest.raises(ValueError, match="lo"):
        pkg.cem_surrogate_features(None, th, np.zeros(2), np.ones(3), np.zeros(16), None)
    with pytest.raises(ValueError, match="scene16"):
        pkg.cem_surrogate_features(None, th, np.zeros(3), np.ones(3), np.zeros(15), None)
    with pytest.raises(TypeError, match="theta: expected a CUDA tensor"):
        pkg.cem_rollout_batch(None, th, 4, torch.zeros(4), torch.zeros(4, dtype=torch.uint8))
    with pytest.raises(ValueError, match="scene16"):
        pkg.cem_solve_screened(None, None, np.zeros(17), pkg.cem_solve_params(), 64)
