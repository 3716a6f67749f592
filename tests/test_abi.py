"""The C-ABI library loads, exports every declared entry point, and its
host-only calls (mesh creation, validation, generators) behave.  No call
here touches the GPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

import workload as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def seg():
    import __graft_entry__ as g

    g.build()
    import paper_1408_2355_gb300 as seg

    return seg


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "seg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(seg_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(seg):
    names = _declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(seg.lib, n), n
    assert set(names) == set(seg.EXPORTED)


def test_no_oracle_in_the_library_path():
    pkg = os.path.join(ROOT, "paper_1408_2355_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("oracle-free", ""), f
                assert "import workload" not in src, f


def test_struct_layouts_match_header(seg):
    assert C.sizeof(seg.seg_params) == 64
    assert C.sizeof(seg.seg_server_params) == 16
    assert C.sizeof(seg.seg_request_info) == 64
    assert C.sizeof(seg.seg_stats) == 64
    assert C.sizeof(seg.seg_tune_result) == 152
    assert C.sizeof(seg.seg_surface) == 32


@pytest.mark.parametrize("level", [0, 1, 3, 5])
def test_native_icosphere_equals_shared_generator(seg, level):
    m = seg.seg_mesh_icosphere(level)
    xyz, tri = seg.seg_mesh_get(m)
    rx, rt = w.icosphere(level)
    assert np.array_equal(tri, rt)
    assert np.abs(xyz - rx).max() < 1e-15


def test_native_torus_and_ellipsoid_equal_shared_generator(seg):
    xyz, tri = seg.seg_mesh_get(seg.seg_mesh_torus(24, 12, 1.0, 0.4))
    rx, rt = w.torus(24, 12, 1.0, 0.4)
    assert np.array_equal(tri, rt) and np.abs(xyz - rx).max() < 1e-14
    xyz, tri = seg.seg_mesh_get(seg.seg_mesh_ellipsoid(3, 1.0, 0.8, 0.6))
    rx, rt = w.ellipsoid(3, 1.0, 0.8, 0.6)
    assert np.array_equal(tri, rt) and np.abs(xyz - rx).max() < 1e-14


def test_native_dziuk_and_refinement_equal_shared_generator(seg):
    for level in (0, 2, 3):
        xyz, tri = seg.seg_mesh_get(seg.seg_mesh_dziuk(level))
        rx, rt = w.dziuk(level)
        assert np.array_equal(tri, rt) and np.abs(xyz - rx).max() < 1e-15
    cases = [
        (w.icosphere(2), ("sphere",), seg.surface(seg.SEG_SURFACE_ELLIPSOID, 1.0, 1.0, 1.0)),
        (w.ellipsoid(2, 1.0, 0.8, 0.6), ("ellipsoid", 1.0, 0.8, 0.6),
         seg.surface(seg.SEG_SURFACE_ELLIPSOID, 1.0, 0.8, 0.6)),
        (w.torus(10, 6, 1.0, 0.4), ("torus", 1.0, 0.4), seg.surface(seg.SEG_SURFACE_TORUS, 1.0, 0.4)),
        (w.dziuk(1), ("dziuk",), seg.surface(seg.SEG_SURFACE_DZIUK)),
        (w.torus(7, 5, 1.0, 0.4), ("none",), seg.surface(seg.SEG_SURFACE_NONE)),
    ]
    for (x, t), wsurf, csurf in cases:
        fine, parents = seg.seg_mesh_refine(seg.seg_create_mesh(x, t), csurf)
        xyz, tri = seg.seg_mesh_get(fine)
        rx, rt, rp = w.refine(x, t, wsurf)
        assert np.array_equal(tri, rt) and np.array_equal(parents, rp), wsurf
        assert np.abs(xyz - rx).max() < 1e-15, wsurf
    with pytest.raises(seg.SegError) as e:
        seg.seg_mesh_refine(seg.seg_mesh_icosphere(1), seg.surface(seg.SEG_SURFACE_TORUS, 0.3, 0.4))
    assert e.value.status == seg.SEG_ERR_ARG
    with pytest.raises(seg.SegError) as e:
        seg.seg_mesh_refine(seg.seg_mesh_icosphere(1), seg.surface(7))
    assert e.value.status == seg.SEG_ERR_ARG


def test_degenerate_meshes(seg):
    xyz, tri = w.icosphere(1)
    with pytest.raises(seg.SegError) as e:  # no triangles
        seg.seg_create_mesh(xyz, tri[:0])
    assert e.value.status == seg.SEG_ERR_ARG
    with pytest.raises(seg.SegError) as e:  # fewer than 3 vertices
        seg.seg_create_mesh(xyz[:2], np.zeros((0, 3), dtype=np.int32))
    assert e.value.status == seg.SEG_ERR_ARG
    # a vertex in no triangle has no mass: the step-1 matrix would be singular
    extra = np.concatenate([xyz, [[0.0, 0.0, 2.0]]])
    with pytest.raises(seg.SegError) as e:
        seg.seg_assemble(seg.seg_create_mesh(extra, tri), 1e-3, 1)
    assert e.value.status == seg.SEG_ERR_MESH
    for tau in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(seg.SegError) as e:
            seg.seg_assemble(seg.seg_create_mesh(xyz, tri), tau, 1)
        assert e.value.status == seg.SEG_ERR_ARG


def test_mesh_validation_errors(seg):
    xyz, tri = w.icosphere(1)
    m = seg.seg_create_mesh(xyz, tri)
    assert seg.seg_mesh_info(m) == (42, 80)
    bad = tri.copy()
    bad[3, 1] = 42
    with pytest.raises(seg.SegError) as e:
        seg.seg_create_mesh(xyz, bad)
    assert e.value.status == seg.SEG_ERR_ARG
    bad = tri.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(seg.SegError) as e:
        seg.seg_create_mesh(xyz, bad)
    assert e.value.status == seg.SEG_ERR_MESH
    flat = xyz.copy()
    flat[tri[5, 1]] = flat[tri[5, 0]]
    with pytest.raises(seg.SegError) as e:
        seg.seg_create_mesh(flat, tri)
    assert e.value.status == seg.SEG_ERR_MESH
    nan = xyz.copy()
    nan[7, 2] = np.nan
    with pytest.raises(seg.SegError) as e:
        seg.seg_create_mesh(nan, tri)
    assert e.value.status == seg.SEG_ERR_ARG
    with pytest.raises(seg.SegError):
        seg.seg_mesh_icosphere(-1)
    with pytest.raises(seg.SegError):
        seg.seg_mesh_torus(8, 8, 0.3, 0.4)
    assert "R > r" in seg.seg_last_error()


def test_noalloc_wrapper_rejects_bad_arguments_before_any_call(seg):
    """seg_s_eps_noalloc's binding checks every argument (kind, dtype,
    contiguity, shape, output length, device) before the library sees a raw
    address; each bad argument below is refused with SEG_ERR_ARG on the host
    (no GPU here: the valid tensors are CPU tensors, refused last for not
    being on a CUDA device)."""
    torch = pytest.importorskip("torch")
    n, m, f = 12, 3, 20
    good = dict(u=torch.zeros((n, m), dtype=torch.float64), xyz=torch.zeros((n, 3), dtype=torch.float64),
                tri=torch.zeros((f, 3), dtype=torch.int32), out=torch.zeros(m + 1, dtype=torch.float64))
    bad_cases = [
        ("u", np.zeros((n, m)), "torch tensor"),
        ("tri", torch.zeros((f, 3), dtype=torch.int64), "torch.int32"),
        ("u", torch.zeros((m, n), dtype=torch.float64).t(), "contiguous"),
        ("u", torch.zeros(n * m, dtype=torch.float64), "(n_vert, m)"),
        ("xyz", torch.zeros((n + 1, 3), dtype=torch.float64), "xyz must be"),
        ("tri", torch.zeros((f, 4), dtype=torch.int32), "tri must be"),
        ("out", torch.zeros(m, dtype=torch.float64), "m + 1"),
        (None, None, "CUDA tensor"),
    ]
    for key, value, words in bad_cases:
        args = dict(good)
        if key is not None:
            args[key] = value
        with pytest.raises(seg.SegError) as err:
            seg.seg_s_eps_noalloc(args["u"], args["xyz"], args["tri"], 0.1, args["out"])
        assert err.value.status == seg.SEG_ERR_ARG
        assert words in str(err.value), (key, str(err.value))


HANDLE_CALLS = [
    "seg_mesh_info", "seg_mesh_get", "seg_problem_info", "seg_state_bytes", "seg_set_u", "seg_get_u",
    "seg_checkpoint_size", "seg_get_checkpoint", "seg_set_checkpoint", "seg_set_wait_limit", "seg_set_wait_stall",
    "seg_step_async", "seg_sync", "seg_step", "seg_substep", "seg_batch_step_async", "seg_batch_sync",
    "seg_batch_step", "seg_batch_set_persistent", "seg_energy", "seg_eigenvalue_estimates", "seg_energy_p",
    "seg_prolong", "seg_labels", "seg_get_stats", "seg_stats_enqueue", "seg_stats_wait", "seg_time_kernel",
    "seg_autotune", "seg_launch_info", "seg_server_submit", "seg_server_tick", "seg_server_info",
    "seg_server_result",
]


@pytest.mark.parametrize("name", HANDLE_CALLS)
def test_null_handle_is_refused_without_touching_the_gpu(seg, name):
    """Every entry point that takes a mesh, problem, state, batch or server
    handle first returns SEG_ERR_ARG for a NULL handle (with a message), before
    any other work -- so also on a machine without a GPU."""
    fn = getattr(seg.lib, name)
    args = []
    for t in fn.argtypes:
        if t in (C.c_int32, C.c_int64, C.c_uint64, C.c_int):
            args.append(0)
        elif t is C.c_double:
            args.append(0.0)
        else:
            args.append(None)  # the handle and every pointer
    assert fn(*args) == seg.SEG_ERR_ARG, name
    assert seg.seg_last_error()
