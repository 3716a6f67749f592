"""Launch-geometry autotuner: it restores the state bitwise, picks the
fastest measured candidate, and later steps agree with an untuned twin up to
the summation order of the partial inner products."""

import numpy as np
import pytest

import workload as w
from tests.gpu_helpers import lib, make_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    return lib()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_autotune_restores_and_agrees(seg, prec, tol):
    xyz, tri = w.icosphere(6)
    tuned = make_state(seg, xyz, tri, 1e-5, 8, 2e-3, prec, 11)
    twin = make_state(seg, xyz, tri, 1e-5, 8, 2e-3, prec, 11)
    assert seg.seg_step(tuned, 5) == 5
    assert seg.seg_step(twin, 5) == 5
    before = seg.seg_get_u(tuned)
    stats0 = seg.seg_get_stats(tuned)
    r = seg.seg_autotune(tuned, 5)
    assert np.array_equal(seg.seg_get_u(tuned), before)
    stats1 = seg.seg_get_stats(tuned)
    assert stats1.pop("graph_peel") == r["cg_peel"]
    stats0.pop("graph_peel")
    assert stats1 == stats0
    grids = [g for g, _ in r["candidates"]]
    assert r["grid_blocks"] in grids and len(grids) >= 2
    assert r["ms_model"] <= min(ms for _, ms in r["candidates"]) * (1 + 1e-12)
    assert set(r["grid_pass"].values()) <= set(grids)
    assert r["grid_pass"]["cg_a"] == r["grid_blocks"]
    assert r["cg_weight"] == pytest.approx(stats0["cg_iterations"] / 5)
    assert seg.seg_launch_info(tuned)["grid_blocks"] == r["grid_blocks"]
    assert seg.seg_step(tuned, 20) == 20
    assert seg.seg_step(twin, 20) == 20
    a, b = seg.seg_get_u(tuned), seg.seg_get_u(twin)
    assert np.abs(a - b).max() <= tol * np.abs(b).max()
    e1, e2 = seg.seg_energy(tuned), seg.seg_energy(twin)
    assert abs(e1["total"] - e2["total"]) <= tol * abs(e2["total"])


def test_autotune_small_mesh_candidates(seg):
    xyz, tri = w.icosphere(2)  # 162 vertices: one block of rows is enough
    st = make_state(seg, xyz, tri, 1e-3, 3, 5e-2, 1, 3)
    r = seg.seg_autotune(st, 3)
    assert [g for g, _ in r["candidates"]] == [1]
    assert r["grid_blocks"] == 1
    assert seg.seg_step(st, 3) == 3
