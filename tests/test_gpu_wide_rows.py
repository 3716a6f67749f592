"""Meshes with high-degree vertices: padded rows of 16 entries (vertex degree
8 to 15) against the oracle, and the supported-degree limit."""

import numpy as np
import pytest

import workload as w
from tests.gpu_helpers import lib, make_state, oracle_run

pytestmark = pytest.mark.gpu


def bipyramid(k, refinements):
    """Spherical bipyramid over a k-gon (two poles of degree k), refined."""
    ang = 2 * np.pi * np.arange(k) / k
    ring = np.stack([np.cos(ang), np.sin(ang), np.zeros(k)], 1)
    xyz = np.concatenate([ring, [[0, 0, 1.0], [0, 0, -1.0]]])
    top, bot = k, k + 1
    tri = []
    for j in range(k):
        a, b = j, (j + 1) % k
        tri.append((a, b, top))
        tri.append((b, a, bot))
    tri = np.array(tri, dtype=np.int32)
    for _ in range(refinements):
        xyz, tri, _ = w.refine(xyz, tri, ("sphere",))
    return xyz, tri


@pytest.fixture(scope="module")
def seg():
    return lib()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_degree_12_vertices_against_oracle(seg, prec, tol):
    xyz, tri = bipyramid(12, 3)
    deg = np.bincount(tri.ravel(), minlength=len(xyz))
    assert deg.max() == 12
    m, eps, tau, steps, seed = 4, 5e-2, 1e-3, 30, 9
    st = make_state(seg, xyz, tri, tau, m, eps, prec, seed, check_every=-1)
    assert seg.seg_launch_info(st)["padded_m"] >= m
    assert seg.seg_step(st, steps) == steps
    U, M, K = oracle_run(xyz, tri, w.initial_values("uniform", seed, len(xyz), m), tau, eps, steps)
    from oracle import seg_oracle as o

    ref = o.energy(xyz, tri, K, U, eps)["total"]
    got = seg.seg_energy(st)["total"]
    assert abs(got - ref) <= tol * abs(ref)
    Ug = seg.seg_get_u(st)
    assert np.abs(Ug - U).max() <= (1e-9 if prec == 0 else 5e-4) * np.abs(U).max()


def test_degree_limit(seg):
    xyz, tri = bipyramid(16, 1)  # poles of degree 16: rows of 17 entries
    with pytest.raises(seg.SegError) as e:
        seg.seg_assemble(seg.seg_create_mesh(xyz, tri), 1e-3, 1)
    assert e.value.status == seg.SEG_ERR_UNSUPPORTED
