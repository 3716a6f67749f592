"""Closed forms of the paper on the GPU: the eigenvalue estimates of the
interpolated two-hemisphere and Y-partition eigenfunctions (Sec. 1: the sums
4 and 45/4 for eps -> 0) equal the oracle's on the same mesh and converge to
the closed form under refinement; the constant state's S_eps."""

import os

import numpy as np
import pytest

import workload as w
from oracle import seg_oracle as o
from tests.gpu_helpers import lib

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


@pytest.fixture(scope="module")
def seg():
    return lib()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_hemispheres_and_y_partition(seg, prec, tol):
    g = _golden()
    cases = {
        "hemispheres_total": lambda x: np.stack([np.maximum(x[:, 2], 0), np.maximum(-x[:, 2], 0)], 1),
        "y_partition_total": o.y_partition,
    }
    for key, make in cases.items():
        errs = []
        for L in (3, 4, 5):
            xyz, tri = w.icosphere(L)
            U = make(xyz)
            m = U.shape[1]
            prob = seg.seg_assemble(seg.seg_create_mesh(xyz, tri), 1e-4, prec)
            st = seg.seg_state_create(prob, m, 1e-2, seg.SEG_INIT_UNIFORM, 1)
            seg.seg_set_u(st, U)
            lam, _ = seg.seg_eigenvalue_estimates(st)
            M, K = o.assemble(xyz, tri)
            ref = o.dirichlet(K, o.normalise(M, U))
            assert np.abs(lam - ref).max() <= tol * np.abs(ref).max(), (key, L)
            errs.append(abs(lam.sum() - g[key]))
        assert errs[2] < errs[1] < errs[0], (key, errs)


@pytest.mark.parametrize("prec,tol,dtol", [(0, 1e-12, 1e-10), (1, 1e-6, 1e-3)])
def test_constant_state_s_eps(seg, prec, tol, dtol):
    xyz, tri = w.icosphere(4)
    m, eps = 5, 0.05
    prob = seg.seg_assemble(seg.seg_create_mesh(xyz, tri), 1e-4, prec)
    st = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, 1)
    seg.seg_set_u(st, np.ones((len(xyz), m)))
    area = seg.seg_problem_info(prob)["area"]
    e = seg.seg_energy(st)
    assert e["s_eps"] == pytest.approx(o.constant_state_s_eps(m, area, eps), rel=tol)
    assert abs(e["dirichlet"]) < dtol  # K annihilates constants (up to the rounding of float32 K)
