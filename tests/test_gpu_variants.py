"""Variants and extensions on the GPU against the oracle: the lumped-mass
variant, the l^p energies of Problem 1.2, P1 prolongation onto a refined
mesh and the continuation of Sec. 3.3 (sphere and surface (D))."""

import math

import numpy as np
import pytest

import workload as w
from oracle import seg_oracle as o
from tests.gpu_helpers import lib, make_state, oracle_run

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}  # relative energy: FP64, mixed


@pytest.fixture(scope="module")
def seg():
    return lib()


def _rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("prec", [0, 1])
def test_lumped_mass_variant_against_oracle(seg, prec):
    xyz, tri = w.icosphere(4)
    m, eps, tau, steps, seed = 3, 1e-2, 1e-4, 100, 71
    prob = seg.seg_assemble_ex(seg.seg_create_mesh(xyz, tri), tau, prec, seg.SEG_ASSEMBLE_LUMPED_MASS)
    p = seg.seg_params()
    p.check_every = -1
    st = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, seed, p)
    assert seg.seg_step(st, steps) == steps
    ML = o.lumped_mass(xyz, tri)
    _, K = o.assemble(xyz, tri)
    U = o.initial_state(ML, w.initial_values("uniform", seed, len(xyz), m))
    for _ in range(steps):
        U = o.step(ML, K, tau, eps, U)
    ref = o.energy(xyz, tri, K, U, eps)
    got = seg.seg_energy(st)
    assert _rel(got["total"], ref["total"]) < TOL[prec]
    assert _rel(got["dirichlet"], ref["dirichlet"]) < TOL[prec]
    Ug = seg.seg_get_u(st)
    assert np.abs(Ug - U).max() <= (1e-9 if prec == 0 else 2e-4) * np.abs(U).max()
    # the lumped state is normalised in the lumped norm
    assert np.allclose(np.einsum("zi,z,zi->i", Ug, ML.diagonal(), Ug), 1.0, rtol=1e-12 if prec == 0 else 1e-5)
    with pytest.raises(seg.SegError):
        seg.seg_assemble_ex(seg.seg_create_mesh(xyz, tri), tau, prec, 4)


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_p_against_oracle(seg, prec):
    xyz, tri = w.icosphere(4)
    m, eps, tau, steps, seed = 4, 2e-2, 1e-4, 40, 5
    st = make_state(seg, xyz, tri, tau, m, eps, prec, seed, check_every=-1)
    seg.seg_step(st, steps)
    U, M, K = oracle_run(xyz, tri, w.initial_values("uniform", seed, len(xyz), m), tau, eps, steps)
    lam = o.energy(xyz, tri, K, U, eps)["D"]
    for p in (1, 2, 5.5, math.inf):
        assert _rel(seg.seg_energy_p(st, p), o.energy_p(lam, p)) < TOL[prec], p
    assert seg.seg_energy_p(st, 1) == pytest.approx(seg.seg_energy(st)["dirichlet"] / m, rel=1e-12)
    with pytest.raises(seg.SegError):
        seg.seg_energy_p(st, 0.5)


@pytest.mark.parametrize("prec", [0, 1])
def test_prolongation_on_the_device(seg, prec):
    x0, t0 = w.icosphere(2)
    coarse = make_state(seg, x0, t0, 1e-3, 5, 0.1, prec, 9, check_every=-1)
    seg.seg_step(coarse, 5)
    fine_mesh, parents = seg.seg_mesh_refine(seg.seg_create_mesh(x0, t0),
                                             seg.surface(seg.SEG_SURFACE_ELLIPSOID, 1.0, 1.0, 1.0))
    x1, t1, p1 = w.refine(x0, t0, ("sphere",))
    assert np.array_equal(parents, p1)
    fine = seg.seg_state_create(seg.seg_assemble(fine_mesh, 5e-4, prec), 5, 0.05, seg.SEG_INIT_UNIFORM, 1)
    seg.seg_prolong(coarse, fine, parents)
    M1, _ = o.assemble(x1, t1)
    ref = o.normalise(M1, o.prolong(seg.seg_get_u(coarse), p1))
    got = seg.seg_get_u(fine)
    assert np.abs(got - ref).max() <= (1e-13 if prec == 0 else 1e-6) * np.abs(ref).max()
    bad = parents.copy()
    bad[-1, 0] = len(x0)
    with pytest.raises(seg.SegError) as e:
        seg.seg_prolong(coarse, fine, bad)
    assert e.value.status == seg.SEG_ERR_ARG


@pytest.mark.parametrize("surface,prec", [("sphere", 0), ("sphere", 1), ("dziuk", 0)])
def test_continuation_against_oracle(seg, surface, prec):
    """Three levels: eps and tau halve per refinement (two bisection levels of
    the sqrt-2 rule of Sec. 3.3); each level starts from the interpolated
    previous state."""
    if surface == "sphere":
        x0, t0 = w.icosphere(2)
        wsurf, csurf = ("sphere",), seg.surface(seg.SEG_SURFACE_ELLIPSOID, 1.0, 1.0, 1.0)
    else:
        x0, t0 = w.dziuk(2)
        wsurf, csurf = ("dziuk",), seg.surface(seg.SEG_SURFACE_DZIUK)
    m, eps, tau, steps, seed = 3, 0.2, 4e-3, 30, 17
    levels = [(x0, t0, None)]
    for _ in range(2):
        x, t, par = w.refine(levels[-1][0], levels[-1][1], wsurf)
        levels.append((x, t, par))
    ref = o.continuation(levels, w.initial_values("uniform", seed, len(x0), m), eps, tau, steps)
    mesh = seg.seg_create_mesh(x0, t0)
    p = seg.seg_params()
    p.check_every = -1
    st = seg.seg_state_create(seg.seg_assemble(mesh, tau, prec), m, eps, seg.SEG_INIT_UNIFORM, seed, p)
    for lvl in range(3):
        if lvl > 0:
            eps, tau = eps / 2, tau / 2
            mesh, _, st = seg.seg_continue(st, mesh, csurf, eps, tau, p)
            xyz, tri = seg.seg_mesh_get(mesh)
            assert np.array_equal(tri, levels[lvl][1]) and np.abs(xyz - levels[lvl][0]).max() < 1e-15
        assert seg.seg_step(st, steps) == steps
        got = seg.seg_energy(st)["total"]
        assert _rel(got, ref[lvl][1]["total"]) < TOL[prec], (lvl, got, ref[lvl][1]["total"])
