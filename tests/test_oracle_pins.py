"""Pins of the FP64 oracle to things other than itself.

Each test checks one part of the oracle against what the paper or the
mathematics fixes: closed forms stated in the paper, textbook routines
(dense LAPACK eigen/linear solves, an ODE integrator), independent
quadrature, exact invariants, or a value printed in the paper (tests/golden).
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import solve_ivp

import workload as w
from oracle import seg_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


@pytest.fixture(scope="module")
def sph3():
    xyz, tri = w.icosphere(3)
    M, K = o.assemble(xyz, tri)
    return xyz, tri, M, K


# ---------------------------------------------------------------- assembly


def test_mass_total_is_polyhedral_area_and_converges_to_4pi():
    errs = []
    for L in (2, 3, 4):
        xyz, tri = w.icosphere(L)
        M, _ = o.assemble(xyz, tri)
        one = np.ones(xyz.shape[0])
        area = o.triangle_areas(xyz, tri).sum()
        assert abs(one @ (M @ one) - area) < 1e-13 * area
        errs.append(4 * math.pi - area)
    # inscribed polyhedron: area below 4 pi, error O(h^2) (factor ~4 per level)
    assert all(e > 0 for e in errs)
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_stiffness_annihilates_constants_and_symmetry(sph3):
    xyz, tri, M, K = sph3
    one = np.ones(xyz.shape[0])
    assert np.abs(K @ one).max() < 1e-13 * abs(K).max()
    assert abs(K - K.T).max() < 1e-15 * abs(K).max()
    assert abs(M - M.T).max() == 0.0


def test_stiffness_equals_cotangent_formula(sph3):
    """Independent closed form: K_ij = -(cot a_ij + cot b_ij)/2 off the diagonal."""
    xyz, tri, M, K = sph3
    n = xyz.shape[0]
    Kc = np.zeros((n, n))
    for f in tri:
        for k in range(3):
            i, j, opp = f[(k + 1) % 3], f[(k + 2) % 3], f[k]
            e1 = xyz[i] - xyz[opp]
            e2 = xyz[j] - xyz[opp]
            cot = np.dot(e1, e2) / np.linalg.norm(np.cross(e1, e2))
            Kc[i, j] -= 0.5 * cot
            Kc[j, i] -= 0.5 * cot
    np.fill_diagonal(Kc, -Kc.sum(axis=1))
    assert np.abs(K.toarray() - Kc).max() < 1e-12 * np.abs(Kc).max()


def test_mass_matches_quadrature_of_basis_products():
    xyz, tri = w.icosphere(1)
    M, _ = o.assemble(xyz, tri)
    n = xyz.shape[0]
    # M_ij = int phi_i phi_j via the degree-4 Gauss rule applied to nodal unit vectors
    E = np.eye(n)
    Uq, W = o.pointwise_at_quadrature(xyz, tri, E)
    Mq = np.einsum("fq,fqi,fqj->ij", W, Uq, Uq)
    assert np.abs(M.toarray() - Mq).max() < 1e-15


def test_sphere_spectrum_l_l_plus_1():
    """Generalised eigenvalues of (K, M) approach l(l+1) with multiplicity 2l+1."""
    errs = []
    for L in (2, 3):
        xyz, tri = w.icosphere(L)
        M, K = o.assemble(xyz, tri)
        lam = sla.eigh(K.toarray(), M.toarray(), eigvals_only=True)[:25]
        exact = np.concatenate([[l * (l + 1)] * (2 * l + 1) for l in range(5)])
        assert abs(lam[0]) < 1e-10
        rel = np.abs(lam[1:] - exact[1:]) / exact[1:]
        errs.append(rel.max())
        # multiplicity 2l+1: the cluster of each l is far tighter than the gaps
        start = 0
        for l in range(5):
            cl = lam[start:start + 2 * l + 1]
            assert np.ptp(cl) < 0.02 * (l + 1)
            start += 2 * l + 1
    assert errs[1] < 0.04
    assert errs[1] < errs[0] / 3  # O(h^2)


# ---------------------------------------------------------------- step 1


def test_heat_step_pcg_equals_dense_solve():
    xyz, tri = w.icosphere(2)
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, w.uniform01(11, xyz.shape[0], 3))
    a = o.heat_step(M, K, 1e-2, U)
    b = o.heat_step(M, K, 1e-2, U, solver="direct")
    assert np.abs(a - b).max() < 1e-13


def test_heat_step_on_discrete_eigenvector(sph3):
    """K v = lam M v  =>  (M + tau K)^{-1} M v = v / (1 + tau lam)."""
    xyz, tri, M, K = sph3
    lam, V = sla.eigh(K.toarray(), M.toarray())
    tau = 3e-3
    idx = [0, 2, 7, 20]
    out = o.heat_step(M, K, tau, V[:, idx])
    expect = V[:, idx] / (1 + tau * lam[idx])[None, :]
    assert np.abs(out - expect).max() < 1e-12 * np.abs(expect).max()


# ---------------------------------------------------------------- step 2


def test_segregation_step_solves_the_nodal_ode():
    """Compare with a numerical integration of the step-2 ODE over [t_k, t_k + tau]."""
    rng = np.random.default_rng(3)
    tau, eps = 2e-3, 0.05
    for m in (2, 3, 5):
        Ut = rng.uniform(-0.2, 1.5, size=(4, m))
        out = o.segregation_step(Ut, tau, eps)
        for z in range(Ut.shape[0]):
            ut = Ut[z]
            coef = np.array([(2.0 / eps ** 2) * sum(ut[j] ** 2 for j in range(m) if j != i) for i in range(m)])
            sol = solve_ivp(lambda t, y: -coef * y, (0.0, tau), ut, rtol=1e-12, atol=1e-14, method="DOP853")
            assert np.abs(sol.y[:, -1] - out[z]).max() < 1e-10


def test_segregation_step_identity_cases():
    rng = np.random.default_rng(4)
    U1 = rng.uniform(size=(20, 1))
    assert np.array_equal(o.segregation_step(U1, 1e-3, 1e-2), U1)  # m = 1: no coupling
    oh = w.initial_values("onehot", 9, 30, 4) * 2.5  # disjoint supports
    assert np.array_equal(o.segregation_step(oh, 1e-3, 1e-2), oh)


# ---------------------------------------------------------------- step 3


def test_normalise_gives_unit_l2_by_quadrature(sph3):
    xyz, tri, M, K = sph3
    Uh = w.uniform01(5, xyz.shape[0], 4) * 3.0
    U = o.normalise(M, Uh)
    Uq, W = o.pointwise_at_quadrature(xyz, tri, U)
    l2 = np.einsum("fq,fqi->i", W, Uq * Uq)
    assert np.abs(l2 - 1).max() < 1e-13


# ---------------------------------------------------------------- full step


def test_constant_state_is_a_fixed_point(sph3):
    xyz, tri, M, K = sph3
    area = o.triangle_areas(xyz, tri).sum()
    U = np.full((xyz.shape[0], 3), 1.0 / math.sqrt(area))
    out = o.step(M, K, 1e-3, 0.1, U)
    assert np.abs(out - U).max() < 1e-13


def test_eigenvector_is_a_fixed_point_without_coupling(sph3):
    xyz, tri, M, K = sph3
    lam, V = sla.eigh(K.toarray(), M.toarray())
    U = V[:, [1, 5]] / np.sqrt(np.einsum("zi,zi->i", V[:, [1, 5]], M @ V[:, [1, 5]]))
    U *= np.sign(U[np.abs(U).argmax(0), [0, 1]])
    out = o.step(M, K, 1e-2, 1e30, U)
    assert np.abs(out - U).max() < 1e-12


def test_step_with_direct_solver_equals_pcg_brute_force():
    xyz, tri = w.icosphere(1)
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, w.uniform01(2, xyz.shape[0], 3))
    a, b = U, U
    for _ in range(5):
        a = o.step(M, K, 1e-2, 0.2, a)
        b = o.step(M, K, 1e-2, 0.2, b, solver="direct")
    assert np.abs(a - b).max() < 1e-13


# ---------------------------------------------------------------- energies


def test_s_eps_constant_state_closed_form(sph3):
    xyz, tri, M, K = sph3
    area = o.triangle_areas(xyz, tri).sum()
    for m, eps in [(3, 0.5), (5, 0.1)]:
        U = np.full((xyz.shape[0], m), 1.0 / math.sqrt(area))
        got = o.s_eps(xyz, tri, U, eps)
        assert abs(got - m * (m - 1) / (eps ** 2 * area)) < 1e-12 * got
        assert abs(o.dirichlet(K, U)).max() < 1e-12


def test_s_eps_single_triangle_monomials():
    """int_T lam_a^2 lam_b^2 = |T|/90 and int_T lam_a^4 = |T|/15 (2|T| a!b!c!/(a+b+c+2)!)."""
    xyz = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.3, 1.7, 0.4]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    area = o.triangle_areas(xyz, tri)[0]
    U = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])  # u1 = lam_0, u2 = lam_1
    assert abs(o.s_eps(xyz, tri, U, 1.0) - 2 * area / 90) < 1e-15
    U = np.array([[1.0, 1.0], [0.0, 0.0], [0.0, 0.0]])  # u1 = u2 = lam_0
    assert abs(o.s_eps(xyz, tri, U, 1.0) - 2 * area / 15) < 1e-15
    U = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    assert abs(o.s_eps(xyz, tri, U, 0.5) - 6 * area / 90 / 0.25) < 1e-14


def test_hemispheres_sum_to_4():
    ref = _golden("closed_forms.txt")["hemispheres_total"]
    errs = []
    for L in (3, 4, 5):
        xyz, tri = w.icosphere(L)
        M, K = o.assemble(xyz, tri)
        U = np.stack([np.maximum(xyz[:, 2], 0), np.maximum(-xyz[:, 2], 0)], 1)
        U = o.normalise(M, U)
        errs.append(abs(o.dirichlet(K, U).sum() - ref))
    assert errs[2] < 0.012 and errs[2] < errs[1] < errs[0]


def test_y_partition_sum_to_45_over_4():
    g = _golden("closed_forms.txt")
    errs = []
    for L in (3, 4, 5):
        xyz, tri = w.icosphere(L)
        M, K = o.assemble(xyz, tri)
        U = o.normalise(M, o.y_partition(xyz))
        D = o.dirichlet(K, U)
        errs.append(abs(D.sum() - g["y_partition_total"]))
        # the three lunes are congruent: equal eigenvalue estimates
        assert np.ptp(D) < 0.1 * abs(D.mean() - g["y_partition_eigenvalue"]) + 0.05
    assert errs[2] < 0.1 and errs[2] < 0.7 * errs[1] < 0.7 * 0.7 * errs[0]


def test_lambda_formula_sums_to_dirichlet_plus_twice_s_eps(sph3):
    xyz, tri, M, K = sph3
    U = o.initial_state(M, w.uniform01(8, xyz.shape[0], 4))
    eps = 0.3
    lam = o.lambda_cl(xyz, tri, K, U, eps)
    e = o.energy(xyz, tri, K, U, eps)
    assert abs(lam.sum() - (e["dirichlet"] + 2 * e["s_eps"])) < 1e-12 * lam.sum()
    assert e["functional"] <= lam.sum()


def functional_pin_errors(energy_fn, xyz, tri, M, K):
    """Relative errors of the functional of Problem 2.1 against two things
    that fix it: (a) half the sum of the eigenvalue estimates of Sec. 1.1
    (summing lambda_i over i gives sum D_i + 2 S_eps, which is twice
    E^{eps,h} = 0.5 sum D_i + S_eps exactly); (b) for m = 1 (no coupling,
    S_eps = 0) and u an M-normalised generalised eigenvector K v = lambda M v
    from LAPACK, E^{eps,h} = lambda / 2 and the total energy = lambda."""
    U = o.initial_state(M, w.uniform01(8, xyz.shape[0], 4))
    eps = 0.3
    e = energy_fn(xyz, tri, K, U, eps)
    lam = o.lambda_cl(xyz, tri, K, U, eps)
    err_a = abs(e["functional"] - 0.5 * lam.sum()) / (0.5 * lam.sum())
    ev, V = sla.eigh(K.toarray(), M.toarray())
    err_b = 0.0
    for k in (1, 4, 9):  # eigenvalues near l(l+1) = 2, 6, 12
        v = V[:, k:k + 1]
        e1 = energy_fn(xyz, tri, K, v, eps)
        err_b = max(err_b, abs(e1["functional"] - 0.5 * ev[k]) / ev[k], abs(e1["total"] - ev[k]) / ev[k])
    return err_a, err_b


def test_functional_is_half_the_eigenvalue_sum_and_half_an_eigenvalue(sph3):
    xyz, tri, M, K = sph3
    err_a, err_b = functional_pin_errors(o.energy, xyz, tri, M, K)
    assert err_a < 1e-13
    assert err_b < 1e-12


def test_table_u_eps_first_row():
    """Flow at eps = 0.5 from random one-hot data reaches the printed energy and S_eps."""
    g = _golden("table_u_eps_row1.txt")
    xyz, tri = w.icosphere(4)
    M, K = o.assemble(xyz, tri)
    U0 = w.initial_values("onehot", 1, xyz.shape[0], int(g["m"]))
    U, k, hist = o.run(xyz, tri, U0, tau=0.1, eps=g["eps"], nsteps=400, tol=1e-9, check_every=10)
    e = o.energy(xyz, tri, K, U, g["eps"])
    assert k < 400
    assert abs(e["total"] - g["energy"]) < 3e-3
    assert abs(e["s_eps"] - g["s_eps"]) < 3e-3


# ---------------------------------------------------------------- invariants


def test_component_permutation_and_vertex_renumbering():
    xyz, tri = w.icosphere(2)
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, w.uniform01(21, xyz.shape[0], 4))
    tau, eps = 1e-3, 0.1
    base = o.step(M, K, tau, eps, U)
    perm = [2, 0, 3, 1]
    permuted = o.step(M, K, tau, eps, U[:, perm])
    assert np.abs(permuted - base[:, perm]).max() < 1e-14
    rng = np.random.default_rng(0)
    p = rng.permutation(xyz.shape[0])
    inv = np.argsort(p)
    xyz2, tri2 = xyz[p], inv[tri].astype(np.int32)
    M2, K2 = o.assemble(xyz2, tri2)
    out2 = o.step(M2, K2, tau, eps, U[p])
    assert np.abs(out2 - base[p]).max() < 1e-13
    e1 = o.energy(xyz, tri, K, base, eps)["total"]
    e2 = o.energy(xyz2, tri2, K2, out2, eps)["total"]
    assert abs(e1 - e2) < 1e-12 * e1


def test_unit_norm_after_every_step_and_energy_decreases(sph3):
    xyz, tri, M, K = sph3
    U = o.initial_state(M, w.initial_values("uniform", 5, xyz.shape[0], 4))
    prev = o.energy(xyz, tri, K, U, 0.05)
    for _ in range(25):
        U = o.step(M, K, 1e-3, 0.05, U)
        assert np.abs(o.l2_norms(M, U) - 1).max() < 1e-14
        e = o.energy(xyz, tri, K, U, 0.05)
        assert e["functional"] <= prev["functional"] + 1e-12
        assert e["total"] <= prev["total"] + 1e-12
        prev = e


def test_labels_ties_and_v_flag():
    U = np.array([[0.5, 0.5, 0.0], [0.1, 0.9, 0.3], [0.4, 0.3, 0.2], [0.0, 0.0, 0.0]])
    am, v = o.labels(U)
    assert am.tolist() == [0, 1, 0, 0]
    # v = u_i - sum_{j != i} u_j: 0 (not > 0), 0.5, -0.1, 0
    assert v.tolist() == [0, 1, 0, 0]


def test_stop_rule_stops_at_first_quiet_check(sph3):
    xyz, tri, M, K = sph3
    area = o.triangle_areas(xyz, tri).sum()
    U0 = np.full((xyz.shape[0], 3), 2.0)  # constant: energy does not change
    U, k, hist = o.run(xyz, tri, U0, tau=1e-2, eps=0.3, nsteps=100, tol=1e-10)
    assert o.check_interval(1e-2) == 10
    assert k == 10 and len(hist) == 2
    assert abs(hist[0] - o.constant_state_s_eps(3, area, 0.3)) < 1e-10


# ------------------------------------------- variants and continuation pins


def test_lumped_mass_is_vertex_quadrature(sph3):
    """M_L = diag(|star(z)|/3) equals the row sums of the consistent mass
    matrix (sum_b |T|(1 + delta_ab)/12 = |T|/3), integrates constants and
    linear functions exactly on every flat triangle (vertex rule)."""
    xyz, tri, M, K = sph3
    ML = o.lumped_mass(xyz, tri)
    assert np.abs(ML.diagonal() - np.asarray(M.sum(axis=1)).ravel()).max() < 1e-16
    assert ML.nnz == xyz.shape[0]
    one = np.ones(xyz.shape[0])
    assert abs(one @ ML @ one - o.triangle_areas(xyz, tri).sum()) < 1e-13
    # a linear function f = c.x: int_Gamma_h f by the exact centroid rule on each
    # flat triangle equals 1^T M_L f
    c = np.array([0.3, -0.7, 0.2])
    f = xyz @ c
    cent = xyz[tri].mean(1) @ c
    assert abs(one @ ML @ f - (o.triangle_areas(xyz, tri) * cent).sum()) < 1e-14


def test_energy_p_power_means():
    lam = np.array([2.0, 6.0, 12.0, 20.0])
    assert o.energy_p(lam, 1) == pytest.approx(lam.mean(), rel=1e-15)
    assert o.energy_p(lam, 2) == pytest.approx(math.sqrt((lam ** 2).mean()), rel=1e-15)
    assert o.energy_p(lam, math.inf) == 20.0
    ps = [1, 1.5, 2, 4, 8, 32]
    vals = [o.energy_p(lam, p) for p in ps]
    assert all(a <= b for a, b in zip(vals, vals[1:]))  # power-mean inequality
    assert o.energy_p(lam, 400) == pytest.approx(20.0 * 0.25 ** (1 / 400), rel=1e-3)
    assert o.energy_p(np.full(5, 7.5), 3.7) == pytest.approx(7.5, rel=1e-14)
    with pytest.raises(ValueError):
        o.energy_p(lam, 0.5)


def test_prolongation_is_p1_interpolation():
    """Before projection the fine vertices are edge midpoints of the coarse
    polyhedron, where a P1 function takes the mean of the edge's end values:
    affine functions are reproduced exactly, constants stay constant."""
    x, t = w.torus(9, 7, 1.0, 0.4)
    xf, tf, par = w.refine(x, t, ("none",))
    A = np.array([[0.5, -1.0], [2.0, 0.25], [-0.3, 0.8]])
    b = np.array([1.5, -2.0])
    U = x @ A + b
    assert np.abs(o.prolong(U, par) - (xf @ A + b)).max() < 1e-14
    assert np.array_equal(o.prolong(np.full((len(x), 3), 0.7), par), np.full((len(xf), 3), 0.7))
    # on the sphere the values are those at the unprojected midpoints
    x, t = w.icosphere(1)
    xf, tf, par = w.refine(x, t, ("sphere",))
    U = x @ A
    mid = 0.5 * (x[par[:, 0]] + x[par[:, 1]])
    assert np.abs(o.prolong(U, par) - mid @ A).max() < 1e-15


def test_continuation_first_level_is_a_plain_run_and_levels_chain():
    x0, t0 = w.icosphere(1)
    x1, t1, p1 = w.refine(x0, t0, ("sphere",))
    U0 = w.initial_values("uniform", 5, len(x0), 3)
    eps, tau, steps = 0.2, 2e-3, 4
    out = o.continuation([(x0, t0, None), (x1, t1, p1)], U0, eps, tau, steps)
    M, K = o.assemble(x0, t0)
    U = o.initial_state(M, U0)
    for _ in range(steps):
        U = o.step(M, K, tau, eps, U)
    assert np.abs(out[0][0] - U).max() < 1e-13
    # level 1 = a plain run from the normalised interpolant with eps/2, tau/2
    M1, K1 = o.assemble(x1, t1)
    V = o.normalise(M1, o.prolong(U, p1))
    for _ in range(steps):
        V = o.step(M1, K1, tau / 2, eps / 2, V)
    assert np.abs(out[1][0] - V).max() < 1e-13
    assert out[1][1]["total"] == pytest.approx(o.energy(x1, t1, K1, V, eps / 2)["total"], rel=1e-14)
