"""The oracle's pins are sensitive: plausible mistakes planted in the oracle fail them.

Each case monkeypatches one oracle function with a wrong variant (a dropped
factor, a wrong index, a wrong norm, a transposed sign) and checks that the
corresponding pin quantity moves far outside its tolerance.  Mistakes are
planted only in the CPU oracle.
"""

import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import solve_ivp

import workload as w
from oracle import seg_oracle as o


@pytest.fixture(scope="module")
def sph2():
    xyz, tri = w.icosphere(2)
    M, K = o.assemble(xyz, tri)
    return xyz, tri, M, K


def _ode_pin_error(seg):
    rng = np.random.default_rng(3)
    tau, eps, m = 2e-3, 0.05, 3
    Ut = rng.uniform(0.1, 1.5, size=(3, m))
    out = seg(Ut, tau, eps)
    err = 0.0
    for z in range(Ut.shape[0]):
        ut = Ut[z]
        coef = np.array([(2.0 / eps ** 2) * sum(ut[j] ** 2 for j in range(m) if j != i) for i in range(m)])
        sol = solve_ivp(lambda t, y: -coef * y, (0.0, tau), ut, rtol=1e-12, atol=1e-14, method="DOP853")
        err = max(err, np.abs(sol.y[:, -1] - out[z]).max())
    return err


def test_exponent_factor_without_the_2_is_caught():
    def wrong(Ut, tau, eps):
        sq = Ut * Ut
        return Ut * np.exp(-(tau / eps ** 2) * (sq.sum(1, keepdims=True) - sq))

    assert _ode_pin_error(o.segregation_step) < 1e-10
    assert _ode_pin_error(wrong) > 1e-3


def test_gauss_seidel_or_self_term_is_caught():
    def self_term(Ut, tau, eps):
        sq = Ut * Ut
        return Ut * np.exp(-(2 * tau / eps ** 2) * sq.sum(1, keepdims=True))

    assert _ode_pin_error(self_term) > 1e-3


def test_rhs_without_mass_matrix_is_caught(sph2):
    xyz, tri, M, K = sph2
    lam, V = sla.eigh(K.toarray(), M.toarray())
    tau = 3e-3
    A = (M + tau * K).toarray()
    wrong = np.linalg.solve(A, V[:, [3]])  # forgot M on the right-hand side
    expect = V[:, [3]] / (1 + tau * lam[3])
    assert np.abs(wrong - expect).max() > 1e-3 * np.abs(expect).max()


def test_wrong_sign_of_stiffness_is_caught(sph2):
    xyz, tri, M, K = sph2
    lam, V = sla.eigh(K.toarray(), M.toarray())
    tau = 3e-3
    wrong = o.heat_step(M, -K, tau, V[:, [3]], solver="direct")
    expect = V[:, [3]] / (1 + tau * lam[3])
    assert np.abs(wrong - expect).max() > 1e-3 * np.abs(expect).max()


def test_euclidean_instead_of_l2_normalisation_is_caught(sph2):
    xyz, tri, M, K = sph2
    Uh = w.uniform01(5, xyz.shape[0], 3)
    wrong = Uh / np.linalg.norm(Uh, axis=0, keepdims=True)
    Uq, W = o.pointwise_at_quadrature(xyz, tri, wrong)
    l2 = np.einsum("fq,fqi->i", W, Uq * Uq)
    assert np.abs(l2 - 1).max() > 0.1


def test_s_eps_missing_eps_or_pair_factor_is_caught(sph2, monkeypatch):
    xyz, tri, M, K = sph2
    area = o.triangle_areas(xyz, tri).sum()
    U = np.full((xyz.shape[0], 3), 1.0 / math.sqrt(area))
    exact = 3 * 2 / (0.25 * area)

    def half_pairs(xyz, tri, U, eps):  # counts each unordered pair once
        Uq, Wq = o.pointwise_at_quadrature(xyz, tri, U)
        sq = Uq * Uq
        pair = 0.5 * (sq.sum(-1) ** 2 - (sq * sq).sum(-1))
        return float((Wq * pair).sum()) / eps ** 2

    assert abs(o.s_eps(xyz, tri, U, 0.5) - exact) < 1e-12 * exact
    assert abs(half_pairs(xyz, tri, U, 0.5) - exact) > 0.4 * exact


def test_transposed_gradient_map_is_caught(monkeypatch):
    """A metric inverse applied on the wrong side breaks the cotangent pin."""
    xyz, tri = w.icosphere(1)

    def wrong_grads(xyz, tri):
        x0, x1, x2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
        G = np.stack([x1 - x0, x2 - x0], axis=2)
        ref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
        return np.einsum("fki,bi->fbk", G, ref)  # dropped the metric inverse

    good_M, good_K = o.assemble(xyz, tri)
    monkeypatch.setattr(o, "p1_gradients", wrong_grads)
    _, bad_K = o.assemble(xyz, tri)
    assert abs(bad_K - good_K).max() > 0.1 * abs(good_K).max()


def test_planted_mistakes_in_the_variants_fail_their_pins(monkeypatch):
    # prolongation taking one parent only: affine functions are no longer reproduced
    x, t = w.torus(9, 7, 1.0, 0.4)
    xf, tf, par = w.refine(x, t, ("none",))
    U = x @ np.array([[0.5], [2.0], [-0.3]])
    good = np.abs(o.prolong(U, par) - xf @ np.array([[0.5], [2.0], [-0.3]])).max()
    monkeypatch.setattr(o, "prolong", lambda U, parents: U[parents[:, 0]])
    bad = np.abs(o.prolong(U, par) - xf @ np.array([[0.5], [2.0], [-0.3]])).max()
    assert good < 1e-14 and bad > 1e-2
    monkeypatch.undo()
    # lumped mass from the consistent diagonal instead of the row sums
    xyz, tri = w.icosphere(2)
    M, _ = o.assemble(xyz, tri)
    rowsum = np.asarray(M.sum(axis=1)).ravel()
    assert np.abs(o.lumped_mass(xyz, tri).diagonal() - rowsum).max() < 1e-16
    assert np.abs(M.diagonal() - rowsum).max() > 1e-3
    # E_p without the 1/m of the mean
    lam = np.array([2.0, 6.0, 12.0])
    wrong = float(np.sum(lam ** 2) ** 0.5)
    assert abs(o.energy_p(lam, 2) - math.sqrt((lam ** 2).mean())) < 1e-14
    assert abs(wrong - math.sqrt((lam ** 2).mean())) > 1.0


def test_functional_without_the_half_is_caught():
    """A functional with the 1/2 of Problem 2.1 dropped fails its pins."""
    from tests.test_oracle_pins import functional_pin_errors

    xyz, tri = w.icosphere(3)
    M, K = o.assemble(xyz, tri)

    def no_half(xyz, tri, K, U, eps):
        e = o.energy(xyz, tri, K, U, eps)
        e["functional"] = e["dirichlet"] + e["s_eps"]
        return e

    good_a, good_b = functional_pin_errors(o.energy, xyz, tri, M, K)
    bad_a, bad_b = functional_pin_errors(no_half, xyz, tri, M, K)
    assert good_a < 1e-13 and good_b < 1e-12
    assert bad_a > 0.1 and bad_b > 0.4
