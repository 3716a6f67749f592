"""FP64 CPU oracle for the eigenfunction-segregation gradient flow.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU library computes.  Only the test-suite, the smoke
check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it; the library never does.  It shares no code with the CUDA path: it
re-derives the finite-element matrices, the time step and the energies from
the paper (Elliott & Ranner, "A computational approach to an optimal
partition problem on surfaces").

Everything is float64.  Arrays are vertex-major: ``U[z, i]`` is component i
at vertex z.  Inputs (meshes, random initial values) come from ``workload``.

Readings of the paper taken here:

* Step 2 exponent factor is 2*tau/eps^2 (the ODE of Algorithm 2.2 step 2 and
  its practical version agree on the 2; the displayed exact solution drops it).
* Consistent mass matrix in steps 1 and 3 (the L2(Gamma_h) norm of step 3 is
  the consistent one; step 1 is the Galerkin form), nodal values in step 2.
* Reported "total energy" = sum_i D_i + S_eps (the tables of Sec. 3 add the
  eigenvalue estimates and S_eps: e.g. 3 * 3.605 + 0.072 = 10.887), with
  D_i = |u_i|_{H^1}^2; the functional of Problem 2.1 = 0.5 sum_i D_i + S_eps.
  Summing the lambda formula of Sec. 1.1 over i gives sum D_i + 2 S_eps,
  twice the functional (the paper prints E + 2 int F, which does not follow
  from its own definitions).
* The quartic S_eps integrand is integrated exactly (the paper is silent).
* The linear solve of step 1 is done to rtol 1e-14 (the paper gives none;
  with this tolerance the result does not depend on the solver's start).

Parity status: every function below is pinned by tests in
``tests/test_oracle_pins.py`` against closed forms, textbook routines,
independent quadrature or values printed in the paper.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# Sec. 2.1: P1 finite elements on the triangulated surface Gamma_h
# ---------------------------------------------------------------------------


def triangle_areas(xyz, tri):
    """|T| for every flat triangle of Gamma_h (Sec. 2.1)."""
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def p1_gradients(xyz, tri):
    """Tangential gradients of the three nodal basis functions on each triangle.

    On T with vertices x0, x1, x2 the affine map from the reference triangle
    has Jacobian G = [x1 - x0, x2 - x0] (3x2); the reference gradients of the
    barycentric coordinates are (-1,-1), (1,0), (0,1).  The surface gradient of
    a function with reference gradient g is G (G^T G)^{-1} g.
    Returns array (F, 3 basis functions, 3 coordinates).
    """
    x0, x1, x2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    G = np.stack([x1 - x0, x2 - x0], axis=2)  # F x 3 x 2
    g = np.einsum("fki,fkj->fij", G, G)  # metric, F x 2 x 2
    ginv = np.linalg.inv(g)
    ref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])  # basis x ref-coord
    # grad_b = G ginv ref_b
    return np.einsum("fki,fij,bj->fbk", G, ginv, ref)


def assemble(xyz, tri):
    """Mass and stiffness matrices of S_h on Gamma_h (Sec. 2.1, Algorithm 2.2).

    M_ij = int phi_i phi_j,  K_ij = int grad phi_i . grad phi_j, summed over
    triangles; on one triangle int phi_a phi_b = |T| (1 + delta_ab) / 12 and
    the gradients are constant.  Returns scipy CSR matrices with sorted
    indices.
    """
    n = xyz.shape[0]
    area = triangle_areas(xyz, tri)
    grads = p1_gradients(xyz, tri)
    Me = area[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None] / 12.0
    Ke = area[:, None, None] * np.einsum("fak,fbk->fab", grads, grads)
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    M.sum_duplicates()
    K.sum_duplicates()
    M.sort_indices()
    K.sort_indices()
    return M, K


# ---------------------------------------------------------------------------
# Algorithm 2.2, step 1: one implicit Euler step of the heat equation
# ---------------------------------------------------------------------------


def pcg(A, b, x0, rtol=1e-14, maxit=10000):
    """Textbook conjugate gradients with the Jacobi (diagonal) preconditioner.

    Stops when ||b - A x||_2 (the recursively updated residual) is at most
    rtol * ||b||_2.  Returns (x, iterations).
    """
    dinv = 1.0 / A.diagonal()
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    k = 0
    while np.linalg.norm(r) > rtol * bnorm and k < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        k += 1
    return x, k


def heat_step(M, K, tau, U, rtol=1e-14, solver="pcg"):
    """Algorithm 2.2 step 1 for every component i.

    The weak form int (u~ - u_k)/tau chi + grad u~ . grad chi = 0 for all chi
    in S_h is the linear system (M + tau K) u~_i = M u_i^k.  The default solver
    is Jacobi-PCG warm-started at u_i^k (the paper uses preconditioned CG);
    solver="direct" uses a dense LU solve (small meshes only).
    """
    A = (M + tau * K).tocsr()
    B = M @ U
    out = np.empty_like(U)
    if solver == "direct":
        Ad = A.toarray()
        return np.linalg.solve(Ad, B)
    for i in range(U.shape[1]):
        out[:, i], _ = pcg(A, B[:, i], U[:, i], rtol=rtol)
    return out


# ---------------------------------------------------------------------------
# Algorithm 2.2, step 2: the segregation ODE solved exactly at every node
# ---------------------------------------------------------------------------


def segregation_step(Ut, tau, eps):
    """Practical version of Algorithm 2.2 step 2 (Jacobi form).

    At each node z: (a) square every component, (b) S = sum of the squares,
    (c) u^_i = u~_i exp(-(2 tau / eps^2) (S - u~_i^2)).  All i use the
    pre-step values u~ (Jacobi, not Gauss-Seidel).
    """
    sq = Ut * Ut
    S = sq.sum(axis=1, keepdims=True)
    return Ut * np.exp(-(2.0 * tau / eps ** 2) * (S - sq))


# ---------------------------------------------------------------------------
# Algorithm 2.2, step 3: L2(Gamma_h) renormalisation
# ---------------------------------------------------------------------------


def l2_norms(M, U):
    """||u_i||_{L2(Gamma_h)} = sqrt(u_i^T M u_i) for every component."""
    return np.sqrt(np.einsum("zi,zi->i", U, M @ U))


def normalise(M, Uh):
    """Algorithm 2.2 step 3: u_i^{k+1} = u^_i / ||u^_i||_{L2(Gamma_h)}."""
    return Uh / l2_norms(M, Uh)[None, :]


def step(M, K, tau, eps, U, rtol=1e-14, solver="pcg"):
    """One full step of Algorithm 2.2: heat step, segregation ODE, normalisation."""
    Ut = heat_step(M, K, tau, U, rtol=rtol, solver=solver)
    Uh = segregation_step(Ut, tau, eps)
    return normalise(M, Uh)


def initial_state(M, U0):
    """Sec. 2.2 initial condition: each component of the drawn values normalised in L2."""
    return normalise(M, U0)


# ---------------------------------------------------------------------------
# Energies (Problem 2.1, eq. (Seps-u), the lambda formula of Sec. 1.1)
# ---------------------------------------------------------------------------


def _gauss_triangle_rule(n=3):
    """Collapsed-coordinate (Duffy) Gauss-Legendre rule on the reference triangle.

    Maps (s, t) in [0,1]^2 to barycentrics (1-s, s(1-t), s t) with Jacobian
    s (relative to the reference area 1/2 normalised to 1: weights sum to 1).
    With n points per direction it integrates polynomials of degree <= 2n-2
    exactly (degree 4 needs n = 3).
    Returns (bary[q, 3], w[q]) with sum(w) == 1 (integral = |T| * sum w f).
    """
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    S, Tt = np.meshgrid(x, x, indexing="ij")
    WS, WT = np.meshgrid(w, w, indexing="ij")
    s = S.ravel()
    t = Tt.ravel()
    bary = np.stack([1.0 - s, s * (1.0 - t), s * t], axis=1)
    wq = (WS * WT).ravel() * s * 2.0  # reference-triangle area 1/2 -> weights sum to 1
    return bary, wq


def pointwise_at_quadrature(xyz, tri, U, n=3):
    """Values of the P1 functions at the quadrature points: (F, q, m) plus weights |T| w_q."""
    bary, wq = _gauss_triangle_rule(n)
    area = triangle_areas(xyz, tri)
    Uq = np.einsum("qa,fam->fqm", bary, U[tri])
    return Uq, area[:, None] * wq[None, :]


def dirichlet(K, U):
    """D_i = int |grad_{Gamma_h} u_i|^2 = u_i^T K u_i (the H^1 semi-norm squared)."""
    return np.einsum("zi,zi->i", U, K @ U)


def s_eps(xyz, tri, U, eps):
    """S_eps = eps^-2 int_{Gamma_h} sum_i sum_{j != i} u_i^2 u_j^2 (eq. (Seps-u)).

    The integrand is a quartic on every flat triangle; the degree-4-exact
    Gauss rule integrates it exactly.
    """
    Uq, W = pointwise_at_quadrature(xyz, tri, U)
    sq = Uq * Uq
    pair = sq.sum(-1) ** 2 - (sq * sq).sum(-1)  # sum_{i != j} u_i^2 u_j^2
    return float((W * pair).sum()) / eps ** 2


def lambda_cl(xyz, tri, K, U, eps):
    """lambda_i = int |grad u_i|^2 + (2/eps^2) (sum_{j != i} u_j^2) u_i^2 (Sec. 1.1)."""
    Uq, W = pointwise_at_quadrature(xyz, tri, U)
    sq = Uq * Uq
    others = sq.sum(-1, keepdims=True) - sq
    coupling = np.einsum("fq,fqi->i", W, others * sq)
    return dirichlet(K, U) + 2.0 * coupling / eps ** 2


def energy(xyz, tri, K, U, eps):
    """Energy record of a normalised state.

    total      = sum_i D_i + S_eps  (the "total energy" of the tables of Sec. 3)
    functional = 0.5 sum_i D_i + S_eps  (E^{eps,h} of Problem 2.1)
    """
    D = dirichlet(K, U)
    S = s_eps(xyz, tri, U, eps)
    return {
        "total": float(D.sum() + S),
        "functional": float(0.5 * D.sum() + S),
        "dirichlet": float(D.sum()),
        "s_eps": S,
        "D": D,
    }


# ---------------------------------------------------------------------------
# Partition read-out (Sec. 1.1 and eq. (vi))
# ---------------------------------------------------------------------------


def labels(U):
    """argmax_i u_i(z) (lowest index on ties) and the flag v_i(z) > 0 for that i.

    v_i = u_i - sum_{j != i} u_j (eq. (vi)).
    """
    am = np.argmax(U, axis=1).astype(np.int32)
    ui = U[np.arange(U.shape[0]), am]
    v = ui - (U.sum(axis=1) - ui)
    return am, (v > 0).astype(np.uint8)


# ---------------------------------------------------------------------------
# Time loop with the stopping rule of Sec. 2.2
# ---------------------------------------------------------------------------


def check_interval(tau):
    """M_tau with M_tau * tau = 0.1, rounded to the nearest integer (at least 1)."""
    return max(1, int(round(0.1 / tau)))


def run(xyz, tri, U0, tau, eps, nsteps, tol=1e-6, check_every=None, rtol=1e-14):
    """Run Algorithm 2.2 from the drawn values U0 for at most nsteps steps.

    The energy is evaluated every M_tau steps; the run stops at the first
    check whose change against the previous check is below tol.
    Returns (U, steps_done, energies at the checks).
    """
    M, K = assemble(xyz, tri)
    U = initial_state(M, U0)
    every = check_interval(tau) if check_every is None else check_every
    history = [energy(xyz, tri, K, U, eps)["total"]]
    k = 0
    while k < nsteps:
        U = step(M, K, tau, eps, U, rtol=rtol)
        k += 1
        if k % every == 0:
            e = energy(xyz, tri, K, U, eps)["total"]
            history.append(e)
            if abs(e - history[-2]) < tol:
                break
    return U, k, history


# ---------------------------------------------------------------------------
# Variants and extensions: lumped mass, l^p energies (Problem 1.2),
# continuation with refinement and prolongation (Sec. 3.3)
# ---------------------------------------------------------------------------


def lumped_mass(xyz, tri):
    """Mass matrix of the vertex quadrature int_T f ~ |T|/3 (f(a) + f(b) + f(c)):
    the lumped-mass variant, M_L = diag(|star(z)| / 3), |star(z)| the area of
    the triangles around z.  (The paper uses the consistent M; this variant
    replaces it in steps 1 and 3.)"""
    n = xyz.shape[0]
    area = triangle_areas(xyz, tri)
    d = np.zeros(n)
    for k in range(3):
        np.add.at(d, tri[:, k], area / 3.0)
    return sp.diags(d).tocsr()


def energy_p(lams, p):
    """E_p of Problem 1.2 from the eigenvalue estimates lambda_i:
    ((1/m) sum lambda_i^p)^(1/p) for 1 <= p < inf, max lambda_i for p = inf."""
    lams = np.asarray(lams, dtype=np.float64)
    if p == math.inf:
        return float(lams.max())
    if p < 1:
        raise ValueError("p must be >= 1")
    top = lams.max()  # scaled by the largest value so that lambda^p cannot overflow
    if top == 0.0:
        return 0.0
    return float(top * np.mean((lams / top) ** p) ** (1.0 / p))


def prolong(U, parents):
    """P1 interpolation onto a refined mesh (Sec. 3.3: the previous minimiser
    is the initial condition on the next level).  A fine vertex with parent
    edge (a, b) takes (U[a] + U[b]) / 2 (its value at the edge midpoint of the
    coarse polyhedron); a coarse vertex (a = b) keeps its value."""
    return 0.5 * (U[parents[:, 0]] + U[parents[:, 1]])


def continuation(levels, U0, eps0, tau0, steps, factor=0.5, rtol=1e-14):
    """The refinement rule of Sec. 3.3 run for a fixed number of steps per level.

    levels: list of (xyz, tri, parents) for level 0, 1, ...; parents of level
    l maps its vertices to level l - 1 (ignored for level 0).  Level 0 starts
    from the drawn values U0; every later level starts from the P1
    interpolation of the previous level's final state, with eps and tau
    multiplied by `factor` per level (one global red refinement = two
    bisection levels, each dividing eps and tau by sqrt 2).  Returns a list of
    (U, energy record) per level.
    """
    out = []
    eps, tau = eps0, tau0
    U = None
    for l, (xyz, tri, parents) in enumerate(levels):
        M, K = assemble(xyz, tri)
        if l == 0:
            U = initial_state(M, U0)
        else:
            eps, tau = eps * factor, tau * factor
            U = normalise(M, prolong(U, parents))
        for _ in range(steps):
            U = step(M, K, tau, eps, U, rtol=rtol)
        out.append((U, energy(xyz, tri, K, U, eps)))
    return out


def constant_state_s_eps(m, area, eps):
    """S_eps of u_i = |Gamma_h|^{-1/2} for all i: m (m - 1) / (eps^2 |Gamma_h|)."""
    return m * (m - 1) / (eps ** 2 * area)


def y_partition(xyz):
    """Nodal values of the Y-partition eigenfunctions of Sec. 3.1 (unnormalised).

    theta is the polar angle, phi the azimuth in (-pi, pi];
    u_1 = sin(3 phi/2) sin(theta)^{3/2} on 0 < phi < 2 pi/3,
    u_2 = -sin(3 phi/2) sin(theta)^{3/2} on -2 pi/3 < phi < 0,
    u_3 = sin(3|phi|/2 - pi) sin(theta)^{3/2} on |phi| > 2 pi/3, zero elsewhere.
    """
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    theta = np.arccos(np.clip(z / np.linalg.norm(xyz, axis=1), -1.0, 1.0))
    phi = np.arctan2(y, x)
    st = np.sin(theta) ** 1.5
    U = np.zeros((xyz.shape[0], 3))
    g1 = (phi > 0) & (phi < 2 * math.pi / 3)
    g2 = (phi < 0) & (phi > -2 * math.pi / 3)
    g3 = np.abs(phi) > 2 * math.pi / 3
    U[g1, 0] = np.sin(1.5 * phi[g1]) * st[g1]
    U[g2, 1] = -np.sin(1.5 * phi[g2]) * st[g2]
    U[g3, 2] = np.sin(1.5 * np.abs(phi[g3]) - math.pi) * st[g3]
    return U
