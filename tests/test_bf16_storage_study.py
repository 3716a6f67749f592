"""Study behind the storage format of the state (no GPU).

BF16 storage of u (FP32 arithmetic, FP64 reductions) is adopted only if the
total energy stays within 1e-5 (relative) of the float64 run.  The oracle's
float64 step with the stored state rounded after every step measures what a
storage format costs: float32 storage stays far inside the bar (the mixed
mode's state format), bfloat16 (8-bit significand) misses it by orders of
magnitude, so the state is not stored in BF16.  The narrower use -- only the
CG search directions p and q = A p (buffers P and Q) in BF16, with the
predicted start of the CUDA path -- misses the bar too (by 1.4x to 5.5x), so
P and Q stay in float32.
"""

import numpy as np
import pytest

import workload as w
from oracle import seg_oracle as o


def _round_bf16(x):
    """Round float64 values to bfloat16 (round to nearest, ties to even) via float32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _round_f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def test_bf16_rounding_is_round_to_nearest_even():
    assert _round_bf16(np.array([1.0]))[0] == 1.0
    assert _round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0  # tie -> even
    assert _round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert _round_bf16(np.array([1.0 + 2.0 ** -7]))[0] == 1.0 + 2.0 ** -7  # representable
    x = np.random.default_rng(0).uniform(0.5, 2.0, 1000)
    assert np.abs(_round_bf16(x) - x).max() <= 2.0 ** -8 * 2.0


@pytest.mark.parametrize("m,eps,tau", [(3, 1e-2, 1e-4), (8, 2e-2, 1e-4)])
def test_storage_format_energy_error(m, eps, tau):
    xyz, tri = w.icosphere(4)
    M, K = o.assemble(xyz, tri)
    U0 = o.initial_state(M, w.initial_values("uniform", 3, len(xyz), m))
    runs = {}
    for name, rnd in (("f64", lambda u: u), ("f32", _round_f32), ("bf16", _round_bf16)):
        U = rnd(U0)
        for _ in range(60):
            U = rnd(o.step(M, K, tau, eps, U, rtol=1e-12))
        runs[name] = o.energy(xyz, tri, K, o.normalise(M, U), eps)["total"]
    err32 = abs(runs["f32"] - runs["f64"]) / runs["f64"]
    err16 = abs(runs["bf16"] - runs["f64"]) / runs["f64"]
    assert err32 < 1e-6
    assert err16 > 1e-4  # the 1e-5 bar is missed by more than 10x: BF16 storage is not adopted


def _pcg_stored_directions(A, b, x0, rnd, rtol):
    """Jacobi-PCG as the oracle's, with the search direction p and q = A p
    rounded by `rnd` where they are formed (the buffers P and Q of the CUDA
    passes); everything else float64."""
    dinv = 1.0 / A.diagonal()
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    z = dinv * r
    p = rnd(z)
    rz = r @ z
    k = 0
    while np.linalg.norm(r) > rtol * bnorm and k < 10000:
        q = rnd(A @ p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = rnd(z + beta * p)
        k += 1
    return x


def _run_with_predicted_start(M, K, tau, eps, U, rnd, rtol, steps):
    """Algorithm 2.2 steps whose solves start, per component, from the
    correction extrapolated from the last three solves (3 y_k - 3 y_{k-1} +
    y_{k-2}) where its residual is smaller than the plain warm start's -- the
    start the CUDA path uses -- with the directions stored through `rnd`."""
    A = (M + tau * K).tocsr()
    hist = []
    for _ in range(steps):
        B = M @ U
        Ut = np.empty_like(U)
        for i in range(U.shape[1]):
            x0 = U[:, i].copy()
            if len(hist) == 3:
                yp = 3 * hist[2][:, i] - 3 * hist[1][:, i] + hist[0][:, i]
                if np.linalg.norm(B[:, i] - A @ (x0 + yp)) < np.linalg.norm(B[:, i] - A @ x0):
                    x0 += yp
            Ut[:, i] = _pcg_stored_directions(A, B[:, i], x0, rnd, rtol)
        hist = (hist + [Ut - U])[-3:]
        U = o.normalise(M, o.segregation_step(Ut, tau, eps))
    return U


@pytest.mark.parametrize("m,eps,tau", [(3, 1e-2, 1e-4), (6, 5e-3, 2e-5)])
def test_search_directions_in_bf16_miss_the_bar(m, eps, tau):
    """The narrower use of BF16: only the CG search directions p and q = A p
    stored in bfloat16 (whose rounding the CG recurrences partly absorb),
    with the predicted start and the mixed mode's tolerance (rtol 1e-7).
    After 120 steps on the level-4 sphere the total energy moves by more
    than the 1e-5 bar (1.4e-5 and 5.5e-5 when written); float32 directions,
    the mixed mode's format, stay below 1e-8.  P and Q stay in float32."""
    xyz, tri = w.icosphere(4)
    M, K = o.assemble(xyz, tri)
    U0 = o.initial_state(M, w.initial_values("uniform", 3, len(xyz), m))
    e = {}
    for name, rnd in (("f64", lambda v: v), ("f32", _round_f32), ("bf16", _round_bf16)):
        U = _run_with_predicted_start(M, K, tau, eps, U0.copy(), rnd, 1e-7, 120)
        e[name] = o.energy(xyz, tri, K, U, eps)["total"]
    assert abs(e["f32"] - e["f64"]) / e["f64"] < 1e-8
    assert abs(e["bf16"] - e["f64"]) / e["f64"] > 1e-5
