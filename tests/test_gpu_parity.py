"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances (written per test):
  FP64 mode   relative total energy <= 1e-10, max |du| <= 1e-9
  mixed mode  relative total energy <= 1e-5, per-component D_i <= 1e-5,
              labels equal off the interface vertices
Inputs are seeded: meshes and initial values from `workload`, expected values
from `oracle` only.
"""

import numpy as np
import pytest

import workload as w
from oracle import seg_oracle as o
from tests.gpu_helpers import check_labels, lib, make_state, oracle_run, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    return lib()


PRECS = [("fp64", 0, 1e-13, 1e-10), ("mixed", 1, 2e-7, 1e-5)]


@pytest.mark.parametrize("name,prec,utol,etol", PRECS)
@pytest.mark.parametrize("m", [1, 2, 3, 5, 16])
def test_initial_state_and_energy(seg, name, prec, utol, etol, m):
    xyz, tri = w.icosphere(3)
    st = make_state(seg, xyz, tri, 1e-4, m, 0.05, prec, seed=77)
    U = seg.seg_get_u(st)
    M, K = o.assemble(xyz, tri)
    Uo = o.initial_state(M, w.uniform01(77, xyz.shape[0], m))
    assert np.abs(U - Uo).max() <= utol * np.abs(Uo).max()
    e = seg.seg_energy(st)
    eo = o.energy(xyz, tri, K, Uo, 0.05)
    for k in ("total", "functional", "dirichlet"):
        assert rel(e[k], eo[k]) <= etol, (k, e[k], eo[k])
    if m > 1:
        assert rel(e["s_eps"], eo["s_eps"]) <= etol
    lam, lam_cl = seg.seg_eigenvalue_estimates(st)
    assert np.abs(lam - eo["D"]).max() <= etol * np.abs(eo["D"]).max()
    lo = o.lambda_cl(xyz, tri, K, Uo, 0.05)
    assert np.abs(lam_cl - lo).max() <= etol * np.abs(lo).max()


def test_onehot_initial_state(seg):
    xyz, tri = w.icosphere(3)
    st = make_state(seg, xyz, tri, 1e-4, 4, 0.05, 0, seed=5, init=seg.SEG_INIT_ONEHOT)
    U = seg.seg_get_u(st)
    M, K = o.assemble(xyz, tri)
    Uo = o.initial_state(M, w.initial_values("onehot", 5, xyz.shape[0], 4))
    assert np.abs(U - Uo).max() < 1e-13


@pytest.mark.parametrize("name,prec,utol,etol", PRECS)
def test_stages_match_algorithm_steps(seg, name, prec, utol, etol):
    """Stage 1 = heat step, stage 2 = nodal ODE, stage 3 = renormalisation."""
    xyz, tri = w.icosphere(4)
    m, tau, eps = 5, 2e-4, 2e-2
    st = make_state(seg, xyz, tri, tau, m, eps, prec, seed=9)
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, w.uniform01(9, xyz.shape[0], m))
    tol = 1e-10 if prec == 0 else 2e-6
    seg.seg_substep(st, 1)
    Ut = o.heat_step(M, K, tau, U)
    assert np.abs(seg.seg_get_u(st) - Ut).max() <= tol * np.abs(Ut).max()
    seg.seg_substep(st, 2)
    Uh = o.segregation_step(Ut, tau, eps)
    assert np.abs(seg.seg_get_u(st) - Uh).max() <= tol * np.abs(Uh).max()
    seg.seg_substep(st, 3)
    Un = o.normalise(M, Uh)
    assert np.abs(seg.seg_get_u(st) - Un).max() <= tol * np.abs(Un).max()
    # the staged state continues exactly like a full step
    seg.seg_step(st, 1)
    U2 = o.step(M, K, tau, eps, Un)
    assert np.abs(seg.seg_get_u(st) - U2).max() <= tol * np.abs(U2).max()


@pytest.mark.parametrize("m", [3, 2])
def test_config_sphere_level4_fp64_500_steps(seg, m):
    """Icosphere level 4, eps 1e-2, tau 1e-4, 500 steps, FP64."""
    xyz, tri = w.icosphere(4)
    tau, eps, steps, seed = 1e-4, 1e-2, 500, 1234
    st = make_state(seg, xyz, tri, tau, m, eps, 0, seed=seed)
    assert seg.seg_step(st, steps) == steps
    U = seg.seg_get_u(st)
    Uo, M, K = oracle_run(xyz, tri, w.uniform01(seed, xyz.shape[0], m), tau, eps, steps)
    assert np.abs(U - Uo).max() <= 1e-9
    e = seg.seg_energy(st)
    eo = o.energy(xyz, tri, K, Uo, eps)
    assert rel(e["total"], eo["total"]) <= 1e-10
    assert rel(e["s_eps"], eo["s_eps"]) <= 1e-9
    assert check_labels(seg, st, tri, Uo, U) > 0.5
    stats = seg.seg_get_stats(st)
    assert stats["steps"] == steps and stats["cg_max"] >= 1 and stats["status_bits"] == 0


@pytest.mark.parametrize("m", [3, 2])
def test_config_sphere_level4_mixed_500_steps(seg, m):
    xyz, tri = w.icosphere(4)
    tau, eps, steps, seed = 1e-4, 1e-2, 500, 1234
    st = make_state(seg, xyz, tri, tau, m, eps, 1, seed=seed)
    assert seg.seg_step(st, steps) == steps
    Uo, M, K = oracle_run(xyz, tri, w.uniform01(seed, xyz.shape[0], m), tau, eps, steps)
    e = seg.seg_energy(st)
    eo = o.energy(xyz, tri, K, Uo, eps)
    assert rel(e["total"], eo["total"]) <= 1e-5
    lam, _ = seg.seg_eigenvalue_estimates(st)
    assert np.abs(lam - eo["D"]).max() <= 1e-5 * np.abs(eo["D"]).max()
    check_labels(seg, st, tri, Uo, seg.seg_get_u(st))


@pytest.mark.parametrize("name,prec,utol,etol", PRECS)
@pytest.mark.parametrize("m", [1, 4, 7, 13, 17, 32])
def test_ragged_component_counts(seg, name, prec, utol, etol, m):
    xyz, tri = w.icosphere(3)
    tau, eps, steps = 5e-4, 5e-2, 6
    st = make_state(seg, xyz, tri, tau, m, eps, prec, seed=m)
    seg.seg_step(st, steps)
    Uo, M, K = oracle_run(xyz, tri, w.uniform01(m, xyz.shape[0], m), tau, eps, steps)
    U = seg.seg_get_u(st)
    assert np.abs(U - Uo).max() <= (1e-10 if prec == 0 else 1e-5) * np.abs(Uo).max()
    e = seg.seg_energy(st)
    assert rel(e["total"], o.energy(xyz, tri, K, Uo, eps)["total"]) <= etol


@pytest.mark.parametrize("name,prec,utol,etol", PRECS)
@pytest.mark.parametrize("surface", ["ico0", "ico1", "torus", "ellipsoid"])
def test_other_surfaces_and_tiny_meshes(seg, name, prec, utol, etol, surface):
    if surface == "ico0":
        xyz, tri = w.icosphere(0)
    elif surface == "ico1":
        xyz, tri = w.icosphere(1)
    elif surface == "torus":
        xyz, tri = w.torus(48, 20, 1.0, 0.4)
    else:
        xyz, tri = w.ellipsoid(3, 1.0, 0.8, 0.6)
    tau, eps, steps, m = 1e-3, 0.1, 8, 6
    st = make_state(seg, xyz, tri, tau, m, eps, prec, seed=3)
    seg.seg_step(st, steps)
    Uo, M, K = oracle_run(xyz, tri, w.uniform01(3, xyz.shape[0], m), tau, eps, steps)
    assert np.abs(seg.seg_get_u(st) - Uo).max() <= (1e-10 if prec == 0 else 1e-5) * np.abs(Uo).max()
    assert rel(seg.seg_energy(st)["total"], o.energy(xyz, tri, K, Uo, eps)["total"]) <= etol


@pytest.mark.parametrize("prec", [0, 1])
def test_constant_state_is_fixed_and_stop_rule_fires(seg, prec):
    xyz, tri = w.icosphere(3)
    tau = 1e-2  # check every 10 steps
    # float32 storage puts a ~1e-7 relative noise floor on the energy, so the
    # mixed-mode stop tolerance must sit above it
    st = make_state(seg, xyz, tri, tau, 3, 0.3, prec, energy_tol=1e-8 if prec == 0 else 1e-5)
    seg.seg_set_u(st, np.full((xyz.shape[0], 3), 2.0))
    done = seg.seg_step(st, 100)
    assert done == 10
    stats = seg.seg_get_stats(st)
    assert stats["converged"] == 1 and stats["checks"] == 2
    area = o.triangle_areas(xyz, tri).sum()
    U = seg.seg_get_u(st)
    assert np.abs(U - 1 / np.sqrt(area)).max() < (1e-13 if prec == 0 else 1e-6)
    e = seg.seg_energy(st)
    assert rel(e["s_eps"], o.constant_state_s_eps(3, area, 0.3)) < (1e-12 if prec == 0 else 1e-6)
    assert seg.seg_step(st, 5) == 0  # converged states stay put


def test_stop_rule_matches_oracle_run(seg):
    xyz, tri = w.icosphere(3)
    tau, eps = 5e-3, 0.3
    U0 = w.uniform01(4, xyz.shape[0], 3)
    st = make_state(seg, xyz, tri, tau, 3, eps, 0, seed=4, energy_tol=1e-4)
    done = seg.seg_step(st, 400)
    Uo, k, hist = o.run(xyz, tri, U0, tau, eps, 400, tol=1e-4)
    assert done == k
    assert np.abs(seg.seg_get_u(st) - Uo).max() < 1e-9


def test_error_statuses(seg):
    xyz, tri = w.icosphere(3)
    st = make_state(seg, xyz, tri, 1e-2, 3, 0.1, 0, cg_maxit=1, cg_rtol=1e-14)
    with pytest.raises(seg.SegError) as e:
        seg.seg_step(st, 2)
    assert e.value.status == seg.SEG_ERR_NOT_CONVERGED
    assert seg.seg_step(st, 2, ok_not_converged=True) == 2
    st = make_state(seg, xyz, tri, 1e-2, 3, 0.1, 0)
    U = np.full((xyz.shape[0], 3), 1.0)
    U[:, 1] = 0.0  # a vanished component cannot be normalised
    seg.seg_set_u(st, U)
    with pytest.raises(seg.SegError) as e:
        seg.seg_step(st, 1)
    assert e.value.status == seg.SEG_ERR_NONFINITE
    U = np.full((xyz.shape[0], 3), 1.0)
    U[17, 2] = np.nan
    seg.seg_set_u(st, U)
    with pytest.raises(seg.SegError) as e:
        seg.seg_step(st, 1)
    assert e.value.status == seg.SEG_ERR_NONFINITE
    # new data recovers the state (no NaN left in its CG work vectors)
    seg.seg_set_u(st, w.initial_values("uniform", 3, xyz.shape[0], 3))
    assert seg.seg_step(st, 3) == 3
    assert np.isfinite(seg.seg_get_u(st)).all() and np.isfinite(seg.seg_energy(st)["total"])
    with pytest.raises(seg.SegError) as e:
        make_state(seg, xyz, tri, 1e-2, 33, 0.1, 0)
    assert e.value.status == seg.SEG_ERR_UNSUPPORTED
    with pytest.raises(seg.SegError):
        make_state(seg, xyz, tri, 1e-2, 3, -1.0, 0)


@pytest.mark.parametrize("prec", [0, 1])
def test_bitwise_reproducible(seg, prec):
    xyz, tri = w.icosphere(4)
    outs = []
    for _ in range(2):
        st = make_state(seg, xyz, tri, 1e-4, 5, 1e-2, prec, seed=11)
        seg.seg_step(st, 20)
        outs.append(seg.seg_get_u(st))
    assert np.array_equal(outs[0], outs[1])


def test_component_permutation_and_vertex_renumbering(seg):
    xyz, tri = w.icosphere(3)
    m, tau, eps = 4, 1e-3, 0.05
    U0 = o.initial_state(o.assemble(xyz, tri)[0], w.uniform01(8, xyz.shape[0], m))
    st = make_state(seg, xyz, tri, tau, m, eps, 0)
    seg.seg_set_u(st, U0)
    seg.seg_step(st, 5)
    base = seg.seg_get_u(st)
    perm = [2, 0, 3, 1]
    st2 = make_state(seg, xyz, tri, tau, m, eps, 0)
    seg.seg_set_u(st2, U0[:, perm])
    seg.seg_step(st2, 5)
    assert np.abs(seg.seg_get_u(st2) - base[:, perm]).max() < 1e-12
    p = np.random.default_rng(0).permutation(xyz.shape[0])
    inv = np.argsort(p)
    st3 = make_state(seg, xyz[p], inv[tri].astype(np.int32), tau, m, eps, 0)
    seg.seg_set_u(st3, U0[p])
    seg.seg_step(st3, 5)
    assert np.abs(seg.seg_get_u(st3) - base[p]).max() < 1e-12


def test_set_get_roundtrip_and_device_pointers(seg):
    import torch

    xyz, tri = w.icosphere(3)
    st = make_state(seg, xyz, tri, 1e-3, 5, 0.05, 0, seed=2)
    seg.seg_step(st, 3)
    U = seg.seg_get_u(st)
    dev = torch.empty((xyz.shape[0], 5), dtype=torch.float64, device="cuda")
    seg.seg_get_u(st, dev, is_device=True)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), U)
    st2 = make_state(seg, xyz, tri, 1e-3, 5, 0.05, 0, seed=99)
    seg.seg_set_u(st2, dev, is_device=True)
    assert np.abs(seg.seg_get_u(st2) - U).max() < 1e-15
    seg.seg_step(st, 2)
    seg.seg_step(st2, 2)
    # st starts its next solve from the CG correction it carries, st2 (just
    # set) from none: the two agree to the solve's tolerance (rtol 1e-12)
    assert np.abs(seg.seg_get_u(st2) - seg.seg_get_u(st)).max() < 1e-10
