"""Request server with continuous batching: requests of different meshes, m and
eps arrive while others are resident, are admitted as memory frees up, run in
shared batched launches, and each result equals the same request stepped
alone (bitwise)."""

import numpy as np
import pytest

import workload as w
from tests.gpu_helpers import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    return lib()


def _problems(seg, prec, tau):
    meshes = [w.icosphere(3), w.icosphere(4), w.torus(48, 24, 1.0, 0.4), w.ellipsoid(3, 1.0, 0.8, 0.6)]
    return [seg.seg_assemble(seg.seg_create_mesh(x, t), tau, prec) for x, t in meshes]


def _params(seg):
    p = seg.seg_params()
    p.check_every = 10
    p.energy_tol = 1e-3
    p.max_steps = 150
    return p


REQS = [(0, 3, 0.05), (1, 6, 0.03), (2, 8, 0.05), (3, 5, 0.04), (1, 2, 0.05), (0, 12, 0.03), (2, 4, 0.02),
        (3, 7, 0.05), (1, 16, 0.04), (0, 6, 0.06)]


@pytest.mark.parametrize("prec", [1, 0])
def test_server_results_equal_alone(seg, prec):
    tau = 1e-3
    probs = _problems(seg, prec, tau)
    prm = _params(seg)
    need = [seg.seg_state_bytes(probs[k], m) for k, m, _ in REQS]
    budget = 2 * max(need)  # the largest fits, not all of them at once
    assert sum(need) > budget
    sp = seg.seg_server_params()
    sp.hbm_budget_bytes = budget
    sp.steps_per_tick = 7
    srv = seg.seg_server_create(sp)
    ids = []
    for i, (k, m, eps) in enumerate(REQS[:5]):
        ids.append(seg.seg_server_submit(srv, probs[k], m, eps, seg.SEG_INIT_UNIFORM, 100 + i, prm))
    max_running = 0
    waited = False
    ticks = 0
    while True:
        running, queued = seg.seg_server_tick(srv)
        resident = [i for i, rid in enumerate(ids) if seg.seg_server_info(srv, rid)["phase"] == 1]
        assert len(resident) == running
        assert sum(need[i] for i in resident) <= budget
        max_running = max(max_running, running)
        waited |= queued > 0
        ticks += 1
        if ticks == 3:  # the rest arrive while the first ones are on the GPU
            for i, (k, m, eps) in enumerate(REQS[5:], start=5):
                ids.append(seg.seg_server_submit(srv, probs[k], m, eps, seg.SEG_INIT_UNIFORM, 100 + i, prm))
        if running == 0 and queued == 0 and ticks > 3:
            break
        assert ticks < 500
    assert max_running > 1 and waited
    for i, rid in enumerate(ids):
        info = seg.seg_server_info(srv, rid)
        assert info["phase"] == 2, info
        assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
        k, m, eps = REQS[i]
        st = seg.seg_state_create(probs[k], m, eps, seg.SEG_INIT_UNIFORM, 100 + i, prm)
        done = seg.seg_step(st, 1000)
        assert done == info["steps"]
        assert np.array_equal(seg.seg_get_u(st), seg.seg_server_result(srv, rid))
        stats = seg.seg_get_stats(st)
        assert stats["converged"] == info["converged"]
        assert stats["last_check_total"] == info["total_energy"]
    seg.seg_server_destroy(srv)


def test_server_rejects_requests_that_cannot_finish(seg):
    probs = _problems(seg, 1, 1e-3)
    srv = seg.seg_server_create()
    p = seg.seg_params()
    p.energy_tol = -1.0
    with pytest.raises(seg.SegError) as e:
        seg.seg_server_submit(srv, probs[0], 3, 0.05, seg.SEG_INIT_UNIFORM, 1, p)
    assert e.value.status == seg.SEG_ERR_ARG


def test_served_requests_converge_and_match_the_oracle(seg):
    """Requests served to the relative stop rule (checks every 0.01 of
    simulated time, |E_k - E_prev| <= 1e-5 |E_k|) on the level-4 sphere,
    eps = 1e-2, tau = 5 eps^2, mixed precision, uniform random data.  Each
    must converge; its result is compared with the FP64 oracle run for the
    same number of steps (relative total energy and per-component D_i within
    1e-5, labels equal off the interface), and the oracle's own energies
    must meet the stop rule at that check and not at the one before (up to
    the float32 noise of the served energies: a relative change within 10%
    of the tolerance counts as either)."""
    from oracle import seg_oracle as o
    from tests.gpu_helpers import check_labels, rel

    xyz, tri = w.icosphere(4)
    eps = 1e-2
    tau = 5 * eps * eps
    every = round(0.01 / tau)
    rtol = 1e-5
    prob = seg.seg_assemble(seg.seg_create_mesh(xyz, tri), tau, seg.SEG_MIXED_FP32)
    p = seg.seg_params()
    p.check_every = every
    p.energy_tol = -1.0
    p.energy_rtol = rtol
    p.max_steps = round(10.0 / tau)
    reqs = [(2, 301), (3, 302)]
    srv = seg.seg_server_create()
    ids = [seg.seg_server_submit(srv, prob, m, eps, seg.SEG_INIT_UNIFORM, sd, p) for m, sd in reqs]
    while True:
        running, queued = seg.seg_server_tick(srv)
        if running == 0 and queued == 0:
            break
    M, K = o.assemble(xyz, tri)
    for (m, sd), rid in zip(reqs, ids):
        info = seg.seg_server_info(srv, rid)
        assert info["phase"] == 2 and info["converged"] == 1, info
        S = info["steps"]
        assert S % every == 0 and S < p.max_steps
        Ug = seg.seg_server_result(srv, rid)
        U = o.initial_state(M, w.uniform01(sd, xyz.shape[0], m))
        energies = {0: o.energy(xyz, tri, K, U, eps)["total"]}
        for k in range(1, S + 1):
            U = o.step(M, K, tau, eps, U)
            if k % every == 0:
                energies[k] = o.energy(xyz, tri, K, U, eps)["total"]
        eo = o.energy(xyz, tri, K, U, eps)
        assert rel(info["total_energy"], eo["total"]) <= 1e-5, (m, info["total_energy"], eo["total"])
        change = {k: abs(energies[k] - energies[k - every]) / abs(energies[k]) for k in energies if k >= every}
        assert change[S] <= 1.1 * rtol, (m, S, change[S])
        assert all(c > 0.9 * rtol for k, c in change.items() if k < S - every), m
        # the served state against the oracle's: energies, D_i, labels
        e_sum = o.energy(xyz, tri, K, Ug, eps)
        assert rel(e_sum["total"], eo["total"]) <= 1e-5
        assert np.abs(e_sum["D"] - eo["D"]).max() <= 1e-5 * np.abs(eo["D"]).max()
        st = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, sd, p)
        seg.seg_set_u(st, Ug)
        check_labels(seg, st, tri, U, Ug)
    seg.seg_server_destroy(srv)


def test_concurrent_classes_with_one_iteration_solves_equal_alone(seg):
    """Requests of three classes (m = 3, 6, 16: three lane layouts, so three
    batches on their own streams, running at the same time) in the regime
    where nearly every solve takes one CG iteration and ends in CG pass A:
    each result is bitwise the request stepped alone.  (A batched pass maps
    its blocks to the members as its blocks start, while other classes'
    kernels hold SMs; no member's flags may change meanwhile.)"""
    xyz, tri = w.icosphere(5)
    tau, steps = 1e-6, 600
    prob = seg.seg_assemble(seg.seg_create_mesh(xyz, tri), tau, 1)
    p = seg.seg_params()
    p.check_every = 1
    p.energy_tol = -1.0
    p.max_steps = steps
    reqs = [(3, 5e-3), (6, 4e-3), (16, 6e-3), (3, 7e-3), (6, 5e-3), (16, 4e-3), (6, 8e-3), (16, 5e-3)]
    sp = seg.seg_server_params()
    sp.steps_per_tick = 64
    srv = seg.seg_server_create(sp)
    ids = [seg.seg_server_submit(srv, prob, m, eps, seg.SEG_INIT_UNIFORM, 400 + i, p) for i, (m, eps) in enumerate(reqs)]
    ticks = 0
    while True:
        running, queued = seg.seg_server_tick(srv)
        ticks += 1
        if running == 0 and queued == 0:
            break
        assert ticks < 100
    one_iteration = 0  # solves of one iteration (the rest here take two, a few at the start more)
    for i, rid in enumerate(ids):
        info = seg.seg_server_info(srv, rid)
        assert info["phase"] == 2 and info["steps"] == steps, info
        m, eps = reqs[i]
        st = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, 400 + i, p)
        assert seg.seg_step(st, steps) == steps
        assert np.array_equal(seg.seg_get_u(st), seg.seg_server_result(srv, rid)), i
        one_iteration += max(0, 2 * steps - seg.seg_get_stats(st)["cg_iterations"])
    assert one_iteration >= 0.1 * steps * len(reqs)  # the regime is the one meant
    seg.seg_server_destroy(srv)
