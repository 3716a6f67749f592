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
