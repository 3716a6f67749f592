"""Checkpoint / resume, side-effect-free reads, and the bounded device wait.

Checkpoint and resume: N steps, a checkpoint, then M steps must give bitwise
the same state, energies and counters as N + M steps without interruption --
whether the checkpoint is restored into a fresh state on the same mesh or
into the state it came from after it has moved on -- in float64 and mixed
precision, with the stop rule's energy history and the predicted start of the
solves (its correction history and the per-component choice of start) in
use.  Reading the state between steps (seg_get_u, seg_energy,
seg_eigenvalue_estimates, seg_labels) must not change the steps that follow.

Bounded wait: every wait of a kernel for data staged by the bulk-copy engine
gives up after the state's wait limit, records SEG_ERR_TIMEOUT and halts the
run (the copies still in flight are drained with the default 1 s limit).
seg_set_wait_stall makes the staged passes wait on a barrier that nothing
completes, so the wait runs out after the limit (1 ms here); the state is
then halted -- alone, when it is stepped in a batch -- and turning the stall
off plus seg_set_u bring it back to normal steps.  No GPU fault or hang is
involved: every copy that was issued completes.
"""

import numpy as np
import pytest

import workload as w
from tests.gpu_helpers import lib, make_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    return lib()


def _snapshot(seg, st):
    e = seg.seg_energy(st)
    lam, lam_cl = seg.seg_eigenvalue_estimates(st)
    s = seg.seg_get_stats(st)
    keep = ("steps", "cg_iterations", "cg_last", "cg_max", "checks", "last_check_total", "status_bits")
    return seg.seg_get_u(st), e, lam, lam_cl, {k: s[k] for k in keep}


def _same(a, b):
    Ua, ea, la, lca, sa = a
    Ub, eb, lb, lcb, sb = b
    assert np.array_equal(Ua, Ub)
    assert ea == eb
    assert np.array_equal(la, lb) and np.array_equal(lca, lcb)
    assert sa == sb


CASES = [
    # (mesh level, m, tau, eps, precision, steps before, steps after, extra params)
    (5, 5, 2e-4, 2e-2, 0, 25, 30, dict(check_every=5, energy_tol=-1.0)),
    (5, 5, 2e-4, 2e-2, 1, 25, 30, dict(check_every=5, energy_tol=-1.0)),
    (7, 16, 2e-5, 2e-3, 1, 40, 24, dict(check_every=1, energy_tol=-1.0)),
    (6, 3, 5e-5, 5e-3, 0, 40, 24, dict()),
]


@pytest.mark.parametrize("level,m,tau,eps,prec,n1,n2,params", CASES)
def test_checkpoint_then_resume_is_bitwise_the_uninterrupted_run(seg, level, m, tau, eps, prec, n1, n2, params):
    xyz, tri = w.icosphere(level)
    mesh = seg.seg_create_mesh(xyz, tri)
    prob = seg.seg_assemble(mesh, tau, prec)
    p = seg.seg_params()
    for k, v in params.items():
        setattr(p, k, v)

    # the uninterrupted run, never read in between
    ref = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, 77, p)
    assert seg.seg_step(ref, n1 + n2) == n1 + n2
    want = _snapshot(seg, ref)

    # the same run with a checkpoint after n1 steps and reads of the state
    a = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, 77, p)
    assert seg.seg_step(a, n1) == n1
    ck = seg.seg_get_checkpoint(a)
    assert ck.nbytes == seg.seg_checkpoint_size(a)
    seg.seg_get_u(a)
    seg.seg_energy(a)
    seg.seg_eigenvalue_estimates(a)
    seg.seg_labels(a)
    assert seg.seg_step(a, n2) == n2
    _same(_snapshot(seg, a), want)

    # restored into a fresh state on the same problem
    b = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, 5, p)
    seg.seg_set_checkpoint(b, ck)
    assert seg.seg_step(b, n2) == n2
    _same(_snapshot(seg, b), want)

    # restored into the state it came from, after that state moved on
    seg.seg_set_checkpoint(a, ck)
    assert seg.seg_step(a, n2) == n2
    _same(_snapshot(seg, a), want)

    # restored into a state on another problem assembled from the same mesh
    prob2 = seg.seg_assemble(mesh, tau, prec)
    c = seg.seg_state_create(prob2, m, eps, seg.SEG_INIT_UNIFORM, 9, p)
    seg.seg_set_checkpoint(c, ck)
    assert seg.seg_step(c, n2) == n2
    _same(_snapshot(seg, c), want)


def test_checkpoint_of_another_shape_is_refused(seg):
    xyz, tri = w.icosphere(3)
    mesh = seg.seg_create_mesh(xyz, tri)
    prob = seg.seg_assemble(mesh, 1e-4, seg.SEG_FP64)
    a = seg.seg_state_create(prob, 3, 0.05, seg.SEG_INIT_UNIFORM, 1)
    ck = seg.seg_get_checkpoint(a)
    for m, eps in ((4, 0.05), (3, 0.06)):
        b = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, 1)
        with pytest.raises(seg.SegError) as err:
            seg.seg_set_checkpoint(b, ck)
        assert err.value.status == seg.SEG_ERR_ARG
    damaged = ck.copy()
    damaged[0] ^= 0xFF
    with pytest.raises(seg.SegError) as err:
        seg.seg_set_checkpoint(a, damaged)
    assert err.value.status == seg.SEG_ERR_ARG
    with pytest.raises(seg.SegError) as err:
        seg.seg_set_checkpoint(a, ck[:-8])
    assert err.value.status == seg.SEG_ERR_ARG


@pytest.mark.parametrize("mode", [0, 1])
def test_bounded_wait_runs_out_and_the_state_recovers(seg, mode):
    xyz, tri = w.icosphere(6)
    m, tau, eps, seed = 16, 5e-5, 5e-3, 11
    ref = make_state(seg, xyz, tri, tau, m, eps, 1, seed=seed, launch_mode=mode)
    U0 = seg.seg_get_u(ref)
    seg.seg_set_u(ref, U0)  # both states start from the same stored values
    assert seg.seg_step(ref, 3) == 3
    want = seg.seg_get_u(ref)

    # every staged pass first waits on a barrier that nothing completes, with
    # a 1 ms limit
    st = make_state(seg, xyz, tri, tau, m, eps, 1, seed=seed, launch_mode=mode, wait_limit_ns=1_000_000)
    seg.seg_set_wait_stall(st, True)
    with pytest.raises(seg.SegError) as err:
        seg.seg_step(st, 3)
    assert err.value.status == seg.SEG_ERR_TIMEOUT
    stats = seg.seg_get_stats(st)
    assert stats["status_bits"] & 4
    assert stats["steps"] == 0  # halted in the first step's start pass
    # the state stays halted: further steps do nothing
    assert seg.seg_step(st, 1) == 0
    assert seg.seg_get_stats(st)["steps"] == 0
    # the waits back to normal and fresh data: the state steps again, bitwise
    # like the reference
    seg.seg_set_wait_stall(st, False)
    seg.seg_set_wait_limit(st, 0)
    seg.seg_set_u(st, U0)
    assert seg.seg_step(st, 3) == 3
    assert seg.seg_get_stats(st)["status_bits"] == 0
    assert np.array_equal(seg.seg_get_u(st), want)


def test_a_member_whose_wait_runs_out_halts_alone_in_a_batch(seg):
    """Two states stepped as a batch, the waits of the second made to run
    out: the batch step reports SEG_ERR_TIMEOUT, the second member is halted
    before its first step, and the first member's steps are bitwise those of
    the same state stepped alone."""
    xyz, tri = w.icosphere(5)
    m, tau, eps = 6, 1e-4, 2e-2
    alone = make_state(seg, xyz, tri, tau, m, eps, 1, seed=21, check_every=1, energy_tol=-1.0)
    assert seg.seg_step(alone, 8) == 8
    a = make_state(seg, xyz, tri, tau, m, eps, 1, seed=21, check_every=1, energy_tol=-1.0)
    b = make_state(seg, xyz, tri, tau, m, eps, 1, seed=22, check_every=1, energy_tol=-1.0,
                   wait_limit_ns=1_000_000)
    seg.seg_set_wait_stall(b, True)
    batch = seg.seg_batch_create([a, b])
    with pytest.raises(seg.SegError) as err:
        seg.seg_batch_step(batch, 8)
    assert err.value.status == seg.SEG_ERR_TIMEOUT
    sb = seg.seg_get_stats(b)
    assert sb["steps"] == 0 and sb["status_bits"] & 4
    assert seg.seg_get_stats(a)["steps"] == 8
    assert np.array_equal(seg.seg_get_u(a), seg.seg_get_u(alone))
    seg.seg_batch_destroy(batch)
