"""Batched stepping: several states (different meshes, m, eps) advanced with
one launch per pass.  Each member's result must be bitwise the same as the
same state stepped alone -- also when the members' grids together exceed the
blocks resident at once, as for the two-instance torus + ellipsoid workload
at full size -- and that workload must match the oracle over 50 steps."""

import numpy as np
import pytest

import workload as w
from oracle import seg_oracle as o
from tests.gpu_helpers import lib, make_state, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    return lib()


def _members(seg, prec):
    specs = [
        (w.icosphere(3), 5, 0.05, 1e-3, 11),
        (w.torus(40, 20, 1.0, 0.4), 6, 0.08, 1e-3, 12),
        (w.ellipsoid(4, 1.0, 0.8, 0.6), 7, 0.03, 5e-4, 13),
        (w.icosphere(2), 6, 0.3, 1e-2, 14),  # constant data: its stop rule fires at step 10
    ]
    states = []
    for (xyz, tri), m, eps, tau, seed in specs:
        st = make_state(seg, xyz, tri, tau, m, eps, prec, seed=seed, check_every=10,
                        energy_tol=1e-8 if prec == 0 else 1e-5)
        if seed == 14:
            seg.seg_set_u(st, np.full((xyz.shape[0], m), 1.0))
        states.append(st)
    return states


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("steps", [30, 100])  # 100: stepped in chunks, the graphs' peels reviewed
def test_batch_members_equal_alone(seg, prec, steps):
    alone = _members(seg, prec)
    done_alone = [seg.seg_step(s, steps) for s in alone]
    assert done_alone[3] == 10 and done_alone[0] > 10
    batched = _members(seg, prec)
    b = seg.seg_batch_create(batched)
    seg.seg_batch_step(b, steps)
    for sa, sb in zip(alone, batched):
        assert np.array_equal(seg.seg_get_u(sa), seg.seg_get_u(sb))
        ta, tb = seg.seg_get_stats(sa), seg.seg_get_stats(sb)
        for k in ("steps", "cg_iterations", "cg_max", "converged", "checks"):
            assert ta[k] == tb[k], k
        assert ta["last_check_total"] == tb["last_check_total"]
    # members remain usable on their own after the batch
    seg.seg_batch_destroy(b)
    seg.seg_step(batched[0], 2)
    seg.seg_step(alone[0], 2)
    assert np.array_equal(seg.seg_get_u(alone[0]), seg.seg_get_u(batched[0]))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("steps", [30, 100])
def test_persistent_batch_members_equal_alone(seg, prec, steps):
    """The persistent mode (one cooperative launch per call, grid barriers
    between the passes, the CG loop and the stop rules decided on the
    device): every member bitwise equal to itself stepped alone, counters
    included; the steps may be split over several calls and the batch may
    go back to the step graph."""
    alone = _members(seg, prec)
    for s_ in alone:
        seg.seg_step(s_, steps)
    batched = _members(seg, prec)
    b = seg.seg_batch_create(batched)
    seg.seg_batch_set_persistent(b, True)
    seg.seg_batch_step(b, steps // 3)
    seg.seg_batch_step(b, steps - steps // 3 - 5)
    seg.seg_batch_set_persistent(b, False)
    seg.seg_batch_step(b, 5)
    for sa, sb in zip(alone, batched):
        assert np.array_equal(seg.seg_get_u(sa), seg.seg_get_u(sb))
        ta, tb = seg.seg_get_stats(sa), seg.seg_get_stats(sb)
        for k in ("steps", "cg_iterations", "cg_max", "converged", "checks"):
            assert ta[k] == tb[k], k
        assert ta["last_check_total"] == tb["last_check_total"]
    seg.seg_batch_destroy(b)


def test_persistent_batch_member_whose_wait_runs_out_halts_alone(seg):
    """In the persistent mode a member whose staged-data waits run out (the
    stall aid, 1 ms limit) halts with SEG_ERR_TIMEOUT in its first step; the
    grid barriers go on and the other member's steps are bitwise those of it
    stepped alone."""
    xyz, tri = w.icosphere(5)
    alone = make_state(seg, xyz, tri, 1e-4, 6, 2e-2, 1, seed=21, check_every=1, energy_tol=-1.0)
    assert seg.seg_step(alone, 8) == 8
    a = make_state(seg, xyz, tri, 1e-4, 6, 2e-2, 1, seed=21, check_every=1, energy_tol=-1.0)
    b = make_state(seg, xyz, tri, 1e-4, 6, 2e-2, 1, seed=22, check_every=1, energy_tol=-1.0, wait_limit_ns=1_000_000)
    seg.seg_set_wait_stall(b, True)
    batch = seg.seg_batch_create([a, b])
    seg.seg_batch_set_persistent(batch, True)
    with pytest.raises(seg.SegError) as err:
        seg.seg_batch_step(batch, 8)
    assert err.value.status == seg.SEG_ERR_TIMEOUT
    sb = seg.seg_get_stats(b)
    assert sb["steps"] == 0 and sb["status_bits"] & 4
    assert seg.seg_get_stats(a)["steps"] == 8
    assert np.array_equal(seg.seg_get_u(a), seg.seg_get_u(alone))
    seg.seg_batch_destroy(batch)


def test_batch_rejects_mixed_classes(seg):
    xyz, tri = w.icosphere(2)
    a = make_state(seg, xyz, tri, 1e-3, 3, 0.1, 1)
    c = make_state(seg, xyz, tri, 1e-3, 16, 0.1, 1)
    d = make_state(seg, xyz, tri, 1e-3, 3, 0.1, 0)
    for pair in ([a, c], [a, d], [a, a]):
        with pytest.raises(seg.SegError) as e:
            seg.seg_batch_create(pair)
        assert e.value.status == seg.SEG_ERR_ARG


@pytest.mark.parametrize("m", [6, 12])
def test_torus_and_ellipsoid_batched_against_oracle(seg, m):
    """Torus R = 1, r = 0.4 on a 1024 x 512 grid and the level-8 ellipsoid
    (1, 0.8, 0.6), eps = 1e-3, tau = 5e-6, mixed precision, two instances in
    one launch per pass."""
    meshes = [w.torus(1024, 512, 1.0, 0.4), w.ellipsoid(8, 1.0, 0.8, 0.6)]
    eps, tau, steps = 1e-3, 5e-6, 2
    states = [make_state(seg, xyz, tri, tau, m, eps, 1, seed=1237 + k, check_every=1, energy_tol=-1.0)
              for k, (xyz, tri) in enumerate(meshes)]
    b = seg.seg_batch_create(states)
    seg.seg_batch_step(b, steps)
    for k, ((xyz, tri), st) in enumerate(zip(meshes, states)):
        M, K = o.assemble(xyz, tri)
        U = o.initial_state(M, w.uniform01(1237 + k, xyz.shape[0], m))
        for _ in range(steps):
            U = o.step(M, K, tau, eps, U)
        Ug = seg.seg_get_u(st)
        assert np.abs(Ug - U).max() <= 1e-4 * np.abs(U).max()
        assert rel(seg.seg_energy(st)["total"], o.energy(xyz, tri, K, U, eps)["total"]) <= 1e-5


def _pair(seg, m, seeds=(1237, 1238)):
    meshes = [w.torus(1024, 512, 1.0, 0.4), w.ellipsoid(8, 1.0, 0.8, 0.6)]
    states = [make_state(seg, xyz, tri, 5e-6, m, 1e-3, 1, seed=sd, check_every=1, energy_tol=-1.0)
              for (xyz, tri), sd in zip(meshes, seeds)]
    return meshes, states


def test_full_size_pair_batched_is_bitwise_the_pair_alone(seg):
    """The two-instance workload (torus 1024 x 512 and the level-8
    ellipsoid, m = 12) in the default launch geometry (two blocks per SM for
    each member, so the two grids together need twice the blocks resident at
    once): 20 steps of each member alone, then 40 batched steps, equal 60
    steps of each member alone."""
    _, alone = _pair(seg, 12)
    _, batched = _pair(seg, 12)
    for sa, sb in zip(alone, batched):
        seg.seg_step(sa, 60)
        seg.seg_step(sb, 20)
        assert seg.seg_launch_info(sa) == seg.seg_launch_info(sb)
    b = seg.seg_batch_create(batched)
    seg.seg_batch_step(b, 40)
    for sa, sb in zip(alone, batched):
        assert np.array_equal(seg.seg_get_u(sa), seg.seg_get_u(sb))
        ta, tb = seg.seg_get_stats(sa), seg.seg_get_stats(sb)
        assert ta["cg_iterations"] == tb["cg_iterations"] and ta["steps"] == tb["steps"]


def test_full_size_pair_persistent_is_bitwise_the_pair_alone(seg):
    """The two full-size instances (torus 1024 x 512 and the level-8
    ellipsoid, m = 12) stepped by the persistent kernel (one block per SM,
    each member's virtual blocks in its own decomposition) for 40 steps after
    20 alone: bitwise the 60 steps of each alone."""
    _, alone = _pair(seg, 12)
    _, batched = _pair(seg, 12)
    for sa, sb in zip(alone, batched):
        seg.seg_step(sa, 60)
        seg.seg_step(sb, 20)
    b = seg.seg_batch_create(batched)
    seg.seg_batch_set_persistent(b, True)
    seg.seg_batch_step(b, 40)
    for sa, sb in zip(alone, batched):
        assert np.array_equal(seg.seg_get_u(sa), seg.seg_get_u(sb))
        ta, tb = seg.seg_get_stats(sa), seg.seg_get_stats(sb)
        assert ta["cg_iterations"] == tb["cg_iterations"] and ta["steps"] == tb["steps"]


def test_full_size_pair_batched_50_steps_against_oracle(seg):
    """Config 4 batched for 50 steps against the FP64 oracle (stored values
    of tests/golden/longrun_torus1024_m12.json and _ellipsoid8_m12.json,
    written by tests/golden/make_longrun.py from the oracle alone): total
    energy and per-component D_i within 1e-5 at steps 25 and 50, sampled rows
    within 1e-4, labels equal off the interface."""
    import json
    import os

    gold = []
    for name in ("torus1024_m12", "ellipsoid8_m12"):
        with open(os.path.join(os.path.dirname(__file__), "golden", f"longrun_{name}.json")) as f:
            gold.append(json.load(f))
    meshes, states = _pair(seg, 12, seeds=(gold[0]["seed"], gold[1]["seed"]))
    b = seg.seg_batch_create(states)
    done = 0
    for k, cp in enumerate(gold[0]["oracle"]["checkpoints"]):
        if cp["step"] > done:
            seg.seg_batch_step(b, cp["step"] - done)
            done = cp["step"]
        for g, st in zip(gold, states):
            ref = g["oracle"]["checkpoints"][k]
            assert ref["step"] == done
            e = seg.seg_energy(st)
            lam, _ = seg.seg_eigenvalue_estimates(st)
            assert rel(e["total"], ref["total"]) <= 1e-5, (g["case"], done, e["total"], ref["total"])
            D = np.array(ref["D"])
            assert np.abs(lam - D).max() <= 1e-5 * np.abs(D).max(), (g["case"], done)
    for g, st in zip(gold, states):
        U = seg.seg_get_u(st)
        idx = np.array(g["sample"]["vertices"])
        Uo = np.array(g["sample"]["u"])
        err = np.abs(U[idx] - Uo).max()
        assert err <= 1e-4 * np.abs(Uo).max(), (g["case"], err)
        am, _ = seg.seg_labels(st)
        srt = np.sort(Uo, axis=1)
        gap = srt[:, -1] - srt[:, -2]
        off = (np.array(g["sample"]["ring_mixed"]) == 0) & (gap > 2 * err + 1e-6 * srt[:, -1])
        assert np.array_equal(am[idx][off], np.array(g["sample"]["label"])[off])
