"""The launch counter of seg_stats matches the step structure: per step the
start, energy-check and finish passes and the CG passes.  The step graph runs
pass A of the first iteration, then (pass B, pass A) for the next peel - 1
iterations as plain nodes, then, while a pass B is needed, two (pass B, pass
A) pairs per evaluation of its loop condition; a solve of one iteration that
ends in pass A needs no pass B.  Direct launches run exactly one (pass A,
pass B) pair per iteration."""

import pytest

import workload as w
from tests.gpu_helpers import lib, make_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    return lib()


@pytest.mark.parametrize("mode", [0, 1])
def test_kernel_launch_counter(seg, mode):
    xyz, tri = w.icosphere(4)
    st = make_state(seg, xyz, tri, 1e-4, 3, 1e-2, 1, 3, launch_mode=mode, check_every=1, energy_tol=-1.0)
    seg.seg_step(st, 1)  # the first step also runs the pending normalisation
    for _ in range(4):
        s0 = seg.seg_get_stats(st)
        seg.seg_step(st, 1)
        s1 = seg.seg_get_stats(st)
        k = s1["cg_last"]
        assert k == s1["cg_iterations"] - s0["cg_iterations"] and k >= 1
        got = s1["kernel_launches"] - s0["kernel_launches"]
        if mode == 1:
            assert got == 3 + 2 * k
            continue
        pl = s0["graph_peel"]

        def graph_launches(n_b):  # n_b: the passes B the solve needs
            in_loop = max(0, n_b - (pl - 1))
            return 3 + (2 * pl - 1) + 4 * ((in_loop + 1) // 2)

        # a one-iteration solve ends in pass A (no pass B) unless its residual
        # was within the rounding margin of the tolerance
        assert got in ({graph_launches(0), graph_launches(1)} if k == 1 else {graph_launches(k)}), (got, k, pl)


def test_step_limit_with_more_blocks_than_resident(seg):
    """The last step under a step limit updates every row even when the grid
    runs in several waves (later blocks start after earlier ones finished)."""
    import numpy as np

    xyz, tri = w.icosphere(6)
    a = make_state(seg, xyz, tri, 1e-4, 8, 2e-2, 0, 5, check_every=-1, max_steps=3, grid_blocks=2048)
    b = make_state(seg, xyz, tri, 1e-4, 8, 2e-2, 0, 5, check_every=-1)
    assert seg.seg_step(a, 10) == 3
    assert seg.seg_get_stats(a)["steps"] == 3
    assert seg.seg_step(b, 3) == 3
    ua, ub = seg.seg_get_u(a), seg.seg_get_u(b)
    assert np.abs(ua - ub).max() <= 1e-12 * np.abs(ub).max()


def test_long_step_reviews_the_graph_without_changing_results(seg):
    """A long seg_step adapts the step graph's peel between chunks of steps;
    the arithmetic is the same as one graph for the whole run (bitwise)."""
    import numpy as np

    xyz, tri = w.icosphere(5)
    a = make_state(seg, xyz, tri, 2e-5, 6, 2e-3, 1, 7, check_every=-1)
    b = make_state(seg, xyz, tri, 2e-5, 6, 2e-3, 1, 7, check_every=-1)
    assert seg.seg_get_stats(a)["graph_peel"] == 4  # the untuned default
    assert seg.seg_step(a, 160) == 160
    seg.seg_step_async(b, 160)
    assert seg.seg_sync(b) == 160
    assert np.array_equal(seg.seg_get_u(a), seg.seg_get_u(b))
    sa, sb = seg.seg_get_stats(a), seg.seg_get_stats(b)
    assert sa["cg_iterations"] == sb["cg_iterations"]
    assert 1 <= sa["graph_peel"] <= max(4, sa["cg_max"])


def test_predicted_start_cuts_the_iterations(seg):
    """The step-1 solve starts from the extrapolated correction once that
    beats a plain warm start: after the first steps from random data the CG
    iterations per step drop well below those of the first steps, and a state
    set to the same data again (no history) starts over."""
    import numpy as np

    xyz, tri = w.icosphere(5)  # tau / h^2 and 2 tau / eps^2 as in the level-8 workload
    st = make_state(seg, xyz, tri, 3e-4, 8, 8e-3, 1, 3, check_every=-1)

    def its(k):
        c0 = seg.seg_get_stats(st)["cg_iterations"]
        seg.seg_step(st, k)
        return (seg.seg_get_stats(st)["cg_iterations"] - c0) / k

    first = its(5)
    its(45)
    late = its(20)
    assert late < 0.75 * first, (first, late)
    U = seg.seg_get_u(st)
    seg.seg_set_u(st, U)  # same state, no history: plain warm start again
    again = its(1)
    assert again > late
    assert np.all(np.isfinite(seg.seg_get_u(st)))


def test_pipelined_statistics_read_every_step(seg):
    """seg_stats_enqueue / seg_stats_wait: the statistics of step k read while
    step k + 1 is queued equal those a synchronous twin reports after step k."""
    xyz, tri = w.icosphere(4)
    a = make_state(seg, xyz, tri, 1e-4, 5, 2e-2, 1, 21, check_every=1, energy_tol=-1.0)
    b = make_state(seg, xyz, tri, 1e-4, 5, 2e-2, 1, 21, check_every=1, energy_tol=-1.0)
    got, want, tickets = [], [], []
    for k in range(12):
        seg.seg_step_async(a, 1)
        tickets.append(seg.seg_stats_enqueue(a))
        if k >= 1:
            got.append(seg.seg_stats_wait(a, tickets[k - 1]))
        seg.seg_step(b, 1)
        want.append(seg.seg_get_stats(b))
    got.append(seg.seg_stats_wait(a, tickets[-1]))
    assert seg.seg_sync(a) == 1  # steps since the last seg_step_async
    assert seg.seg_get_stats(a)["steps"] == 12
    for g, w_ in zip(got, want):
        for key in ("steps", "cg_iterations", "cg_last", "checks", "last_check_total", "status_bits"):
            assert g[key] == w_[key], key
    # a ticket overwritten by SEG_STATS_RING newer copies is refused
    for _ in range(seg.SEG_STATS_RING):
        seg.seg_stats_enqueue(a)
    with pytest.raises(seg.SegError) as e:
        seg.seg_stats_wait(a, tickets[-1])
    assert e.value.status == seg.SEG_ERR_ARG
