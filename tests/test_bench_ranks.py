"""Host-side logic of bench.py on CPU: the replica ranks' barrier and
max-over-ranks timing with the gloo backend (world size 2), and the JSON line
of the reference arm (the oracle) alone and under two ranks."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    class A:
        pass

    r, ws, local = bench.dist_setup(A())
    bench.barrier(ws)
    m = bench.max_over_ranks(1.5 + rank, ws)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{r} {ws} {m}\n")
    import torch.distributed as dist

    dist.destroy_process_group()


def test_max_over_ranks_with_gloo(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        r, ws, m = open(tmp_path / f"rank{rank}.txt").read().split()
        assert int(r) == rank and int(ws) == 2 and float(m) == 2.5


REF_ARGS = ["--impl", "reference", "--level", "3", "--components", "4", "--steps", "2", "--warmup", "1",
            "--reference-budget-seconds", "2"]


def _check_reference_line(line):
    d = json.loads(line)
    assert d["impl"] == "reference" and d["unit"] == "DoF-steps/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + REF_ARGS, capture_output=True,
                       text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    _check_reference_line(lines[0])


def test_reference_arm_under_two_ranks_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"), "--gpus", "2"]
    r = subprocess.run(cmd + REF_ARGS, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    _check_reference_line(lines[0])


def test_kernel_byte_model_matches_the_design_table():
    """The algorithmic bytes per launch that bench.py divides by the measured
    times (level-8 sphere, m = 16, float32, ELL width 8): V = N * 16 * 4."""
    sys.path.insert(0, ROOT)
    import bench

    n, ntri = 655362, 1310720
    kb = bench.kernel_bytes(n, ntri, 16, 4)
    V = n * 16 * 4
    ell = n * 8 * 4
    assert kb["k_start"] == 3 * V + ell + 3 * n * 8 * 4 + n * 4
    assert kb["k_cg_a_first"] == 2 * V + ell + n * 8 * 4 + n * 4
    assert kb["k_cg_a_even"] == 5 * V + ell + n * 8 * 4
    assert kb["k_cg_a_odd"] == 8 * V + ell + n * 8 * 4
    assert kb["k_cg_b"] == 3 * V + 2 * n * 4
    assert kb["k_cg_b_first"] == 4 * V + 2 * n * 4
    assert (kb["k_finish_one"], kb["k_finish_two"]) == (8 * V, 9 * V)
    assert kb["k_energy_check"] == V + ntri * 16
    # the per-launch figures, MB: start 212.3, CG pass A 128.5 / 251.7 / 377.5
    # (first / even / odd form), CG pass B 131.1 / 173.0 (later / first
    # iteration), finish 335.5 / 377.5, energy 62.9
    quoted = {"k_start": 212.3, "k_cg_a_first": 128.5, "k_cg_a_even": 251.7, "k_cg_a_odd": 377.5,
              "k_cg_b": 131.1, "k_cg_b_first": 173.0, "k_finish_one": 335.5, "k_finish_two": 377.5,
              "k_energy_check": 62.9}
    for k, mb in quoted.items():
        assert abs(kb[k] / 1e6 - mb) < 0.06, (k, kb[k] / 1e6)


def test_pass_counts_per_step():
    """Launches per step of each form of the CG passes and of the finish
    pass: a solve of one iteration ends in CG pass A (no pass B); one of k >= 2
    runs pass B k times, the first in its first-iteration form."""
    sys.path.insert(0, ROOT)
    import bench

    one = bench.pass_counts(1.0)
    assert (one["first"], one["odd"], one["even"], one["fin_one"], one["fin_two"]) == (1, 0, 0, 1, 0)
    assert (one["b_first"], one["b_later"]) == (0, 0)
    two = bench.pass_counts(2.0)
    assert (two["b_first"], two["b_later"]) == (1, 1)
    three = bench.pass_counts(3.0)
    assert (three["b_first"], three["b_later"]) == (1, 2)
    four = bench.pass_counts(4.0)  # first, odd, even, odd
    assert (four["first"], four["odd"], four["even"], four["fin_one"], four["fin_two"]) == (1, 2, 1, 1, 0)
    five = bench.pass_counts(5.0)  # first, odd, even, odd, even; two pending updates at the end
    assert (five["first"], five["odd"], five["even"], five["fin_one"], five["fin_two"]) == (1, 2, 2, 0, 1)
    half = bench.pass_counts(1.5)
    assert half["first"] == 1 and half["odd"] == 0.5 and half["even"] == 0
    for k in (0.0, 0.7, 2.3, 7.9):
        c = bench.pass_counts(k)
        assert abs(c["first"] + c["odd"] + c["even"] - k) < 1e-12 or k < 1
