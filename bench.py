"""Benchmark of the segregation gradient flow on one GB300 (or N replicas).

Workload (default): unit-sphere icosphere level 8 (N = 655 362 vertices,
1 310 720 triangles), m = 16 components, eps = 1e-3, tau = 5e-6, seeded
uniform[0,1) initial data; mixed precision (float32 vectors and matrices,
inner products / norms / CG scalars / energies accumulated to float64).
One bench step = one step of Algorithm 2.2 (heat step by Jacobi-PCG, nodal
ODE, renormalisation) plus the energy evaluation of the stop rule, i.e. every
hot-path pass runs in every step.  Metric: DoF-steps/s = N * m * steps / s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank runs an independent replica on its own GPU
(weak scaling); ranks meet only at a host barrier and a max-reduction of the
timings (gloo), never in the data path.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal
# DRAM bytes (read + write) per launch of each form of the hot-path kernels,
# from one ncu capture of the level-8 sphere, m = 16, mixed precision, 1000
# steps in, default geometry of 304 blocks: dram__bytes_read.sum +
# dram__bytes_write.sum of the bench's own kernel timing launches (selected by
# their NVTX range), mean of the second and third launch; valid only for the
# kernel versions captured.
TRAFFIC = {"k_start": 196.1e6, "k_cg_a_first": 97.0e6, "k_cg_b": 90.6e6, "k_cg_b_first": 113.8e6,
           "k_finish_one": 279.5e6, "k_energy_check": 63.0e6}
KERNEL_ROLE = {
    "k_start": "start pass: r0 = -tau K X - A y for the predicted correction y, z0 = D^-1 r0, norms "
               "(issue and latency bound: three sparse products and three float-float sums per row)",
    "k_cg_a": "CG pass A: p = z + beta p, q = A z + beta q, p.q; the solve's correction updated every "
              "second iteration (its first, odd and later even forms weighted by their launches per step)",
    "k_cg_b": "CG pass B: z -= alpha D^-1 q, r.z, |r|^2, convergence and beta",
    "k_finish": "finish pass: x = X + y, nodal segregation ODE, next predicted correction (its forms with "
                "one and two pending updates weighted by their launches per step)",
    "k_energy_check": "S_eps by the degree-4 rule and the stop rule",
}
METRIC = "DoF-steps/s (N*m*steps) sphere 655k m=16 FP32-mix vs FP64; p50/p99 latency"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--launch-mode", default="graph", choices=["graph", "direct"],
                    help="direct: kernels launched one by one (for profilers that cannot see graph kernels)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=8)
    ap.add_argument("--components", dest="m", type=int, default=16, help="number of components m")
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--tau", type=float, default=5e-6)
    ap.add_argument("--seed", type=int, default=1236)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch geometry")
    ap.add_argument("--grid-blocks", type=int, default=0, help="row-kernel blocks (0: default / autotuned)")
    ap.add_argument("--batch-steps", type=int, default=200, help="0 disables the two-instance batch run")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests served (the first ones of the seeded 256-request stream); 0 disables")
    ap.add_argument("--serve-compare", type=int, default=24)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-eps-min", type=float, default=5e-3,
                    help="eps of the requests log-uniform in [eps-min, 1e-2]")
    ap.add_argument("--serve-tau-factor", type=float, default=5.0, help="tau = factor * eps^2")
    ap.add_argument("--serve-check-dt", type=float, default=0.01,
                    help="stop-rule checks every round(dt / tau) steps (simulated time dt)")
    ap.add_argument("--serve-rtol", type=float, default=1e-5,
                    help="stop when the energy changes by at most rtol (relative) between checks")
    ap.add_argument("--serve-t-max", type=float, default=10.0, help="step budget: simulated time t_max / tau")
    ap.add_argument("--serve-compare-steps", type=int, default=400,
                    help="steps per request of the burst / alone throughput comparison")
    ap.add_argument("--serve-quantum", type=int, default=64)
    ap.add_argument("--cpu-sample-seconds", type=float, default=20.0)
    ap.add_argument("--setup-steps", type=int, default=1000,
                    help="steps of the run before the autotuner and the timed window (not timed): the "
                         "solves' predicted start settles over the first ~1000 steps of the 10000-step run, "
                         "so a window after them matches the whole run's rate (full_run)")
    ap.add_argument("--run-steps", type=int, default=10000,
                    help="the configured run length: one fresh state runs it whole (0 disables)")
    ap.add_argument("--other-m", default="8,32", help="further component counts timed at the same level")
    ap.add_argument("--reference-budget-seconds", type=float, default=150.0)
    return ap.parse_args()


def workload_name(a):
    n = 10 * 4 ** a.level + 2
    return f"unit sphere icosphere level {a.level} (N={n}), m={a.m}, eps={a.eps:g}, tau={a.tau:g}, seeded uniform init"


# --------------------------------------------------------------- distributed


def dist_setup(a):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle


def oracle_sample(level, m, eps, tau, seed, budget_s, max_cols=None):
    """Time the FP64 oracle on a bounded sample of the workload.

    A sample step is the oracle's Algorithm 2.2 step restricted to the first
    c components (c columns of the heat step, the nodal ODE and the
    normalisation over those c columns); its cost is proportional to c, and
    its DoF count is N * c.  c is chosen so that the sample takes about
    budget_s seconds.  Returns (DoF-steps/s, c, seconds, threads).
    """
    import numpy as np

    import workload as w
    from oracle import seg_oracle as o

    xyz, tri = w.icosphere(level)
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, w.uniform01(seed, xyz.shape[0], m))
    t0 = time.perf_counter()
    o.heat_step(M, K, tau, U[:, :1])
    t_col = time.perf_counter() - t0
    c = int(max(1, min(max_cols or m, budget_s // max(t_col, 1e-9))))
    t0 = time.perf_counter()
    o.step(M, K, tau, eps, U[:, :c])
    dt = time.perf_counter() - t0
    return xyz.shape[0] * c / dt, c, dt, 1


def oracle_sample_all_cores(level, m, eps, tau, seed, steps, workers):
    """Time the FP64 oracle with its m step-1 solves spread over `workers`
    processes (oracle.parallel; steps 2 and 3 in the parent): `steps` full
    steps of all m components.  Returns (DoF-steps/s, seconds, workers)."""
    import workload as w
    from oracle import parallel
    from oracle import seg_oracle as o

    xyz, tri = w.icosphere(level)
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, w.uniform01(seed, xyz.shape[0], m))
    with parallel.ColumnPool(M, K, tau, m, workers) as pool:
        U = pool.step(U, eps)  # warm-up (workers started, caches filled)
        t0 = time.perf_counter()
        for _ in range(steps):
            U = pool.step(U, eps)
        dt = time.perf_counter() - t0
        used = pool.workers
    return xyz.shape[0] * m * steps / dt, dt, used


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                model = line.split(":", 1)[1].strip()
                if model:
                    break
        else:
            model = None
    except OSError:
        model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform

    return f"{model or 'unknown'} ({platform.machine()})"


def cpu_baseline(a):
    """The oracle on the host cores: one thread, and all cores (the m step-1
    solves in parallel worker processes)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    ncores = os.cpu_count() or 1
    code = (f"import json,sys; sys.path.insert(0,{ROOT!r}); import bench; "
            f"r=bench.oracle_sample({a.level},{a.m},{a.eps},{a.tau},{a.seed},{a.cpu_sample_seconds}); "
            f"print(json.dumps(r))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return {"value": None, "unit": "DoF-steps/s", "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    rate1, c, dt1, _ = json.loads(r.stdout.strip().splitlines()[-1])
    code = (f"import json,sys; sys.path.insert(0,{ROOT!r}); import bench; "
            f"r=bench.oracle_sample_all_cores({a.level},{a.m},{a.eps},{a.tau},{a.seed},2,{ncores}); "
            f"print(json.dumps(r))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    single = {"value": rate1, "cores": 1,
              "sample": f"one oracle step (FP64 numpy/scipy, one thread) of the first {c} of {a.m} components "
                        f"on the level-{a.level} sphere, {dt1:.1f} s"}
    if r.returncode != 0:
        return {"value": rate1, "unit": "DoF-steps/s", "cores": 1, "kind": "oracle", "sample": single["sample"],
                "cpu_model": cpu_model(), "nproc": ncores, "all_cores_error": r.stderr[-300:]}
    rate, dt, used = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": rate, "unit": "DoF-steps/s", "cores": used, "kind": "oracle",
            "sample": f"2 oracle steps (FP64 numpy/scipy) of all {a.m} components on the level-{a.level} sphere, "
                      f"the {a.m} step-1 solves spread over {used} worker processes (one BLAS thread each), "
                      f"after one warm-up step, {dt:.1f} s",
            "cpu_model": cpu_model(), "nproc": ncores, "single_thread": single}


# ---------------------------------------------------------------- our arm


class nvtx_range:
    """An NVTX push/pop range (a no-op where NVTX is unavailable): the kernel
    timing launches run inside "time_<kernel>", so that a profiler capture
    can select them (ncu --nvtx --nvtx-include "time_<kernel>/")."""

    def __init__(self, name):
        self.name, self.pushed = name, False

    def __enter__(self):
        try:
            import torch

            torch.cuda.nvtx.range_push(self.name)
            self.pushed = True
        except Exception:
            pass
        return self

    def __exit__(self, *exc):
        if self.pushed:
            import torch

            torch.cuda.nvtx.range_pop()
        return False


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def kernel_bytes(n, ntri, m_pad, s, W=8):
    """Algorithmic bytes per launch of each hot-path kernel.

    V = N * m_pad * s is one state-sized vector.  Gathered neighbour rows
    count once (each unique row is needed once); the padded-ELL matrix rows
    are W int32 columns plus W values per vertex, the Jacobi diagonal N * s.
      k_start  read X and the carried correction Y, write Z, columns + K + M + A values,
               Jacobi inverse diagonal
      k_cg_a   first iteration of a solve: read z and the diagonal of A; write q = A z
               (p = z stays in Z); columns + A values; later even iterations also read
               p_old and q_old and write p; odd iterations also read Y and p_{j-2} and
               write Y (two solution updates)
      k_cg_b   read Z, q; write Z; diagonal of A and its inverse; in the first iteration of
               a solve that goes on also write p_1 = z_0
      k_finish read X, Y, the last two corrections and p (with two pending updates, after an
               odd count of 3 or more, also p of the iteration before); write X, the next
               step's predicted correction Y and this step's correction (over the older of the
               two)
      k_energy_check / k_energy  read X, triangle corners (3 int32) and areas
    """
    V = n * m_pad * s
    ell = n * W * 4
    return {
        "k_start": 3 * V + ell + 3 * n * W * s + n * s,
        "k_cg_a_first": 2 * V + ell + n * W * s + n * s,
        "k_cg_a_even": 5 * V + ell + n * W * s,
        "k_cg_a_odd": 8 * V + ell + n * W * s,
        "k_cg_b": 3 * V + 2 * n * s,
        "k_cg_b_first": 4 * V + 2 * n * s,
        "k_finish_one": 8 * V,
        "k_finish_two": 9 * V,
        "k_energy_check": V + ntri * (12 + s),
        "k_energy": V + ntri * (12 + s),
    }


def pass_counts(kcg):
    """Launches per step of each form of the CG passes and of the finish pass
    for a mean of kcg CG iterations per step (linear between the two integer
    counts around it): a solve of k >= 1 iterations runs pass A once in its
    first form, floor(k / 2) times in its odd form and ceil(k / 2) - 1 times in
    its later even form; pass B not at all when k = 1 (the first pass A ends
    the solve), else once in its first form and k - 1 times in its later form;
    the finish pass has two pending updates when k is odd and at least 3.
    (A solve of one iteration whose residual lies within the first pass A's
    rounding margin of the tolerance also runs pass B; not counted.)"""
    def at(k):
        if k <= 0:
            return {"first": 0.0, "odd": 0.0, "even": 0.0, "b_first": 0.0, "b_later": 0.0,
                    "fin_one": 1.0, "fin_two": 0.0}
        return {"first": 1.0, "odd": float(k // 2), "even": float((k + 1) // 2 - 1),
                "b_first": 1.0 if k >= 2 else 0.0, "b_later": float(k - 1) if k >= 2 else 0.0,
                "fin_one": 0.0 if (k % 2 == 1 and k >= 3) else 1.0,
                "fin_two": 1.0 if (k % 2 == 1 and k >= 3) else 0.0}
    lo = int(math.floor(kcg))
    f = kcg - lo
    a, b = at(lo), at(lo + 1)
    return {k: (1 - f) * a[k] + f * b[k] for k in a}


def run_ours(a, rank, ws, local):
    import numpy as np
    import torch

    import paper_1408_2355_gb300 as seg
    import workload as w

    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    xyz, tri = w.icosphere(a.level)
    n = xyz.shape[0]
    mesh = seg.seg_create_mesh(xyz, tri)
    stream = torch.cuda.Stream()

    tunes = {}

    problems = {}

    def make(prec, m=None, rtol=0.0, tune=True):
        m = a.m if m is None else m
        if prec not in problems:
            problems[prec] = seg.seg_assemble(mesh, a.tau, prec)
        prob = problems[prec]
        prm = seg.seg_params()
        prm.check_every = 1      # energy + stop-rule pass in every step
        prm.energy_tol = -1.0    # ... but never stop: time exactly K steps
        prm.launch_mode = 1 if a.launch_mode == "direct" else 0
        prm.grid_blocks = a.grid_blocks
        prm.cg_rtol = rtol
        st = seg.seg_state_create(prob, m, a.eps, seg.SEG_INIT_UNIFORM, a.seed, prm, stream.cuda_stream)
        # the first steps of the run (set-up, not timed), then the launch
        # geometry by measurement
        seg.seg_step(st, a.setup_steps)
        if tune and not a.no_autotune:
            tunes[(prec, m, rtol)] = seg.seg_autotune(st, 10)
        return prob, st

    def timed(st, K, W, before=None):
        seg.seg_step(st, W)
        if before is not None:
            before(st)
        s0 = seg.seg_get_stats(st)
        barrier(ws)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with nvtx_range("timed_window"):
            seg.seg_step(st, K)  # the public call: enqueues in chunks, reviewing the step graph as it goes
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        ms = e0.elapsed_time(e1)
        s1 = seg.seg_get_stats(st)
        return ms, s0, s1

    # clocks sampled from the set-up on: the timed window alone (K steps of
    # ~0.3 ms) is shorter than nvidia-smi's 200 ms sampling period
    clocks = ClockSampler(dev_index)
    clocks.start()
    prob, st = make(seg.SEG_MIXED_FP32)
    info = seg.seg_problem_info(prob)
    li = seg.seg_launch_info(st)
    kept = {}

    def keep_checkpoint(st_):
        # the state at the start of the timed window, in pinned host memory:
        # the end-to-end run below starts from it
        buf = torch.empty(seg.seg_checkpoint_size(st_), dtype=torch.uint8).pin_memory()
        seg.seg_get_checkpoint(st_, buf.numpy())
        kept["ck"] = buf

    ms, s0, s1 = timed(st, a.steps, a.warmup, keep_checkpoint)
    clk = clocks.stop()
    clk["window"] = "the set-up steps, the autotuner and the timed steps of the headline state"
    ms = max_over_ranks(ms, ws)
    dcg = s1["cg_iterations"] - s0["cg_iterations"]
    launches = s1["kernel_launches"] - s0["kernel_launches"]  # counted on the device
    value = ws * n * a.m * a.steps / (ms / 1e3)
    e_final = seg.seg_energy(st)

    e2e = None
    if not a.no_e2e:
        # the same K steps end to end through the public API: the state at the
        # start of the window comes from pinned host memory (a checkpoint:
        # the stored state, the corrections its next solves start from and
        # the control block), every step's statistics (the energy of its
        # stop-rule check) are read back -- step k's while step k + 1 runs --
        # and the final state goes out to pinned host memory
        ck = kept["ck"].numpy()
        Uout = torch.empty((n, a.m), dtype=torch.float64).pin_memory()
        barrier(ws)
        t0 = time.perf_counter()
        seg.seg_set_checkpoint(st, ck)
        energies = []
        prev = None
        for _ in range(a.steps):
            seg.seg_step_async(st, 1)
            ticket = seg.seg_stats_enqueue(st)
            if prev is not None:
                energies.append(seg.seg_stats_wait(st, prev)["last_check_total"])
            prev = ticket
        energies.append(seg.seg_stats_wait(st, prev)["last_check_total"])
        seg.seg_sync(st)
        seg.seg_get_u(st, Uout)
        t1 = time.perf_counter()
        dt = max_over_ranks(t1 - t0, ws)
        assert len(energies) == a.steps and all(math.isfinite(e) for e in energies)
        # the same steps as the device-timed window: the same final energy
        e_check = seg.seg_energy(st)["total"]
        e2e = {"value": ws * n * a.m * a.steps / dt, "unit": "DoF-steps/s",
               "h2d_bytes_per_step": ck.nbytes / a.steps,
               "d2h_bytes_per_step": n * a.m * 8 / a.steps + seg.SEG_STATS_COPY_BYTES,
               "same_final_energy_as_device_window": e_check == e_final["total"],
               "note": "seg_set_checkpoint from pinned host (the state at the start of the timed window); "
                       "K x (seg_step_async + seg_stats_enqueue, then seg_stats_wait of the step before: every "
                       "step's statistics read back while the next step runs); seg_get_u to pinned host"}

    # live per-launch durations of the hot-path kernels with CUDA events on
    # the state's stream (same launch geometry as inside the step graph)
    peak, peak_kind = measured_peak()
    kb = kernel_bytes(n, int(tri.shape[0]), li["padded_m"], 4)
    kern = {}
    # seg_time_kernel selectors of each kernel form
    names = {"k_start": 0, "k_cg_a_first": 1, "k_cg_b": 2, "k_finish_one": 3, "k_energy_check": 4, "k_energy": 5,
             "k_cg_a_odd": 6, "k_finish_two": 7, "k_cg_a_even": 8, "k_cg_b_first": 9}
    for name, which in names.items():
        with nvtx_range("time_" + name):
            t = seg.seg_time_kernel(st, which, 20)
        kern[name] = {"ms": t, "bytes": kb[name], "GBps": kb[name] / (t / 1e3) / 1e9,
                      "frac": kb[name] / (t / 1e3) / 1e9 / peak}
    seg.seg_set_checkpoint(st, kept["ck"].numpy())  # the timing launches overwrote the state
    # per-step kernel time: each form of CG pass A and of the finish pass
    # weighted by its launches per step at the measured CG iterations per step
    # (pass_counts); the energy check runs every step here
    kcg = dcg / a.steps
    pc = pass_counts(kcg)

    def mix(forms):
        # (mean ms, mean bytes, launches per step, the form with the most launches)
        c = sum(w for _, w in forms)
        top = max(forms, key=lambda fw: fw[1])[0]
        if c <= 0:
            return kern[forms[0][0]]["ms"], kb[forms[0][0]], 0.0, forms[0][0]
        return (sum(kern[f]["ms"] * w for f, w in forms) / c, sum(kb[f] * w for f, w in forms) / c, c, top)

    per = {
        "k_start": (kern["k_start"]["ms"], kb["k_start"], 1.0, "k_start"),
        "k_energy_check": (kern["k_energy_check"]["ms"], kb["k_energy_check"], 1.0, "k_energy_check"),
        "k_cg_a": mix([("k_cg_a_first", pc["first"]), ("k_cg_a_odd", pc["odd"]), ("k_cg_a_even", pc["even"])]),
        "k_cg_b": mix([("k_cg_b_first", pc["b_first"]), ("k_cg_b", pc["b_later"])]),
        "k_finish": mix([("k_finish_one", pc["fin_one"]), ("k_finish_two", pc["fin_two"])]),
    }
    share = {k: t * c for k, (t, _, c, _) in per.items()}
    tot_share = sum(share.values())

    def roofline_of(name):
        t, b, c, form = per[name]
        got = b / (t / 1e3) / 1e9
        # the captured traffic of the form the figures are (mostly) of, if only that form runs
        single = (t == kern[form]["ms"])
        return {"bound": "hbm", "kernel": f"{name} ({KERNEL_ROLE[name]})", "achieved": got, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": got / peak,
                "traffic": TRAFFIC.get(form) if single else None, "form": form,
                "frac_of_nominal": got / HBM_NOMINAL_GBS, "peak_nominal": HBM_NOMINAL_GBS,
                "bytes_per_launch": b, "launch_ms": t, "launches_per_step": c,
                "share_of_kernel_time": share[name] / tot_share}

    dominant = max(share, key=share.get)

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "DoF-steps/s",
        "n_gpus": ws,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "impl": "ours",
        "config": {
            "workload": workload_name(a),
            "n_vert": n,
            "n_tri": int(tri.shape[0]),
            "nnz": info["nnz"],
            "m": a.m,
            "precision": "mixed: f32 vectors/matrices/exp, inner products and CG scalars to f64 accuracy",
            "cg_rtol": 1e-7,
            "energy_every_step": True,
            "l2": "inputs larger than L2: 8 state vectors x 42 MB + 84 MB of padded-ELL matrices > 129 MB L2",
            "grid_blocks": li["grid_blocks"],
            "launch_mode": a.launch_mode,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
        },
        "cg_iterations_per_step": dcg / a.steps,
        "final_total_energy": e_final["total"],
        "gpu_launches": launches,
        "clocks": clk,
        # the kernel with the largest share of the kernel time per step, and
        # CG pass A, the bandwidth-bound pass of the solve
        "roofline": roofline_of(dominant),
        "roofline_cg_a": roofline_of("k_cg_a"),
        "step_roofline": {"bytes_per_step": sum(b * c for _, b, c, _ in per.values()),
                          "achieved": sum(b * c for _, b, c, _ in per.values()) / (ms / a.steps / 1e3) / 1e9,
                          "peak": peak, "unit": "GB/s",
                          "frac": sum(b * c for _, b, c, _ in per.values()) / (ms / a.steps / 1e3) / 1e9 / peak,
                          "bytes": "this design's streams (per-kernel model above) x launches per step"},
        "step_roofline_method": method_roofline(n, int(tri.shape[0]), info["nnz"], li["padded_m"], 4, kcg,
                                                ms / a.steps, peak),
        "kernels": kern,
    }

    if e2e is not None:
        out["e2e"] = e2e

    out["config"]["autotune"] = tunes.get((seg.SEG_MIXED_FP32, a.m, 0.0))
    out["config"]["setup_steps"] = a.setup_steps
    out["config"]["timed_steps"] = f"steps {a.setup_steps + a.warmup + 1}..{a.setup_steps + a.warmup + a.steps} of the run"
    del st

    def arm(prec, m=None, rtol=0.0):
        _, s_ = make(prec, m, rtol)
        ms_, s0_, s1_ = timed(s_, a.steps, a.warmup)
        ms_ = max_over_ranks(ms_, ws)
        mm = a.m if m is None else m
        return {"value": ws * n * mm * a.steps / (ms_ / 1e3), "unit": "DoF-steps/s", "steps": a.steps,
                "ms_per_step": ms_ / a.steps,
                "cg_iterations_per_step": (s1_["cg_iterations"] - s0_["cg_iterations"]) / a.steps,
                "grid_blocks": seg.seg_launch_info(s_)["grid_blocks"]}

    if not a.no_fp64:
        out["fp64"] = arm(seg.SEG_FP64)
        out["fp64"]["cg_rtol"] = 1e-12
        out["mixed_over_fp64"] = out["value"] / out["fp64"]["value"]
        out["mixed_over_fp64_is"] = ("precision (f32 vs f64 vectors) + CG tolerance (1e-7 vs 1e-12) + predictor "
                                     "order (quadratic vs cubic): each mode at its own default")
        out["fp64_rtol_1e-7"] = arm(seg.SEG_FP64, rtol=1e-7)
        out["mixed_over_fp64_same_rtol"] = out["value"] / out["fp64_rtol_1e-7"]["value"]
    others = {}
    for mm in [int(x) for x in a.other_m.split(",") if x.strip()]:
        if mm != a.m and 1 <= mm <= 32:
            others[str(mm)] = arm(seg.SEG_MIXED_FP32, m=mm)
    if others:
        out["other_m"] = others
    if a.run_steps > 0:
        out["full_run"] = full_run(a, seg, problems[seg.SEG_MIXED_FP32], stream, n, ws)
    return out


def method_roofline(n, ntri, nnz, m_pad, s, kcg, ms_step, peak):
    """Bytes per step of the method (not of this design), per the scope of the
    hot path: B_step = k_CG (A_b + 8V) + 4V + K_b + M_b with V = N m s one
    state vector, A_b = K_b = M_b = 4 (N + 1) + nnz (4 + s) one CSR matrix, plus
    the stop-rule energy pass V + 12 F (three corner indices per triangle),
    which the bench runs every step."""
    V = n * m_pad * s
    Ab = 4 * (n + 1) + nnz * (4 + s)
    b = kcg * (Ab + 8 * V) + 4 * V + 2 * Ab + V + 12 * ntri
    got = b / (ms_step / 1e3) / 1e9
    return {"bytes_per_step": b, "cg_iterations_per_step": kcg, "achieved": got, "unit": "GB/s", "peak": peak,
            "frac": got / peak, "frac_of_nominal": got / HBM_NOMINAL_GBS,
            "model": "k_CG (A_b + 8V) + 4V + K_b + M_b + (V + 12F), A_b = 4(N+1) + nnz(4+s), V = N m s"}


def full_run(a, seg, prob, stream, n, ws):
    """The configured run whole: a fresh state from the seeded initial data,
    autotuned after --setup-steps, then stepped to --run-steps in chunks of
    500 steps timed with CUDA events (the set-up and the autotuner's own
    launches are outside the chunks).  Reports DoF-steps/s over all chunks
    and, per chunk, ms per step and CG iterations per step: the solves start
    from a correction predicted from the last ones, whose benefit grows over
    the first hundreds of steps."""
    import torch

    prm = seg.seg_params()
    prm.check_every = 1
    prm.energy_tol = -1.0
    st = seg.seg_state_create(prob, a.m, a.eps, seg.SEG_INIT_UNIFORM, a.seed, prm, stream.cuda_stream)
    t_ms, chunks, done = 0.0, [], 0
    first = min(a.setup_steps, a.run_steps)

    def chunk(k):
        s0 = seg.seg_get_stats(st)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        seg.seg_step(st, k)
        e1.record(stream)
        torch.cuda.synchronize()
        s1 = seg.seg_get_stats(st)
        return e0.elapsed_time(e1), (s1["cg_iterations"] - s0["cg_iterations"]) / k

    if first:
        ms_, cg_ = chunk(first)
        t_ms += ms_
        chunks.append([first, round(ms_ / first, 4), round(cg_, 2)])
        done = first
    if not a.no_autotune:
        seg.seg_autotune(st, 10)
    while done < a.run_steps:
        k = min(500, a.run_steps - done)
        ms_, cg_ = chunk(k)
        t_ms += ms_
        done += k
        chunks.append([done, round(ms_ / k, 4), round(cg_, 2)])
    t_ms = max_over_ranks(t_ms, ws)
    return {"steps": a.run_steps, "value": ws * n * a.m * a.run_steps / (t_ms / 1e3), "unit": "DoF-steps/s",
            "ms_per_step": t_ms / a.run_steps, "final_total_energy": seg.seg_energy(st)["total"],
            "chunks": "[last step, ms per step, CG iterations per step] per chunk",
            "per_chunk": chunks}


SERVE_MESHES = [("sphere", 4), ("sphere", 5), ("sphere", 6), ("sphere", 7), ("torus", 128, 64),
                ("torus", 256, 128), ("torus", 512, 256), ("ellipsoid", 5), ("ellipsoid", 6), ("ellipsoid", 7)]


def _serve_mesh(spec):
    import workload as w

    if spec[0] == "sphere":
        return w.icosphere(spec[1])
    if spec[0] == "torus":
        return w.torus(spec[1], spec[2], 1.0, 0.4)
    return w.ellipsoid(spec[1], 1.0, 0.8, 0.6)


SERVE_STREAM_LEN = 256


def serve_eps(a, level):
    """eps of level 0..7: geometric between --serve-eps-min and 1e-2."""
    return a.serve_eps_min * (1e-2 / a.serve_eps_min) ** (level / 7)


def serve_stream(a):
    """The seeded request stream of the serving benchmark: 256 requests, of
    which the first --serve-requests are served.

    Each request picks a mesh from SERVE_MESHES, m uniform in {2..24} and eps
    log-uniform in [--serve-eps-min, 1e-2], drawn from 8 geometric levels so
    that the (mesh, tau) problems are assembled once, before the stream
    starts, and shared; tau = --serve-tau-factor * eps^2.  Arrival times are a
    Poisson process of rate --serve-rate.
    """
    import numpy as np

    rng = np.random.default_rng(a.seed + 5)
    arrivals = np.cumsum(rng.exponential(1.0 / a.serve_rate, SERVE_STREAM_LEN))
    reqs = [(int(rng.integers(len(SERVE_MESHES))), int(rng.integers(2, 25)), int(rng.integers(8)))
            for _ in range(SERVE_STREAM_LEN)]
    n = min(a.serve_requests, SERVE_STREAM_LEN)
    return arrivals[:n], reqs[:n]


def serve_problems(seg, a, reqs, prec):
    """{(mesh index, eps level): (problem, eps, tau)} for the requests' pairs."""
    problems, meshes = {}, {}
    for mi, _, ci in reqs:
        if (mi, ci) in problems:
            continue
        if mi not in meshes:
            meshes[mi] = seg.seg_create_mesh(*_serve_mesh(SERVE_MESHES[mi]))
        eps = serve_eps(a, ci)
        tau = a.serve_tau_factor * eps * eps
        problems[(mi, ci)] = (seg.seg_assemble(meshes[mi], tau, prec), eps, tau)
    return problems


def serve_params(seg, a, tau, converge=True):
    """A request's parameters: checks every dt of simulated time, the relative
    stop rule, a budget of t_max simulated time (converge=False: a fixed step
    count and no stop rule, for throughput comparisons)."""
    prm = seg.seg_params()
    if converge:
        prm.check_every = max(1, round(a.serve_check_dt / tau))
        prm.energy_tol = -1.0
        prm.energy_rtol = a.serve_rtol
        prm.max_steps = max(1, round(a.serve_t_max / tau))
    else:
        prm.check_every = max(1, round(a.serve_check_dt / tau))
        prm.energy_tol = -1.0
        prm.max_steps = a.serve_compare_steps
    return prm


def run_serving(a, seg, prec, stream):
    """Requests through the continuous-batching server.

    stream=True: each request is submitted at its Poisson arrival time (real
    time on the server clock); stream=False: all are submitted at once (a
    burst, for throughput).  Every request runs to its stop rule (|change of
    the total energy| < --serve-tol between checks --serve-check-every steps
    apart) or --serve-max-steps.  Latency = completion - arrival.
    """
    import numpy as np

    arrivals, reqs = serve_stream(a)
    if not stream:
        arrivals, reqs = np.zeros(a.serve_compare), reqs[:a.serve_compare]
    problems = serve_problems(seg, a, reqs, prec)
    sp = seg.seg_server_params()
    sp.steps_per_tick = a.serve_quantum
    srv = seg.seg_server_create(sp)
    n_req = len(reqs)
    ids = [None] * n_req
    nxt = 0
    t_start = seg.seg_server_clock(srv)
    while True:
        now = seg.seg_server_clock(srv) - t_start
        while nxt < n_req and arrivals[nxt] <= now:
            mi, m, ci = reqs[nxt]
            prob, eps, tau = problems[(mi, ci)]
            ids[nxt] = seg.seg_server_submit(srv, prob, m, eps, seg.SEG_INIT_UNIFORM,
                                             a.seed + 1000 + nxt, serve_params(seg, a, tau, converge=stream))
            nxt += 1
        running, queued = seg.seg_server_tick(srv)
        if nxt == n_req and running == 0 and queued == 0:
            break
        if running == 0 and queued == 0:
            time.sleep(max(0.0, min(0.01, arrivals[nxt] - now)))
    makespan = seg.seg_server_clock(srv) - t_start
    lat, lat_conv, dof_steps, conv, failed, steps = [], [], 0.0, 0, 0, []
    for k, rid in enumerate(ids):
        info = seg.seg_server_info(srv, rid)
        if info["phase"] != 2:
            failed += 1
            continue
        t = info["t_done"] - t_start - arrivals[k]
        lat.append(t)
        if info["converged"]:
            lat_conv.append(t)
        steps.append(info["steps"])
        dof_steps += info["n_vert"] * info["m"] * info["steps"]
        conv += info["converged"]
    seg.seg_server_destroy(srv)
    lat = np.array(lat)
    out = {
        "value": dof_steps / makespan, "unit": "DoF-steps/s", "completed": int(len(lat)), "failed": failed,
        "converged_fraction": conv / max(1, len(lat)),
        "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "latency": "arrival to completion (stop rule met, or the step budget)",
        "makespan_s": makespan, "dof_steps": dof_steps,
        "steps_p50": float(np.percentile(steps, 50)) if steps else None,
        "steps_max": int(max(steps)) if steps else None,
    }
    if stream:
        out["p50_time_to_converged_s"] = float(np.percentile(lat_conv, 50)) if lat_conv else None
        out["p99_time_to_converged_s"] = float(np.percentile(lat_conv, 99)) if lat_conv else None
    return out


def run_alone(a, seg, prec):
    """The burst's requests, one after another, each stepped alone (seg_step)."""
    import torch

    reqs = serve_stream(a)[1][:a.serve_compare]
    problems = serve_problems(seg, a, reqs, prec)
    dof_steps = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, (mi, m, ci) in enumerate(reqs):
        prob, eps, tau = problems[(mi, ci)]
        st = seg.seg_state_create(prob, m, eps, seg.SEG_INIT_UNIFORM, a.seed + 1000 + k,
                                  serve_params(seg, a, tau, converge=False))
        steps = seg.seg_step(st, a.serve_compare_steps)
        seg.seg_get_u(st)
        dof_steps += seg.seg_problem_info(prob)["n_vert"] * m * steps
        del st
    dt = time.perf_counter() - t0
    return {"value": dof_steps / dt, "unit": "DoF-steps/s", "seconds": dt, "dof_steps": dof_steps}


def batched_section(a):
    """Two instances in one launch per pass: torus 1024 x 512 (R = 1, r = 0.4)
    and the level-8 ellipsoid (semi-axes 1, 0.8, 0.6), m = 12, eps = 1e-3,
    tau = 5e-6, mixed precision; each member autotuned first.  DoF-steps/s of
    the batch against the two states stepped one after the other."""
    import torch

    import paper_1408_2355_gb300 as seg
    import workload as w

    meshes = [w.torus(1024, 512, 1.0, 0.4), w.ellipsoid(a.level, 1.0, 0.8, 0.6)]
    m, steps = 12, a.batch_steps
    prm = seg.seg_params()
    prm.check_every = 1
    prm.energy_tol = -1.0
    states, probs, dof = [], [], 0
    for k, (xyz, tri) in enumerate(meshes):
        prob = seg.seg_assemble(seg.seg_create_mesh(xyz, tri), a.tau, seg.SEG_MIXED_FP32)
        st = seg.seg_state_create(prob, m, a.eps, seg.SEG_INIT_UNIFORM, a.seed + 10 + k, prm)
        seg.seg_step(st, 20)
        seg.seg_autotune(st, 5)
        probs.append(prob)
        states.append(st)
        dof += xyz.shape[0] * m
    # both arms run the same steps from the same state (a checkpoint of each
    # member after the set-up), so they do the same work
    cks = [seg.seg_get_checkpoint(st) for st in states]
    batch = seg.seg_batch_create(states)
    seg.seg_batch_step(batch, 3)  # warm-up (builds the batch's graph)
    for st, ck in zip(states, cks):
        seg.seg_set_checkpoint(st, ck)
    it0 = [seg.seg_get_stats(st)["cg_iterations"] for st in states]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seg.seg_batch_step(batch, steps)
    t_batch = time.perf_counter() - t0
    e_batch = [seg.seg_energy(st)["total"] for st in states]
    it_batch = [seg.seg_get_stats(st)["cg_iterations"] for st in states]
    # the same batch in the persistent mode: one cooperative launch for all
    # the steps
    seg.seg_batch_set_persistent(batch, True)
    seg.seg_batch_step(batch, 3)  # warm-up
    for st, ck in zip(states, cks):
        seg.seg_set_checkpoint(st, ck)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seg.seg_batch_step(batch, steps)
    t_persist = time.perf_counter() - t0
    e_persist = [seg.seg_energy(st)["total"] for st in states]
    it_persist = [seg.seg_get_stats(st)["cg_iterations"] for st in states]
    del batch
    for st, ck in zip(states, cks):
        seg.seg_step(st, 3)  # warm-up (builds the member's own graph)
        seg.seg_set_checkpoint(st, ck)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for st in states:
        seg.seg_step(st, steps)
    t_alone = time.perf_counter() - t0
    e_alone = [seg.seg_energy(st)["total"] for st in states]
    it_alone = [seg.seg_get_stats(st)["cg_iterations"] for st in states]
    return {"workload": "torus 1024x512 + ellipsoid level %d, m = 12, eps = %g, tau = %g, mixed" % (a.level, a.eps, a.tau),
            "steps": steps, "value": dof * steps / t_batch, "unit": "DoF-steps/s",
            "alone_one_after_the_other": dof * steps / t_alone, "batch_over_alone": t_alone / t_batch,
            "same_results": e_batch == e_alone and it_batch == it_alone,
            "persistent": {"value": dof * steps / t_persist, "persistent_over_alone": t_alone / t_persist,
                           "same_results": e_persist == e_alone and it_persist == it_alone},
            "small_instances": small_batch_arms(seg, torch),
            "cg_iterations_per_step": [(i - c) / steps for i, c in zip(it_batch, it0)],
            "timing": "host clock around synchronous calls, every arm from the same checkpoint of the members "
                      "after 20 set-up steps and the autotuner, energy check every step"}


def small_batch_arms(seg, torch, level=4, n=8, m=8, steps=400):
    """Eight small instances (level-4 spheres, N = 2562, m = 8, eps = 2e-2,
    tau = 1e-4, seeds 50..57, mixed): ms per step of the batch's step graph,
    of its persistent kernel and of the instances stepped one after the
    other, all from the same checkpoints."""
    import workload as w

    xyz, tri = w.icosphere(level)
    prob = seg.seg_assemble(seg.seg_create_mesh(xyz, tri), 1e-4, seg.SEG_MIXED_FP32)
    prm = seg.seg_params()
    prm.check_every = 1
    prm.energy_tol = -1.0
    states = [seg.seg_state_create(prob, m, 2e-2, seg.SEG_INIT_UNIFORM, 50 + k, prm) for k in range(n)]
    for st in states:
        seg.seg_step(st, 20)
    cks = [seg.seg_get_checkpoint(st) for st in states]
    out, finals = {}, {}
    batch = seg.seg_batch_create(states)
    for arm in ("graph", "persistent", "alone"):
        if arm == "persistent":
            seg.seg_batch_set_persistent(batch, True)
        for st, ck in zip(states, cks):
            seg.seg_set_checkpoint(st, ck)
        if arm == "alone":
            for st in states:
                seg.seg_step(st, 3)
        else:
            seg.seg_batch_step(batch, 3)
        for st, ck in zip(states, cks):
            seg.seg_set_checkpoint(st, ck)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if arm == "alone":
            for st in states:
                seg.seg_step(st, steps)
        else:
            seg.seg_batch_step(batch, steps)
        out[arm + "_ms_per_step"] = (time.perf_counter() - t0) / steps * 1e3
        finals[arm] = [seg.seg_energy(st)["total"] for st in states]
    del batch
    out["same_results"] = finals["graph"] == finals["alone"] and finals["persistent"] == finals["alone"]
    out["workload"] = f"{n} x sphere level {level} (N = {xyz.shape[0]}), m = {m}, eps = 2e-2, tau = 1e-4, mixed, {steps} steps"
    return out


def serving_section(a):
    """Serving benchmark: the Poisson stream (latency), and the first
    --serve-compare requests as a burst through the server in mixed precision
    against the same requests each stepped alone in FP64 and in mixed
    precision (throughput)."""
    import paper_1408_2355_gb300 as seg

    out = {"requests": min(a.serve_requests, SERVE_STREAM_LEN),
           "stream": f"the first {min(a.serve_requests, SERVE_STREAM_LEN)} of a seeded {SERVE_STREAM_LEN}-request "
                     f"stream, Poisson arrivals at {a.serve_rate:g}/s",
           "mix": "meshes " + ", ".join("-".join(map(str, s)) for s in SERVE_MESHES)
                  + f"; m ~ U{{2..24}}; eps log-uniform in [{a.serve_eps_min:g}, 1e-2] on 8 levels; "
                    f"tau = {a.serve_tau_factor:g} eps^2; uniform random initial data",
           "stop_rule": {"check_every": f"round({a.serve_check_dt:g} / tau) steps",
                         "energy_rtol": a.serve_rtol,
                         "meaning": "|E_k - E_prev| <= rtol |E_k| between checks",
                         "budget": f"round({a.serve_t_max:g} / tau) steps"},
           "compared_requests": a.serve_compare,
           "compare_steps": a.serve_compare_steps,
           "steps_per_tick": a.serve_quantum}
    out["stream_mixed"] = run_serving(a, seg, seg.SEG_MIXED_FP32, True)
    out["burst_mixed"] = run_serving(a, seg, seg.SEG_MIXED_FP32, False)
    out["alone_mixed"] = run_alone(a, seg, seg.SEG_MIXED_FP32)
    out["alone_fp64"] = run_alone(a, seg, seg.SEG_FP64)
    out["burst_mixed_over_alone_fp64"] = out["burst_mixed"]["value"] / out["alone_fp64"]["value"]
    out["burst_mixed_over_alone_mixed"] = out["burst_mixed"]["value"] / out["alone_mixed"]["value"]
    return out


def run_reference(a, rank, ws):
    """The oracle as the reference arm, timed on the host cores (rank 0 only)."""
    import numpy as np

    import workload as w
    from oracle import seg_oracle as o

    xyz, tri = w.icosphere(a.level)
    n = xyz.shape[0]
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, w.uniform01(a.seed, n, a.m))
    t0 = time.perf_counter()
    o.heat_step(M, K, a.tau, U[:, :1])
    t_col = time.perf_counter() - t0
    per_step = a.reference_budget_seconds / max(1, a.steps + a.warmup)
    c = int(max(1, min(a.m, per_step // max(t_col, 1e-9))))
    for _ in range(a.warmup):
        U[:, :c] = o.step(M, K, a.tau, a.eps, U[:, :c])
    t0 = time.perf_counter()
    for _ in range(a.steps):
        U[:, :c] = o.step(M, K, a.tau, a.eps, U[:, :c])
    dt = time.perf_counter() - t0
    value = n * c * a.steps / dt
    sample = (f"each step: one FP64 oracle step (numpy/scipy, single thread) of the first {c} of {a.m} "
              f"components on the level-{a.level} sphere")
    return {
        "metric": METRIC, "value": value, "unit": "DoF-steps/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(a), "n_vert": n, "m": a.m, "components_per_sample": c},
        "cpu_baseline": {"value": value, "unit": "DoF-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DoF-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    a = parse()
    rank, ws, local = dist_setup(a)
    if a.impl == "reference":
        if rank == 0:
            os.environ.setdefault("OMP_NUM_THREADS", "1")
            print(json.dumps(run_reference(a, rank, ws)), flush=True)
        return
    out = run_ours(a, rank, ws, local)
    if rank == 0:
        if a.batch_steps > 0 and ws == 1:
            out["batched"] = batched_section(a)
        if a.serve_requests > 0 and ws == 1:
            out["serving"] = serving_section(a)
        if not a.no_cpu_baseline and ws == 1:  # the oracle baseline at N = 1 only
            out["cpu_baseline"] = cpu_baseline(a)
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
