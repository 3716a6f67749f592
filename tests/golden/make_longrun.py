"""Writes the stored expected values of the long-run parity tests.

Every number in the files this script writes comes from the FP64 oracle
(``oracle/``, run column-parallel by ``oracle.parallel``, bitwise the
oracle's own steps) on the seeded inputs of ``workload``; nothing comes from
the CUDA library.  Run from the repository root:

    python tests/golden/make_longrun.py [case ...] [--workers N]

Cases (Algorithm 2.2 from uniform random initial data, Sec. 2.2):

  sphere7_m3, sphere7_m2   icosphere level 7 (N = 163 842), eps = 2e-3,
                           tau = 1e-5, 5000 steps (t = 0.05), seed 1235
  sphere8_m16              icosphere level 8 (N = 655 362), m = 16,
                           eps = 1e-3, tau = 5e-6, 1000 steps (t = 5e-3),
                           seed 1236
  torus1024_m12,           the two-instance batched workload: the torus
  ellipsoid8_m12           R = 1, r = 0.4 on a 1024 x 512 grid and the
                           level-8 ellipsoid (1, 0.8, 0.6), m = 12,
                           eps = 1e-3, tau = 5e-6, 50 steps, seeds 1237, 1238

Each file ``longrun_<case>.json`` holds, at every checkpoint, the energy
record of the oracle's state (total, functional, Dirichlet sum, S_eps, the
per-component D_i) and, at the last one, the full rows of u at a seeded
sample of vertices, the oracle label of each sampled vertex and whether its
1-ring holds more than one label (an interface vertex).  The same record is
also kept for a second oracle run started from the initial values rounded
to float32 (the values a float32 state starts from): the difference between
the two runs is the spread that the problem itself gives to a relative
perturbation of 3e-8 of the initial data.
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workload as w  # noqa: E402
from oracle import parallel  # noqa: E402
from oracle import seg_oracle as o  # noqa: E402

CASES = {
    "sphere7_m3": dict(mesh=("sphere", 7), m=3, eps=2e-3, tau=1e-5, steps=5000, every=500, seed=1235, samples=2048),
    "sphere7_m2": dict(mesh=("sphere", 7), m=2, eps=2e-3, tau=1e-5, steps=5000, every=500, seed=1235, samples=2048),
    "sphere8_m16": dict(mesh=("sphere", 8), m=16, eps=1e-3, tau=5e-6, steps=1000, every=100, seed=1236, samples=384),
    "torus1024_m12": dict(mesh=("torus", 1024, 512, 1.0, 0.4), m=12, eps=1e-3, tau=5e-6, steps=50, every=25,
                          seed=1237, samples=384),
    "ellipsoid8_m12": dict(mesh=("ellipsoid", 8, 1.0, 0.8, 0.6), m=12, eps=1e-3, tau=5e-6, steps=50, every=25,
                           seed=1238, samples=384),
}


def make_mesh(spec):
    kind = spec[0]
    if kind == "sphere":
        return w.icosphere(spec[1]), f"icosphere level {spec[1]}"
    if kind == "torus":
        return w.torus(*spec[1:]), "torus %dx%d R=%g r=%g" % spec[1:]
    return w.ellipsoid(*spec[1:]), "ellipsoid level %d semi-axes (%g, %g, %g)" % spec[1:]


def one_ring_mixed(tri, labels, n):
    """True where the closed 1-ring of a vertex holds two or more labels."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], 0)
    A = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n)).tocsr()
    A = (A + A.T).tocsr()
    lab_nb = labels[A.indices]
    row = np.repeat(np.arange(n), np.diff(A.indptr))
    differ = np.zeros(n, dtype=bool)
    np.logical_or.at(differ, row, lab_nb != labels[row])
    return differ


def record(xyz, tri, K, U, eps):
    e = o.energy(xyz, tri, K, U, eps)
    return {
        "total": e["total"],
        "functional": e["functional"],
        "dirichlet": e["dirichlet"],
        "s_eps": e["s_eps"],
        "D": [float(v) for v in e["D"]],
    }


def run_case(name, spec, workers):
    (xyz, tri), mesh_name = make_mesh(spec["mesh"])
    n, m = xyz.shape[0], spec["m"]
    M, K = o.assemble(xyz, tri)
    U0 = w.uniform01(spec["seed"], n, m)
    out = {
        "case": name,
        "mesh": mesh_name,
        "n_vert": n,
        "m": m,
        "eps": spec["eps"],
        "tau": spec["tau"],
        "seed": spec["seed"],
        "init": "uniform",
        "steps": spec["steps"],
        "oracle": "oracle.seg_oracle via oracle.parallel.ColumnPool, pcg rtol 1e-14",
    }
    for label, start in (("oracle", U0), ("oracle_f32_start", U0.astype(np.float32).astype(np.float64))):
        U = o.initial_state(M, start)
        checkpoints = [dict(step=0, **record(xyz, tri, K, U, spec["eps"]))]
        t0 = time.time()
        with parallel.ColumnPool(M, K, spec["tau"], m, workers) as pool:
            for k in range(1, spec["steps"] + 1):
                U = pool.step(U, spec["eps"])
                if k % spec["every"] == 0:
                    checkpoints.append(dict(step=k, **record(xyz, tri, K, U, spec["eps"])))
                    print(f"{name} {label} step {k} total {checkpoints[-1]['total']:.15g} "
                          f"({time.time() - t0:.0f} s)", flush=True)
        out[label] = {"checkpoints": checkpoints}
        if label == "oracle":
            rng = np.random.default_rng(spec["seed"])
            idx = np.sort(rng.choice(n, size=spec["samples"], replace=False))
            lab = np.argmax(U, axis=1)
            mixed = one_ring_mixed(tri, lab, n)
            out["sample"] = {
                "vertices": [int(v) for v in idx],
                "u": [[float(x) for x in U[v]] for v in idx],
                "label": [int(lab[v]) for v in idx],
                "ring_mixed": [int(mixed[v]) for v in idx],
            }
    path = os.path.join(HERE, f"longrun_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0, separators=(",", ":"))
        f.write("\n")
    print("wrote", path, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cases", nargs="*", default=list(CASES))
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    for name in args.cases:
        run_case(name, CASES[name], args.workers)


if __name__ == "__main__":
    main()
