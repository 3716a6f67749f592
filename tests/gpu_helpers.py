"""Shared helpers of the GPU parity tests (inputs from `workload`, expected
values from `oracle` only)."""

import numpy as np
import scipy.sparse as sp

import workload as w
from oracle import seg_oracle as o


def lib():
    import __graft_entry__ as g

    g.build()
    import paper_1408_2355_gb300 as seg

    return seg


def make_state(seg, xyz, tri, tau, m, eps, prec, seed=1234, init=None, **params):
    mesh = seg.seg_create_mesh(xyz, tri)
    prob = seg.seg_assemble(mesh, tau, prec)
    p = seg.seg_params()
    for k, v in params.items():
        setattr(p, k, v)
    init = seg.SEG_INIT_UNIFORM if init is None else init
    return seg.seg_state_create(prob, m, eps, init, seed, p)


def oracle_run(xyz, tri, U0, tau, eps, steps):
    M, K = o.assemble(xyz, tri)
    U = o.initial_state(M, U0)
    for _ in range(steps):
        U = o.step(M, K, tau, eps, U)
    return U, M, K


def interface_mask(tri, U, n):
    """Vertices whose 1-ring holds >= 2 distinct oracle labels, or whose
    top-two gap is below 1e-6 of the row maximum (the label-comparison
    exclusion of the design notes)."""
    am = np.argmax(U, axis=1)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], 0)
    A = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n)).tocsr()
    A = A + A.T + sp.eye(n)
    A = A.tocsr()
    mixed = np.zeros(n, dtype=bool)
    for z in range(n):
        nb = A.indices[A.indptr[z]:A.indptr[z + 1]]
        mixed[z] = len(np.unique(am[nb])) > 1
    srt = np.sort(U, axis=1)
    gap = srt[:, -1] - (srt[:, -2] if U.shape[1] > 1 else 0)
    mixed |= gap < 1e-6 * np.abs(srt[:, -1])
    return mixed


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)
