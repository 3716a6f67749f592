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


def interface_mask(tri, U, n, gap_tol=0.0):
    """Vertices whose 1-ring holds >= 2 distinct oracle labels, or whose
    top-two gap is below max(1e-6 of the row maximum, gap_tol): the vertices
    on or next to an interface between components, where the argmax label is
    not determined by the solution to within the numerical error (pass gap_tol
    = twice the observed max |u_gpu - u_oracle|, so that no decision within
    that error is compared)."""
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
    mixed |= gap < np.maximum(1e-6 * np.abs(srt[:, -1]), gap_tol)
    return mixed


def check_labels(seg, st, tri, U, Ug):
    """argmax labels equal off the interface; the v > 0 flag equal wherever
    |v| exceeds the error bound 2 m max|du|.  Returns the compared fraction."""
    n, m = U.shape
    err = float(np.abs(Ug - U).max())
    am, vp = seg.seg_labels(st)
    off = ~interface_mask(tri, U, n, gap_tol=2 * err)
    amo = np.argmax(U, axis=1)
    assert np.array_equal(am[off], amo[off])
    ui = U[np.arange(n), amo]
    v = ui - (U.sum(1) - ui)
    sure = off & (np.abs(v) > 2 * m * err)
    assert np.array_equal(vp[sure], (v[sure] > 0).astype(np.uint8))
    # labels must always be valid component indices
    assert am.min() >= 0 and am.max() < m
    return off.mean()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)
