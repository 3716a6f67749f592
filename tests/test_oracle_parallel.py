"""The column-parallel oracle driver gives bitwise the oracle's own steps."""

import numpy as np

import workload as w
from oracle import parallel
from oracle import seg_oracle as o


def test_column_pool_steps_are_bitwise_the_oracle_steps():
    xyz, tri = w.icosphere(3)
    M, K = o.assemble(xyz, tri)
    m, tau, eps = 5, 2e-4, 5e-2
    U = o.initial_state(M, w.uniform01(3, xyz.shape[0], m))
    Us = U.copy()
    with parallel.ColumnPool(M, K, tau, m, workers=2) as pool:
        for _ in range(6):
            U = pool.step(U, eps)
            Us = o.step(M, K, tau, eps, Us)
            assert np.array_equal(U, Us)
        assert pool.last_iterations.shape == (m,) and pool.last_iterations.min() >= 1
