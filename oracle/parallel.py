"""Column-parallel driver of the FP64 oracle's time loop.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the test-suite, the
scripts that write stored expected values under ``tests/golden/`` and the
CPU-baseline leg of ``bench.py`` may use it; the library never does.

Step 1 of Algorithm 2.2 is m independent linear solves, one per component:
(M + tau K) u~_i = M u_i^k.  This module runs those solves in worker
processes.  Each worker calls ``seg_oracle.pcg`` exactly as
``seg_oracle.heat_step`` does -- the same matrix A = M + tau K, the column i of
the same right-hand side M U and the same start u_i^k, as strided views of
C-ordered (n, m) arrays -- and steps 2 and 3 run in the parent with
``seg_oracle.segregation_step`` and ``seg_oracle.normalise``.  The arithmetic
is therefore that of ``seg_oracle.step``; the results are bitwise the same
(tested on a small mesh) except where a multithreaded BLAS in the calling
process splits the dot products of a long vector differently from the
workers' single BLAS thread, which changes their rounding only.  The workers are started with the ``spawn`` method,
so the pool may be created in a process that has already used a GPU.
"""

from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np
import scipy.sparse as sp

from . import seg_oracle as o

_W = {}
_BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _attach(name, shape):
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=np.float64, buffer=shm.buf)


def _worker_init(a_parts, n, m, names, rtol):
    data, indices, indptr = a_parts
    _W["A"] = sp.csr_matrix((data, indices, indptr), shape=(n, n))
    _W["rtol"] = rtol
    _W["shm"] = []
    for key, name in zip(("B", "U", "OUT"), names):
        shm, arr = _attach(name, (n, m))
        _W["shm"].append(shm)
        _W[key] = arr


def _worker_solve(cols):
    A, B, U, OUT = _W["A"], _W["B"], _W["U"], _W["OUT"]
    its = []
    for i in cols:
        x, k = o.pcg(A, B[:, i], U[:, i], rtol=_W["rtol"])
        OUT[:, i] = x
        its.append(k)
    return its


class ColumnPool:
    """Worker processes that solve step 1 of Algorithm 2.2 column by column.

    ``heat_step(U)`` equals ``seg_oracle.heat_step(M, K, tau, U, rtol)`` bitwise
    and ``step(U, eps)`` equals ``seg_oracle.step(M, K, tau, eps, U, rtol)``.
    Use as a context manager (the workers and the shared buffers are
    released on exit).
    """

    def __init__(self, M, K, tau, m, workers, rtol=1e-14):
        self.M, self.K, self.tau, self.m, self.rtol = M, K, tau, int(m), rtol
        self.n = M.shape[0]
        A = (M + tau * K).tocsr()  # as in seg_oracle.heat_step
        self.workers = max(1, min(int(workers), self.m))
        nbytes = self.n * self.m * 8
        self._shm = [shared_memory.SharedMemory(create=True, size=nbytes) for _ in range(3)]
        self.B, self.U, self.OUT = (np.ndarray((self.n, self.m), dtype=np.float64, buffer=s.buf) for s in self._shm)
        ctx = mp.get_context("spawn")
        # one BLAS thread per worker: the workers already fill the cores
        saved = {k: os.environ.get(k) for k in _BLAS_THREAD_VARS}
        os.environ.update({k: "1" for k in _BLAS_THREAD_VARS})
        try:
            self._pool = ctx.Pool(
                self.workers,
                initializer=_worker_init,
                initargs=((A.data, A.indices, A.indptr), self.n, self.m, [s.name for s in self._shm], rtol),
            )
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        # components dealt round-robin, so that every worker gets a similar share
        self._cols = [list(range(w, self.m, self.workers)) for w in range(self.workers)]
        self.last_iterations = None

    def heat_step(self, U):
        """Algorithm 2.2 step 1 for every component (the solves in parallel)."""
        self.U[...] = U
        self.B[...] = self.M @ U  # the right-hand side as seg_oracle.heat_step forms it
        its = self._pool.map(_worker_solve, self._cols)
        per = np.zeros(self.m, dtype=np.int64)
        for cols, k in zip(self._cols, its):
            per[cols] = k
        self.last_iterations = per
        return np.array(self.OUT, copy=True)

    def step(self, U, eps):
        """One full step of Algorithm 2.2 (steps 2 and 3 as seg_oracle.step does them)."""
        Ut = self.heat_step(U)
        Uh = o.segregation_step(Ut, self.tau, eps)
        return o.normalise(self.M, Uh)

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
        for s in self._shm:
            s.close()
            s.unlink()
        self._shm = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False
