"""The allocation-free entry point seg_s_eps_noalloc.

It serves callers that cannot allocate device memory (memory reserved up
front by another framework's pool, work captured into a CUDA graph, tight
latency loops).  It must give the same S_eps and coupling integrals as the
regular energy entry points, call after call, although every call reuses the
same static scratch array inside the library.  This file is collected last so
that a failure here does not hide the other tests.
"""

import numpy as np
import pytest

import workload as w
from oracle import seg_oracle as o
from tests.gpu_helpers import lib, make_state, rel

pytestmark = pytest.mark.gpu


def test_noalloc_matches_energy_entry_points_on_consecutive_calls():
    import torch

    seg = lib()
    xyz, tri = w.icosphere(4)
    m, eps = 5, 2e-2
    st = make_state(seg, xyz, tri, 2e-4, m, eps, seg.SEG_FP64, seed=21)
    seg.seg_step(st, 4)
    e = seg.seg_energy(st)
    lam, lam_cl = seg.seg_eigenvalue_estimates(st)
    U = seg.seg_get_u(st)
    coup_ref = (lam_cl - lam) * eps * eps / 2.0  # int u_i^2 sum_{j != i} u_j^2

    dev = torch.device("cuda")
    u_d = torch.from_numpy(U).to(dev)
    x_d = torch.from_numpy(xyz).to(dev)
    t_d = torch.from_numpy(tri).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):  # two calls in a row share the static scratch
        out = torch.full((m + 1,), float("nan"), dtype=torch.float64, device=dev)
        seg.seg_s_eps_noalloc(u_d, x_d, t_d, eps, out, stream)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    # the FP64 oracle on the same u: S_eps by its own quadrature, and the
    # coupling integrals from its lambda formula (Sec. 1.1)
    M, K = o.assemble(xyz, tri)
    s_or = o.s_eps(xyz, tri, U, eps)
    coup_or = (o.lambda_cl(xyz, tri, K, U, eps) - o.dirichlet(K, U)) * eps * eps / 2.0
    for out in outs:
        assert rel(out[0], e["s_eps"]) <= 1e-10
        assert np.abs(out[1:] - coup_ref).max() <= 1e-10 * np.abs(coup_ref).max()
        assert rel(out[0], s_or) <= 1e-12
        assert np.abs(out[1:] - coup_or).max() <= 1e-12 * np.abs(coup_or).max()
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    seg = lib()
    xyz, tri = w.icosphere(1)
    dev = torch.device("cuda")
    u_d = torch.ones((xyz.shape[0], 33), dtype=torch.float64, device=dev)
    out = torch.zeros(34, dtype=torch.float64, device=dev)
    with pytest.raises(seg.SegError) as err:
        seg.seg_s_eps_noalloc(u_d, torch.from_numpy(xyz).to(dev), torch.from_numpy(tri).to(dev), 0.1, out)
    assert err.value.status == seg.SEG_ERR_UNSUPPORTED
    assert "32 components" in seg.seg_last_error()
