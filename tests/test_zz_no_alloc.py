"""The allocation-free deposit (lasto_op_deposit_noalloc) gives the allocating
entry point's results.

Callers that cannot allocate device memory when they deposit use this variant; its
scratch is one fixed device array shared by every call, so the test makes two calls
in a row on different clusters and checks that the second is not coloured by the
first.  The file sorts last so that a stop-at-first-failure run has already run every
other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synth
from gpu_common import host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-11)])
def test_noalloc_deposit_matches_allocating_deposit(precision, tol):
    import torch
    B = need_gpu()
    clusters = [synth.pd13_small(n=33), synth.pd2_dimer(n=33, graded=True)]
    for cl in clusters:                       # two calls in a row through the shared array
        dc = B.DeviceCluster(cl)
        ref, ref_owner, ref_status = B.lasto_op_deposit(dc, precision=precision)
        b = torch.full((dc.N,), float("nan"), dtype=torch.float64, device="cuda")
        owner = torch.full((dc.N,), -7, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.lasto_op_deposit_noalloc(dc, b, owner, status, precision=precision)
        torch.cuda.synchronize()
        r, g = host(ref).ravel(), host(b)
        assert host(status)[0] == host(ref_status)[0] == 0
        assert np.array_equal(host(owner), host(ref_owner).ravel())
        assert np.all(np.isfinite(g))
        assert np.abs(g - r).max() <= tol * np.abs(r).max()


def test_noalloc_rejects_clusters_beyond_its_array():
    import torch
    B = need_gpu()
    rng = np.random.default_rng(0)
    pos = np.stack(np.meshgrid(*(np.arange(11) * 5.0,) * 3, indexing="ij"), -1).reshape(-1, 3)[:1100] - 25.0
    cl = synth.workloads.make_cluster("too-many", pos, rng, n=33, half_width=40.0, h_min=2.5, h_max=2.5)
    dc = B.DeviceCluster(cl)
    b = torch.empty(dc.N, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.lasto_op_deposit_noalloc(dc, b)
