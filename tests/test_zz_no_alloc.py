"""The allocation-free deposit (lasto_op_deposit_noalloc) gives the allocating
entry point's results.

Callers that cannot allocate device memory when they deposit (a fixed device-memory
budget set at start-up, a device heap owned by another framework's allocator, a
real-time loop that forbids allocation) use this variant; its scratch is one fixed
device array shared by every call, so the test makes two calls in a row on different
clusters and checks that the second is not coloured by the first, and that no call
draws on the device's stream-ordered memory pool (where the allocating variant takes
its scratch).  The file sorts last so that a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_common import host, need_gpu

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the CUDA driver API
_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8


class _DefaultPool:
    """Current and high-water use of device 0's default stream-ordered memory pool, read
    through the driver API (the pool cudaMallocAsync draws from)."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def used(self):
        return self._get(_USED_MEM_CURRENT)

    def high(self):
        return self._get(_USED_MEM_HIGH)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-11)])
def test_noalloc_deposit_matches_allocating_deposit(precision, tol):
    import torch
    B = need_gpu()
    pool = _DefaultPool()
    clusters = [synth.pd13_small(n=33), synth.pd2_dimer(n=33, graded=True)]
    for cl in clusters:                       # two calls in a row through the shared array
        dc = B.DeviceCluster(cl)
        ref, ref_owner, ref_status = B.lasto_op_deposit(dc, precision=precision)
        b = torch.full((dc.N,), float("nan"), dtype=torch.float64, device="cuda")
        owner = torch.full((dc.N,), -7, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        used0 = pool.used()
        pool.reset_high()
        B.lasto_op_deposit_noalloc(dc, b, owner, status, precision=precision)
        torch.cuda.synchronize()
        assert pool.high() <= used0, "the allocation-free deposit drew on the stream-ordered pool"
        r, g = host(ref).ravel(), host(b)
        assert host(status)[0] == host(ref_status)[0] == 0
        assert np.array_equal(host(owner), host(ref_owner).ravel())
        assert np.all(np.isfinite(g))
        assert np.abs(g - r).max() <= tol * np.abs(r).max()


def test_pool_probe_sees_the_allocating_deposit():
    """The pool counters do see the allocating entry point's scratch (so the check above can fail)."""
    import torch
    B = need_gpu()
    pool = _DefaultPool()
    dc = B.DeviceCluster(synth.pd13_small(n=33))
    torch.cuda.synchronize()
    used0 = pool.used()
    pool.reset_high()
    B.lasto_op_deposit(dc)
    torch.cuda.synchronize()
    assert pool.high() > used0


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


def test_noalloc_checks_caller_buffers_before_launch():
    import torch
    B = need_gpu()
    dc = B.DeviceCluster(synth.pd13_small(n=33))
    ok = torch.zeros(dc.N, dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(dc.N - 1, dtype=torch.float64, device="cuda"),     # too short
                torch.zeros(dc.N, dtype=torch.float32, device="cuda"),         # wrong type
                torch.zeros((dc.N, 2), dtype=torch.float64, device="cuda")[:, 0],   # not contiguous
                torch.zeros(dc.N, dtype=torch.float64)):                       # on the host
        with pytest.raises(ValueError):
            B.lasto_op_deposit_noalloc(dc, bad)
    with pytest.raises(ValueError):
        B.lasto_op_deposit_noalloc(dc, ok, owner=torch.zeros(dc.N, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        B.lasto_op_deposit_noalloc(dc, ok, status=torch.zeros(0, dtype=torch.int32, device="cuda"))
