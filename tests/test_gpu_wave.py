"""The FP32 wavefront red-black sweep (lasto_op_smooth_wave_f32) against the in-place half
sweeps and the FP64 oracle, and the bounded device wait.

The wavefront pass updates the first colour of plane k+1 and then the second colour of plane
k from row chunks staged in shared memory by cp.async; every node update is the in-place kernels'
expression with the same operands, so the two are compared bit for bit, on graded grids
with ragged tiles in x, y and z, non-cubic shapes, the smallest accepted rows (69 nodes),
both colour orders, and the 385^3 grid of the largest workload (where every thread block's
span crosses tile columns).  The oracle pins the FP32 result to FP32 rounding.
"""
import numpy as np
import pytest

from gpu_common import dev, graded_axis, host, need_gpu

pytestmark = pytest.mark.gpu


def _grid(n, seed):
    return (graded_axis(n[0], 6.0, 3.0, seed, 0.1), graded_axis(n[1], 5.0, 2.0, seed + 1, 0.1),
            graded_axis(n[2], 7.0, 4.0, seed + 2, 0.1))


def _fields(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    u = torch.as_tensor(rng.normal(size=n[::-1]).astype(np.float32)).cuda()
    b = torch.as_tensor(rng.normal(size=n[::-1]).astype(np.float32)).cuda()
    return u, b


SHAPES = [(69, 69, 69), (71, 37, 13), (97, 5, 9), (129, 129, 129), (193, 97, 65)]
TILES = [(60, 16), (48, 8), (17, 16), (60, 12)]


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("tile", TILES)
def test_wave_sweep_equals_in_place_sweeps(n, tile):
    import torch
    B = need_gpu()
    x, y, z = _grid(n, 31)
    u, b = _fields(n, 32)
    u_keep = u.clone()
    for sweeps in (1, 3):
        out = torch.full_like(u, float("nan"))
        B.lasto_op_smooth_wave(dev(x), dev(y), dev(z), u, out, b, sweeps=sweeps, first=0, tile=tile)
        ref = B.lasto_op_smooth(dev(x), dev(y), dev(z), u.clone(), b, sweeps=sweeps, threads=256)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (n, tile, sweeps)
    assert torch.equal(u, u_keep)                      # u_in is not modified


@pytest.mark.parametrize("n", [(69, 69, 69), (97, 71, 33)])
def test_wave_sweep_reversed_colour_order(n):
    """first = 1 (the post-smoothing order of the symmetric cycle): bitwise the fused slab
    passes with the same order, which equal in-place sweeps in that order."""
    import torch
    B = need_gpu()
    x, y, z = _grid(n, 33)
    u, b = _fields(n, 34)
    out = torch.empty_like(u)
    B.lasto_op_smooth_wave(dev(x), dev(y), dev(z), u, out, b, sweeps=2, first=1, tile=(60, 16))
    ref = torch.empty_like(u)
    B.lasto_op_smooth_slab(dev(x), dev(y), dev(z), u, ref, b, sweeps=2, ns=2, first=1, tile=(32, 8, 16))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert not torch.equal(out, B.lasto_op_smooth(dev(x), dev(y), dev(z), u.clone(), b, sweeps=2))


def test_wave_sweep_against_oracle(orc):
    import torch
    B = need_gpu()
    n = (73, 41, 29)
    x, y, z = _grid(n, 35)
    u, b = _fields(n, 36)
    ref = host(u).astype(np.float64)
    b64 = host(b).astype(np.float64)
    for _ in range(2):
        orc.rbgs_half(x, y, z, ref, b64, 0)
        orc.rbgs_half(x, y, z, ref, b64, 1)
    out = torch.empty_like(u)
    B.lasto_op_smooth_wave(dev(x), dev(y), dev(z), u, out, b, sweeps=2, tile=(60, 16))
    got = host(out).astype(np.float64)
    assert np.abs(got - ref).max() < 4e-5 * np.abs(ref).max()
    for face in (np.s_[0], np.s_[-1], np.s_[:, 0], np.s_[:, -1], np.s_[:, :, 0], np.s_[:, :, -1]):
        assert np.array_equal(host(out)[face], host(u)[face])


def test_wave_sweep_at_385():
    """The largest workload's grid (57 M nodes, graded as the Pd561 mesh): one pass, against
    the in-place half sweeps."""
    import torch
    B = need_gpu()
    n = 385
    ax = B.lasto_mesh_axis(n, 0.0, 35.4, 0.12, 0.6, 6.0)
    g = torch.Generator("cuda").manual_seed(3)
    u = torch.rand(n ** 3, dtype=torch.float32, device="cuda", generator=g)
    b = torch.rand(n ** 3, dtype=torch.float32, device="cuda", generator=g)
    for tile in ((60, 16), (48, 8)):
        out = torch.empty_like(u)
        B.lasto_op_smooth_wave(ax, ax, ax, u, out, b, sweeps=1, tile=tile)
        ref = B.lasto_op_smooth(ax, ax, ax, u.clone(), b, sweeps=1, threads=0)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), tile
    del u, b, out, ref
    torch.cuda.empty_cache()


def test_wave_sweep_rejects_bad_arguments():
    import torch
    B = need_gpu()
    n = (69, 9, 9)
    x, y, z = _grid(n, 37)
    u, b = _fields(n, 38)
    out = torch.empty_like(u)
    for kw in (dict(tile=(61, 16)), dict(tile=(60, 10)), dict(tile=(8, 16)), dict(sweeps=0)):
        args = dict(sweeps=1, tile=(60, 16))
        args.update(kw)
        with pytest.raises(RuntimeError, match="INVALID_ARG"):
            B.lasto_op_smooth_wave(dev(x), dev(y), dev(z), u, out, b, **args)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):          # u_in == u_out
        B.lasto_op_smooth_wave(dev(x), dev(y), dev(z), u, u, b)
    short = (67, 9, 9)                                               # rows below 69 nodes
    xs, ys, zs = _grid(short, 39)
    us, bs = _fields(short, 40)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.lasto_op_smooth_wave(dev(xs), dev(ys), dev(zs), us, torch.empty_like(us), bs)


def test_solve_with_the_wave_smoother_forced():
    """A whole mixed-precision solve whose 97^3 level is smoothed by wavefront passes gives
    bitwise the in-place solve (same iterate every sweep, same iteration count)."""
    import torch

    import synth
    B = need_gpu()
    cl = synth.pd13_small(n=97)
    dc = B.DeviceCluster(cl)
    out = {}
    for name, choice in (("inplace", "0 256 0 0 0 0"), ("wave", "2 256 60 16 8 1"), ("wave8", "2 256 48 8 8 1")):
        solver = B.Poisson(n_max=97, max_atoms=13, precision=B.LASTO_PREC_MIXED)
        solver.set_tune_table(f"97 97 97 4 {choice} 0\n49 49 49 4 0 256 0 0 0 0 0\n")
        v = torch.empty((13, 25), dtype=torch.float64, device="cuda")
        s = solver.solve(dc, v)[0]
        torch.cuda.synchronize()
        assert s.status == 0 and s.rel_resid <= 1e-10
        out[name] = (v.clone(), s.cycles)
        solver.close()
    assert torch.equal(out["inplace"][0], out["wave"][0]) and out["inplace"][1] == out["wave"][1]
    assert torch.equal(out["inplace"][0], out["wave8"][0])


def test_bounded_wait_runs_out_and_reports_timeout():
    """A device wait that nothing ends gives up after its limit, raises LASTO_ERR_TIMEOUT in
    the status word, and leaves the context and the stream usable."""
    import time

    import torch
    B = need_gpu()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    B.lasto_selftest_bounded_wait(0.05, status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(status.item()) == B.LASTO_ERR_TIMEOUT
    assert 0.04 < dt < 5.0
    # the stream still runs work afterwards
    x = torch.arange(1000, dtype=torch.float64, device="cuda")
    assert float((x * 2).sum().item()) == 999000.0
    n = (69, 9, 9)
    xs, ys, zs = _grid(n, 41)
    u, b = _fields(n, 42)
    out = torch.empty_like(u)
    B.lasto_op_smooth_wave(dev(xs), dev(ys), dev(zs), u, out, b)
    ref = B.lasto_op_smooth(dev(xs), dev(ys), dev(zs), u.clone(), b, sweeps=1)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.lasto_selftest_bounded_wait(0.0, status)
