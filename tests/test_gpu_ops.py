"""GPU parity of each kernel family against the FP64 oracle, through the C ABI.

Inputs are seeded and made here (graded axes with several tiles and a ragged
tail, random fields); both sides get the same arrays.  Tolerances: FP64 kernels
agree to a few units of rounding of their largest term (the two sides differ only
in FMA contraction and summation order); the FP32 smoother to FP32 rounding.
"""
import numpy as np
import pytest

import synth
from gpu_common import dev, graded_axis, host, need_gpu

pytestmark = pytest.mark.gpu

SIZES = [(33, 33, 33), (65, 33, 49), (97, 97, 97)]


def _grid(n, seed):
    x = graded_axis(n[0], 6.0, 3.0, seed, 0.1)
    y = graded_axis(n[1], 5.0, 2.0, seed + 1, 0.1)
    z = graded_axis(n[2], 7.0, 4.0, seed + 2, 0.1)
    return x, y, z


def _coef_scale(x, y, z):
    h = min(np.diff(x).min(), np.diff(y).min(), np.diff(z).min())
    return 12.0 / (h * h)


@pytest.mark.parametrize("n", SIZES)
def test_apply_and_residual(orc, n):
    B = need_gpu()
    x, y, z = _grid(n, 1)
    rng = np.random.default_rng(2)
    u, b = rng.normal(size=n[::-1]), rng.normal(size=n[::-1])
    tol = 1e-13 * _coef_scale(x, y, z) * np.abs(u).max()
    Au = host(B.lasto_op_apply(dev(x), dev(y), dev(z), dev(u)))
    assert np.abs(Au - orc.apply_A(x, y, z, u)).max() < tol
    r = host(B.lasto_op_residual(dev(x), dev(y), dev(z), dev(u), dev(b)))
    assert np.abs(r - orc.residual(x, y, z, u, b)).max() < tol


@pytest.mark.parametrize("n", SIZES)
def test_red_black_sweeps(orc, n):
    B = need_gpu()
    x, y, z = _grid(n, 3)
    rng = np.random.default_rng(4)
    u, b = rng.normal(size=n[::-1]), rng.normal(size=n[::-1])
    ref = u.copy()
    for _ in range(2):
        orc.rbgs_half(x, y, z, ref, b, 0)
        orc.rbgs_half(x, y, z, ref, b, 1)
    got = host(B.lasto_op_smooth(dev(x), dev(y), dev(z), dev(u), dev(b), sweeps=2))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_red_black_sweep_fp32(orc):
    B = need_gpu()
    import torch
    n = (65, 33, 49)
    x, y, z = _grid(n, 5)
    rng = np.random.default_rng(6)
    u, b = rng.normal(size=n[::-1]), rng.normal(size=n[::-1])
    ref = u.copy()
    orc.rbgs_half(x, y, z, ref, b, 0)
    orc.rbgs_half(x, y, z, ref, b, 1)
    u32 = torch.as_tensor(u.astype(np.float32)).cuda()
    b32 = torch.as_tensor(b.astype(np.float32)).cuda()
    got = B.lasto_op_smooth(dev(x), dev(y), dev(z), u32, b32, sweeps=1).cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()


SLAB_CASES = [((33, 33, 33), 1, 0, (62, 6, 16)), ((65, 33, 49), 2, 0, (16, 4, 8)), ((65, 33, 49), 2, 1, (64, 16, 16)),
              ((97, 97, 97), 2, 1, (40, 6, 11)), ((37, 7, 5), 1, 1, (62, 1, 1)), ((135, 9, 33), 1, 0, (62, 6, 16)), ((5, 5, 5), 2, 0, (2, 1, 1)),
              ((3, 3, 3), 1, 0, (62, 4, 8)), ((65, 65, 17), 1, 1, (62, 2, 5))]


def _sweeps_ref(orc, x, y, z, u, b, ns, first):
    ref = u.copy()
    for _ in range(ns):
        orc.rbgs_half(x, y, z, ref, b, first)
        orc.rbgs_half(x, y, z, ref, b, 1 - first)
    return ref


@pytest.mark.parametrize("n,ns,first,tile", SLAB_CASES)
def test_slab_smoother_fp64(orc, n, ns, first, tile):
    """Fused z-slab passes (ragged tiles, tiles wider than the grid, one-node tiles) equal
    the oracle's in-place half sweeps; faces are copied unchanged."""
    B = need_gpu()
    import torch
    x, y, z = _grid(n, 11)
    rng = np.random.default_rng(12)
    u, b = rng.normal(size=n[::-1]), rng.normal(size=n[::-1])
    ref = _sweeps_ref(orc, x, y, z, u, b, ns, first)
    out = torch.full(n[::-1], float("nan"), dtype=torch.float64, device="cuda")
    B.lasto_op_smooth_slab(dev(x), dev(y), dev(z), dev(u), out, dev(b), ns=ns, first=first, tile=tile)
    got = host(out)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    for face in (np.s_[0], np.s_[-1], np.s_[:, 0], np.s_[:, -1], np.s_[:, :, 0], np.s_[:, :, -1]):
        assert np.array_equal(got[face], u[face])


def test_slab_smoother_fp32(orc):
    """FP32 passes: within FP32 rounding of the oracle, and bitwise the same for two tilings
    and for the in-place half-sweep kernel."""
    B = need_gpu()
    import torch
    n = (65, 33, 49)
    x, y, z = _grid(n, 13)
    rng = np.random.default_rng(14)
    u, b = rng.normal(size=n[::-1]), rng.normal(size=n[::-1])
    u32 = torch.as_tensor(u.astype(np.float32)).cuda()
    b32 = torch.as_tensor(b.astype(np.float32)).cuda()
    outs = []
    for ns, tile in ((2, (32, 8, 16)), (2, (24, 5, 7)), (1, (62, 14, 8))):
        o = torch.empty_like(u32)
        B.lasto_op_smooth_slab(dev(x), dev(y), dev(z), u32, o, b32, sweeps=2, ns=ns, first=0, tile=tile)
        outs.append(o)
    ref = _sweeps_ref(orc, x, y, z, u, b, 2, 0)
    assert np.abs(outs[0].cpu().numpy().astype(np.float64) - ref).max() < 4e-5 * np.abs(ref).max()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    inplace = B.lasto_op_smooth(dev(x), dev(y), dev(z), u32.clone(), b32, sweeps=2)
    assert torch.equal(outs[0], inplace)
    # five sweeps as 2 + 2 + 1 fused passes through the op's scratch grid
    o5 = torch.empty_like(u32)
    B.lasto_op_smooth_slab(dev(x), dev(y), dev(z), u32, o5, b32, sweeps=5, ns=2, first=0, tile=(32, 8, 16))
    assert torch.equal(o5, B.lasto_op_smooth(dev(x), dev(y), dev(z), u32.clone(), b32, sweeps=5))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_row_mapped_half_sweeps(dtype):
    """One block per (j, k) row gives bitwise the flat-index half sweeps (any block size)."""
    B = need_gpu()
    import torch
    n = (65, 33, 49)
    x, y, z = _grid(n, 21)
    rng = np.random.default_rng(22)
    t = torch.float32 if dtype == "f32" else torch.float64
    u = torch.as_tensor(rng.normal(size=n[::-1])).to(t).cuda()
    b = torch.as_tensor(rng.normal(size=n[::-1])).to(t).cuda()
    outs = [B.lasto_op_smooth(dev(x), dev(y), dev(z), u.clone(), b, sweeps=3, threads=th) for th in (0, 128, 512)]
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    for bad in (-1, 16, 100, 1024):
        with pytest.raises(RuntimeError):
            B.lasto_op_smooth(dev(x), dev(y), dev(z), u.clone(), b, sweeps=1, threads=bad)


def test_slab_smoother_rejects_bad_arguments():
    B = need_gpu()
    import torch
    n = (9, 9, 9)
    x, y, z = _grid(n, 15)
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(u)
    for kw in (dict(u_out=u), dict(ns=3), dict(tile=(400, 400, 4)), dict(sweeps=0), dict(tile=(7, 4, 4))):
        args = dict(u_in=u, u_out=torch.empty_like(u), b=b, ns=1, first=0, tile=(8, 8, 8))
        args.update(kw)
        with pytest.raises(RuntimeError, match="INVALID_ARG"):
            B.lasto_op_smooth_slab(dev(x), dev(y), dev(z), **args)


@pytest.mark.parametrize("n", SIZES)
def test_restriction_and_prolongation(orc, n):
    B = need_gpu()
    x, y, z = _grid(n, 7)
    rng = np.random.default_rng(8)
    r = rng.normal(size=n[::-1])
    bc = host(B.lasto_op_restrict(dev(x), dev(y), dev(z), dev(r)))
    ref = orc.restrict(x, y, z, r)
    assert np.abs(bc - ref).max() < 1e-13 * np.abs(ref).max()
    nc = tuple((v + 1) // 2 for v in n)
    ec = rng.normal(size=nc[::-1])
    ec[0] = ec[-1] = 0; ec[:, 0] = ec[:, -1] = 0; ec[:, :, 0] = ec[:, :, -1] = 0
    u = rng.normal(size=n[::-1])
    got = host(B.lasto_op_prolong_add(dev(x), dev(y), dev(z), dev(ec), dev(u)))
    refu = orc.prolong_add(x, y, z, ec, u.copy())
    assert np.abs(got - refu).max() < 1e-14 * np.abs(refu).max() * 10


@pytest.mark.parametrize("n", [(9, 9, 9), (7, 9, 5), (5, 5, 5), (3, 3, 3)])
def test_coarse_solve(orc, n):
    B = need_gpu()
    x, y, z = _grid(n, 9) if min(n) > 3 else (np.array([-1, 0.2, 1.0]),) * 3
    b = np.random.default_rng(10).normal(size=n[::-1])
    e = host(B.lasto_op_coarse_solve(dev(x), dev(y), dev(z), dev(b)))
    ref = orc.coarse_solve(x, y, z, b)
    assert np.abs(e - ref).max() < 1e-12 * np.abs(ref).max()


def test_mesh_axis(orc):
    B = need_gpu()
    for (n, L, hmin, hmax) in [(65, 12.0, 0.375, 0.375), (129, 22.8, 0.12, 0.6), (385, 38.4, 0.12, 0.6),
                               (97, 18.0, 0.15, 0.6)]:
        x, info = B.lasto_mesh_axis(n, 0.0, L, hmin, hmax, 6.0, info=True)
        ref, rinfo = orc.mesh_axis(n, 0.0, L, hmin, hmax, 6.0)
        assert np.abs(host(x) - ref).max() <= 4e-16 * L
        assert np.allclose(host(info), rinfo, rtol=1e-14, atol=1e-15)


@pytest.fixture(scope="module")
def small_clusters():
    return [synth.pd13_small(n=33), synth.pd2_dimer(n=33, graded=True), synth.pd13_uniform65()]


def test_sphere_params(orc, small_clusters):
    B = need_gpu()
    for cl in small_clusters:
        dc = B.DeviceCluster(cl)
        q, rhoR, drhoR, coef, status = (host(t) for t in B.lasto_op_sphere_params(dc))
        rq, rr, rd, rc = orc.sphere_params(cl)
        assert status[0] == 0
        assert np.abs(q - rq).max() < 1e-12 * np.abs(rq).max()
        assert np.abs(rhoR - rr).max() < 1e-12 * np.abs(rr).max()
        assert np.abs(drhoR - rd).max() < 1e-11 * np.abs(rd).max()
        assert np.abs(coef - rc).max() < 1e-11 * np.abs(rc).max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-11)])
def test_deposit(orc, small_clusters, precision, tol):
    """FP64 and FP32-pair deposits against the oracle.  The GPU cancels each atom's own
    spherical terms analytically (the oracle subtracts them), and the FP32-pair form
    carries about 44 bits, so both agree to far below the 1e-8 solve tolerance."""
    B = need_gpu()
    for cl in small_clusters:
        x, y, z = orc.mesh(cl)
        assert np.abs(host(B.DeviceCluster(cl).x) - x).max() < 1e-14 * cl.half_width
        dc = B.DeviceCluster(cl, axes=(x, y, z))   # both sides on the oracle's nodes
        b, owner, status = B.lasto_op_deposit(dc, precision=precision)
        ref, rowner = orc.deposit(cl, x, y, z)
        assert host(status)[0] == 0
        assert np.array_equal(host(owner), rowner)
        b = host(b)
        assert np.abs(b - ref).max() < tol * np.abs(ref).max()
        # node by node where the density matters; far out the GPU drops Slater terms below
        # e^-40 (FP64) or e^-37 (FP32 pairs) of their weight, which the oracle keeps
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        assert np.abs((b - ref)[big] / ref[big]).max() < 1e-10


def test_deposit_far_apart_atoms_non_cubic(orc):
    """Two atoms 50 bohr apart on a 49 x 41 x 45 mesh: tiles at either end of the box lie
    farther than the cut-off (37 / zeta_min = 24.7 bohr) from the other atom, so the FP32-pair
    deposit drops that atom for the whole tile; ragged 8 x 8 x 4 tiles on every axis.  Both
    precisions against the oracle node by node."""
    B = need_gpu()
    from synth import clusters, workloads
    cl = workloads.make_cluster("far-dimer", clusters.dimer(50.0), np.random.default_rng(21), n=49, half_width=36.0,
                                h_min=1.5, h_max=1.5)
    x, y, z = orc.mesh(cl)
    y = np.ascontiguousarray(y[4:-4])
    z = np.ascontiguousarray(z[2:-2])
    assert (len(x), len(y), len(z)) == (49, 41, 45)
    dc = B.DeviceCluster(cl, axes=(x, y, z))
    dc.n = (len(x), len(y), len(z))
    ref, rowner = orc.deposit(cl, x, y, z)
    for precision, tol in ((0, 1e-12), (1, 1e-11)):
        b, owner, status = B.lasto_op_deposit(dc, precision=precision)
        assert host(status)[0] == 0
        assert np.array_equal(host(owner), rowner)
        b = host(b)
        assert b.shape == ref.shape
        assert np.abs(b - ref).max() < tol * np.abs(ref).max()
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        assert np.abs((b - ref)[big] / ref[big]).max() < 1e-10


def test_multipoles_and_faces(orc, small_clusters):
    B = need_gpu()
    for cl in small_clusters:
        x, y, z = orc.mesh(cl)
        dc = B.DeviceCluster(cl, axes=(x, y, z))
        b, _, _ = B.lasto_op_deposit(dc)
        bh = host(b)
        Q = host(B.lasto_op_multipoles(dc.x, dc.y, dc.z, b))
        rQ = orc.multipoles(x, y, z, bh)
        assert np.abs(Q - rQ).max() < 1e-12 * np.abs(rQ).max()
        import torch
        u = torch.zeros_like(b)
        B.lasto_op_boundary_fill(dc.x, dc.y, dc.z, dev(rQ), u)
        ref = orc.boundary_fill(x, y, z, rQ, np.zeros(bh.shape))
        assert np.abs(host(u) - ref).max() < 1e-13 * np.abs(ref).max()


def test_projection(orc):
    B = need_gpu()
    cl = synth.pd13_small(n=33)
    x, y, z = orc.mesh(cl)
    dc = B.DeviceCluster(cl, axes=(x, y, z))
    u = np.random.default_rng(11).normal(size=(33, 33, 33))
    vlm, status = B.lasto_op_project(dc.x, dc.y, dc.z, dev(u), dc.pos, dc.R)
    ref = orc.project(x, y, z, u, cl.pos, cl.R)
    assert host(status)[0] == 0
    assert np.abs(host(vlm) - ref).max() < 1e-13 * np.abs(ref).max()
