"""The learned initial guess, end to end on the GPU.

Training with the library's own kernels lowers the loss; the shipped network (trained on
20 000 potentials the solver produced) lowers the CG iteration count on held-out clusters
while every solve still reaches the same 1e-10 residual and the same sphere coefficients:
the guess changes how fast the solver gets there, never where it ends."""
import os

import numpy as np
import pytest

import synth
from gpu_common import host, need_gpu

pytestmark = pytest.mark.gpu
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0806_1723_gb300", "weights",
                       "unet_pd_33.npz")


def test_training_lowers_the_loss():
    import torch
    B = need_gpu()
    from paper_0806_1723_gb300 import train_unet as T
    from paper_0806_1723_gb300 import unet as U
    clusters = synth.workloads.guess_training_set(48, seed=5)
    net = U.UNet(n=33, nb=8, seed=1)
    X, Y = T.build_dataset(net, clusters, batch=16, log=None)
    T.set_scales(net, X, Y)
    hist = T.train(net, X, Y, epochs=8, lr=2e-3, log=None)
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.7 * hist[0], hist


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="trained weights not shipped")
def test_learned_guess_saves_iterations_and_keeps_the_answer():
    import torch
    B = need_gpu()
    from paper_0806_1723_gb300 import unet as U
    net = U.UNet.load(WEIGHTS, nb=1)
    solver = B.Poisson(n_max=129, max_atoms=147, precision=B.LASTO_PREC_MIXED)
    zero, learned = [], []
    for c in synth.workloads.guess_training_set(8, seed=77):      # not in the training set (seed 3)
        dc = B.DeviceCluster(c)
        v0 = torch.empty((c.n_atoms, 25), dtype=torch.float64, device="cuda")
        v1 = torch.empty_like(v0)
        s0 = solver.solve(dc, v0)[0]
        torch.cuda.synchronize()
        g = U.learned_guess(net, dc)
        s1 = solver.solve(dc, v1, guess=g)[0]
        torch.cuda.synchronize()
        assert s0.status == 0 and s1.status == 0 and s1.rel_resid <= 1e-10
        a, b = host(v0), host(v1)
        assert np.abs(a - b).max() <= 1e-8 * np.abs(a).max()
        zero.append(s0.cycles)
        learned.append(s1.cycles)
    assert np.mean(learned) < np.mean(zero), (zero, learned)


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="trained weights not shipped")
def test_guess_inside_the_solve_graph():
    """The network loaded into the handle runs inside the solve's graph (one batched pass
    for all clusters): same iteration counts as the guess computed outside, same answer as
    the zero start, stats flag the learned start; a 97^3 mesh (no 33^3 level in its
    hierarchy) goes through the resampled subgrid."""
    import torch
    B = need_gpu()
    from paper_0806_1723_gb300 import unet as U
    net = U.UNet.load(WEIGHTS, nb=1)
    cls = synth.workloads.guess_training_set(3, seed=78)
    pos = synth.clusters.cuboctahedron13()
    c97 = synth.workloads.make_cluster("Pd13-graded-97", pos, np.random.default_rng(79), n=97,
                                       half_width=synth.workloads.graded_box(pos), h_min=0.12, h_max=0.6)
    dcs = [B.DeviceCluster(c) for c in cls] + [B.DeviceCluster(c97)]
    na = sum(d.n_atoms for d in dcs)
    plain = B.Poisson(n_max=129, max_atoms=147, max_batch=4, precision=B.LASTO_PREC_MIXED)
    learned = B.Poisson(n_max=129, max_atoms=147, max_batch=4, precision=B.LASTO_PREC_MIXED)
    learned.set_guess(WEIGHTS)
    v0 = torch.empty((na, 25), dtype=torch.float64, device="cuda")
    v1 = torch.empty_like(v0)
    s0 = plain.solve(dcs, v0)
    s1 = learned.solve(dcs, v1)
    torch.cuda.synchronize()
    assert all(s.status == 0 and s.rel_resid <= 1e-10 for s in list(s0) + list(s1))
    assert [s.guess for s in s0] == [0, 0, 0, 0] and [s.guess for s in s1] == [1, 1, 1, 1]
    a, b = host(v0), host(v1)
    assert np.abs(a - b).max() <= 1e-8 * np.abs(a).max()
    # the in-graph guess matches the one computed outside the solve (the same network; the
    # in-graph pass sums the small grids' convolution taps in groups, so the last bits differ)
    single = B.Poisson(n_max=129, max_atoms=147, precision=B.LASTO_PREC_MIXED)
    for k, dc in enumerate(dcs[:3]):
        v = torch.empty((dc.n_atoms, 25), dtype=torch.float64, device="cuda")
        st = single.solve(dc, v, guess=U.learned_guess(net, dc))[0]
        torch.cuda.synchronize()
        assert abs(st.cycles - s1[k].cycles) <= 1, (k, st.cycles, s1[k].cycles)
    assert sum(s.cycles for s in s1[:3]) < sum(s.cycles for s in s0[:3])
    # replaying the captured graph gives the same counts
    s2 = learned.solve(dcs, v1)
    torch.cuda.synchronize()
    assert [s.cycles for s in s2] == [s.cycles for s in s1]
