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
