"""Train the learned-initial-guess network on potentials the solver itself produces.

    python -m paper_0806_1723_gb300.train_unet --samples 20000 --epochs 4 --out unet.npz

Data: perturbed Pd13 / Pd55 / Pd147 clusters on graded 129^3 meshes, each solved to 1e-10 by
the library (batched, one graph launch per batch).  Inputs are the coarse-grid (33^3)
right-hand side, faces and mesh size; targets are the converged potential at the same nodes.
Training runs the library's forward / backward kernels with Adam.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

from . import binding as B
from . import unet as U


def solve_batch(solver, clusters):
    dcs = [B.DeviceCluster(c) for c in clusters]
    vlm = torch.empty((sum(c.n_atoms for c in clusters), 25), dtype=torch.float64, device="cuda")
    pot = torch.empty(sum(d.N for d in dcs), dtype=torch.float64, device="cuda")
    st = solver.solve(dcs, vlm, potential=pot)
    torch.cuda.synchronize()
    return dcs, pot, st


def build_dataset(net, clusters, batch=32, log=print):
    """Features [count, N, 3] and targets [count, N] (FP32, device) for the coarse grid."""
    n_max = max(c.n for c in clusters)
    solver = B.Poisson(n_max=n_max, max_atoms=max(c.n_atoms for c in clusters), max_batch=batch,
                       precision=B.LASTO_PREC_MIXED)
    nc = 33
    N = nc ** 3
    X = torch.empty(len(clusters), N, 3, dtype=torch.float32, device="cuda")
    Y = torch.empty(len(clusters), N, dtype=torch.float32, device="cuda")
    t0 = time.time()
    raw = torch.empty(N, 16, dtype=torch.float32, device="cuda")
    for s0 in range(0, len(clusters), batch):
        chunk = clusters[s0:s0 + batch]
        dcs, pot, st = solve_batch(solver, chunk)
        assert all(s.status == 0 for s in st), [s.status for s in st]
        off = 0
        for k, (c, dc) in enumerate(zip(chunk, dcs)):
            b_c, faces, crs, mid, Q = U.coarse_problem(dc)
            U.features(net, b_c, faces, crs, out=raw)
            X[s0 + k] = raw[:, :3]
            u = pot[off:off + dc.N].view(c.n, c.n, c.n)[::4, ::4, ::4]
            Y[s0 + k] = u.reshape(-1).float()
            off += dc.N
        if log and (s0 // batch) % 10 == 0:
            log(f"dataset {s0 + len(chunk)}/{len(clusters)}  {time.time() - t0:.1f}s")
    solver.close()
    return X, Y


def set_scales(net, X, Y):
    """Standardise the inputs and targets with fixed per-channel factors taken from the data."""
    interior = X[:, :, 0] != 0
    s0 = 1.0 / float(X[:, :, 0][interior].std())
    faces = X[:, :, 1] != 0
    s1 = 1.0 / float(X[:, :, 1][faces].abs().mean())
    out = 1.0 / float(Y.std())
    net.scales = {"s0": s0, "s1": s1, "h_ref": 1.0, "out": out}
    X[:, :, 0] *= s0
    X[:, :, 1] *= s1
    Y *= out


def interior_mask(n, nb, device="cuda"):
    m = torch.zeros(n, n, n, dtype=torch.float32, device=device)
    m[1:-1, 1:-1, 1:-1] = 1.0
    return m.reshape(-1).repeat(nb)


def train(net, X, Y, epochs=4, lr=1e-3, log=print, seed=0):
    nb, n = net.nb, net.n
    N = n ** 3
    mask = interior_mask(n, nb)
    net._mask_count = float(mask.sum().item())
    x32 = torch.zeros(nb * N, 16, dtype=torch.float32, device="cuda")
    tgt = torch.empty(nb * N, dtype=torch.float32, device="cuda")
    g = torch.Generator().manual_seed(seed)
    hist = []
    t0 = time.time()
    steps = 0
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], generator=g)
        tot = torch.zeros((), dtype=torch.float64, device="cuda")
        cnt = 0
        for s0 in range(0, X.shape[0] - nb + 1, nb):
            idx = perm[s0:s0 + nb].cuda()
            x32.view(nb, N, 16)[:, :, :3] = X[idx]
            tgt.copy_(Y[idx].reshape(-1))
            net.forward(x32)
            loss = net.loss_and_grad(tgt, mask)
            net.backward(net.dpred)
            net.adam(lr * (0.5 ** (ep // 2)))
            steps += 1
            tot += loss.reshape(())        # summed on the device: no host sync per step
            cnt += 1
        hist.append(float(tot.item()) / max(cnt, 1))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.4e}  ({time.time() - t0:.1f}s, {steps} steps)")
    return hist


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--samples", type=int, default=20000)
    p.add_argument("--epochs", type=int, default=4)
    p.add_argument("--batch", type=int, default=8)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--seed", type=int, default=3)
    p.add_argument("--out", default="unet.npz")
    p.add_argument("--wmma", action="store_true", help="train on the warp-level MMA kernels instead of tcgen05")
    a = p.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import synth
    clusters = synth.workloads.guess_training_set(a.samples, seed=a.seed)
    net = U.UNet(n=33, nb=a.batch, seed=a.seed, tc=not a.wmma)
    X, Y = build_dataset(net, clusters)
    set_scales(net, X, Y)
    hist = train(net, X, Y, epochs=a.epochs, lr=a.lr)
    net.save(a.out)
    print(json.dumps({"samples": a.samples, "epochs": a.epochs, "loss": hist, "out": a.out}))


if __name__ == "__main__":
    main()
