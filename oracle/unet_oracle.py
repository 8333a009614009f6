"""FP64 CPU oracle of the learned-initial-guess network (3-D U-Net) and its operations.

TEST INFRASTRUCTURE ONLY: used by the tests to check the GPU network kernels (forward,
data gradient, weight gradient, down/up-sampling and their adjoints) and the whole
network's gradients.  The paper has no such network; the definitions here are the plain
textbook ones, written independently of the CUDA code:
  * 3x3x3 convolution (cross-correlation), zero padding, channels-last [b, z, y, x, c],
    weights [27, cin, cout], tap = (dz+1)*9 + (dy+1)*3 + (dx+1);
  * down-sampling onto every other node: full weighting (1/4, 1/2, 1/4) per axis, the two
    boundary nodes using (2/3, 1/3) so constants are preserved;
  * up-sampling: linear interpolation per axis (trilinear in 3-D);
  * ReLU, masked mean-square error.
The down/up operators are built as explicit per-axis matrices, so their adjoints are the
matrix transposes.
"""
from __future__ import annotations

import numpy as np

TAPS = [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def conv3d(x, w, bias=None):
    nb, D, H, W, cin = x.shape
    cout = w.shape[2]
    pad = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((nb, D, H, W, cout))
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = pad[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :]
        y += np.einsum("bzyxc,co->bzyxo", xs, w[t])
    if bias is not None:
        y += bias
    return y


def conv3d_backward(x, w, dy):
    """Gradients of sum(dy * conv3d(x, w, b)) with respect to x, w and b."""
    nb, D, H, W, cin = x.shape
    pad = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    dpad = np.zeros_like(pad)
    dw = np.zeros_like(w)
    for t, (dz, dyy, dx) in enumerate(TAPS):
        sl = (slice(None), slice(1 + dz, 1 + dz + D), slice(1 + dyy, 1 + dyy + H), slice(1 + dx, 1 + dx + W), slice(None))
        dw[t] = np.einsum("bzyxc,bzyxo->co", pad[sl], dy)
        dpad[sl] += np.einsum("bzyxo,co->bzyxc", dy, w[t])
    return dpad[:, 1:-1, 1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1, 2, 3))


def down_matrix(n):
    """Per-axis full weighting from n (odd) nodes onto (n+1)/2."""
    nc = (n + 1) // 2
    M = np.zeros((nc, n))
    for I in range(nc):
        if I == 0:
            M[I, 0], M[I, 1] = 2 / 3, 1 / 3
        elif I == nc - 1:
            M[I, n - 1], M[I, n - 2] = 2 / 3, 1 / 3
        else:
            M[I, 2 * I - 1], M[I, 2 * I], M[I, 2 * I + 1] = 0.25, 0.5, 0.25
    return M


def up_matrix(n):
    """Per-axis linear interpolation from (n+1)/2 nodes onto n."""
    nc = (n + 1) // 2
    M = np.zeros((n, nc))
    for f in range(n):
        if f % 2 == 0:
            M[f, f // 2] = 1.0
        else:
            M[f, f // 2] = M[f, f // 2 + 1] = 0.5
    return M


def _apply_axes(x, Mz, My, Mx):
    return np.einsum("Zz,Yy,Xx,bzyxc->bZYXc", Mz, My, Mx, x)


def down(x):
    _, D, H, W, _ = x.shape
    return _apply_axes(x, down_matrix(D), down_matrix(H), down_matrix(W))


def down_adjoint(y, fine):
    D, H, W = fine
    return _apply_axes(y, down_matrix(D).T, down_matrix(H).T, down_matrix(W).T)


def up(x, fine):
    D, H, W = fine
    return _apply_axes(x, up_matrix(D), up_matrix(H), up_matrix(W))


def up_adjoint(y):
    _, D, H, W, _ = y.shape
    return _apply_axes(y, up_matrix(D).T, up_matrix(H).T, up_matrix(W).T)


def relu(x):
    return np.maximum(x, 0.0)


# ---------------------------------------------------------------- the network
# (name, cin, cout, relu); encoder 16-32-64-64 on grids n, (n+1)/2, ... ; decoder inputs are
# [up-sampled, skip] concatenations.
LAYERS = [("e1a", 16, 16, 1), ("e1b", 16, 16, 1), ("e2a", 16, 32, 1), ("e2b", 32, 32, 1), ("e3a", 32, 64, 1),
          ("e3b", 64, 64, 1), ("bta", 64, 64, 1), ("btb", 64, 64, 1), ("d3a", 128, 64, 1), ("d3b", 64, 64, 1),
          ("d2a", 96, 32, 1), ("d2b", 32, 32, 1), ("d1a", 48, 16, 1), ("d1b", 16, 16, 1), ("out", 16, 16, 0)]


def init_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    P = {}
    for name, cin, cout, _ in LAYERS:
        P[name + ".w"] = rng.normal(0.0, scale * np.sqrt(2.0 / (27 * cin)), size=(27, cin, cout))
        P[name + ".b"] = rng.normal(0.0, 0.01, size=cout)
    return P


def forward(P, x):
    """x [nb, n, n, n, 16] -> (prediction = channel 0 of the output layer, cache)."""
    cache = {}

    def conv(name, inp, act):
        y = conv3d(inp, P[name + ".w"], P[name + ".b"])
        if act:
            y = relu(y)
        cache[name] = (inp, y)
        return y

    e1 = conv("e1b", conv("e1a", x, 1), 1)
    e2 = conv("e2b", conv("e2a", down(e1), 1), 1)
    e3 = conv("e3b", conv("e3a", down(e2), 1), 1)
    bt = conv("btb", conv("bta", down(e3), 1), 1)
    d3 = conv("d3b", conv("d3a", np.concatenate([up(bt, e3.shape[1:4]), e3], axis=-1), 1), 1)
    d2 = conv("d2b", conv("d2a", np.concatenate([up(d3, e2.shape[1:4]), e2], axis=-1), 1), 1)
    d1 = conv("d1b", conv("d1a", np.concatenate([up(d2, e1.shape[1:4]), e1], axis=-1), 1), 1)
    o = conv("out", d1, 0)
    cache["shapes"] = (e1.shape, e2.shape, e3.shape)
    return o[..., 0], cache


def backward(P, cache, dpred):
    """Gradients of sum(dpred * prediction) with respect to every parameter."""
    G = {}
    acts = {name: act for name, _, _, act in LAYERS}

    def back(name, dy):
        inp, y = cache[name]
        if acts[name]:
            dy = dy * (y > 0)
        dx, dw, db = conv3d_backward(inp, P[name + ".w"], dy)
        G[name + ".w"], G[name + ".b"] = dw, db
        return dx

    s1, s2, s3 = cache["shapes"]
    do = np.zeros(dpred.shape + (16,))
    do[..., 0] = dpred
    dcat1 = back("d1a", back("d1b", back("out", do)))
    c_up1 = dcat1.shape[-1] - s1[-1]
    de1 = dcat1[..., c_up1:]
    dcat2 = back("d2a", back("d2b", up_adjoint(dcat1[..., :c_up1])))
    c_up2 = dcat2.shape[-1] - s2[-1]
    de2 = dcat2[..., c_up2:]
    dcat3 = back("d3a", back("d3b", up_adjoint(dcat2[..., :c_up2])))
    c_up3 = dcat3.shape[-1] - s3[-1]
    de3 = dcat3[..., c_up3:]
    dp3 = back("bta", back("btb", up_adjoint(dcat3[..., :c_up3])))
    de3 = de3 + down_adjoint(dp3, s3[1:4])
    dp2 = back("e3a", back("e3b", de3))
    de2 = de2 + down_adjoint(dp2, s2[1:4])
    dp1 = back("e2a", back("e2b", de2))
    de1 = de1 + down_adjoint(dp1, s1[1:4])
    back("e1a", back("e1b", de1))
    return G


def mse(pred, target, mask):
    d = (pred - target) * mask
    return float((d * d).sum() / mask.sum()), 2.0 * d / mask.sum()
