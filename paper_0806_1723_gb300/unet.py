"""Learned initial guess: a 3-D U-Net on the 33^3 coarse grid, run and trained with the
library's own kernels (lasto_nn_*: BF16 tensor-core convolutions with FP32 accumulation,
their data and weight gradients, sampling operators, Adam).

The network maps the restricted right-hand side, the Dirichlet faces and the local mesh
size on the coarse grid (the every-fourth-node level of a 129^3 hierarchy) to the coarse
potential; prolonged to the fine grid it is the multigrid initial guess.  Multigrid always
runs to the same residual, so the guess changes only the iteration count.

This module only sequences kernel calls and moves pointers (PyTorch provides device
memory); every arithmetic step runs in liblasto_poisson.so.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import binding as B

# (name, cin, cout, relu) -- encoder 16-32-64-64 on n, (n+1)/2, ..., decoder on [up, skip]
LAYERS = [("e1a", 16, 16, 1), ("e1b", 16, 16, 1), ("e2a", 16, 32, 1), ("e2b", 32, 32, 1), ("e3a", 32, 64, 1),
          ("e3b", 64, 64, 1), ("bta", 64, 64, 1), ("btb", 64, 64, 1), ("d3a", 128, 64, 1), ("d3b", 64, 64, 1),
          ("d2a", 96, 32, 1), ("d2b", 32, 32, 1), ("d1a", 48, 16, 1), ("d1b", 16, 16, 1), ("out", 16, 16, 0)]


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(st, what):
    if st != 0:
        raise RuntimeError(f"{what} failed with status {st}")


class UNet:
    """Parameters, Adam state and activation buffers for batches of nb grids of n^3 nodes.

    tc=True runs every convolution of training on the fifth-generation tensor cores (tcgen05:
    the forward pass on weights packed into the operand tiles after each update, the data
    gradient as the forward kernel on the flipped weights, the weight gradient as a GEMM over
    the nodes); tc=False on the warp-level MMA kernels."""

    def __init__(self, n=33, nb=8, seed=0, device="cuda", tc=False):
        self.L = B.load()
        self.n, self.nb, self.dev, self.tc = n, nb, device, tc
        self.dims = [n, (n + 1) // 2, ((n + 1) // 2 + 1) // 2, (((n + 1) // 2 + 1) // 2 + 1) // 2]
        for d in self.dims[:3]:
            assert d % 2 == 1, "every level but the last must have an odd node count"
        g = torch.Generator().manual_seed(seed)
        self.w32, self.b32, self.w16, self.gw, self.gb, self.m, self.v = {}, {}, {}, {}, {}, {}, {}
        for name, cin, cout, _ in LAYERS:
            w = torch.randn(27, cin, cout, generator=g, dtype=torch.float64) * np.sqrt(2.0 / (27 * cin))
            self.w32[name] = w.to(device=device, dtype=torch.float32).contiguous()
            self.b32[name] = torch.zeros(cout, device=device, dtype=torch.float32)
            self.w16[name] = self.w32[name].to(torch.bfloat16).contiguous()
            self.gw[name] = torch.zeros_like(self.w32[name])
            self.gb[name] = torch.zeros_like(self.b32[name])
            for st in (self.m, self.v):
                st[name + ".w"] = torch.zeros_like(self.w32[name])
                st[name + ".b"] = torch.zeros_like(self.b32[name])
        self.step_count = 0
        self.wflip = torch.empty(27 * 128 * 64, dtype=torch.bfloat16, device=device)
        self.wpk_flip = torch.empty(27 * 128 * 64, dtype=torch.bfloat16, device=device)
        self.wpk = {name: torch.empty_like(self.w16[name]) for name in self.w16}
        self.packed = False
        self.tc_err = torch.zeros(1, dtype=torch.int32, device=device)
        self._alloc(nb)
        self.scales = {"s0": 1.0, "s1": 1.0, "h_ref": 1.0, "out": 1.0}

    # ------------------------------------------------------------ buffers
    def _alloc(self, nb):
        self.nb = nb
        f32 = lambda *s: torch.empty(*s, dtype=torch.float32, device=self.dev)
        bf = lambda *s: torch.empty(*s, dtype=torch.bfloat16, device=self.dev)
        N = [nb * d ** 3 for d in self.dims]
        self.N = N
        self.act = {}   # name -> (input bf16, output f32)
        self.x16 = bf(N[0], 16)
        shapes = {"e1a": 0, "e1b": 0, "e2a": 1, "e2b": 1, "e3a": 2, "e3b": 2, "bta": 3, "btb": 3, "d3a": 2, "d3b": 2,
                  "d2a": 1, "d2b": 1, "d1a": 0, "d1b": 0, "out": 0}
        self.level = shapes
        for name, cin, cout, _ in LAYERS:
            lv = shapes[name]
            self.act[name] = (bf(N[lv], cin), f32(N[lv], cout))
        self.cat32 = {3: f32(N[2], 128), 2: f32(N[1], 96), 1: f32(N[0], 48)}
        self.pool32 = {1: f32(N[1], 16), 2: f32(N[2], 32), 3: f32(N[3], 64)}
        self.g32 = {lv: f32(N[lv], 128) for lv in range(4)}      # gradient scratch per level
        self.g16 = {lv: bf(N[lv], 128) for lv in range(4)}
        self.gskip = {1: f32(N[0], 16), 2: f32(N[1], 32), 3: f32(N[2], 64)}
        self.gtmp = {lv: f32(N[lv], 128) for lv in range(4)}
        self.pred = f32(N[0])
        self.dpred = f32(N[0])
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)

    def _d3(self, lv):
        d = self.dims[lv]
        return (ctypes.c_int * 3)(d, d, d)

    # ------------------------------------------------------------ building blocks
    def _pack(self):
        if not self.packed:
            for name, cin, cout, _ in LAYERS:
                _chk(self.L.lasto_nn_pack_weights(cin, cout, _p(self.w16[name]), _p(self.wpk[name]), _s()), "pack")
            self.packed = True

    def _conv(self, name, x16, y32, ldy=None, off=0):
        _, cin, cout, relu = next(l for l in LAYERS if l[0] == name)
        lv = self.level[name]
        if self.tc:
            self._pack()
            _chk(self.L.lasto_nn_conv3d_fwd_tc(self.nb, self._d3(lv), cin, cout, _p(x16), _p(self.wpk[name]),
                                               _p(self.b32[name]), relu, _p(y32), ldy or cout, off, None, 0, 0,
                                               _p(self.tc_err), _s()), "conv_tc " + name)
            return
        _chk(self.L.lasto_nn_conv3d_fwd(self.nb, self._d3(lv), cin, cout, _p(x16), _p(self.w16[name]),
                                        _p(self.b32[name]), relu, _p(y32), ldy or cout, off, None, 0, 0, _s()),
             "conv " + name)

    def _tobf(self, src, dst):
        _chk(self.L.lasto_nn_to_bf16(src.numel(), _p(src), _p(dst), _s()), "to_bf16")

    def _copy(self, nodes, C, src, lds, soff, dst, ldd, doff, acc=0):
        _chk(self.L.lasto_nn_copy_channels(nodes, C, _p(src), lds, soff, _p(dst), ldd, doff, acc, _s()), "copy")

    def _layer(self, name, x16):
        """Run one convolution: stores its input (bf16) and output (f32) for the backward pass."""
        xin, y = self.act[name]
        if xin.data_ptr() != x16.data_ptr():
            xin.copy_(x16)
        self._conv(name, xin, y)
        return y

    # ------------------------------------------------------------ forward
    def forward(self, x32):
        """x32: FP32 [nb * n^3][16] input features -> FP32 [nb * n^3] prediction."""
        L = self.L
        self._tobf(x32, self.x16)
        a = self._layer("e1a", self.x16)
        self._tobf(a, self.act["e1b"][0])
        e1 = self._layer("e1b", self.act["e1b"][0])
        fine = lambda lv: self._d3(lv)
        _chk(L.lasto_nn_down(self.nb, fine(0), 16, _p(e1), _p(self.pool32[1]), 0, _s()), "down1")
        self._tobf(self.pool32[1], self.act["e2a"][0])
        a = self._layer("e2a", self.act["e2a"][0])
        self._tobf(a, self.act["e2b"][0])
        e2 = self._layer("e2b", self.act["e2b"][0])
        _chk(L.lasto_nn_down(self.nb, fine(1), 32, _p(e2), _p(self.pool32[2]), 0, _s()), "down2")
        self._tobf(self.pool32[2], self.act["e3a"][0])
        a = self._layer("e3a", self.act["e3a"][0])
        self._tobf(a, self.act["e3b"][0])
        e3 = self._layer("e3b", self.act["e3b"][0])
        _chk(L.lasto_nn_down(self.nb, fine(2), 64, _p(e3), _p(self.pool32[3]), 0, _s()), "down3")
        self._tobf(self.pool32[3], self.act["bta"][0])
        a = self._layer("bta", self.act["bta"][0])
        self._tobf(a, self.act["btb"][0])
        bt = self._layer("btb", self.act["btb"][0])
        # decoder: [up(lower), skip]
        for lv, low, skip, cup, cs, na, nb_ in ((3, bt, e3, 64, 64, "d3a", "d3b"), (2, None, e2, 64, 32, "d2a", "d2b"),
                                                (1, None, e1, 32, 16, "d1a", "d1b")):
            if low is None:
                low = self.act[{"d2a": "d3b", "d1a": "d2b"}[na]][1]
            cat = self.cat32[lv]
            ctot = cup + cs
            _chk(L.lasto_nn_up(self.nb, fine(lv - 1), cup, _p(low), _p(cat), ctot, 0, 0, _s()), "up")
            self._copy(self.N[lv - 1], cs, skip, cs, 0, cat, ctot, cup)
            self._tobf(cat, self.act[na][0])
            a = self._layer(na, self.act[na][0])
            self._tobf(a, self.act[nb_][0])
            self._layer(nb_, self.act[nb_][0])
        d1 = self.act["d1b"][1]
        self._tobf(d1, self.act["out"][0])
        o = self._layer("out", self.act["out"][0])
        self._copy(self.N[0], 1, o, 16, 0, self.pred.view(-1, 1), 1, 0)
        return self.pred

    # ------------------------------------------------------------ backward
    def _back(self, name, dy32):
        """dy32: FP32 gradient of the layer output -> FP32 gradient of its input (in gtmp)."""
        _, cin, cout, relu = next(l for l in LAYERS if l[0] == name)
        lv = self.level[name]
        xin, y = self.act[name]
        n = self.N[lv] * cout
        dpre32 = self.g32[lv][: self.N[lv]].view(-1)[:n]
        dpre16 = self.g16[lv][: self.N[lv]].view(-1)[:n]
        if relu:
            _chk(self.L.lasto_nn_relu_grad(n, _p(y), _p(dy32), _p(dpre32), _p(dpre16), _s()), "relu_grad")
        else:
            dpre32.copy_(dy32.view(-1)[:n])
            self._tobf(dpre32, dpre16)
        dx = self.gtmp[lv].view(-1)[: self.N[lv] * cin]
        if self.tc:
            _chk(self.L.lasto_nn_conv3d_wgrad_tc(self.nb, self._d3(lv), cin, cout, _p(xin), _p(dpre16), _p(dpre32),
                                                 _p(self.gw[name]), _p(self.gb[name]), _p(self.tc_err), _s()),
                 "wgrad_tc " + name)
            _chk(self.L.lasto_nn_conv3d_dgrad_tc(self.nb, self._d3(lv), cin, cout, _p(dpre16), _p(self.w16[name]),
                                                 _p(self.wflip), _p(self.wpk_flip), _p(dx), _p(self.tc_err), _s()),
                 "dgrad_tc " + name)
            return dx.clone()
        _chk(self.L.lasto_nn_conv3d_wgrad(self.nb, self._d3(lv), cin, cout, _p(xin), _p(dpre16), _p(dpre32),
                                          _p(self.gw[name]), _p(self.gb[name]), _s()), "wgrad " + name)
        _chk(self.L.lasto_nn_conv3d_dgrad(self.nb, self._d3(lv), cin, cout, _p(dpre16), _p(self.w16[name]),
                                          _p(self.wflip), _p(dx), _s()), "dgrad " + name)
        return dx.clone()

    def backward(self, dpred):
        L = self.L
        for name in self.gw:
            self.gw[name].zero_()
            self.gb[name].zero_()
        fine = lambda lv: self._d3(lv)
        do = torch.zeros(self.N[0], 16, dtype=torch.float32, device=self.dev)
        self._copy(self.N[0], 1, dpred.view(-1, 1), 1, 0, do, 16, 0)
        g = self._back("out", do)
        g = self._back("d1b", g)
        dcat = self._back("d1a", g).view(self.N[0], 48)
        de1 = dcat[:, 32:].contiguous()
        dlow = torch.empty(self.N[1], 32, dtype=torch.float32, device=self.dev)
        _chk(L.lasto_nn_up(self.nb, fine(0), 32, _p(dcat), _p(dlow), 48, 0, 1, _s()), "up_adj1")
        g = self._back("d2b", dlow)
        dcat = self._back("d2a", g).view(self.N[1], 96)
        de2 = dcat[:, 64:].contiguous()
        dlow = torch.empty(self.N[2], 64, dtype=torch.float32, device=self.dev)
        _chk(L.lasto_nn_up(self.nb, fine(1), 64, _p(dcat), _p(dlow), 96, 0, 1, _s()), "up_adj2")
        g = self._back("d3b", dlow)
        dcat = self._back("d3a", g).view(self.N[2], 128)
        de3 = dcat[:, 64:].contiguous()
        dlow = torch.empty(self.N[3], 64, dtype=torch.float32, device=self.dev)
        _chk(L.lasto_nn_up(self.nb, fine(2), 64, _p(dcat), _p(dlow), 128, 0, 1, _s()), "up_adj3")
        g = self._back("btb", dlow)
        dp3 = self._back("bta", g).view(self.N[3], 64)
        tmp = torch.empty(self.N[2], 64, dtype=torch.float32, device=self.dev)
        _chk(L.lasto_nn_down(self.nb, fine(2), 64, _p(dp3), _p(tmp), 1, _s()), "down_adj3")
        de3 += tmp
        g = self._back("e3b", de3)
        dp2 = self._back("e3a", g).view(self.N[2], 32)
        tmp = torch.empty(self.N[1], 32, dtype=torch.float32, device=self.dev)
        _chk(L.lasto_nn_down(self.nb, fine(1), 32, _p(dp2), _p(tmp), 1, _s()), "down_adj2")
        de2 += tmp
        g = self._back("e2b", de2)
        dp1 = self._back("e2a", g).view(self.N[1], 16)
        tmp = torch.empty(self.N[0], 16, dtype=torch.float32, device=self.dev)
        _chk(L.lasto_nn_down(self.nb, fine(0), 16, _p(dp1), _p(tmp), 1, _s()), "down_adj1")
        de1 += tmp
        g = self._back("e1b", de1)
        self._back("e1a", g)

    def loss_and_grad(self, target, mask):
        """Masked MSE of the current prediction; returns the loss (device scalar) and fills dpred."""
        self.loss.zero_()
        cnt = float(mask.sum().item()) if not hasattr(self, "_mask_count") else self._mask_count
        _chk(self.L.lasto_nn_mse(self.N[0], _p(self.pred), _p(target), _p(mask), 1.0 / cnt, _p(self.dpred),
                                 _p(self.loss), _s()), "mse")
        return self.loss

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        self.packed = False
        for name in self.w32:
            _chk(self.L.lasto_nn_adam(self.w32[name].numel(), _p(self.w32[name]), _p(self.gw[name]),
                                      _p(self.m[name + ".w"]), _p(self.v[name + ".w"]), lr, b1, b2, eps,
                                      self.step_count, _p(self.w16[name]), _s()), "adam")
            _chk(self.L.lasto_nn_adam(self.b32[name].numel(), _p(self.b32[name]), _p(self.gb[name]),
                                      _p(self.m[name + ".b"]), _p(self.v[name + ".b"]), lr, b1, b2, eps,
                                      self.step_count, None, _s()), "adam")

    # ------------------------------------------------------------ parameters
    def set_params(self, P):
        """Load parameters from a dict of numpy arrays name.w [27, cin, cout], name.b [cout]."""
        for name in self.w32:
            self.w32[name].copy_(torch.as_tensor(P[name + ".w"], dtype=torch.float32))
            self.b32[name].copy_(torch.as_tensor(P[name + ".b"], dtype=torch.float32))
            self.w16[name].copy_(self.w32[name].to(torch.bfloat16))
        self.packed = False

    def get_params(self):
        P = {}
        for name in self.w32:
            P[name + ".w"] = self.w32[name].double().cpu().numpy()
            P[name + ".b"] = self.b32[name].double().cpu().numpy()
        return P

    def grads(self):
        G = {}
        for name in self.w32:
            G[name + ".w"] = self.gw[name].double().cpu().numpy()
            G[name + ".b"] = self.gb[name].double().cpu().numpy()
        return G

    def save(self, path):
        P = self.get_params()
        np.savez(path, scales=json.dumps(self.scales), n=self.n, **{k: v.astype(np.float32) for k, v in P.items()})

    @classmethod
    def load(cls, path, nb=1, device="cuda"):
        z = np.load(path)
        net = cls(n=int(z["n"]), nb=nb, device=device)
        net.set_params({k: z[k] for k in z.files if k.endswith(".w") or k.endswith(".b")})
        net.scales = json.loads(str(z["scales"]))
        return net


# ---------------------------------------------------------------- coarse-grid data of a cluster
def coarse_problem(dc, b=None, stream=None):
    """For a DeviceCluster on a 129^3-type hierarchy: the right-hand side restricted twice
    (full weighting, physical coordinates), the Dirichlet faces at the every-fourth nodes,
    the coarse and middle axes and the boundary multipoles Q_lm (FP64 device tensors)."""
    if b is None:
        b, _, _ = B.lasto_op_deposit(dc, precision=B.LASTO_PREC_MIXED)
    ax = [dc.x, dc.y, dc.z]
    mid = [a[::2].contiguous() for a in ax]
    crs = [a[::4].contiguous() for a in ax]
    b_mid = B.lasto_op_restrict(*ax, b.view(-1))
    b_c = B.lasto_op_restrict(*mid, b_mid.view(-1))
    Q = B.lasto_op_multipoles(*ax, b)
    faces = torch.zeros_like(b_c)
    B.lasto_op_boundary_fill(*crs, Q, faces, centre=dc.centre)
    return b_c, faces, crs, mid, Q


def features(net, b_c, faces, crs, out=None):
    n = b_c.shape[-1]
    N = b_c.numel()
    out = out if out is not None else torch.empty(N, 16, dtype=torch.float32, device=b_c.device)
    s = net.scales
    _chk(net.L.lasto_nn_guess_features((ctypes.c_int * 3)(n, n, n), _p(b_c), _p(faces), _p(crs[0]), _p(crs[1]),
                                       _p(crs[2]), s["s0"], s["s1"], s["h_ref"], _p(out), _s()), "features")
    return out


def learned_guess(net, dc, b=None):
    """Fine-grid initial guess for one cluster: network on the coarse grid, then trilinear
    prolongation (physical coordinates) to the middle and fine grids."""
    assert net.nb == 1
    b_c, faces, crs, mid, Q = coarse_problem(dc, b)
    x32 = features(net, b_c, faces, crs)
    pred = net.forward(x32)
    n = b_c.shape[-1]
    u_c = torch.empty_like(b_c)
    _chk(net.L.lasto_nn_guess_grid((ctypes.c_int * 3)(n, n, n), _p(pred), 1, net.scales["out"], _p(faces), _p(u_c),
                                   _s()), "guess_grid")
    nm = mid[0].numel()
    u_mid = torch.zeros((nm, nm, nm), dtype=torch.float64, device=b_c.device)
    B.lasto_op_boundary_fill(*mid, Q, u_mid, centre=dc.centre)      # Dirichlet faces of the middle grid
    B.lasto_op_prolong_add(*mid, u_c.view(-1), u_mid)                # interior: coarse guess interpolated
    u_fine = torch.zeros(dc.N, dtype=torch.float64, device=b_c.device)
    B.lasto_op_prolong_add(dc.x, dc.y, dc.z, u_mid, u_fine)
    return u_fine
