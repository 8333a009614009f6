"""GPU network kernels (lasto_nn_*) against the FP64 oracle (oracle/unet_oracle.py).

Inputs are rounded to BF16 first and the oracle runs on those values in FP64, so the only
differences are FP32 accumulation (convolutions) and, for the whole network, the BF16
rounding of intermediate activations (loose tolerance, as for any BF16 network)."""
import ctypes

import numpy as np
import pytest

from gpu_common import need_gpu
from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)


def _f64(t):
    return t.float().double().cpu().numpy()


def _d3(dims):
    return (ctypes.c_int * 3)(*dims)


@pytest.mark.parametrize("cin,cout,relu", [(16, 16, 1), (48, 64, 0), (128, 32, 1)])
def test_conv_forward(cin, cout, relu):
    import torch
    B = need_gpu()
    L = B.load()
    rng = np.random.default_rng(cin + cout)
    nb, D, H, W = 2, 5, 7, 9
    x = _bf16(rng.normal(size=(nb, D, H, W, cin))).cuda()
    w = _bf16(rng.normal(size=(27, cin, cout)) * 0.1).cuda()
    bias = torch.as_tensor(rng.normal(size=cout), dtype=torch.float32).cuda()
    y = torch.empty(nb * D * H * W, cout, dtype=torch.float32, device="cuda")
    st = L.lasto_nn_conv3d_fwd(nb, _d3((W, H, D)), cin, cout, B._ptr(x), B._ptr(w), B._ptr(bias), relu, B._ptr(y),
                               cout, 0, None, 0, 0, B._stream())
    torch.cuda.synchronize()
    assert st == 0
    ref = U.conv3d(_f64(x), _f64(w), bias.double().cpu().numpy())
    if relu:
        ref = np.maximum(ref, 0)
    got = y.double().cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (48, 16), (32, 64), (128, 64), (96, 32), (64, 48),
                                      (32, 128)])
def test_conv_forward_tensor_memory(cin, cout):
    """The tcgen05 convolution (packed weights, accumulator in tensor memory) against the
    FP64 oracle, with a ragged last tile (630 nodes = 4 tiles of 128 + 118)."""
    import torch
    B = need_gpu()
    L = B.load()
    rng = np.random.default_rng(3 * cin + cout)
    nb, D, H, W = 2, 5, 7, 9
    x = _bf16(rng.normal(size=(nb, D, H, W, cin))).cuda()
    w = _bf16(rng.normal(size=(27, cin, cout)) * 0.1).cuda()
    wpk = torch.empty_like(w)
    bias = torch.as_tensor(rng.normal(size=cout), dtype=torch.float32).cuda()
    y = torch.full((nb * D * H * W, cout), float("nan"), dtype=torch.float32, device="cuda")
    y16 = torch.empty(nb * D * H * W, cout, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.lasto_nn_pack_weights(cin, cout, B._ptr(w), B._ptr(wpk), B._stream()) == 0
    st = L.lasto_nn_conv3d_fwd_tc(nb, _d3((W, H, D)), cin, cout, B._ptr(x), B._ptr(wpk), B._ptr(bias), 1, B._ptr(y),
                                  cout, 0, B._ptr(y16), cout, 0, B._ptr(err), B._stream())
    torch.cuda.synchronize()
    assert st == 0 and int(err.item()) == 0
    ref = np.maximum(U.conv3d(_f64(x), _f64(w), bias.double().cpu().numpy()), 0)
    got = y.double().cpu().numpy().reshape(ref.shape)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    assert torch.equal(y16, y.to(torch.bfloat16))


@pytest.mark.parametrize("cin,cout", [(16, 32), (64, 16), (96, 32)])
def test_conv_gradients(cin, cout):
    import torch
    B = need_gpu()
    L = B.load()
    rng = np.random.default_rng(7 * cin + cout)
    nb, D, H, W = 2, 5, 6, 7
    x = _bf16(rng.normal(size=(nb, D, H, W, cin))).cuda()
    w = _bf16(rng.normal(size=(27, cin, cout)) * 0.1).cuda()
    dy32 = torch.as_tensor(rng.normal(size=(nb * D * H * W, cout)), dtype=torch.float32).cuda()
    dy16 = dy32.to(torch.bfloat16)
    dy32 = dy16.float()
    dx = torch.empty(nb * D * H * W, cin, dtype=torch.float32, device="cuda")
    wf = torch.empty(27 * cin * cout, dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros(27, cin, cout, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    assert L.lasto_nn_conv3d_dgrad(nb, _d3((W, H, D)), cin, cout, B._ptr(dy16), B._ptr(w), B._ptr(wf), B._ptr(dx),
                                   B._stream()) == 0
    assert L.lasto_nn_conv3d_wgrad(nb, _d3((W, H, D)), cin, cout, B._ptr(x), B._ptr(dy16), B._ptr(dy32), B._ptr(dw),
                                   B._ptr(db), B._stream()) == 0
    torch.cuda.synchronize()
    rdx, rdw, rdb = U.conv3d_backward(_f64(x), _f64(w), _f64(dy16).reshape(nb, D, H, W, cout))
    assert np.abs(dx.double().cpu().numpy().reshape(rdx.shape) - rdx).max() <= 2e-5 * np.abs(rdx).max()
    assert np.abs(dw.double().cpu().numpy() - rdw).max() <= 2e-5 * np.abs(rdw).max()
    assert np.abs(db.double().cpu().numpy() - rdb).max() <= 2e-5 * np.abs(rdb).max()


@pytest.mark.parametrize("cin,cout,dims", [(16, 32, (7, 6, 5)), (64, 16, (7, 6, 5)), (96, 32, (7, 6, 5)),
                                           (48, 64, (9, 5, 7)), (128, 128, (5, 5, 5)), (32, 48, (33, 9, 11))])
def test_conv_gradients_tensor_memory(cin, cout, dims):
    """The tcgen05 data gradient (flipped weights through the tcgen05 forward kernel) and
    weight gradient (GEMM over the nodes, both operands read MN-major from the channels-last
    rows) against the FP64 oracle; node counts that leave a ragged last K step and a ragged
    last chunk (33 x 9 x 11 x 2 = 6534 nodes = 3 chunks of 2048 + 390), tap tiles with padding
    rows (cin 48 and 96) and the largest channel counts."""
    import torch
    B = need_gpu()
    L = B.load()
    rng = np.random.default_rng(11 * cin + cout)
    nb, (W, H, D) = 2, dims
    x = _bf16(rng.normal(size=(nb, D, H, W, cin))).cuda()
    w = _bf16(rng.normal(size=(27, cin, cout)) * 0.1).cuda()
    dy16 = _bf16(rng.normal(size=(nb * D * H * W, cout))).cuda()
    dy32 = dy16.float()
    dx = torch.full((nb * D * H * W, cin), float("nan"), dtype=torch.float32, device="cuda")
    wf = torch.empty(27 * cin * cout, dtype=torch.bfloat16, device="cuda")
    wpk = torch.empty_like(wf)
    dw = torch.zeros(27, cin, cout, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.lasto_nn_conv3d_dgrad_tc(nb, _d3((W, H, D)), cin, cout, B._ptr(dy16), B._ptr(w), B._ptr(wf), B._ptr(wpk),
                                      B._ptr(dx), B._ptr(err), B._stream()) == 0
    assert L.lasto_nn_conv3d_wgrad_tc(nb, _d3((W, H, D)), cin, cout, B._ptr(x), B._ptr(dy16), B._ptr(dy32),
                                      B._ptr(dw), B._ptr(db), B._ptr(err), B._stream()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    rdx, rdw, rdb = U.conv3d_backward(_f64(x), _f64(w), _f64(dy16).reshape(nb, D, H, W, cout))
    assert np.abs(dx.double().cpu().numpy().reshape(rdx.shape) - rdx).max() <= 2e-5 * np.abs(rdx).max()
    assert np.abs(dw.double().cpu().numpy() - rdw).max() <= 2e-5 * np.abs(rdw).max()
    assert np.abs(db.double().cpu().numpy() - rdb).max() <= 2e-5 * np.abs(rdb).max()


def test_sampling_and_adjoints():
    import torch
    B = need_gpu()
    L = B.load()
    rng = np.random.default_rng(3)
    nb, D, H, W, C = 2, 9, 5, 7, 16
    Dc, Hc, Wc = 5, 3, 4
    x = rng.normal(size=(nb, D, H, W, C))
    xc = rng.normal(size=(nb, Dc, Hc, Wc, C))
    t = lambda a: torch.as_tensor(a.reshape(-1, C), dtype=torch.float32).cuda()
    f = _d3((W, H, D))
    out_c = torch.empty(nb * Dc * Hc * Wc, C, dtype=torch.float32, device="cuda")
    out_f = torch.empty(nb * D * H * W, C, dtype=torch.float32, device="cuda")
    assert L.lasto_nn_down(nb, f, C, B._ptr(t(x)), B._ptr(out_c), 0, B._stream()) == 0
    torch.cuda.synchronize()
    assert np.abs(out_c.double().cpu().numpy() - U.down(x).reshape(-1, C)).max() < 1e-5
    assert L.lasto_nn_down(nb, f, C, B._ptr(t(xc)), B._ptr(out_f), 1, B._stream()) == 0
    torch.cuda.synchronize()
    assert np.abs(out_f.double().cpu().numpy() - U.down_adjoint(xc, (D, H, W)).reshape(-1, C)).max() < 1e-5
    wide = torch.zeros(nb * D * H * W, 2 * C, dtype=torch.float32, device="cuda")
    assert L.lasto_nn_up(nb, f, C, B._ptr(t(xc)), B._ptr(wide), 2 * C, C, 0, B._stream()) == 0
    torch.cuda.synchronize()
    assert np.abs(wide[:, C:].double().cpu().numpy() - U.up(xc, (D, H, W)).reshape(-1, C)).max() < 1e-5
    wide[:, C:] = t(x)
    assert L.lasto_nn_up(nb, f, C, B._ptr(wide), B._ptr(out_c), 2 * C, C, 1, B._stream()) == 0
    torch.cuda.synchronize()
    assert np.abs(out_c.double().cpu().numpy() - U.up_adjoint(x).reshape(-1, C)).max() < 1e-5


@pytest.mark.parametrize("tc", [False, True])
def test_whole_network_matches_oracle(tc):
    """Forward, loss and every parameter gradient of the U-Net on a batch of two 17^3 grids, on
    the warp-level MMA kernels and on the tcgen05 kernels (forward, data and weight gradients)."""
    import torch
    B = need_gpu()
    from paper_0806_1723_gb300 import unet
    rng = np.random.default_rng(5)
    P = U.init_params(seed=6)
    net = unet.UNet(n=17, nb=2, tc=tc)
    net.set_params(P)
    x = rng.normal(size=(2, 17, 17, 17, 16)) * 0.5
    x[..., 3:] = 0
    target = rng.normal(size=(2, 17, 17, 17))
    mask = np.zeros_like(target)
    mask[:, 1:-1, 1:-1, 1:-1] = 1
    xb = np.asarray(_f64(_bf16(x)))
    pred = net.forward(torch.as_tensor(x.reshape(-1, 16), dtype=torch.float32).cuda())
    net._mask_count = float(mask.sum())
    net.loss_and_grad(torch.as_tensor(target.reshape(-1), dtype=torch.float32).cuda(),
                      torch.as_tensor(mask.reshape(-1), dtype=torch.float32).cuda())
    net.backward(net.dpred)
    torch.cuda.synchronize()
    assert int(net.tc_err.item()) == 0
    rpred, cache = U.forward(P, xb)
    assert np.linalg.norm(pred.double().cpu().numpy() - rpred.reshape(-1)) <= 2e-2 * np.linalg.norm(rpred)
    loss, dpred = U.mse(rpred, target, mask)
    assert abs(float(net.loss.item()) - loss) <= 2e-2 * loss
    G = U.backward(P, cache, dpred)
    Gg = net.grads()
    for k in G:
        a, b = Gg[k].ravel(), G[k].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        assert cos > 0.99 and np.linalg.norm(a - b) <= 0.1 * np.linalg.norm(b), (k, cos)
