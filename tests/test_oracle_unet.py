"""Pins of the network oracle (oracle/unet_oracle.py): the convolution against scipy's
correlate, the sampling operators' exactness properties, and every gradient against
central finite differences in FP64."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet_oracle as U


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 5, 6, 7, 2))
    w = rng.normal(size=(27, 2, 3))
    y = U.conv3d(x, w)
    for co in range(3):
        ref = np.zeros((5, 6, 7))
        for ci in range(2):
            k = w[:, ci, co].reshape(3, 3, 3)   # tap = (dz, dy, dx) lexicographic
            ref += ndimage.correlate(x[0, ..., ci], k, mode="constant", cval=0.0)
        assert np.abs(y[0, ..., co] - ref).max() < 1e-12


def test_sampling_operators():
    n = 9
    D, Up = U.down_matrix(n), U.up_matrix(n)
    assert np.allclose(D.sum(1), 1.0)                        # constants preserved
    t = np.linspace(-1, 1, (n + 1) // 2)
    assert np.allclose(Up @ t, np.linspace(-1, 1, n))        # linear functions reproduced
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 9, 5, 7, 3))
    yc = rng.normal(size=(2, 5, 3, 4, 3))
    assert abs((U.down(x) * yc).sum() - (x * U.down_adjoint(yc, (9, 5, 7))).sum()) < 1e-12
    assert abs((U.up(yc, (9, 5, 7)) * x).sum() - (yc * U.up_adjoint(x)).sum()) < 1e-12


def test_conv_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 4, 3, 5, 2))
    w = rng.normal(size=(27, 2, 3))
    b = rng.normal(size=3)
    dy = rng.normal(size=(1, 4, 3, 5, 3))
    dx, dw, db = U.conv3d_backward(x, w, dy)
    f = lambda xx, ww, bb: (U.conv3d(xx, ww, bb) * dy).sum()
    h = 1e-6
    for _ in range(10):
        i = tuple(rng.integers(0, s) for s in x.shape)
        e = np.zeros_like(x); e[i] = h
        assert abs((f(x + e, w, b) - f(x - e, w, b)) / (2 * h) - dx[i]) < 1e-6
        j = tuple(rng.integers(0, s) for s in w.shape)
        e = np.zeros_like(w); e[j] = h
        assert abs((f(x, w + e, b) - f(x, w - e, b)) / (2 * h) - dw[j]) < 1e-6
    e = np.zeros(3); e[1] = h
    assert abs((f(x, w, b + e) - f(x, w, b - e)) / (2 * h) - db[1]) < 1e-6


@pytest.mark.slow
def test_network_gradients_by_finite_differences():
    """Whole U-Net on a 9^3 grid (levels 9, 5, 3, 2 are not all odd, so use 17^3 -> 9 -> 5 -> 3)."""
    rng = np.random.default_rng(3)
    P = U.init_params(seed=4)
    x = rng.normal(size=(1, 17, 17, 17, 16)) * 0.5
    target = rng.normal(size=(1, 17, 17, 17))
    mask = np.ones_like(target)
    pred, cache = U.forward(P, x)
    loss, dpred = U.mse(pred, target, mask)
    G = U.backward(P, cache, dpred)
    h = 1e-5
    for name in ("e1a.w", "bta.w", "d2a.b", "out.w", "e3b.w"):
        for _ in range(2):
            j = tuple(rng.integers(0, s) for s in P[name].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][j] += h
            Pm[name][j] -= h
            lp = U.mse(U.forward(Pp, x)[0], target, mask)[0]
            lm = U.mse(U.forward(Pm, x)[0], target, mask)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[name][j]) <= 1e-6 + 1e-4 * abs(fd), (name, j, fd, G[name][j])
