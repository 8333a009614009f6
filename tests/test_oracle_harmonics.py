"""Pins of the oracle's real spherical harmonics (Eq. 3.1's y_LM, l <= 4) and quadrature.

The paper names real spherical harmonics without a convention; the reading is the
orthonormal set without Condon-Shortley phase (m > 0 ~ cos m phi, m < 0 ~ sin |m| phi).
Pinned against scipy's complex harmonics and against orthonormality on an
independent product quadrature.
"""
import numpy as np
import pytest
import scipy.special as sp


def _scipy_real_ylm(l, m, theta, phi):
    if hasattr(sp, "sph_harm_y"):
        Y = sp.sph_harm_y(l, abs(m), theta, phi)
    else:  # older scipy: sph_harm(m, l, azimuth, polar)
        Y = sp.sph_harm(abs(m), l, phi, theta)
    if m == 0:
        return Y.real
    # scipy includes the Condon-Shortley phase (-1)^m; remove it
    s = np.sqrt(2.0) * (-1.0) ** abs(m)
    return s * (Y.real if m > 0 else Y.imag)


def test_matches_scipy(orc):
    rng = np.random.default_rng(0)
    for _ in range(40):
        v = rng.normal(size=3)
        r = np.linalg.norm(v)
        theta, phi = np.arccos(v[2] / r), np.arctan2(v[1], v[0])
        S = orc.solid_harmonics(*v)
        for l in range(5):
            for m in range(-l, l + 1):
                ref = _scipy_real_ylm(l, m, theta, phi) * r ** l
                assert abs(S[l * l + l + m] - ref) < 1e-13 * max(1.0, r ** l), (l, m)


def test_orthonormal_on_sphere(orc):
    t, w = np.polynomial.legendre.leggauss(12)
    nph = 24
    G = np.zeros((25, 25))
    for ct, wt in zip(t, w):
        st = np.sqrt(1 - ct * ct)
        for k in range(nph):
            ph = 2 * np.pi * k / nph
            S = orc.solid_harmonics(st * np.cos(ph), st * np.sin(ph), ct)
            G += wt * (2 * np.pi / nph) * np.outer(S, S)
    assert np.abs(G - np.eye(25)).max() < 1e-13


def test_homogeneous_and_harmonic(orc):
    rng = np.random.default_rng(1)
    ls = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)
    for _ in range(5):
        v = rng.normal(size=3)
        lam = 1.7
        assert np.allclose(orc.solid_harmonics(*(lam * v)), lam ** ls * orc.solid_harmonics(*v), rtol=1e-13, atol=1e-14)
        # Laplacian of a polynomial of degree <= 4 by the 5-point rule is exact up to rounding
        h = 1e-2
        lap = np.zeros(25)
        for a in range(3):
            e = np.zeros(3); e[a] = h
            f = lambda s: orc.solid_harmonics(*(v + s * e))
            lap += (-f(2) + 16 * f(1) - 30 * f(0) + 16 * f(-1) - f(-2)) / (12 * h * h)
        assert np.abs(lap).max() < 1e-8


@pytest.mark.parametrize("n", [1, 2, 16, 64])
def test_gauss_legendre(orc, n):
    t, w = orc.gauss_legendre(n)
    tr, wr = np.polynomial.legendre.leggauss(n)
    assert np.abs(t - tr).max() < 1e-14 and np.abs(w - wr).max() < 1e-14
