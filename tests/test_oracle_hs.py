"""Pins of the interstitial overlap and Hamiltonian contributions (Eq. 3.11-3.14, grid-point
form) of Table 1's Slater-type basis.

The kinetic part of Eq. 3.14's phi~ is checked against a finite-difference Laplacian of the
sampled functions (not the analytic form the oracle uses), S against the analytic radial
overlap beyond the sphere and the orthogonality of the harmonics, and the potential term by
the exact identity H(V + c) = H(V) + c S."""
import numpy as np
import pytest
from scipy import special

LS = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)


def _uniform_box(n, L):
    x = np.linspace(-L, L, n)
    return x, x, x


def _basis_on_grid(orc, pos, x, y, z, basis):
    """phi_a at every node (closed form r^(n-1) e^{-zeta r} y_lm), atom-major, table order."""
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    out = []
    for p in pos:
        d = np.stack([Xg - p[0], Yg - p[1], Zg - p[2]], axis=-1)
        r = np.linalg.norm(d, axis=-1)
        S = np.apply_along_axis(lambda v: orc.solid_harmonics(*v), -1, d)
        for n, l, zt in basis:
            for m in range(-l, l + 1):
                out.append(r ** (n - 1 - l) * np.exp(-zt * r) * S[..., l * l + l + m])
    return np.array(out)


def test_kinetic_part_against_a_finite_difference_laplacian(orc):
    """V = 0: H_ab = 1/2 sum (phi_a T phi_b + phi_b T phi_a) vol with T = -1/2 Lap; with T from
    a fourth-order central difference on a fine uniform grid the two agree to O(h^4).  The
    exponents are steep enough (zeta >= 2.2) that the functions are below 1e-4 of their peak on
    the two outer node layers, which the difference stencil leaves out."""
    basis = [(5, 0, 2.5), (5, 1, 2.5), (4, 2, 2.2), (4, 3, 2.5)]
    pos = np.array([[0.1, -0.05, 0.02]])
    R = np.array([2.4])
    h = 0.1
    n = 161
    x, y, z = _uniform_box(n, (n - 1) / 2 * h)
    S, H = orc.interstitial_hs(pos, R, x, y, z, np.zeros((n, n, n)), basis)
    phi = _basis_on_grid(orc, pos, x, y, z, basis)
    lap = np.zeros_like(phi)
    c = [-1 / 12, 4 / 3, -5 / 2, 4 / 3, -1 / 12]
    for ax in (1, 2, 3):
        for k, w in zip(range(-2, 3), c):
            lap += w * np.roll(phi, k, axis=ax)
    lap /= h * h
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt((Xg - pos[0, 0]) ** 2 + (Yg - pos[0, 1]) ** 2 + (Zg - pos[0, 2]) ** 2)
    inner = np.zeros(phi.shape[1:], bool)
    inner[2:-2, 2:-2, 2:-2] = True
    W = np.where((r >= R[0]) & inner, h ** 3, 0.0).reshape(-1)
    P = phi.reshape(len(phi), -1)
    Tm = (-0.5 * lap).reshape(len(phi), -1)
    Hfd = 0.5 * ((P * W) @ Tm.T + (Tm * W) @ P.T)
    scale = np.sqrt(np.outer(np.diag(S), np.diag(S)))
    assert (np.abs(H - Hfd) / scale).max() < 1e-4


def test_overlap_against_the_radial_integral(orc):
    """One atom: S_ab = delta_ll' delta_mm' int_R^inf r^(n+n') e^{-(zeta+zeta') r} dr.  The grid
    sum's error comes from the sphere's staircase boundary (O(h), of either sign from one
    resolution to the next); a wrong power, exponent or harmonic would be O(1)."""
    basis = [(5, 0, 1.0), (6, 0, 2.0), (5, 1, 1.0), (4, 2, 2.2)]
    pos = np.array([[0.0, 0.0, 0.0]])
    R = np.array([2.4])
    errs = []
    for n in (61, 121):
        x, y, z = _uniform_box(n, 15.0)
        S, _ = orc.interstitial_hs(pos, R, x, y, z, np.zeros((n, n, n)), basis)
        ls = [0, 0] + [1] * 3 + [2] * 5
        ns = [5, 6] + [5] * 3 + [4] * 5
        zs = [1.0, 2.0] + [1.0] * 3 + [2.2] * 5
        ms = [0, 0, -1, 0, 1, -2, -1, 0, 1, 2]
        exact = np.zeros_like(S)
        for a in range(len(ls)):
            for b in range(len(ls)):
                if ls[a] == ls[b] and ms[a] == ms[b]:
                    p, zz = ns[a] + ns[b], zs[a] + zs[b]
                    exact[a, b] = special.gamma(p + 1) / zz ** (p + 1) * special.gammaincc(p + 1, zz * R[0])
        scale = np.sqrt(np.outer(np.diag(exact), np.diag(exact)))
        errs.append(np.abs(S - exact).max() / scale.max())
    assert max(errs) < 1e-3


def test_potential_term_and_symmetry(orc):
    """H(V + c) - H(V) = c S exactly (up to rounding), S and H symmetric."""
    from synth import clusters
    pos = clusters.dimer()
    R = np.array([2.4, 2.4])
    x, y, z = _uniform_box(21, 9.0)
    rng = np.random.default_rng(0)
    V = rng.normal(size=(21, 21, 21))
    S, H = orc.interstitial_hs(pos, R, x, y, z, V)
    S2, H2 = orc.interstitial_hs(pos, R, x, y, z, V + 0.75)
    assert S.shape == (50, 50)
    assert np.abs(S - S2).max() < 1e-14 * np.abs(S).max()
    assert np.abs(H2 - H - 0.75 * S).max() < 1e-12 * np.abs(H).max()
    assert np.abs(S - S.T).max() < 1e-14 * np.abs(S).max() and np.abs(H - H.T).max() < 1e-14 * np.abs(H).max()
