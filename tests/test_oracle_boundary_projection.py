"""Pins of the boundary multipoles (Eq. 2.7 decay via the exterior expansion), the
sphere-surface projection (Eq. 3.6) and the whole oracle pipeline.

Whole pipeline: outside the spheres the pseudo-density has the same potential as
the true density (same monopole inside each sphere, shell theorem), which for
the Slater model is known in closed form; so the exact V_LM(R_i) of Eq. 3.6 is a
surface quadrature done here, and the oracle's discrete answer must approach it
at second order in h.
"""
import numpy as np
import pytest
from scipy import integrate

import synth

LS = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)


def test_offcentre_gaussian_moments(orc):
    """A spherical charge centred at d has Q_lm = Q S_lm(d) (mean-value property); the trapezoid sum is spectral."""
    Q, a, L = 2.0, 1.5, 8.0
    d = np.array([0.7, -0.4, 1.1])
    x = np.linspace(-L, L, 65)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r2 = (X - d[0]) ** 2 + (Y - d[1]) ** 2 + (Z - d[2]) ** 2
    b = 4 * np.pi * Q * (a * a / np.pi) ** 1.5 * np.exp(-a * a * r2)
    Qlm = orc.multipoles(x, x, x, b)
    assert np.abs(Qlm - Q * orc.solid_harmonics(*d)).max() < 1e-9


def test_boundary_values_are_point_multipoles(orc):
    """Faces get -sum 4pi/(2l+1) Q_lm y_lm / r^(l+1); for a point charge at d this is the l<=4 truncation of -Q/|x-d|."""
    Q = 1.3
    d = np.array([0.5, 0.3, -0.6])
    Qlm = Q * orc.solid_harmonics(*d)
    x = np.linspace(-6, 6, 17)
    u = orc.boundary_fill(x, x, x, Qlm, np.zeros((17,) * 3))
    for k, j, i in [(0, 3, 5), (16, 8, 8), (4, 0, 12), (9, 16, 2), (7, 11, 0), (13, 2, 16)]:
        p = np.array([x[i], x[j], x[k]])
        r, rd = np.linalg.norm(p), np.linalg.norm(d)
        exact = -Q / np.linalg.norm(p - d)
        assert abs(u[k, j, i] - exact) < 2 * Q / r * (rd / r) ** 5
    assert np.all(u[1:-1, 1:-1, 1:-1] == 0)


@pytest.mark.parametrize("lm", [0, 1, 2, 3])
def test_projection_exact_for_linear(orc, lm):
    """V = S_lm(x - X) with l <= 1 is reproduced exactly by trilinear interpolation: V_LM = R^l delta."""
    x = np.linspace(-6, 6, 33)
    y = np.linspace(-5, 7, 33)
    centre, R = np.array([0.3, 1.1, -0.2]), 2.4
    Z, Y, X = np.meshgrid(x, y, x, indexing="ij")
    u = np.vectorize(lambda a, b_, c: orc.solid_harmonics(a, b_, c)[lm])(X - centre[0], Y - centre[1], Z - centre[2])
    vlm = orc.project(x, y, x, u, centre[None, :], np.array([R]))
    ref = np.zeros(25)
    ref[lm] = R ** LS[lm]
    assert np.abs(vlm[0] - ref).max() < 1e-12


def test_projection_second_order_for_higher_l(orc):
    centre, R = np.array([0.1, -0.2, 0.3]), 2.4
    errs = []
    for n in (33, 65):
        x = np.linspace(-6, 6, n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        S = np.zeros((n, n, n))
        for idx in np.ndindex(S.shape):
            S[idx] = orc.solid_harmonics(X[idx] - centre[0], Y[idx] - centre[1], Z[idx] - centre[2])[18]
        vlm = orc.project(x, x, x, S, centre[None, :], np.array([R]))[0]
        errs.append(abs(vlm[18] - R ** 4))
    assert errs[1] < errs[0] / 3.0 and errs[1] < 0.02 * R ** 4


def _exact_surface_potential(orc, cl, p):
    """Continuum potential of the Slater-model cluster at p (outside every sphere interior)."""
    u = 0.0
    for j in range(cl.n_atoms):
        d = p - cl.pos[j]
        r = np.linalg.norm(d)
        for w, z in zip(cl.slater_w[j], cl.slater_zeta[j]):
            u += w * np.exp(-z * r) * (1 / r + z / 2)      # nucleus Z plus its normalised Slater shells
        R, z1 = cl.R[j], cl.slater_zeta[j, 0]
        S = orc.solid_harmonics(*d)
        for lm in range(1, 25):
            l = LS[lm]
            rad = integrate.quad(lambda s: z1 ** 3 / (8 * np.pi) * np.exp(-z1 * s) * (1 - s * s / R / R) ** 2 * s ** (2 * l + 2),
                                 0, R, epsabs=1e-15, epsrel=1e-13)[0]
            u -= 4 * np.pi / (2 * l + 1) * cl.c_lm[j, lm - 1] * rad / R ** l * S[lm] / r ** (2 * l + 1)
    return u


def _exact_vlm(orc, cl, i, nt=20, nph=40):
    t, w = np.polynomial.legendre.leggauss(nt)
    acc = np.zeros(25)
    for ct, wt in zip(t, w):
        st = np.sqrt(1 - ct * ct)
        for k in range(nph):
            ph = 2 * np.pi * k / nph
            nrm = np.array([st * np.cos(ph), st * np.sin(ph), ct])
            acc += wt * 2 * np.pi / nph * _exact_surface_potential(orc, cl, cl.pos[i] + cl.R[i] * nrm) * orc.solid_harmonics(*nrm)
    return acc


@pytest.mark.slow
def test_pipeline_approaches_the_continuum_answer(orc):
    """Pd2 at the paper's 4.802 au: oracle V_LM(R_i) -> exact continuum value at O(h^2).

    The box half-width (15 bohr) keeps the atoms' exponential tails at the faces far
    below the discretisation error, so the l <= 4 multipole faces do not set a floor.
    """
    base = synth.pd2_dimer(n=33, half_width=15.0)
    exact = _exact_vlm(orc, base, 0)
    errs = []
    for n in (33, 65, 129):
        cl = synth.pd2_dimer(n=n, half_width=15.0)
        out = orc.poisson_solve(cl, tol=1e-12, max_cycles=40)
        assert out["status"] == 0
        errs.append(np.abs(out["vlm"][0] - exact).max())
    assert errs[2] < errs[1] < errs[0]
    assert errs[0] / errs[2] > 12.0          # two halvings of h at second order: 16
    assert errs[2] < 1e-2 * np.abs(exact).max()
