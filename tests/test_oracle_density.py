"""Pins of the density model, the sphere monopoles and the pseudo-density.

Pseudo-density (Section 3, the constraints beside Eq. 3.2-3.3): inside each
sphere it carries the same charge as rho - Z delta and meets the spherical part
of rho in value and slope at R; Fig. 3 shows it finite and negative at the
centre.  Everything here is checked against quadratures done in this file
(scipy / numpy), not against the oracle's own Gauss-Legendre.
"""

import numpy as np
import pytest
from scipy import integrate

import synth
from synth.workloads import make_cluster


pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _single_atom(seed=5):
    rng = np.random.default_rng(seed)
    return make_cluster("Pd1", np.zeros((1, 3)), rng, n=33, half_width=12.0, h_min=0.75, h_max=0.75)


def _angular_rule(nt=24, nph=48):
    t, w = np.polynomial.legendre.leggauss(nt)
    st = np.sqrt(1 - t * t)
    ph = 2 * np.pi * np.arange(nph) / nph
    dirs = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(t, np.ones(nph))], -1).reshape(-1, 3)
    wts = np.outer(w, np.full(nph, 2 * np.pi / nph)).reshape(-1)
    return dirs, wts


def _sphere_mean(orc, cl, centre, r, dirs, wts):
    vals = np.array([orc.density(cl, *(centre + r * d)) for d in dirs])
    return (wts * vals).sum() / (4 * np.pi)


def test_atom_holds_Z_electrons(orc):
    """A lone atom's density integrates to sum(w) = 46 (normalised Slater terms; zero-monopole l >= 1 part)."""
    cl = _single_atom()
    dirs, wts = _angular_rule(8, 16)
    f = lambda r: r * r * (wts * np.array([orc.density(cl, *(r * d)) for d in dirs])).sum()
    total = sum(integrate.quad(f, a, b, epsabs=1e-13, epsrel=1e-13, limit=200)[0]
                for a, b in [(0, 1), (1, 2.4), (2.4, 10), (10, 40)])
    assert abs(total - 46.0) < 1e-9


def test_nonspherical_moments(orc):
    """int rho S_lm dV = c_lm R^-l int_0^R slater1 (1 - r^2/R^2)^2 r^(2l+2) dr (reading of the l >= 1 profile)."""
    cl = _single_atom()
    R, z1 = cl.R[0], cl.slater_zeta[0, 0]
    dirs, wts = _angular_rule(10, 20)
    S_dirs = np.array([orc.solid_harmonics(*d) for d in dirs])  # unit-sphere y_lm
    def moment(r):
        rho = np.array([orc.density(cl, *(r * d)) for d in dirs])
        return r * r * (wts[:, None] * rho[:, None] * S_dirs * r ** np.array([0] + [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)).sum(0)
    gl, gw = np.polynomial.legendre.leggauss(40)
    rr = 0.5 * R * (gl + 1)
    got = sum(0.5 * R * w * moment(r) for r, w in zip(rr, gw))
    for l in range(1, 5):
        radial = integrate.quad(lambda r: z1 ** 3 / (8 * np.pi) * np.exp(-z1 * r) * (1 - r * r / R / R) ** 2 * r ** (2 * l + 2),
                                0, R, epsabs=1e-15, epsrel=1e-14)[0]
        for m in range(-l, l + 1):
            lm = l * l + l + m
            assert abs(got[lm] - cl.c_lm[0, lm - 1] * radial / R ** l) < 1e-12


@pytest.mark.parametrize("i,r", [(0, 0.35), (0, 2.4), (5, 1.1), (12, 2.4), (7, 1e-5)])
def test_monopole_is_spherical_average(orc, i, r):
    cl = synth.pd13_uniform65()
    dirs, wts = _angular_rule()
    ref = _sphere_mean(orc, cl, cl.pos[i], r, dirs, wts)
    rho0, _ = orc.monopole(cl, i, r)
    assert abs(rho0 - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("i,r", [(0, 0.8), (3, 2.4)])
def test_monopole_slope(orc, i, r):
    cl = synth.pd13_uniform65()
    h = 1e-3
    f = lambda s: orc.monopole(cl, i, s)[0]
    fd = (8 * (f(r + h) - f(r - h)) - (f(r + 2 * h) - f(r - 2 * h))) / (12 * h)
    assert abs(orc.monopole(cl, i, r)[1] - fd) < 1e-8 * abs(fd)


def test_sphere_charge_and_pseudo_density_constraints(orc):
    cl = synth.pd13_uniform65()
    q, rhoR, drhoR, coef = orc.sphere_params(cl)
    for i in range(cl.n_atoms):
        R = cl.R[i]
        own = sum(w * (1 - np.exp(-z * R) * (1 + z * R + (z * R) ** 2 / 2))
                  for w, z in zip(cl.slater_w[i], cl.slater_zeta[i]))
        # electrons inside sphere i: own Slater terms in closed form + neighbours by adaptive quadrature
        total = integrate.quad(lambda r: 4 * np.pi * r * r * orc.monopole(cl, i, r)[0], 0, R,
                               epsabs=1e-13, epsrel=1e-14, limit=200)[0]
        assert 0.0 < total - own < 3.0  # neighbour tails add a little charge inside
        assert abs(q[i] - (total - cl.Z[i])) < 1e-11
        # rho_tilde = a + b r^2 + c r^4 meets the three constraints
        poly = np.polynomial.Polynomial([coef[i, 0], 0, coef[i, 1], 0, coef[i, 2]])
        charge = 4 * np.pi * (poly * np.polynomial.Polynomial([0, 0, 1])).integ()(R)
        assert abs(charge - q[i]) < 1e-11 * abs(q[i])
        assert abs(poly(R) - rhoR[i]) < 1e-13 * abs(rhoR[i]) + 1e-15
        assert abs(poly.deriv()(R) - drhoR[i]) < 1e-12 * abs(drhoR[i]) + 1e-15
        rho_ref, drho_ref = orc.monopole(cl, i, R)
        assert rhoR[i] == rho_ref and drhoR[i] == drho_ref
        # Fig. 3: the pseudo-density is finite and negative at the centre (net positive charge inside)
        assert q[i] < 0 and coef[i, 0] < 0


def test_deposit_swaps_only_the_monopole(orc):
    cl = synth.pd13_small(n=17)
    x, y, z = orc.mesh(cl)
    b, owner = orc.deposit(cl, x, y, z)
    q, rhoR, drhoR, coef = orc.sphere_params(cl)
    rng = np.random.default_rng(3)
    for flat in rng.choice(b.size, 200, replace=False):
        k, j, i = np.unravel_index(flat, b.shape)
        p = np.array([x[i], y[j], z[k]])
        d = np.linalg.norm(cl.pos - p, axis=1)
        inside = np.nonzero(d < cl.R)[0]
        ne = orc.density(cl, *p)
        if len(inside) == 0:
            assert owner[k, j, i] == -1 and b[k, j, i] == pytest.approx(4 * np.pi * ne, rel=1e-15)
        else:
            a = inside[0]
            r = d[a]
            assert owner[k, j, i] == a
            pseudo = coef[a, 0] + coef[a, 1] * r * r + coef[a, 2] * r ** 4
            assert abs(b[k, j, i] - 4 * np.pi * (ne - orc.monopole(cl, a, r)[0] + pseudo)) < 1e-12 * (1 + abs(4 * np.pi * ne))


def test_deposit_is_neutral_for_a_neutral_cluster(orc):
    """int rho_tilde_grid = sum_i q_i + electrons outside spheres = 0 for neutral atoms; the node sum -> 0 at O(h^2)."""
    errs = []
    for n in (33, 65):
        cl = synth.pd2_dimer(n=n, half_width=14.0)
        x, y, z = orc.mesh(cl)
        b, _ = orc.deposit(cl, x, y, z)
        v = orc.dual_lengths(x)
        errs.append(abs(np.einsum("kji,i,j,k->", b / (4 * np.pi), v, v, v)))
    assert errs[1] < errs[0] / 3.0
