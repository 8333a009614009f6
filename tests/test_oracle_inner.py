"""Pins of the oracle's inside-the-sphere functions (Section 3, Eq. 3.4-3.7): the radial mesh,
the surface projection of the density at each radius (Eq. 3.7) and the inner Dirichlet
solve (Eq. 3.4 in the Green's-function form of Eq. 3.5).

Each check is tied to something other than the oracle's own formula: exact solutions of
the radial equation (homogeneous, point charge, uniform sphere), the equation itself through
finite differences, the closed-form potential of an isolated Slater atom, and closed-form
projections of the synthetic density."""
import numpy as np
import pytest

import synth

SQ4PI = np.sqrt(4 * np.pi)
L_OF = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)


def test_radial_mesh(orc):
    r = orc.radial_mesh(429, 1e-5, 2.4)
    assert r[0] == pytest.approx(1e-5, rel=1e-12) and r[-1] == 2.4
    ratio = r[1:] / r[:-1]
    assert np.allclose(ratio, ratio[0], rtol=1e-12)   # logarithmic: constant ratio


def test_homogeneous_and_point_charge(orc):
    """rho = 0: V_LM(r) = V_LM(R) (r/R)^L; a bare nucleus adds sqrt(4pi) Z (1/r - 1/R) to
    V_00 (the potential Z/r of +Z, zero shift at R)."""
    rng = np.random.default_rng(0)
    R = np.array([2.4, 2.0])
    Z = np.array([0.0, 46.0])
    vR = rng.normal(size=(2, 25))
    rho = np.zeros((2, 25, 429))
    v = orc.inner_solve(R, Z, rho, vR)
    for a in range(2):
        r = orc.radial_mesh(429, 1e-5, R[a])
        for lm in range(25):
            ref = vR[a, lm] * (r / R[a]) ** L_OF[lm]
            if lm == 0:
                ref = ref + SQ4PI * Z[a] * (1 / r - 1 / R[a])
            assert np.allclose(v[a, lm], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("rho0", [0.37, -2.0])
def test_uniform_sphere_and_order(orc, rho0):
    """A uniform density rho0: V_00 = V_00(R) + sqrt(4pi) (2pi/3) rho0 (r^2 - R^2) (the interior
    solution of Lap V = 4pi rho0); the quadrature error falls 16-fold per halving of dx.  The
    cubic rule in x = ln r integrates r^4 with error ~ (19/720) h^4 4^4 per unit of the
    integral: about 5e-6 at 429 points (h = 0.029)."""
    R = np.array([2.4])
    vR = np.zeros((1, 25))
    vR[0, 0] = 1.3
    errs = []
    for n in (108, 215, 429):
        rho = np.zeros((1, 25, n))
        rho[0, 0] = SQ4PI * rho0
        v = orc.inner_solve(R, np.zeros(1), rho, vR)
        r = orc.radial_mesh(n, 1e-5, 2.4)
        ref = 1.3 + SQ4PI * 2 * np.pi / 3 * rho0 * (r ** 2 - 2.4 ** 2)
        errs.append(np.abs(v[0, 0] - ref).max() / np.abs(ref).max())
    assert errs[-1] < 5e-6
    assert 10 < errs[0] / errs[1] < 24 and 10 < errs[1] / errs[2] < 24


@pytest.mark.parametrize("lm", [0, 2, 6, 12, 20])
def test_radial_equation_residual(orc, lm):
    """V from the inner solve satisfies (d2/dr2 + 2/r d/dr - L(L+1)/r^2) V = 4 pi rho (Eq. 3.4)
    at the mesh points (central differences in x = ln r) and V(R) = V_R."""
    L = L_OF[lm]
    n = 2049
    R = np.array([2.4])
    r = orc.radial_mesh(n, 1e-4, 2.4)
    rho = np.zeros((1, 25, n))
    rho[0, lm] = r ** L * np.exp(-1.3 * r) * (1 + 0.5 * r)
    vR = np.zeros((1, 25))
    vR[0, lm] = -0.7
    v = orc.inner_solve(R, np.zeros(1), rho, vR, r_min=1e-4)[0, lm]
    assert v[-1] == pytest.approx(-0.7, abs=1e-14)
    h = np.log(r[1] / r[0])
    vx = (v[2:] - v[:-2]) / (2 * h)
    vxx = (v[2:] - 2 * v[1:-1] + v[:-2]) / h ** 2
    rr = r[1:-1]
    lhs = (vxx - vx) / rr ** 2 + 2 * vx / rr ** 2 - L * (L + 1) * v[1:-1] / rr ** 2
    rhs = 4 * np.pi * rho[0, lm, 1:-1]
    sel = rr > 0.05
    assert np.abs(lhs - rhs)[sel].max() < 2e-4 * np.abs(rhs[sel]).max()


def _isolated_atom(clm_sigma=0.0, seed=1):
    rng = np.random.default_rng(seed)
    return synth.workloads.make_cluster("Pd1", np.zeros((1, 3)), rng, n=33, half_width=8.0, h_min=0.5, h_max=0.5,
                                        clm_sigma=clm_sigma)


def test_isolated_atom_potential(orc):
    """One Pd atom (Z = 46, three normalised Slater shells): the projection of its density is
    sqrt(4pi) n_e(r) and, with V_00(R) from the closed-form potential
    Phi(r) = Z/r - sum_k w_k [1/r - e^{-zeta_k r}(1/r + zeta_k/2)], the inner solve returns
    sqrt(4pi) Phi(r) inside the sphere."""
    cl = _isolated_atom()
    rho = orc.sphere_density(cl)
    r = orc.radial_mesh(429, 1e-5, cl.R[0])
    w, z = cl.slater_w[0], cl.slater_zeta[0]
    ne = sum(w[k] * z[k] ** 3 / (8 * np.pi) * np.exp(-z[k] * r) for k in range(3))
    assert np.allclose(rho[0, 0], SQ4PI * ne, rtol=1e-12)
    assert np.abs(rho[0, 1:]).max() < 1e-12 * np.abs(rho[0, 0]).max()
    phi = lambda x: 46.0 / x - sum(w[k] * (1 / x - np.exp(-z[k] * x) * (1 / x + z[k] / 2)) for k in range(3))
    vR = np.zeros((1, 25))
    vR[0, 0] = SQ4PI * phi(cl.R[0])
    v = orc.inner_solve(cl.R, cl.Z, rho, vR)
    ref = SQ4PI * phi(r)
    sel = r > 1e-3
    assert np.abs(v[0, 0] - ref)[sel].max() < 1e-8 * np.abs(ref[sel]).max()


def test_nonspherical_projection(orc):
    """Inside its own sphere an atom's l >= 1 density is c_lm f(r) (r/R)^l y_lm with
    f = zeta_1^3/(8 pi) e^{-zeta_1 r} (1 - r^2/R^2)^2: the projection returns each c_lm
    times f(r) (r/R)^l (the rule integrates these polynomials on the sphere exactly)."""
    cl = _isolated_atom(clm_sigma=1e-2, seed=2)
    rho = orc.sphere_density(cl)
    r = orc.radial_mesh(429, 1e-5, cl.R[0])
    R = cl.R[0]
    f = cl.slater_zeta[0, 0] ** 3 / (8 * np.pi) * np.exp(-cl.slater_zeta[0, 0] * r) * (1 - r ** 2 / R ** 2) ** 2
    for lm in range(1, 25):
        ref = cl.c_lm[0, lm - 1] * f * (r / R) ** L_OF[lm]
        # rounding of 512-point sums of a density whose spherical part is ~1e3 times larger
        assert np.abs(rho[0, lm] - ref).max() < 1e-13 * np.abs(rho[0, 0]).max()


def test_monopole_projection_with_a_neighbour(orc):
    """Two atoms: the L = 0 projection about atom 0 equals sqrt(4pi) times the closed-form
    spherical average (own shells + the neighbour's shells averaged over the sphere)."""
    cl = synth.pd2_dimer()
    rho = orc.sphere_density(cl)
    r = orc.radial_mesh(429, 1e-5, cl.R[0])
    ref = np.array([orc.monopole(cl, 0, x)[0] for x in r[::16]])
    assert np.abs(rho[0, 0, ::16] - SQ4PI * ref).max() < 1e-9 * np.abs(ref).max()
