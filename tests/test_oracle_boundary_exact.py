"""Pins of the exact-superposition Dirichlet values (the alternative to Eq. 3.3's zero faces
and to the truncated multipole expansion) and of what each choice costs in accuracy.

The face values are the model density's continuum potential.  The spherical part is checked
against the Coulomb integral of the density done numerically (not the closed form the oracle
uses), the nonspherical part against multipoles whose moments come from a 3-D quadrature of
the density."""
import numpy as np
import pytest
from scipy import integrate

import synth

LS = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)


def _atom(clm_sigma, seed):
    rng = np.random.default_rng(seed)
    return synth.workloads.make_cluster("Pd1", np.array([[0.3, -0.2, 0.1]]), rng, n=17, half_width=9.0, h_min=1.1,
                                        h_max=1.2, clm_sigma=clm_sigma)


def _faces(u):
    m = np.zeros(u.shape, bool)
    m[0] = m[-1] = True
    m[:, 0] = m[:, -1] = True
    m[:, :, 0] = m[:, :, -1] = True
    return m


def test_spherical_atom_faces_are_its_coulomb_potential(orc):
    cl = _atom(0.0, 1)
    x, y, z = orc.mesh(cl)
    u = orc.boundary_exact(cl, x, y, z)
    w, zt = cl.slater_w[0], cl.slater_zeta[0]
    rho = lambda r: sum(w[k] * zt[k] ** 3 / (8 * np.pi) * np.exp(-zt[k] * r) for k in range(3))

    def pot(r):
        inner = integrate.quad(lambda s: 4 * np.pi * s * s * rho(s), 0, r, epsabs=0, epsrel=1e-13, limit=200)[0]
        outer = integrate.quad(lambda s: 4 * np.pi * s * rho(s), r, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
        return 46.0 / r - inner / r - outer

    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    m = _faces(u)
    pts = np.stack([Xg[m], Yg[m], Zg[m]], axis=1)[::37]
    ref = np.array([pot(np.linalg.norm(p - cl.pos[0])) for p in pts])
    # the neutral atom's potential at the faces is the small remainder of Z/r and the shells'
    # potentials (~1e-5 of Z/r): compare on the scale of the cancelling terms, then relatively
    assert np.abs(u[m][::37] - ref).max() < 1e-14 * 46.0 / 9.0
    assert np.abs(u[m][::37] - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.all(u[~m] == 0.0)


def test_nonspherical_faces_are_its_multipoles(orc):
    """c_lm != 0 minus c_lm = 0 (same shells): -4pi/(2l+1) q_lm S_lm(d)/|d|^(2l+1), with
    q_lm = int rho_ns S_lm dV from a Gauss-Legendre (radius) x product (sphere) quadrature of
    the oracle's point density."""
    cl1, cl0 = _atom(5e-2, 2), _atom(0.0, 2)
    cl0.slater_w[:] = cl1.slater_w
    x, y, z = orc.mesh(cl1)
    du = orc.boundary_exact(cl1, x, y, z) - orc.boundary_exact(cl0, x, y, z)
    R, c = cl1.R[0], cl1.pos[0]
    tr, wr = np.polynomial.legendre.leggauss(48)
    tc, wc = np.polynomial.legendre.leggauss(12)
    q = np.zeros(25)
    for r_, w_ in zip(0.5 * R * (tr + 1), 0.5 * R * wr):
        for ct, wct in zip(tc, wc):
            st = np.sqrt(1 - ct * ct)
            for k in range(24):
                ph = 2 * np.pi * k / 24
                u = np.array([st * np.cos(ph), st * np.sin(ph), ct])
                p = c + r_ * u
                rns = orc.density(cl1, *p) - orc.density(cl0, *p)
                q += w_ * r_ * r_ * wct * 2 * np.pi / 24 * rns * orc.solid_harmonics(*(r_ * u))
    m = _faces(du)
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([Xg[m], Yg[m], Zg[m]], axis=1)[::29]
    ref = []
    for p in pts:
        d = p - c
        S = orc.solid_harmonics(*d)
        dn = np.linalg.norm(d)
        ref.append(sum(-4 * np.pi / (2 * LS[lm] + 1) * q[lm] * S[lm] / dn ** (2 * LS[lm] + 1) for lm in range(1, 25)))
    ref = np.array(ref)
    assert np.abs(du[m][::29] - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.slow
def test_boundary_choice_and_box_size(orc):
    """Pd2 (4.802 au, a neutral cluster) at h = 0.375 on boxes of half-width 9 and 12 bohr: the
    error each choice of faces adds, measured against the exact-faces solve on the same grid
    (the shared discretisation error cancels).  Zero faces (Eq. 3.3) cost only the atoms'
    exponential tails at the faces, which fall steeply with the box (e^{-zeta_1 d}).  The l <= 4
    multipole faces take the moments of the grid charge, whose O(h^2) quadrature error acts as
    a spurious net charge; their error does not fall with the box and, for a neutral cluster,
    exceeds the zero faces' on the larger box."""
    out = {}
    for hw in (9.0, 12.0):
        n = int(round(2 * hw / 0.375)) + 1
        n += 1 - n % 2
        cl = synth.pd2_dimer(n=n, half_width=hw)
        for bc in ("zero", "multipole", "exact"):
            o = orc.poisson_solve(cl, tol=1e-12, max_cycles=60, bc=bc)
            assert o["status"] == 0
            out[bc, hw] = o["vlm"][0]
    d = {k: np.abs(out[k] - out["exact", k[1]]).max() / np.abs(out["exact", k[1]]).max() for k in out}
    assert d["zero", 9.0] > 30 * d["zero", 12.0]                 # tails e^{-1.5 d}, d 3 bohr longer
    assert 0.3 < d["multipole", 9.0] / d["multipole", 12.0] < 3   # set by h, not by the box
    assert d["multipole", 12.0] > d["zero", 12.0]
