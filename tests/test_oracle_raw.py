"""Pins of the raw-density path (Eq. 3.1's representation: a grid density plus each sphere's
spherical component rho_00 on the logarithmic radial mesh, Eq. 3.7 at every radius).

Fed with the synthetic model's own density, the raw path must reproduce the model path's
pseudo-density constraints and deposit (both pinned elsewhere against closed forms) up to
its radial quadrature and interpolation; its radial interpolation is exact for cubics in
ln r."""
import numpy as np

import synth

SQ4PI = np.sqrt(4 * np.pi)


def _model_tables(orc, cl):
    x, y, z = orc.mesh(cl)
    ne = orc.density_grid(cl, x, y, z)
    rho00 = orc.sphere_density(cl)[:, 0, :]
    return x, y, z, ne, rho00


def test_sphere_constraints_from_the_table(orc):
    cl = synth.pd13_small(n=17)
    _, _, _, _, rho00 = _model_tables(orc, cl)
    q, rr, dr, coef = orc.raw_sphere_params(cl.Z, cl.R, rho00)
    mq, mr, md, mc = orc.sphere_params(cl)
    # q = sqrt(4pi) int rho_00 r^2 dr - Z is a small difference (about 43.8 electrons against
    # Z = 46): the 4th-order rule's ~2e-7 on the electron count becomes ~4e-6 on q
    assert np.abs(q - mq).max() < 2e-5 * np.abs(mq).max()
    # the surface projection of the neighbours' tails at R (16 x 32 rule): ~1e-11
    assert np.abs(rr - mr).max() < 1e-10 * np.abs(mr).max()
    # one-sided 4th-order difference in ln r at R (the zeta = 3 shell's derivatives dominate)
    assert np.abs(dr - md).max() < 1e-4 * np.abs(md).max()
    # the quartic meets the three constraints (Section 3) exactly
    R = cl.R
    assert np.allclose(4 * np.pi * (coef[:, 0] * R ** 3 / 3 + coef[:, 1] * R ** 5 / 5 + coef[:, 2] * R ** 7 / 7), q,
                       rtol=1e-12, atol=1e-12 * np.abs(q).max())
    assert np.allclose(coef[:, 0] + coef[:, 1] * R ** 2 + coef[:, 2] * R ** 4, rr, rtol=1e-12)
    assert np.allclose(2 * coef[:, 1] * R + 4 * coef[:, 2] * R ** 3, dr, rtol=1e-11)


def test_raw_deposit_reproduces_the_model_deposit(orc):
    cl = synth.pd13_small(n=33)
    x, y, z, ne, rho00 = _model_tables(orc, cl)
    b, owner = orc.raw_deposit(cl.pos, cl.Z, cl.R, x, y, z, ne, rho00)
    ref, rowner = orc.deposit(cl, x, y, z)
    assert np.array_equal(owner, rowner)
    # inside the spheres the quartic inherits q's and rho'(R)'s quadrature errors (~1e-5)
    assert np.abs(b - ref).max() < 1e-5 * np.abs(ref).max()
    assert np.array_equal(b[owner < 0], ref[owner < 0])          # outside the spheres: the grid density


def test_radial_interpolation_is_exact_for_cubics_in_log_r(orc):
    """rho_00 = sqrt(4pi) p(ln r) with p cubic and ne = 0: inside the sphere the deposit is
    4pi (pseudo(r) - p(ln r)), the pseudo-density from the same table."""
    cl = synth.pd2_dimer(n=33)
    x, y, z = orc.mesh(cl)
    r = orc.radial_mesh(429, 1e-5, cl.R[0])
    p = lambda t: 0.3 + 0.05 * t - 0.02 * t ** 2 + 0.001 * t ** 3
    rho00 = np.stack([SQ4PI * p(np.log(r)), SQ4PI * p(np.log(r))])
    ne = np.zeros((33, 33, 33))
    b, owner = orc.raw_deposit(cl.pos, cl.Z, cl.R, x, y, z, ne, rho00)
    _, _, _, coef = orc.raw_sphere_params(cl.Z, cl.R, rho00)
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    for a in range(2):
        m = owner == a
        rr = np.sqrt((Xg - cl.pos[a, 0]) ** 2 + (Yg - cl.pos[a, 1]) ** 2 + (Zg - cl.pos[a, 2]) ** 2)[m]
        c = coef[a]
        ref = 4 * np.pi * (c[0] + c[1] * rr ** 2 + c[2] * rr ** 4 - p(np.log(np.maximum(rr, 1e-5))))
        assert np.abs(b[m] - ref).max() < 1e-12 * np.abs(ref).max()
