"""Pins of the oracle's finite-difference operator and multigrid pieces (Section 3:
"a finite difference scheme and a multigrid method").

Operator: on a uniform mesh it must be the textbook 7-point Laplacian; on any
graded mesh the 3-point nonuniform difference is exact for quadratics, and
vol * A is symmetric negative definite.  Smoother: Gauss-Seidel zeroes the
residual of the colour just relaxed.  Transfers: uniform full weighting is the
textbook (1,2,1)/4 stencil; prolongation is exact for trilinear functions; the
restriction is the volume-weighted adjoint of the prolongation.  Solver: equals
a sparse direct solve, converges at O(h^2) on a manufactured solution and on the
Gaussian charge whose potential is Q erf(a r)/r.
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla
from scipy.special import erf


def _graded(orc, n, L=6.0, ratio=4.0):
    m = (n - 1) / 2
    hmin = L / m / 1.8
    return orc.mesh_axis(n, 0.0, L, hmin, hmin * ratio)[0]


def _vol(x, y, z):
    d = lambda c: np.concatenate([[c[1] - c[0]], c[2:] - c[:-2], [c[-1] - c[-2]]]) / 2
    return np.einsum("k,j,i->kji", d(z), d(y), d(x))


def _interior(a):
    return a[1:-1, 1:-1, 1:-1]


def _dense_A(orc, x, y, z):
    """Columns of the interior operator with zero boundary values."""
    nx, ny, nz = len(x), len(y), len(z)
    m = (nx - 2) * (ny - 2) * (nz - 2)
    M = np.zeros((m, m))
    e = np.zeros((nz, ny, nx))
    for c in range(m):
        k, j, i = np.unravel_index(c, (nz - 2, ny - 2, nx - 2))
        e[k + 1, j + 1, i + 1] = 1.0
        M[:, c] = _interior(orc.apply_A(x, y, z, e)).ravel()
        e[k + 1, j + 1, i + 1] = 0.0
    return M


def test_uniform_operator_is_textbook_laplacian(orc):
    n, h = 9, 0.5
    x = -2.0 + h * np.arange(n)
    T = (np.diag(np.full(n, -2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h ** 2
    I = np.eye(n)
    Lap = np.kron(np.kron(T, I), I) + np.kron(np.kron(I, T), I) + np.kron(np.kron(I, I), T)
    u = np.random.default_rng(0).normal(size=(n, n, n))
    ref = (Lap @ u.ravel()).reshape(n, n, n)
    got = orc.apply_A(x, x, x, u)
    assert np.abs(_interior(got - ref)).max() < 1e-12 * np.abs(ref).max()


def test_graded_operator_exact_for_quadratics(orc):
    x, y, z = _graded(orc, 17), _graded(orc, 17, L=5.0, ratio=3.0), _graded(orc, 17, L=7.0)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = 1.5 * X ** 2 - 0.7 * Y ** 2 + 0.25 * Z ** 2 + 0.3 * X * Y - 2.0 * Y * Z + X - 4.0
    Au = orc.apply_A(x, y, z, u)
    assert np.abs(_interior(Au) - 2 * (1.5 - 0.7 + 0.25)).max() < 1e-11


def test_volume_weighted_operator_is_symmetric_negative_definite(orc):
    x = _graded(orc, 7)
    M = _dense_A(orc, x, x, x)
    VM = _interior(_vol(x, x, x)).ravel()[:, None] * M
    assert np.abs(VM - VM.T).max() < 1e-12 * np.abs(VM).max()
    assert np.linalg.eigvalsh(0.5 * (VM + VM.T)).max() < 0


def test_gauss_seidel_zeroes_the_relaxed_colour(orc):
    x = _graded(orc, 17)
    rng = np.random.default_rng(1)
    u, b = rng.normal(size=(17,) * 3), rng.normal(size=(17,) * 3)
    k, j, i = np.meshgrid(*(np.arange(17),) * 3, indexing="ij")
    colour = (i + j + k) % 2
    inner = np.zeros_like(u, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    for c in (0, 1):
        orc.rbgs_half(x, x, x, u, b, c)
        r = orc.residual(x, x, x, u, b)
        assert np.abs(r[inner & (colour == c)]).max() < 1e-12 * np.abs(b).max() * 50
        assert np.abs(r[inner & (colour != c)]).max() > 1e-3


def test_coarse_solve_matches_dense_solve(orc):
    x = _graded(orc, 9)
    b = np.random.default_rng(2).normal(size=(9,) * 3)
    e = orc.coarse_solve(x, x, x, b)
    ref = np.linalg.solve(_dense_A(orc, x, x, x), _interior(b).ravel())
    assert np.abs(_interior(e).ravel() - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.all(e[0] == 0) and np.all(e[:, :, -1] == 0)


def test_uniform_full_weighting_is_textbook(orc):
    n = 17
    x = np.linspace(-4, 4, n)
    r = np.random.default_rng(3).normal(size=(n,) * 3)
    r[0] = r[-1] = 0; r[:, 0] = r[:, -1] = 0; r[:, :, 0] = r[:, :, -1] = 0
    bc = orc.restrict(x, x, x, r)
    w1 = np.array([0.25, 0.5, 0.25])
    W = np.einsum("a,b,c->abc", w1, w1, w1)
    for K in range(1, 8):
        for J in range(1, 8):
            for I in range(1, 8):
                ref = (W * r[2 * K - 1:2 * K + 2, 2 * J - 1:2 * J + 2, 2 * I - 1:2 * I + 2]).sum()
                assert abs(bc[K, J, I] - ref) < 1e-14


def test_prolongation_exact_for_trilinear(orc):
    x, y, z = _graded(orc, 17), _graded(orc, 17, L=4.0), _graded(orc, 17, ratio=2.0)
    rng = np.random.default_rng(4)
    a = rng.normal(size=6)
    f = lambda X, Y, Z: (a[0] + a[1] * X) * (a[2] + a[3] * Y) * (a[4] + a[5] * Z)
    ec = f(*np.meshgrid(x[::2], y[::2], z[::2], indexing="ij")).transpose(2, 1, 0).copy()
    u = np.zeros((17, 17, 17))
    orc.prolong_add(x, y, z, ec, u)
    ref = f(*np.meshgrid(x, y, z, indexing="ij")).transpose(2, 1, 0)
    assert np.abs(_interior(u - ref)).max() < 1e-13 * np.abs(ref).max()
    assert np.all(u[0] == 0)


def test_restriction_is_volume_adjoint_of_prolongation(orc):
    x, y, z = _graded(orc, 33), _graded(orc, 33, L=5.0), _graded(orc, 33, ratio=2.5)
    rng = np.random.default_rng(5)
    r = np.zeros((33,) * 3)
    r[1:-1, 1:-1, 1:-1] = rng.normal(size=(31,) * 3)
    ec = np.zeros((17,) * 3)
    ec[1:-1, 1:-1, 1:-1] = rng.normal(size=(15,) * 3)
    Pe = orc.prolong_add(x, y, z, ec, np.zeros((33,) * 3))
    lhs = (_vol(x[::2], y[::2], z[::2]) * orc.restrict(x, y, z, r) * ec).sum()
    rhs = (_vol(x, y, z) * r * Pe).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def _sparse_A(x, y, z):
    """The nonuniform 3-point difference per axis, assembled in the test with scipy."""
    def T(c):
        n = len(c) - 2
        hm, hp = c[1:-1] - c[:-2], c[2:] - c[1:-1]
        s = 2.0 / (hm + hp)
        return sps.diags([(s / hm)[1:], -s * (1 / hm + 1 / hp), (s / hp)[:-1]], [-1, 0, 1], shape=(n, n))
    Ix, Iy, Iz = (sps.identity(len(c) - 2) for c in (x, y, z))
    return (sps.kron(sps.kron(Iz, Iy), T(x)) + sps.kron(sps.kron(Iz, T(y)), Ix) + sps.kron(sps.kron(T(z), Iy), Ix)).tocsc()


def _boundary_term(x, y, z, u):
    """b_eff = b - (contribution of the Dirichlet faces) on the interior, via the same difference."""
    w = u.copy()
    w[1:-1, 1:-1, 1:-1] = 0
    out = np.zeros_like(u[1:-1, 1:-1, 1:-1])
    for ax, c in ((2, x), (1, y), (0, z)):
        hm, hp = c[1:-1] - c[:-2], c[2:] - c[1:-1]
        s = 2.0 / (hm + hp)
        sl = [slice(1, -1)] * 3
        lo, hi = list(sl), list(sl)
        lo[ax], hi[ax] = slice(0, -2), slice(2, None)
        shape = [1, 1, 1]
        shape[ax] = -1
        out += (s / hm).reshape(shape) * w[tuple(lo)] + (s / hp).reshape(shape) * w[tuple(hi)]
    return out


@pytest.mark.parametrize("n", [9, 17, 33])
def test_multigrid_equals_direct_solve(orc, n):
    x, y, z = _graded(orc, n), _graded(orc, n, L=5.0), _graded(orc, n, ratio=2.0)
    rng = np.random.default_rng(6)
    b = rng.normal(size=(n,) * 3)
    u = np.zeros((n,) * 3)
    u[0] = u[-1] = u[:, 0] = u[:, -1] = u[:, :, 0] = u[:, :, -1] = 0.0
    faces = rng.normal(size=(n,) * 3)
    for sl in ((0,), (-1,), (slice(None), 0), (slice(None), -1), (Ellipsis, 0), (Ellipsis, -1)):
        u[sl] = faces[sl]
    rhs = _interior(b).ravel() - _boundary_term(x, y, z, u).ravel()
    ref = spla.spsolve(_sparse_A(x, y, z), rhs)
    st, cyc, hist = orc.mg_solve(x, y, z, b, u, tol=1e-14, max_cycles=200)
    assert st == 0 and hist[-1] <= 1e-14
    assert np.abs(_interior(u).ravel() - ref).max() < 1e-11 * np.abs(ref).max()


def _manufactured(X, Y, Z, L):
    k = np.pi / (2 * L)
    u = np.sin(k * X + 0.3) * np.cos(0.7 * k * Y) * np.exp(0.1 * Z)
    lap = u * (-(k ** 2) - (0.7 * k) ** 2 + 0.01)
    return u, lap


@pytest.mark.parametrize("graded", [False, True])
def test_second_order_on_manufactured_solution(orc, graded):
    errs = []
    L = 6.0
    for n in (17, 33, 65):
        m = (n - 1) / 2
        x = orc.mesh_axis(n, 0.0, L, L / m / (1.6 if graded else 1.0), L / m * (1.8 if graded else 1.0))[0]
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        ue, lap = _manufactured(X, Y, Z, L)
        u = ue.copy()
        u[1:-1, 1:-1, 1:-1] = 0.0
        st, cyc, hist = orc.mg_solve(x, x, x, lap, u, tol=1e-13, max_cycles=100)
        assert st == 0
        errs.append(np.abs(u - ue).max())
    rates = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((rates > 3.4) & (rates < 4.6)), rates


def test_gaussian_charge_potential_is_erf_over_r(orc):
    """b = 4 pi Q (a^2/pi)^{3/2} e^{-a^2 r^2} gives u = -Q erf(a r)/r (electron-sign charge, Eq. 2.6 sign)."""
    Q, a, L = 3.0, 1.2, 8.0
    errs = []
    for n in (33, 65):
        x = np.linspace(-L, L, n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r = np.sqrt(X * X + Y * Y + Z * Z)
        rho = Q * (a * a / np.pi) ** 1.5 * np.exp(-a * a * r * r)
        exact = -Q * np.where(r > 0, erf(a * r) / np.where(r > 0, r, 1), 2 * a / np.sqrt(np.pi))
        b = 4 * np.pi * rho
        u = exact.copy()
        u[1:-1, 1:-1, 1:-1] = 0.0
        st, _, _ = orc.mg_solve(x, x, x, b, u, tol=1e-13, max_cycles=60)
        assert st == 0
        errs.append(np.abs(u - exact).max())
    assert 3.4 < errs[0] / errs[1] < 4.6
    # multipole moments of the same grid charge: only the monopole, Q_00 = -Q... in electron sign +Q y00
    x = np.linspace(-L, L, 65)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    rho = Q * (a * a / np.pi) ** 1.5 * np.exp(-a * a * (X * X + Y * Y + Z * Z))
    Qlm = orc.multipoles(x, x, x, 4 * np.pi * rho)
    assert abs(Qlm[0] - Q / np.sqrt(4 * np.pi)) < 1e-10
    assert np.abs(Qlm[1:]).max() < 1e-12


@pytest.mark.parametrize("n", [17, 33, 65, 97, 129, 161, 193, 385])
def test_level_count(orc, n):
    """Coarsen every other node until every axis has at most 9 nodes."""
    L = orc.num_levels(n, n, n)
    c = n
    for _ in range(L - 1):
        assert (c - 1) % 2 == 0
        c = (c + 1) // 2
    assert c <= 9 and (L == 1 or (2 * c - 1) > 9)
