"""ctypes wrapper of the FP64 CPU oracle (``lasto_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg.  The CUDA library and its Python binding never
import this package.  Every function here is a marshalling shim over the C
oracle; the arithmetic lives in ``lasto_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liblasto_oracle.so")
_lib = None

OK, INVALID_ARG, GEOMETRY, NONFINITE, NOT_CONVERGED = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP over independent node loops)."""
    src = os.path.join(_HERE, "lasto_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "lasto_oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _declare(L):
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "or_solid_harmonics": (None, [d, d, d, _D]),
        "or_gauss_legendre": (i, [i, _D, _D]),
        "or_mesh_axis": (i, [i, d, d, d, d, d, _D, _D]),
        "or_dual_lengths": (None, [i, _D, _D]),
        "or_density": (d, [i, _D, _D, _D, _D, _D, d, d, d]),
        "or_density_grid": (None, [i, _D, _D, _D, _D, _D, i, i, i, _D, _D, _D, _D]),
        "or_monopole": (None, [i, _D, _D, _D, i, d, _D, _D]),
        "or_sphere_params": (None, [i, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
        "or_deposit": (i, [i, _D, _D, _D, _D, _D, _D, i, i, i, _D, _D, _D, _D, _I]),
        "or_multipoles": (None, [i, i, i, _D, _D, _D, _D, d, d, d, _D]),
        "or_boundary_fill": (None, [i, i, i, _D, _D, _D, d, d, d, _D, _D]),
        "or_apply_A": (None, [i, i, i, _D, _D, _D, _D, _D]),
        "or_residual": (None, [i, i, i, _D, _D, _D, _D, _D, _D]),
        "or_norm2_interior": (d, [i, i, i, _D]),
        "or_rbgs_half": (None, [i, i, i, _D, _D, _D, _D, _D, i]),
        "or_restrict": (None, [i, i, i, _D, _D, _D, _D, _D]),
        "or_prolong_add": (None, [i, i, i, _D, _D, _D, _D, _D]),
        "or_coarse_solve": (i, [i, i, i, _D, _D, _D, _D, _D]),
        "or_num_levels": (i, [i, i, i]),
        "or_mg_solve": (i, [i, i, i, _D, _D, _D, _D, _D, i, i, i, d, i, _D, _I]),
        "or_project": (i, [i, i, i, _D, _D, _D, _D, i, _D, _D, i, i, _D]),
        "or_poisson_solve": (i, [i, _D, _D, _D, _D, _D, _D, _D, _I, d, _D, _D, _D, _D]),
        "or_radial_mesh": (None, [i, d, d, _D]),
        "or_sphere_density": (i, [i, _D, _D, _D, _D, _D, i, d, i, i, _D]),
        "or_inner_solve": (i, [i, _D, _D, i, d, _D, _D, _D]),
        "or_boundary_exact": (None, [i, _D, _D, _D, _D, _D, _D, i, i, i, _D, _D, _D, _D]),
        "or_raw_sphere_params": (i, [i, _D, _D, i, d, _D, _D, _D, _D, _D]),
        "or_interstitial_hs": (i, [i, _D, _D, i, _I, _I, _D, i, i, i, _D, _D, _D, _D, _D, _D]),
        "or_raw_deposit": (i, [i, _D, _D, _D, i, i, i, _D, _D, _D, _D, i, d, _D, _D, _I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ thin wrappers
def solid_harmonics(x, y, z) -> np.ndarray:
    out = np.zeros(25)
    lib().or_solid_harmonics(float(x), float(y), float(z), _p(out))
    return out


def gauss_legendre(n):
    t, w = np.zeros(n), np.zeros(n)
    lib().or_gauss_legendre(n, _p(t), _p(w))
    return t, w


def mesh_axis(n, c, L, h_min, h_max, p_max=6.0):
    x, info = np.zeros(n), np.zeros(5)
    st = lib().or_mesh_axis(n, c, L, h_min, h_max, p_max, _p(x), _p(info))
    if st != OK:
        raise ValueError(f"mesh_axis status {st}")
    return x, info


def mesh(cl):
    """The three axes of a cluster's cubic box."""
    return tuple(mesh_axis(cl.n, cl.centre[a], cl.half_width, cl.h_min, cl.h_max, cl.p_max)[0] for a in range(3))


def dual_lengths(x):
    x = _f64(x)
    v = np.zeros_like(x)
    lib().or_dual_lengths(len(x), _p(x), _p(v))
    return v


def _atoms(cl):
    return cl.n_atoms, _p(cl.pos), _p(cl.Z), _p(cl.R), _p(cl.slater_w), _p(cl.slater_zeta), _p(cl.c_lm)


def density(cl, x, y, z) -> float:
    return lib().or_density(cl.n_atoms, _p(cl.pos), _p(cl.R), _p(cl.slater_w), _p(cl.slater_zeta), _p(cl.c_lm),
                            float(x), float(y), float(z))


def density_grid(cl, x, y, z):
    x, y, z = _f64(x), _f64(y), _f64(z)
    out = np.zeros((len(z), len(y), len(x)))
    lib().or_density_grid(cl.n_atoms, _p(cl.pos), _p(cl.R), _p(cl.slater_w), _p(cl.slater_zeta), _p(cl.c_lm),
                          len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(out))
    return out


def monopole(cl, i, r):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_monopole(cl.n_atoms, _p(cl.pos), _p(cl.slater_w), _p(cl.slater_zeta), i, float(r),
                      ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def sphere_params(cl):
    na = cl.n_atoms
    q, rhoR, drhoR, coef = np.zeros(na), np.zeros(na), np.zeros(na), np.zeros((na, 3))
    lib().or_sphere_params(na, _p(cl.pos), _p(cl.Z), _p(cl.R), _p(cl.slater_w), _p(cl.slater_zeta),
                           _p(q), _p(rhoR), _p(drhoR), _p(coef))
    return q, rhoR, drhoR, coef


def deposit(cl, x, y, z):
    x, y, z = _f64(x), _f64(y), _f64(z)
    b = np.zeros((len(z), len(y), len(x)))
    owner = np.zeros(b.shape, dtype=np.int32)
    lib().or_deposit(*_atoms(cl), len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(b),
                     owner.ctypes.data_as(_I))
    return b, owner


def multipoles(x, y, z, b, centre=(0.0, 0.0, 0.0)):
    x, y, z, b = _f64(x), _f64(y), _f64(z), _f64(b)
    Q = np.zeros(25)
    lib().or_multipoles(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(b), *map(float, centre), _p(Q))
    return Q


def boundary_fill(x, y, z, Q, u, centre=(0.0, 0.0, 0.0)):
    """Writes the six faces of u (float64 C-contiguous [nz, ny, nx]) in place."""
    x, y, z, Q = _f64(x), _f64(y), _f64(z), _f64(Q)
    assert u.dtype == np.float64 and u.flags.c_contiguous
    lib().or_boundary_fill(len(x), len(y), len(z), _p(x), _p(y), _p(z), *map(float, centre), _p(Q), _p(u))
    return u


def apply_A(x, y, z, u):
    x, y, z, u = _f64(x), _f64(y), _f64(z), _f64(u)
    out = np.zeros_like(u)
    lib().or_apply_A(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(u), _p(out))
    return out


def residual(x, y, z, u, b):
    x, y, z, u, b = _f64(x), _f64(y), _f64(z), _f64(u), _f64(b)
    out = np.zeros_like(u)
    lib().or_residual(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(u), _p(b), _p(out))
    return out


def norm2_interior(r):
    r = _f64(r)
    nz, ny, nx = r.shape
    return lib().or_norm2_interior(nx, ny, nz, _p(r))


def rbgs_half(x, y, z, u, b, colour):
    """In place on u (float64 C-contiguous)."""
    x, y, z, b = _f64(x), _f64(y), _f64(z), _f64(b)
    assert u.dtype == np.float64 and u.flags.c_contiguous
    lib().or_rbgs_half(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(u), _p(b), int(colour))
    return u


def restrict(x, y, z, r):
    x, y, z, r = _f64(x), _f64(y), _f64(z), _f64(r)
    bc = np.zeros(((len(z) + 1) // 2, (len(y) + 1) // 2, (len(x) + 1) // 2))
    lib().or_restrict(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(r), _p(bc))
    return bc


def prolong_add(x, y, z, ec, u):
    """u += P ec in place (x, y, z are the FINE coordinates)."""
    x, y, z, ec = _f64(x), _f64(y), _f64(z), _f64(ec)
    assert u.dtype == np.float64 and u.flags.c_contiguous
    lib().or_prolong_add(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(ec), _p(u))
    return u


def coarse_solve(x, y, z, b):
    x, y, z, b = _f64(x), _f64(y), _f64(z), _f64(b)
    e = np.zeros_like(b)
    st = lib().or_coarse_solve(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(b), _p(e))
    if st != OK:
        raise ValueError(f"coarse_solve status {st}")
    return e


def num_levels(nx, ny, nz):
    return lib().or_num_levels(nx, ny, nz)


def mg_solve(x, y, z, b, u, nu1=2, nu2=2, n_f=1, tol=1e-13, max_cycles=60):
    """Multigrid in place on u; returns (status, cycles, history)."""
    x, y, z, b = _f64(x), _f64(y), _f64(z), _f64(b)
    assert u.dtype == np.float64 and u.flags.c_contiguous
    hist = np.zeros(max_cycles + 1)
    cyc = ctypes.c_int()
    st = lib().or_mg_solve(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(b), _p(u), nu1, nu2, n_f, tol,
                           max_cycles, _p(hist), ctypes.byref(cyc))
    return st, cyc.value, hist[:cyc.value + 1]


def project(x, y, z, u, pos, R, n_theta=16, n_phi=32):
    x, y, z, u, pos, R = _f64(x), _f64(y), _f64(z), _f64(u), _f64(pos), _f64(R)
    vlm = np.zeros((len(R), 25))
    st = lib().or_project(len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(u), len(R), _p(pos), _p(R),
                          n_theta, n_phi, _p(vlm))
    if st != OK:
        raise ValueError(f"project status {st}")
    return vlm


def boundary_exact(cl, x, y, z, u=None):
    """u with its six faces set to the exact superposition of the atoms' potentials."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    u = np.zeros((len(z), len(y), len(x))) if u is None else u
    lib().or_boundary_exact(*_atoms(cl), len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(u))
    return u


# Table 1's LASTO basis per Pd atom: (n, l, zeta) of 4d 5d 5s 5p 6s 6p 4f
LASTO_BASIS = [(4, 2, 2.20), (5, 2, 2.60), (5, 0, 1.00), (5, 1, 1.00), (6, 0, 2.00), (6, 1, 2.00), (4, 3, 1.60)]


def interstitial_hs(pos, R, x, y, z, V, basis=LASTO_BASIS):
    """(S, H) [M][M] over the nodes outside every sphere (Eq. 3.11-3.14, grid-point form)."""
    pos, R, x, y, z, V = (_f64(a) for a in (pos, R, x, y, z, V))
    bn = np.array([b[0] for b in basis], dtype=np.int32)
    bl = np.array([b[1] for b in basis], dtype=np.int32)
    bz = np.array([b[2] for b in basis], dtype=np.float64)
    M = len(R) * int(sum(2 * l + 1 for l in bl))
    S, H = np.zeros((M, M)), np.zeros((M, M))
    st = lib().or_interstitial_hs(len(R), _p(pos), _p(R), len(basis), bn.ctypes.data_as(_I), bl.ctypes.data_as(_I),
                                  _p(bz), len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(V), _p(S), _p(H))
    if st != OK:
        raise ValueError(f"interstitial_hs status {st}")
    return S, H


def raw_sphere_params(Z, R, rho00, r_min=1e-5):
    """(q, rho(R), rho'(R), coef [na][3]) of each sphere from its rho_00 radial table."""
    Z, R, rho00 = _f64(Z), _f64(R), _f64(rho00)
    na = len(R)
    q, rr, dr, coef = np.zeros(na), np.zeros(na), np.zeros(na), np.zeros((na, 3))
    st = lib().or_raw_sphere_params(na, _p(Z), _p(R), rho00.shape[1], r_min, _p(rho00), _p(q), _p(rr), _p(dr), _p(coef))
    if st != OK:
        raise ValueError(f"raw_sphere_params status {st}")
    return q, rr, dr, coef


def raw_deposit(pos, Z, R, x, y, z, ne, rho00, r_min=1e-5):
    """b = 4 pi rho~_grid from a grid density ne [nz][ny][nx] and rho_00 tables [na][n_rad]."""
    pos, Z, R, x, y, z, ne, rho00 = (_f64(a) for a in (pos, Z, R, x, y, z, ne, rho00))
    b = np.zeros((len(z), len(y), len(x)))
    owner = np.zeros(b.shape, dtype=np.int32)
    st = lib().or_raw_deposit(len(R), _p(pos), _p(Z), _p(R), len(x), len(y), len(z), _p(x), _p(y), _p(z), _p(ne),
                              rho00.shape[1], r_min, _p(rho00), _p(b), owner.ctypes.data_as(_I))
    if st != OK:
        raise ValueError(f"raw_deposit status {st}")
    return b, owner


def radial_mesh(n, r_min, R):
    """Logarithmic radial mesh of a sphere (Section 4: 429 points; last point on the sphere)."""
    r = np.zeros(n)
    lib().or_radial_mesh(n, r_min, R, _p(r))
    return r


def sphere_density(cl, n_rad=429, r_min=1e-5, n_theta=16, n_phi=32):
    """rho_LM(r_j) [na][25][n_rad] by the surface projection of Eq. 3.7 at each radius."""
    out = np.zeros((cl.n_atoms, 25, n_rad))
    st = lib().or_sphere_density(cl.n_atoms, _p(_f64(cl.pos)), _p(_f64(cl.R)), _p(_f64(cl.slater_w)),
                                 _p(_f64(cl.slater_zeta)), _p(_f64(cl.c_lm)), n_rad, r_min, n_theta, n_phi, _p(out))
    if st != OK:
        raise ValueError(f"sphere_density status {st}")
    return out


def inner_solve(R, Z, rho_lm, v_R, r_min=1e-5):
    """V_LM(r_j) [na][25][n_rad] inside each sphere (Eq. 3.4 with the Green's form of Eq. 3.5)."""
    R, Z, rho_lm, v_R = _f64(R), _f64(Z), _f64(rho_lm), _f64(v_R)
    v = np.zeros_like(rho_lm)
    st = lib().or_inner_solve(len(R), _p(R), _p(Z), rho_lm.shape[2], r_min, _p(rho_lm), _p(v_R), _p(v))
    if st != OK:
        raise ValueError(f"inner_solve status {st}")
    return v


BC = {"multipole": 0, "zero": 1, "exact": 2}


def poisson_solve(cl, nu1=2, nu2=2, n_f=1, tol=1e-13, max_cycles=60, n_theta=16, n_phi=32, want_u=False,
                  bc="multipole"):
    """The whole step on one cluster.  Returns dict(status, cycles, rel_resid, vlm, hist[, u]).
    bc: Dirichlet values from the l <= 4 multipole expansion of the grid charge, zero (Eq. 3.3),
    or the exact superposition of the atoms' potentials."""
    n = cl.n
    meshp = np.array([n, *cl.centre, cl.half_width, cl.h_min, cl.h_max, cl.p_max], dtype=np.float64)
    ctl = np.array([nu1, nu2, n_f, max_cycles, n_theta, n_phi, BC[bc]], dtype=np.int32)
    vlm = np.zeros((cl.n_atoms, 25))
    u = np.zeros((n, n, n)) if want_u else None
    stats, hist = np.zeros(3), np.zeros(max_cycles + 1)
    st = lib().or_poisson_solve(*_atoms(cl), _p(meshp), ctl.ctypes.data_as(_I), tol, _p(vlm),
                                _p(u) if want_u else None, _p(stats), _p(hist))
    out = dict(status=st, cycles=int(stats[0]), rel_resid=stats[1], vlm=vlm, hist=hist[:int(stats[0]) + 1])
    if want_u:
        out["u"] = u
    return out
