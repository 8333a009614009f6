"""Seeded synthetic inputs for the LASTO interstitial Poisson step.

This module draws the random numbers and lays out the geometry; it holds none of
the method's arithmetic (no density, pseudo-density, mesh or solver formulas).
Both the FP64 oracle and the CUDA path read the same ``Cluster`` records, so a
difference between them can never come from the inputs.

Density model parameters per atom (the paper's real Pd densities are not
available; the model stands in for the density update of Eq. 3.15):
  * nuclear charge Z = 46, sphere radius R = 2.4 bohr;
  * three Slater exponents zeta = (1.5, 3.0, 8.0) / bohr with weights
    w_k = 46 u_k / sum(u), u_k ~ U(0.5, 1.5) (one draw per atom and term), so
    every atom is neutral;
  * 24 nonspherical coefficients c_lm (l = 1..4, index lm = l*l + l + m - 1)
    drawn from N(0, 1e-3^2).
Mesh parameters per cluster (the mesh itself is built by the method):
  n nodes per axis, box centre, half-width L = cluster radius + R + vacuum,
  h_min (spacing at the centre), h_max (spacing at the box edge) and the
  largest grading exponent p_max.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import clusters

Z_PD = 46.0
R_SPHERE = 2.4
ZETA = (1.5, 3.0, 8.0)
N_CLM = 24
P_MAX = 6.0


@dataclass
class Cluster:
    """One free-standing cluster and the mesh parameters of its box."""
    name: str
    pos: np.ndarray          # [n_atoms, 3] bohr
    Z: np.ndarray            # [n_atoms]
    R: np.ndarray            # [n_atoms] sphere radii
    slater_w: np.ndarray     # [n_atoms, 3] electrons per Slater term
    slater_zeta: np.ndarray  # [n_atoms, 3] 1/bohr
    c_lm: np.ndarray         # [n_atoms, 24]
    n: int                   # nodes per axis (cubic box)
    half_width: float        # L
    h_min: float
    h_max: float
    p_max: float = P_MAX
    centre: tuple = (0.0, 0.0, 0.0)
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    def contiguous(self) -> "Cluster":
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        return replace(self, pos=f(self.pos), Z=f(self.Z), R=f(self.R), slater_w=f(self.slater_w),
                       slater_zeta=f(self.slater_zeta), c_lm=f(self.c_lm))


def draw_density(n_atoms: int, rng: np.random.Generator, clm_sigma: float = 1e-3):
    """Seeded Slater weights (normalised to Z electrons per atom) and nonspherical coefficients."""
    u = rng.uniform(0.5, 1.5, size=(n_atoms, 3))
    w = Z_PD * u / u.sum(axis=1, keepdims=True)
    c = rng.normal(0.0, clm_sigma, size=(n_atoms, N_CLM))
    return w, c


def make_cluster(name, pos, rng, n, half_width, h_min, h_max, p_max=P_MAX, clm_sigma=1e-3, **meta) -> Cluster:
    na = len(pos)
    w, c = draw_density(na, rng, clm_sigma)
    return Cluster(name=name, pos=np.asarray(pos, float), Z=np.full(na, Z_PD), R=np.full(na, R_SPHERE),
                   slater_w=w, slater_zeta=np.tile(np.array(ZETA), (na, 1)), c_lm=c,
                   n=n, half_width=float(half_width), h_min=float(h_min), h_max=float(h_max),
                   p_max=float(p_max), meta=dict(meta)).contiguous()


def graded_box(pos, vacuum=10.0):
    """Half-width of the box: cluster radius + sphere radius + vacuum."""
    return clusters.cluster_radius(pos) + R_SPHERE + vacuum


def potential_energy(pos, x, y, z, seed: int = 0) -> np.ndarray:
    """A seeded potential-energy field at the nodes [nz][ny][nx] (x fastest) for the H and S
    contributions: a screened attraction to every atom, A e^{-k r} / max(r, 0.5) with
    A ~ U(8, 12) hartree bohr and k ~ U(0.5, 0.8) / bohr per atom, plus N(0, 0.05^2) noise.
    It stands in for the SCF potential, which is not available."""
    rng = np.random.default_rng(seed)
    V = np.zeros((len(z), len(y), len(x)))
    zz, yy, xx = z[:, None, None], y[None, :, None], x[None, None, :]
    for p in np.asarray(pos, float):
        r = np.sqrt((xx - p[0]) ** 2 + (yy - p[1]) ** 2 + (zz - p[2]) ** 2)
        V -= rng.uniform(8.0, 12.0) * np.exp(-rng.uniform(0.5, 0.8) * r) / np.maximum(r, 0.5)
    return V + 0.05 * rng.normal(size=V.shape)


# ---------------------------------------------------------------- the five workloads
def pd13_uniform65(seed: int = 0) -> Cluster:
    """Pd13 cuboctahedron, uniform 65^3 box of side 24 bohr (h = 0.375)."""
    rng = np.random.default_rng(seed)
    return make_cluster("Pd13-uniform-65", clusters.cuboctahedron13(), rng, n=65, half_width=12.0,
                        h_min=0.375, h_max=0.375)


def pd55_graded129(seed: int = 1) -> Cluster:
    """Pd55 Mackay icosahedron, graded 129^3 mesh, 0.12 bohr at the centre to 0.6 at the edge, 10 bohr vacuum."""
    rng = np.random.default_rng(seed)
    pos = clusters.mackay_icosahedron(2)
    return make_cluster("Pd55-graded-129", pos, rng, n=129, half_width=graded_box(pos), h_min=0.12, h_max=0.6)


BATCH_SIZES = (65, 97, 129, 161, 193)


def batch64(seed: int = 2, count: int = 64, sizes=BATCH_SIZES) -> list[Cluster]:
    """Random mix of Pd13/Pd55/Pd147 with atoms displaced N(0, 0.1^2) bohr per coordinate.

    Each cluster draws its grid size uniformly from the sizes whose graded mesh
    is feasible (edge spacing 0.6 bohr must cover the half-width).  A draw whose
    spheres come closer than 2R + 0.24 bohr has the atoms involved redrawn.
    """
    rng = np.random.default_rng(seed)
    shapes = {13: clusters.cuboctahedron13(), 55: clusters.mackay_icosahedron(2), 147: clusters.mackay_icosahedron(3)}
    out = []
    for c in range(count):
        kind = int(rng.choice([13, 55, 147]))
        pos = shapes[kind] + rng.normal(0.0, 0.1, size=shapes[kind].shape)
        for _ in range(10000):
            bad = clusters.close_atoms(pos, 2 * R_SPHERE + 0.24)
            if len(bad) == 0:
                break
            pos[bad] = shapes[kind][bad] + rng.normal(0.0, 0.1, size=(len(bad), 3))
        else:
            raise RuntimeError("could not place atoms without sphere overlap")
        L = graded_box(pos)
        feasible = [n for n in sizes if 0.6 * (n - 1) / 2 > L * 1.05]
        n = int(rng.choice(feasible))
        out.append(make_cluster(f"batch{c}-Pd{kind}-{n}", pos, rng, n=n, half_width=L, h_min=0.12, h_max=0.6))
    return out


def pd561_graded385(seed: int = 4, n_densities: int = 8, n: int = 385) -> list[Cluster]:
    """Pd561 five-shell icosahedron, graded 385^3, a sequence of SCF-like densities.

    Density s+1 is density s with every Slater draw scaled by (1 + 0.01 N(0,1))
    (then renormalised to 46 electrons) and every c_lm scaled likewise.
    """
    rng = np.random.default_rng(seed)
    pos = clusters.mackay_icosahedron(5)
    base = make_cluster("Pd561-graded-385-s0", pos, rng, n=n, half_width=graded_box(pos), h_min=0.12, h_max=0.6)
    seq = [base]
    w, c = base.slater_w.copy(), base.c_lm.copy()
    for s in range(1, n_densities):
        w = w * (1.0 + 0.01 * rng.normal(size=w.shape))
        w = Z_PD * w / w.sum(axis=1, keepdims=True)
        c = c * (1.0 + 0.01 * rng.normal(size=c.shape))
        seq.append(replace(base, name=f"Pd561-graded-385-s{s}", slater_w=w.copy(), c_lm=c.copy()))
    return seq


def guess_training_set(count: int, seed: int = 3, n: int = 129) -> list[Cluster]:
    """Training clusters of the learned initial guess: perturbed Pd13 / Pd55 / Pd147 on graded
    n^3 meshes (same recipe as the 64-cluster batch, one mesh size)."""
    rng = np.random.default_rng(seed)
    shapes = {13: clusters.cuboctahedron13(), 55: clusters.mackay_icosahedron(2), 147: clusters.mackay_icosahedron(3)}
    out = []
    for c in range(count):
        kind = int(rng.choice([13, 55, 147]))
        pos = shapes[kind] + rng.normal(0.0, 0.1, size=shapes[kind].shape)
        for _ in range(10000):
            bad = clusters.close_atoms(pos, 2 * R_SPHERE + 0.24)
            if len(bad) == 0:
                break
            pos[bad] = shapes[kind][bad] + rng.normal(0.0, 0.1, size=(len(bad), 3))
        out.append(make_cluster(f"guess{c}-Pd{kind}", pos, rng, n=n, half_width=graded_box(pos), h_min=0.12,
                                h_max=0.6))
    return out


# ---------------------------------------------------------------- small test cases
def pd2_dimer(seed: int = 10, n: int = 33, half_width: float = 9.0, graded: bool = False) -> Cluster:
    """Pd2 at the paper's GGA bond length 4.802 au (Table 2), in a small box."""
    rng = np.random.default_rng(seed)
    m = (n - 1) / 2
    h_min = 0.5 * half_width / m if graded else half_width / m
    h_max = 1.6 * half_width / m if graded else half_width / m
    return make_cluster(f"Pd2-{'graded' if graded else 'uniform'}-{n}", clusters.dimer(), rng, n=n,
                        half_width=half_width, h_min=h_min, h_max=h_max)


def pd13_small(seed: int = 11, n: int = 33, graded: bool = True, vacuum: float = 6.0) -> Cluster:
    rng = np.random.default_rng(seed)
    pos = clusters.cuboctahedron13()
    L = graded_box(pos, vacuum)
    m = (n - 1) / 2
    h_max = 1.5 * L / m if graded else L / m
    h_min = 0.6 * L / m if graded else L / m
    return make_cluster(f"Pd13-{'graded' if graded else 'uniform'}-{n}", pos, rng, n=n, half_width=L,
                        h_min=h_min, h_max=h_max)
