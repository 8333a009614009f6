"""Cluster geometries for the synthetic Pd workloads (atom centres only).

Pure geometry: no part of the Poisson method lives here.  The paper tests its
method on small Pd clusters (Section 4, Table 3 and the cluster figure beside
it: Pd2 at 4.802 au, Pd4 at 4.72 au, Pd8 at 4.88 au); the larger benchmark
clusters below (cuboctahedral Pd13, Mackay icosahedra Pd55/Pd147/Pd561) are
the usual closed-shell Pd cluster shapes and stand in for the paper's
free-standing clusters.  Lengths are in bohr.
"""
from __future__ import annotations

import itertools

import numpy as np

PD_NN = 5.20  # fcc Pd nearest-neighbour distance in bohr (2.75 Angstrom)


def dimer(d: float = 4.802) -> np.ndarray:
    """Pd2 along z, bond length from the paper's Table 2 / cluster figure (Section 4)."""
    return np.array([[0.0, 0.0, -d / 2], [0.0, 0.0, d / 2]])


def square4(d: float = 4.72) -> np.ndarray:
    """Pd4 square in the xy-plane, edge from the paper's cluster figure (Section 4)."""
    h = d / 2
    return np.array([[-h, -h, 0.0], [h, -h, 0.0], [h, h, 0.0], [-h, h, 0.0]])


def cube8(d: float = 4.88) -> np.ndarray:
    """Pd8 cube, edge from the paper's cluster figure (Section 4)."""
    h = d / 2
    return np.array(list(itertools.product((-h, h), repeat=3)), dtype=float)


def cuboctahedron13(d: float = PD_NN) -> np.ndarray:
    """Centre atom plus its 12 fcc nearest neighbours at (+-a, +-a, 0) and permutations, a = d/sqrt(2)."""
    a = d / np.sqrt(2.0)
    pts = [(0.0, 0.0, 0.0)]
    for s1 in (-a, a):
        for s2 in (-a, a):
            pts += [(s1, s2, 0.0), (s1, 0.0, s2), (0.0, s1, s2)]
    return np.array(pts, dtype=float)


def _icosahedron_unit() -> tuple[np.ndarray, list[tuple[int, int]], list[tuple[int, int, int]]]:
    """Unit-circumradius icosahedron: 12 vertices, 30 edges, 20 faces."""
    g = (1.0 + np.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-g, g):
            v += [(0.0, s1, s2), (s1, s2, 0.0), (s2, 0.0, s1)]
    v = np.array(v)
    v /= np.linalg.norm(v[0])
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    edge2 = np.min(d2[d2 > 1e-12])
    adj = np.abs(d2 - edge2) < 1e-9
    edges = [(i, j) for i in range(12) for j in range(i + 1, 12) if adj[i, j]]
    faces = [(i, j, k) for i in range(12) for j in range(i + 1, 12) for k in range(j + 1, 12)
             if adj[i, j] and adj[j, k] and adj[i, k]]
    assert len(edges) == 30 and len(faces) == 20
    return v, edges, faces


def mackay_icosahedron(shells: int, d: float = PD_NN) -> np.ndarray:
    """Mackay icosahedron with the given number of shells around a centre atom.

    Shell k has its 12 vertices at radius k*d; its 30 edges carry k-1 atoms each
    and its 20 flat faces (k-1)(k-2)/2 atoms each, 10k^2+2 atoms in all, so that
    1, 2, 3, 5 shells give Pd13, Pd55, Pd147, Pd561.
    """
    v, edges, faces = _icosahedron_unit()
    pts = [np.zeros(3)]
    for k in range(1, shells + 1):
        vk = v * (k * d)
        pts += list(vk)
        for i, j in edges:
            for t in range(1, k):
                pts.append(vk[i] + (t / k) * (vk[j] - vk[i]))
        for i, j, l in faces:
            for a in range(1, k):
                for b in range(1, k - a):
                    pts.append(vk[i] + (a / k) * (vk[j] - vk[i]) + (b / k) * (vk[l] - vk[i]))
    out = np.array(pts)
    assert len(out) == 1 + sum(10 * k * k + 2 for k in range(1, shells + 1))
    return out


def min_pair_distance(pos: np.ndarray) -> float:
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    d2[np.diag_indices(len(pos))] = np.inf
    return float(np.sqrt(d2.min()))


def cluster_radius(pos: np.ndarray, centre=(0.0, 0.0, 0.0)) -> float:
    return float(np.sqrt(((pos - np.asarray(centre)) ** 2).sum(-1)).max())


def close_atoms(pos: np.ndarray, dmin: float) -> np.ndarray:
    """Indices of the atoms that have a partner closer than dmin (the later atom of each pair)."""
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    iu = np.triu_indices(len(pos), 1)
    bad = d2[iu] < dmin * dmin
    return np.unique(iu[1][bad])
