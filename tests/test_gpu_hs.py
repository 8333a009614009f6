"""The interstitial overlap and Hamiltonian contributions (Eq. 3.11-3.14, grid-point form) on
the GPU against the oracle, element by element.

Tolerance, from the arithmetic: the GPU evaluates the basis in FP32 (a few roundings per value)
and forms FP32 products summed per 32-node step into FP64, so an element of S errs by at most a
few 1e-7 of sum |phi_a phi_b| Vol <= sqrt(S_aa S_bb) (Cauchy-Schwarz); the test allows 1e-5 of
that.  For H the same holds with |phi~_b| <= c |phi_b|, c = max |kinetic factor| (its terms
taken in absolute value) + max |V| over the interstitial nodes."""
import numpy as np
import pytest

import synth
from gpu_common import dev, host, need_gpu

pytestmark = pytest.mark.gpu

PD = [(4, 2, 2.20), (5, 2, 2.60), (5, 0, 1.00), (5, 1, 1.00), (6, 0, 2.00), (6, 1, 2.00), (4, 3, 1.60)]
L4 = [(5, 4, 1.4), (3, 1, 1.8), (5, 0, 0.9)]


def _axes(orc, cl):
    return orc.mesh(cl)


def _potential(cl, x, y, z, seed):
    return synth.potential_energy(cl.pos, x, y, z, seed)


def _outside(cl, x, y, z):
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    out = np.ones(Xg.shape, bool)
    for p, R in zip(cl.pos, cl.R):
        out &= np.sqrt((Xg - p[0]) ** 2 + (Yg - p[1]) ** 2 + (Zg - p[2]) ** 2) >= R
    return out


def _scale(S, V, basis, R, diag):
    """Per-element error scale: sqrt(S_aa S_bb) and (c_a + c_b) sqrt(S_aa S_bb) for H (V: its
    values at the interstitial nodes)."""
    r = np.linspace(min(R), diag, 4000)
    per = []
    for n, l, zt in basis:
        k = 0.5 * (abs(l * (l + 1) - n * (n - 1)) / r ** 2 + 2 * zt * n / r + zt * zt)
        per += [k.max()] * (2 * l + 1)
    c = np.tile(np.array(per), len(S) // len(per)) + np.abs(V).max()
    d = np.sqrt(np.abs(np.diag(S)))
    sS = np.outer(d, d)
    return sS, sS * (c[:, None] + c[None, :])


def _compare(orc, cl, basis, seed, mode=0):
    B = need_gpu()
    x, y, z = _axes(orc, cl)
    V = _potential(cl, x, y, z, seed)
    S, H = B.lasto_op_interstitial_hs(dev(x), dev(y), dev(z), dev(cl.pos), dev(cl.R), dev(V), basis=basis, mode=mode)
    S, H = host(S), host(H)
    Sr, Hr = orc.interstitial_hs(cl.pos, cl.R, x, y, z, V, basis)
    diag = np.sqrt((x[-1] - x[0]) ** 2 + (y[-1] - y[0]) ** 2 + (z[-1] - z[0]) ** 2)
    sS, sH = _scale(Sr, V[_outside(cl, x, y, z)], basis, cl.R, diag)
    assert np.array_equal(S, S.T) and np.array_equal(H, H.T)
    assert np.all(np.abs(S - Sr) <= 1e-5 * sS)
    assert np.all(np.abs(H - Hr) <= 1e-5 * sH)
    return S, H, Sr, Hr


MODES = [0, 1, 2]   # default (tensor cores), FP32 SIMT, tensor cores


@pytest.mark.parametrize("mode", MODES)
def test_pd2_table_basis(orc, mode):
    """Pd2 (50 functions: one ragged tile), uniform 33^3 box."""
    _compare(orc, synth.pd2_dimer(n=33), PD, seed=1, mode=mode)


@pytest.mark.parametrize("mode", MODES[1:])
def test_pd13_graded(orc, mode):
    """Pd13 on a graded 49^3 mesh: 325 functions (six 64-wide or three 128-wide tiles per side,
    the last ragged), about 70k interstitial nodes (several 4096-node work units per tile)."""
    S, H, Sr, Hr = _compare(orc, synth.pd13_small(n=49), PD, seed=2, mode=mode)
    assert np.linalg.eigvalsh(S).min() > 0


@pytest.mark.parametrize("mode", MODES[1:])
def test_l4_basis_single_atom(orc, mode):
    """Every l <= 4 harmonic (a g-type entry) on one off-centre atom."""
    cl = synth.pd2_dimer(n=33)
    cl.pos = np.ascontiguousarray(cl.pos[:1] + np.array([0.3, -0.2, 0.1]))
    cl.R = np.ascontiguousarray(cl.R[:1])
    _compare(orc, cl, L4, seed=3, mode=mode)


def test_modes_agree(orc):
    """The tensor-core (FP16 pairs) and SIMT (FP32) contractions of the same tables agree to their
    rounding."""
    B = need_gpu()
    cl = synth.pd13_small(n=33)
    x, y, z = _axes(orc, cl)
    V = _potential(cl, x, y, z, 6)
    args = [dev(a) for a in (x, y, z, cl.pos, cl.R, V)]
    S1, H1 = (host(t) for t in B.lasto_op_interstitial_hs(*args, mode=1))
    S2, H2 = (host(t) for t in B.lasto_op_interstitial_hs(*args, mode=2))
    diag = np.sqrt(3) * 2 * cl.half_width
    sS, sH = _scale(S1, V[_outside(cl, x, y, z)], PD, cl.R, diag)
    assert np.all(np.abs(S1 - S2) <= 1e-5 * sS)
    assert np.all(np.abs(H1 - H2) <= 1e-5 * sH)


def test_potential_shift_on_the_gpu(orc):
    """H(V + c) - H(V) = c S on the GPU's own outputs, to the rounding of the two H's; S does
    not depend on V."""
    B = need_gpu()
    cl = synth.pd2_dimer(n=33)
    x, y, z = _axes(orc, cl)
    V = _potential(cl, x, y, z, 4)
    args = [dev(a) for a in (x, y, z, cl.pos, cl.R)]
    S0, H0 = (host(t) for t in B.lasto_op_interstitial_hs(*args, dev(V)))
    S1, H1 = (host(t) for t in B.lasto_op_interstitial_hs(*args, dev(V + 0.75)))
    diag = np.sqrt(3) * 2 * cl.half_width
    sS, sH = _scale(S0, np.abs(V[_outside(cl, x, y, z)]) + 0.75, PD, cl.R, diag)
    assert np.all(np.abs(S1 - S0) <= 1e-6 * sS)
    assert np.all(np.abs(H1 - H0 - 0.75 * S0) <= 2e-5 * sH)


@pytest.mark.parametrize("sub,locs", [((2, 5), (10, 15, 16, 17)), ((0,), (0, 1, 2, 3, 4))],
                         ids=["5s+6p", "4d"])
def test_full_size_pd55_sub_basis(orc, sub, locs):
    """Pd55 on the graded 129^3 mesh with the whole Table 1 basis (1375 functions) on the GPU;
    the entries of a sub-basis (5s and 6p; 4d) checked against the oracle run on that
    sub-basis."""
    B = need_gpu()
    cl = synth.pd55_graded129()
    x, y, z = _axes(orc, cl)
    V = _potential(cl, x, y, z, 5)
    S, H = B.lasto_op_interstitial_hs(dev(x), dev(y), dev(z), dev(cl.pos), dev(cl.R), dev(V), basis=PD)
    sub = [PD[q] for q in sub]
    Sr, Hr = orc.interstitial_hs(cl.pos, cl.R, x, y, z, V, sub)
    # within an atom's 25 functions: 4d 0-4, 5d 5-9, 5s 10, 5p 11-13, 6s 14, 6p 15-17, 4f 18-24
    pick = np.array([a * 25 + loc for a in range(cl.n_atoms) for loc in locs])
    S, H = host(S)[np.ix_(pick, pick)], host(H)[np.ix_(pick, pick)]
    diag = np.sqrt(3) * 2 * cl.half_width
    sS, sH = _scale(Sr, V[_outside(cl, x, y, z)], sub, cl.R, diag)
    assert np.all(np.abs(S - Sr) <= 1e-5 * sS)
    assert np.all(np.abs(H - Hr) <= 1e-5 * sH)


def test_rejects_bad_arguments():
    B = need_gpu()
    import torch
    x = torch.linspace(-5, 5, 9, dtype=torch.float64, device="cuda")
    pos = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    R = torch.full((1,), 1.0, dtype=torch.float64, device="cuda")
    V = torch.zeros((9, 9, 9), dtype=torch.float64, device="cuda")
    for basis in ([(2, 2, 1.0)], [(5, 5, 1.0)], [(3, 1, 0.0)], [(3, 1, 1.0)] * 9, [(5, 4, 1.0)] * 8):
        with pytest.raises(RuntimeError):
            B.lasto_op_interstitial_hs(x, x, x, pos, R, V, basis=basis)
    for mode in (-1, 3):
        with pytest.raises(RuntimeError):
            B.lasto_op_interstitial_hs(x, x, x, pos, R, V, mode=mode)


@pytest.mark.parametrize("mode", MODES[1:])
def test_no_interstitial_nodes(orc, mode):
    """A sphere that holds the whole box leaves no interstitial node: S = H = 0 (the oracle's
    sums are empty too)."""
    B = need_gpu()
    cl = synth.pd2_dimer(n=17)
    x, y, z = _axes(orc, cl)
    pos, R = np.zeros((1, 3)), np.array([100.0])
    V = _potential(cl, x, y, z, 7)
    S, H = B.lasto_op_interstitial_hs(dev(x), dev(y), dev(z), dev(pos), dev(R), dev(V), basis=PD, mode=mode)
    Sr, Hr = orc.interstitial_hs(pos, R, x, y, z, V, PD)
    assert not np.any(Sr) and not np.any(Hr)
    assert not np.any(host(S)) and not np.any(host(H))


@pytest.mark.parametrize("mode", MODES[1:])
def test_non_cubic_box(orc, mode):
    """Axes of different lengths (33, 29, 25 nodes; every other coordinate dropped where
    needed) keep the node indexing right."""
    B = need_gpu()
    cl = synth.pd2_dimer(n=33)
    x, y, z = _axes(orc, cl)
    y = np.ascontiguousarray(np.concatenate([y[:14], y[18:]]))
    z = np.ascontiguousarray(np.concatenate([z[:12], z[20:]]))
    assert (len(x), len(y), len(z)) == (33, 29, 25)
    V = _potential(cl, x, y, z, 8)
    S, H = B.lasto_op_interstitial_hs(dev(x), dev(y), dev(z), dev(cl.pos), dev(cl.R), dev(V), basis=PD, mode=mode)
    Sr, Hr = orc.interstitial_hs(cl.pos, cl.R, x, y, z, V, PD)
    diag = np.sqrt((x[-1] - x[0]) ** 2 + (y[-1] - y[0]) ** 2 + (z[-1] - z[0]) ** 2)
    sS, sH = _scale(Sr, V[_outside(cl, x, y, z)], PD, cl.R, diag)
    assert np.all(np.abs(host(S) - Sr) <= 1e-5 * sS)
    assert np.all(np.abs(host(H) - Hr) <= 1e-5 * sH)
