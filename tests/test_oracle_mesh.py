"""Pins of the graded tensor-product mesh (Section 3: fine near the atoms, coarse far away)."""
import numpy as np
import pytest

import synth


def test_uniform_box_of_side_24(orc):
    cl = synth.pd13_uniform65()
    x, info = orc.mesh_axis(cl.n, 0.0, cl.half_width, cl.h_min, cl.h_max)
    assert np.array_equal(x, -12.0 + 0.375 * np.arange(65))
    assert info[1] == 0.0


@pytest.mark.parametrize("n,L,hmin,hmax", [(129, 22.8, 0.12, 0.6), (97, 17.6, 0.12, 0.6), (33, 9.0, 0.2, 0.8)])
def test_graded_properties(orc, n, L, hmin, hmax):
    x, (A, B, p, hc, he) = orc.mesh_axis(n, 0.0, L, hmin, hmax)
    m = (n - 1) // 2
    assert x[0] == -L and x[-1] == L
    assert np.all(np.diff(x) > 0)
    assert np.abs(x + x[::-1]).max() < 1e-13 * L
    assert abs(x[m]) < 1e-15
    # slopes of x(xi) at the centre and the ends are h_min*m and h_max*m
    assert abs(A - hmin * m) < 1e-12 and abs(A + p * B - hmax * m) < 1e-12 and abs(A + B - L) < 1e-12
    # the discrete spacings approach those slopes
    assert abs(hc - (hmin + B / m ** p)) < 1e-12
    assert abs(he - hmax) < p * (p - 1) / (2 * m) * hmax + 1e-12
    # the deviation from linear is a pure power |xi|^p
    xi = (np.arange(n) - m) / m
    dev = (x - A * xi)[m + 1:]
    slope = np.diff(np.log(dev)) / np.diff(np.log(xi[m + 1:]))
    assert np.abs(slope - p).max() < 1e-8


def test_steep_grading_is_clamped(orc):
    # Pd561 box: with h_min = 0.15 the exponent would be 9 > p_max = 6; keep h_max, lower p
    x, (A, B, p, hc, he) = orc.mesh_axis(385, 0.0, 38.4, 0.15, 0.6, 6.0)
    assert p == 6.0 and abs(A + 6 * B - 0.6 * 192) < 1e-12 and abs(A + B - 38.4) < 1e-12


def test_infeasible_mesh_rejected(orc):
    with pytest.raises(ValueError):
        orc.mesh_axis(65, 0.0, 30.0, 0.12, 0.6)   # edge spacing cannot cover the box
    with pytest.raises(ValueError):
        orc.mesh_axis(64, 0.0, 10.0, 0.12, 0.6)   # even node count has no centre node


def test_dual_lengths_sum_to_box(orc):
    x, _ = orc.mesh_axis(129, 0.0, 22.8, 0.12, 0.6)
    v = orc.dual_lengths(x)
    assert abs(v.sum() - 2 * 22.8) < 1e-12
