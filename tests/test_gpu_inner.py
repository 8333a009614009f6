"""Inside the spheres on the GPU (Eq. 3.4-3.7) against the oracle: the density's harmonic
components on the logarithmic radial mesh, the inner Dirichlet solve on the oracle's own
inputs, and the whole chain from the interstitial solve's sphere coefficients."""
import numpy as np
import pytest

import synth
from gpu_common import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [lambda: synth.pd13_small(n=33), lambda: synth.pd2_dimer(n=33),
                                  lambda: synth.pd55_graded129()], ids=["pd13", "pd2", "pd55-full"])
def test_sphere_density(orc, make):
    B = need_gpu()
    cl = make()
    dc = B.DeviceCluster(cl)
    rho, status = B.lasto_op_sphere_density(dc, n_rad=429)
    ref = orc.sphere_density(cl, n_rad=429)
    got = host(rho)
    assert int(host(status)[0]) == 0
    # FP32-pair Slater sums (~44 bits), the far tails (zeta r > 20) in FP32: ~1e-13 of the
    # density scale
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n_rad", [4, 64, 429])
def test_inner_solve_on_oracle_inputs(orc, n_rad):
    B = need_gpu()
    rng = np.random.default_rng(n_rad)
    R = np.array([2.4, 2.2, 2.0])
    Z = np.array([46.0, 0.0, 12.0])
    r = [orc.radial_mesh(n_rad, 1e-5, x) for x in R]
    L = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9)
    rho = np.stack([np.stack([rng.normal() * r[a] ** L[lm] * np.exp(-r[a]) for lm in range(25)]) for a in range(3)])
    vR = rng.normal(size=(3, 25))
    ref = orc.inner_solve(R, Z, rho, vR)
    got = host(B.lasto_op_inner_solve(dev(R), dev(Z), dev(rho), dev(vR)))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_inner_chain_from_the_interstitial_solve(orc):
    """GPU interstitial solve -> sphere coefficients -> GPU density projection -> GPU inner
    solve, against the same chain in the oracle: the inner potential inherits the 1e-8
    parity of V_LM(R)."""
    import torch
    B = need_gpu()
    cl = synth.pd13_small(n=33)
    dc = B.DeviceCluster(cl)
    solver = B.Poisson(n_max=33, max_atoms=13, precision=B.LASTO_PREC_MIXED)
    vlm = torch.empty((13, 25), dtype=torch.float64, device="cuda")
    st = solver.solve(dc, vlm)[0]
    torch.cuda.synchronize()
    assert st.status == 0
    rho, _ = B.lasto_op_sphere_density(dc)
    v = host(B.lasto_op_inner_solve(dc.R, dc.Z, rho, vlm))
    out = orc.poisson_solve(cl, tol=1e-13, max_cycles=200)
    ref = orc.inner_solve(cl.R, cl.Z, orc.sphere_density(cl), out["vlm"])
    assert np.abs(v - ref).max() < 1e-8 * np.abs(ref).max()
    # on the sphere the inner solution is the boundary data
    assert np.allclose(v[:, :, -1], host(vlm), rtol=0, atol=1e-14 * np.abs(host(vlm)).max())
