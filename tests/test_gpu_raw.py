"""The raw-density entry point on the GPU (a grid density plus each sphere's rho_00 table,
Eq. 3.1's representation) against the oracle's raw path, and through the whole solve."""
import numpy as np
import pytest

import synth
from gpu_common import dev, host, need_gpu

pytestmark = pytest.mark.gpu


def _raw_inputs(orc, cl, B, dc):
    x, y, z = orc.mesh(cl)
    ne = orc.density_grid(cl, x, y, z)
    rho00 = orc.sphere_density(cl)[:, 0, :]
    rc = B.RawCluster(cl.pos, cl.Z, cl.R, dc.x, dc.y, dc.z, cl.centre, ne, rho00)
    return x, y, z, ne, rho00, rc


@pytest.mark.parametrize("make", [lambda: synth.pd13_small(n=33), lambda: synth.pd2_dimer(n=33)])
def test_raw_deposit(orc, make):
    B = need_gpu()
    cl = make()
    dc = B.DeviceCluster(cl, axes=orc.mesh(cl))
    x, y, z, ne, rho00, rc = _raw_inputs(orc, cl, B, dc)
    b, owner, status = B.lasto_op_raw_deposit(rc)
    ref, rowner = orc.raw_deposit(cl.pos, cl.Z, cl.R, x, y, z, ne, rho00)
    assert int(host(status)[0]) == 0
    assert np.array_equal(host(owner).reshape(rowner.shape), rowner)
    assert np.abs(host(b).reshape(ref.shape) - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_raw_solve_matches_the_oracle_chain(orc, precision):
    """Raw solve on the GPU against the oracle's raw deposit followed by its multipoles, faces,
    multigrid and projection; and, since the raw inputs are the model's own density, within the
    raw path's quadrature error (~1e-5) of the model solve."""
    import torch
    B = need_gpu()
    cl = synth.pd13_small(n=33)
    dc = B.DeviceCluster(cl, axes=orc.mesh(cl))
    x, y, z, ne, rho00, rc = _raw_inputs(orc, cl, B, dc)
    prec = B.LASTO_PREC_MIXED if precision == "mixed" else B.LASTO_PREC_FP64
    solver = B.Poisson(n_max=33, max_atoms=13, precision=prec)
    v = torch.empty((13, 25), dtype=torch.float64, device="cuda")
    st = solver.solve_raw(rc, v)[0]
    torch.cuda.synchronize()
    assert st.status == 0 and st.rel_resid <= 1e-10
    b, _ = orc.raw_deposit(cl.pos, cl.Z, cl.R, x, y, z, ne, rho00)
    Q = orc.multipoles(x, y, z, b)
    u = orc.boundary_fill(x, y, z, Q, np.zeros(b.shape))
    stt, _, _ = orc.mg_solve(x, y, z, b, u, tol=1e-13, max_cycles=200)
    ref = orc.project(x, y, z, u, cl.pos, cl.R)
    got = host(v)
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()
    model = orc.poisson_solve(cl, tol=1e-13, max_cycles=200)["vlm"]
    assert np.abs(got - model).max() < 1e-4 * np.abs(model).max()
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.Poisson(n_max=33, max_atoms=13, boundary=B.LASTO_BC_EXACT).solve_raw(rc, v)
