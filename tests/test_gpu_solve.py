"""Whole-step GPU parity against the FP64 oracle, through lasto_poisson_solve.

Bar (the target of the step): every sphere-surface coefficient within 1e-8 of the
oracle relative to the largest |V_LM|, and the GPU's own true residual
||b - A u|| / ||b_eff|| <= 1e-10.  The oracle solves the same discretisation to its
floor (1e-13), so the two answers differ by at most the GPU's stopping error.
"""
import numpy as np
import pytest

import synth
from gpu_common import host, need_gpu

pytestmark = pytest.mark.gpu

_ORACLE_CACHE = {}


def oracle_vlm(orc, cl):
    import hashlib
    h = hashlib.sha1()
    for a in (cl.pos, cl.slater_w, cl.slater_zeta, cl.c_lm, cl.R, cl.Z):
        h.update(np.ascontiguousarray(a).tobytes())
    key = (cl.name, cl.n, cl.half_width, cl.h_min, cl.h_max, h.hexdigest())
    if key not in _ORACLE_CACHE:
        out = orc.poisson_solve(cl, tol=1e-13, max_cycles=200)
        assert out["status"] == 0, out["status"]
        _ORACLE_CACHE[key] = out["vlm"]
    return _ORACLE_CACHE[key]


def gpu_solve(B, cl, **kw):
    import torch
    solver = B.Poisson(n_max=cl.n, max_atoms=cl.n_atoms, **kw)
    dc = B.DeviceCluster(cl)
    vlm = torch.empty((cl.n_atoms, 25), dtype=torch.float64, device="cuda")
    pot = torch.empty(dc.N, dtype=torch.float64, device="cuda")
    st = solver.solve(dc, vlm, potential=pot)
    torch.cuda.synchronize()
    return solver, dc, host(vlm), host(pot), st[0]


CASES = [
    ("small-graded", lambda: synth.pd13_small(n=33)),
    ("dimer-graded", lambda: synth.pd2_dimer(n=65, half_width=12.0, graded=True)),
    ("pd13-uniform-65", synth.pd13_uniform65),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("precision,cycle", [(0, 2), (1, 2), (0, 0), (0, 1)])
def test_solve_matches_oracle(orc, name, make, precision, cycle):
    B = need_gpu()
    cl = make()
    ref = oracle_vlm(orc, cl)
    maxc = 50 if cycle == 2 else 120
    _, _, vlm, _, st = gpu_solve(B, cl, precision=precision, cycle=cycle, max_cycles=maxc)
    assert st.status == 0, (st.status, st.cycles, st.rel_resid)
    assert st.rel_resid <= 1e-10
    assert np.abs(vlm - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.slow
@pytest.mark.parametrize("precision", [0, 1])
def test_pd55_graded_129(orc, precision):
    """The benchmark workload (Pd55, graded 129^3) at full size, both precisions."""
    B = need_gpu()
    cl = synth.pd55_graded129()
    ref = oracle_vlm(orc, cl)
    _, _, vlm, pot, st = gpu_solve(B, cl, precision=precision)
    assert st.status == 0 and st.rel_resid <= 1e-10, (st.status, st.cycles, st.rel_resid)
    assert np.abs(vlm - ref).max() <= 1e-8 * np.abs(ref).max()
    # the returned potential satisfies the residual bound when checked by the oracle's operator
    x, y, z = orc.mesh(cl)
    u = pot.reshape(cl.n, cl.n, cl.n)
    b, _ = orc.deposit(cl, x, y, z)
    r = orc.residual(x, y, z, u, b)
    ub = u.copy()
    ub[1:-1, 1:-1, 1:-1] = 0
    assert orc.norm2_interior(r) <= 2e-10 * orc.norm2_interior(orc.residual(x, y, z, ub, b))


@pytest.mark.parametrize("precision", [0, 1])
def test_direct_launch_matches_graph(orc, precision):
    """The profiling launch mode runs the same kernels: same answer bit for bit."""
    B = need_gpu()
    cl = synth.pd13_small(n=33)
    _, _, v_graph, _, st_g = gpu_solve(B, cl, precision=precision)
    _, _, v_direct, _, st_d = gpu_solve(B, cl, precision=precision, launch=1)
    assert st_g.status == 0 and st_d.status == 0 and st_g.cycles == st_d.cycles
    assert np.array_equal(v_graph, v_direct)


def test_replay_is_deterministic_and_tracks_new_density(orc):
    import torch
    B = need_gpu()
    cl = synth.pd13_small(n=33)
    solver = B.Poisson(n_max=33, max_atoms=cl.n_atoms)
    dc = B.DeviceCluster(cl)
    vlm = torch.empty((cl.n_atoms, 25), dtype=torch.float64, device="cuda")
    solver.solve(dc, vlm)
    torch.cuda.synchronize()
    a = host(vlm).copy()
    solver.solve(dc, vlm)            # replays the captured graph
    torch.cuda.synchronize()
    assert np.array_equal(a, host(vlm))
    # change the density in place: the replay must follow it
    cl2 = synth.pd13_small(n=33, seed=99)
    dc.w.copy_(torch.as_tensor(cl2.slater_w))
    dc.clm.copy_(torch.as_tensor(cl2.c_lm))
    st = solver.solve(dc, vlm)
    torch.cuda.synchronize()
    cl_mod = synth.workloads.replace(cl, slater_w=cl2.slater_w, c_lm=cl2.c_lm)
    ref = oracle_vlm(orc, cl_mod)
    assert st[0].status == 0
    assert np.abs(host(vlm) - ref).max() <= 1e-8 * np.abs(ref).max()


def test_single_level_grid(orc):
    """n = 9: the whole grid is the coarsest level (one exact solve)."""
    import torch
    B = need_gpu()
    cl = synth.workloads.make_cluster("tiny", np.zeros((1, 3)), np.random.default_rng(0), n=9, half_width=8.0,
                                      h_min=2.0, h_max=2.0)
    ref = oracle_vlm(orc, cl)
    _, _, vlm, _, st = gpu_solve(B, cl, cycle=0)
    assert st.status == 0 and st.cycles <= 2
    assert np.abs(vlm - ref).max() <= 1e-8 * np.abs(ref).max()


def test_error_statuses(orc):
    import torch
    B = need_gpu()
    # overlapping spheres -> GEOMETRY
    pos = np.array([[0.0, 0.0, -1.5], [0.0, 0.0, 1.5]])
    cl = synth.workloads.make_cluster("overlap", pos, np.random.default_rng(1), n=33, half_width=9.0,
                                      h_min=9.0 / 16, h_max=9.0 / 16)
    _, _, _, _, st = gpu_solve(B, cl)
    assert st.status == B.LASTO_ERR_GEOMETRY
    # a sphere poking out of the box -> GEOMETRY
    cl = synth.workloads.make_cluster("outside", np.array([[7.5, 0.0, 0.0]]), np.random.default_rng(1), n=33,
                                      half_width=9.0, h_min=9.0 / 16, h_max=9.0 / 16)
    _, _, _, _, st = gpu_solve(B, cl)
    assert st.status == B.LASTO_ERR_GEOMETRY
    # NaN in the density -> NONFINITE
    cl = synth.pd13_small(n=33)
    cl.slater_w[3, 1] = np.nan
    _, _, _, _, st = gpu_solve(B, cl)
    assert st.status == B.LASTO_ERR_NONFINITE
    # cycle cap -> NOT_CONVERGED, outputs still written
    cl = synth.pd13_small(n=33)
    _, _, vlm, _, st = gpu_solve(B, cl, max_cycles=2)
    assert st.status == B.LASTO_ERR_NOT_CONVERGED and st.cycles == 2 and np.all(np.isfinite(vlm))
    # host-detected bad arguments
    with pytest.raises(RuntimeError):
        B.Poisson(n_max=64)
    solver = B.Poisson(n_max=33)
    big = synth.pd13_small(n=65)
    dc = B.DeviceCluster(big)
    with pytest.raises(RuntimeError):
        solver.solve(dc, torch.empty((13, 25), dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_of_uneven_clusters(orc, precision):
    """Several clusters with different grids and atom counts in one solve call (one graph
    launch, each cluster an independent branch): every cluster matches its own oracle solve."""
    import torch
    B = need_gpu()
    batch = [synth.pd13_small(n=33), synth.pd2_dimer(n=65, half_width=12.0, graded=True), synth.pd13_uniform65(),
             synth.pd13_small(n=65, seed=21), synth.pd2_dimer(n=33, seed=22)]
    n_max = max(c.n for c in batch)
    atoms = sum(c.n_atoms for c in batch)
    solver = B.Poisson(n_max=n_max, max_atoms=max(c.n_atoms for c in batch), max_batch=len(batch),
                       precision=precision)
    dcs = [B.DeviceCluster(c) for c in batch]
    vlm = torch.empty((atoms, 25), dtype=torch.float64, device="cuda")
    pot = torch.empty(sum(d.N for d in dcs), dtype=torch.float64, device="cuda")
    for rep in range(2):                       # capture, then replay
        st = solver.solve(dcs, vlm, potential=pot)
        torch.cuda.synchronize()
        got = host(vlm)
        off = 0
        for c, s in zip(batch, st):
            ref = oracle_vlm(orc, c)
            assert s.status == 0 and s.rel_resid <= 1e-10, (c.name, s.status, s.rel_resid)
            assert np.abs(got[off:off + c.n_atoms] - ref).max() <= 1e-8 * np.abs(ref).max(), c.name
            off += c.n_atoms


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_smoother_tuning_and_forced_choices(precision):
    """The first solve measures the smoother of every level the cycle smooths with separate
    launches; whatever the table says (in-place half sweeps over the flat index or one block per
    row, fused register-column passes, fused two-sweep z-slab passes) the converged solution is
    bitwise the same."""
    B = need_gpu()
    import torch
    prec = B.LASTO_PREC_MIXED if precision == "mixed" else B.LASTO_PREC_FP64
    cl = synth.pd13_small(n=65)
    dc = B.DeviceCluster(cl)
    auto = B.Poisson(n_max=65, max_atoms=13, precision=prec)
    v_auto = torch.empty((13, 25), dtype=torch.float64, device="cuda")
    st = auto.solve(dc, v_auto)[0]
    torch.cuda.synchronize()
    assert st.status == 0
    rows = [line.split() for line in auto.tune_table().strip().splitlines()]
    elem = 4 if precision == "mixed" else 8
    shapes = sorted({tuple(int(v) for v in r[:3]) for r in rows if int(r[3]) == elem})
    assert (65, 65, 65) in shapes and (33, 33, 33) in shapes
    col_ty = 14 if elem == 4 else 6
    forms = {"inplace": "0 256 0 0 0 0", "rows": "0 0 0 0 0 0", "column": f"1 256 62 {col_ty} 32 1",
             "slab": "1 256 64 16 32 2"}
    out = {}
    for name, choice in forms.items():
        solver = B.Poisson(n_max=65, max_atoms=13, precision=prec)
        solver.set_tune_table("\n".join(f"{a} {b} {c} {elem} {choice} 0" for a, b, c in shapes) + "\n")
        v = torch.empty((13, 25), dtype=torch.float64, device="cuda")
        s = solver.solve(dc, v)[0]
        torch.cuda.synchronize()
        assert s.status == 0 and s.rel_resid <= 1e-10
        out[name] = (v.clone(), s.cycles)
        assert all(line.split()[4:10] == choice.split() for line in solver.tune_table().strip().splitlines()
                   if int(line.split()[3]) == elem and tuple(int(x) for x in line.split()[:3]) in shapes)
    for name in ("rows", "column", "slab"):
        assert torch.equal(out["inplace"][0], out[name][0]) and out["inplace"][1] == out[name][1], name
    assert torch.equal(out["inplace"][0], v_auto)


def test_tune_table_rejects_bad_lines():
    B = need_gpu()
    solver = B.Poisson(n_max=65, max_atoms=13, precision=B.LASTO_PREC_MIXED)
    for bad in ("65 65 65 4 1 256 62 14 32 3 0\n", "not a table\n", "65 65 65 2 0 256 0 0 0 0 0\n",
                "65 65 65 4 0 100 0 0 0 0 0\n"):
        with pytest.raises(RuntimeError, match="INVALID_ARG"):
            solver.set_tune_table(bad)
    solver.set_tune_table("\n  \n")   # empty is fine


def test_boundary_exact_op(orc):
    B = need_gpu()
    import torch
    for cl in (synth.pd13_small(n=33), synth.pd2_dimer(n=33)):
        x, y, z = orc.mesh(cl)
        dc = B.DeviceCluster(cl, axes=(x, y, z))
        u = torch.zeros((cl.n,) * 3, dtype=torch.float64, device="cuda")
        got = host(B.lasto_op_boundary_exact(dc, u))
        ref = orc.boundary_exact(cl, x, y, z)
        # the faces carry the small remainder of the nuclei's Z/r and the shells' potentials
        assert np.abs(got - ref).max() < 1e-14 * 46.0 * cl.n_atoms / cl.half_width * 10


@pytest.mark.parametrize("bc", ["zero", "exact"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_boundary_choices(orc, bc, precision):
    """Zero faces (Eq. 3.3) and exact-superposition faces through the whole solve, against the
    oracle with the same faces."""
    B = need_gpu()
    import torch
    cl = synth.pd13_small(n=33)
    dc = B.DeviceCluster(cl)
    prec = B.LASTO_PREC_MIXED if precision == "mixed" else B.LASTO_PREC_FP64
    code = B.LASTO_BC_ZERO if bc == "zero" else B.LASTO_BC_EXACT
    solver = B.Poisson(n_max=33, max_atoms=13, precision=prec, boundary=code)
    v = torch.empty((13, 25), dtype=torch.float64, device="cuda")
    st = solver.solve(dc, v)[0]
    torch.cuda.synchronize()
    assert st.status == 0 and st.rel_resid <= 1e-10
    ref = orc.poisson_solve(cl, tol=1e-13, max_cycles=200, bc=bc)["vlm"]
    assert np.abs(host(v) - ref).max() < 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("nu_coarse", [0, 1, 4])
def test_coarse_level_sweeps(orc, nu_coarse):
    """The one-block coarse levels of the mixed-precision cycle with 0, 1 or 4 (default) sweeps:
    the solve converges to the same V_LM (against the oracle)."""
    B = need_gpu()
    import torch
    cl = synth.pd13_small(n=65)
    dc = B.DeviceCluster(cl)
    solver = B.Poisson(n_max=65, max_atoms=13, precision=B.LASTO_PREC_MIXED, nu_coarse=nu_coarse)
    v = torch.empty((13, 25), dtype=torch.float64, device="cuda")
    st = solver.solve(dc, v)[0]
    torch.cuda.synchronize()
    assert st.status == 0 and st.rel_resid <= 1e-10
    ref = oracle_vlm(orc, cl)
    assert np.abs(host(v) - ref).max() < 1e-8 * np.abs(ref).max()


def test_back_to_back_solves_on_one_handle_keep_their_stats(orc):
    """Solves enqueued one after another on the same handle, with no synchronisation between
    them, each deliver their own stats (every call carries its own destination)."""
    import torch
    B = need_gpu()
    cls = [synth.pd13_small(n=33, seed=s) for s in (11, 12, 13)]
    solver = B.Poisson(n_max=33, max_atoms=13, precision=B.LASTO_PREC_MIXED)
    dcs = [B.DeviceCluster(c) for c in cls]
    outs = [torch.empty((13, 25), dtype=torch.float64, device="cuda") for _ in cls]
    solver.solve(dcs[0], outs[0])
    torch.cuda.synchronize()
    sts = [solver.solve(d, o) for d, o in zip(dcs, outs)]      # no sync in between
    torch.cuda.synchronize()
    for c, st, o in zip(cls, sts, outs):
        s = st[0]
        assert s.status == 0 and 0 < s.rel_resid <= 1e-10 and s.cycles > 0, (s.status, s.rel_resid, s.cycles)
        ref = oracle_vlm(orc, c)
        assert np.abs(host(o) - ref).max() <= 1e-8 * np.abs(ref).max()


def test_dropped_stats_arrays_are_kept_until_written():
    """Solves whose returned stats the caller drops at once (no synchronisation), with new
    pointers every few calls (recapture while earlier solves run): the library writes every
    stats array after its solve, the binding keeps each alive until then, nothing crashes, and
    the last solve is right."""
    import torch
    B = need_gpu()
    cls = [synth.pd13_small(n=33, seed=s) for s in (31, 32, 33)]
    solver = B.Poisson(n_max=33, max_atoms=13, precision=B.LASTO_PREC_MIXED)
    dcs = [B.DeviceCluster(c) for c in cls]
    outs = [torch.empty((13, 25), dtype=torch.float64, device="cuda") for _ in cls]
    for r in range(24):
        solver.solve(dcs[(r // 4) % 3], outs[(r // 4) % 3])      # result dropped immediately
    st = solver.solve(dcs[0], outs[0])
    torch.cuda.synchronize()
    assert st[0].status == 0 and 0 < st[0].rel_resid <= 1e-10
    solver.close()
