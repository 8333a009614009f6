"""Colour-split storage of the finest FP32 level (lasto_op_smooth_split_f32 and the solver's
fused = 3 smoother choice) against natural storage.

Every neighbour of a node has the other colour, so with the red nodes stored first and the
black ones after them a half sweep reads only the other half and its own right-hand side.
Each node update keeps the in-place kernels' expression and operands, and every kernel that
touches the split arrays (restriction of the residual, prolongation, the inner CG's operator,
dots and updates, the FP64 defect and correction) walks the nodes in flat order, so a whole
solve over split storage equals the natural-storage solve bit for bit, and both match the
FP64 oracle.
"""
import numpy as np
import pytest

import synth
from gpu_common import dev, graded_axis, host, need_gpu

pytestmark = pytest.mark.gpu


def _grid(n, seed):
    return (graded_axis(n[0], 6.0, 3.0, seed, 0.1), graded_axis(n[1], 5.0, 2.0, seed + 1, 0.1),
            graded_axis(n[2], 7.0, 4.0, seed + 2, 0.1))


@pytest.mark.parametrize("n", [(5, 3, 7), (33, 33, 33), (71, 37, 13), (129, 129, 129), (97, 5, 9), (9, 9, 9),
                               (35, 17, 21), (97, 99, 9), (513, 11, 9)])
@pytest.mark.parametrize("threads", [128, 256, 512, 0, 1])
def test_split_sweeps_equal_natural_sweeps(n, threads):
    """threads = 1 is the plane-staged kernel: tiles of 8 rows (ragged last tile), plane chunks
    of one plane up to many, rows of 9 to 513 nodes; it takes no axis shorter than 9."""
    import torch
    B = need_gpu()
    x, y, z = _grid(n, 51)
    rng = np.random.default_rng(52)
    u = torch.as_tensor(rng.normal(size=n[::-1]).astype(np.float32)).cuda().reshape(-1)
    b = torch.as_tensor(rng.normal(size=n[::-1]).astype(np.float32)).cuda().reshape(-1)
    if threads == 0 and n[0] > 1023 or threads == 1 and min(n) < 9:
        with pytest.raises(RuntimeError, match="INVALID_ARG"):
            B.lasto_op_smooth_split(dev(x), dev(y), dev(z), B.split_colours(u), B.split_colours(b), threads=threads)
        return
    for sweeps in (1, 3):
        ref = B.lasto_op_smooth(dev(x), dev(y), dev(z), u.clone(), b, sweeps=sweeps, threads=256)
        us, bs = B.split_colours(u), B.split_colours(b)
        B.lasto_op_smooth_split(dev(x), dev(y), dev(z), us, bs, sweeps=sweeps, threads=threads)
        torch.cuda.synchronize()
        assert torch.equal(B.merge_colours(us), ref), (n, threads, sweeps)


def test_split_layout_helpers_round_trip():
    import torch
    B = need_gpu()
    for N in (1, 2, 7, 8, 105):
        a = torch.arange(N, dtype=torch.float32, device="cuda")
        s = B.split_colours(a)
        assert host(s).tolist() == list(range(0, N, 2)) + list(range(1, N, 2))
        assert torch.equal(B.merge_colours(s), a)


def test_split_op_rejects_bad_input():
    import torch
    B = need_gpu()
    x = dev(np.linspace(-1, 1, 9))
    x8 = dev(np.linspace(-1, 1, 8))
    u = torch.zeros(9 * 9 * 8, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.lasto_op_smooth_split(x, x, x8, u, u.clone())        # an even axis
    u = torch.zeros(9 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.lasto_op_smooth_split(x, x, x, u, u.clone(), threads=100)
    # the staged kernel copies 16-byte runs: arrays that do not start on 16 bytes are refused
    big = torch.zeros(9 ** 3 + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.lasto_op_smooth_split(x, x, x, big[1:1 + 9 ** 3], u.clone(), threads=1)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        B.lasto_op_smooth_split(x, x, x, u, big[2:2 + 9 ** 3], threads=1)
    B.lasto_op_smooth_split(x, x, x, big[4:4 + 9 ** 3], u.clone(), threads=1)


def _solve(B, cls, table, n_max, guess=False):
    import torch
    solver = B.Poisson(n_max=n_max, max_atoms=max(c.n_atoms for c in cls), max_batch=len(cls),
                       precision=B.LASTO_PREC_MIXED)
    if guess:
        solver.set_guess()
    if table is not None:
        solver.set_tune_table(table)
    dcs = [B.DeviceCluster(c) for c in cls]
    v = torch.empty((sum(c.n_atoms for c in cls), 25), dtype=torch.float64, device="cuda")
    st = solver.solve(dcs if len(dcs) > 1 else dcs[0], v)
    torch.cuda.synchronize()
    tab = solver.tune_table()
    solver.close()
    return v, st, tab


def test_solve_over_split_storage_equals_natural_storage(orc):
    """Pd13 on 65^3 (its 33^3 level below): the finest level forced to each split kernel (flat
    blocks of 128 and 256, one warp per row, plane-staged), then natural; the V_LM, iteration
    counts and residuals agree bit for bit, and match the oracle."""
    B = need_gpu()
    cl = synth.pd13_small(n=65)
    rest = "33 33 33 4 0 256 0 0 0 0 0\n"
    v0, st0, _ = _solve(B, [cl], "65 65 65 4 0 256 0 0 0 0 0\n" + rest, 65)
    assert st0[0].status == 0 and st0[0].rel_resid <= 1e-10
    for nt in (128, 256, 0, 1):
        v, st, _ = _solve(B, [cl], f"65 65 65 4 3 {nt} 0 0 0 0 0\n" + rest, 65)
        assert st[0].status == 0 and st[0].cycles == st0[0].cycles and st[0].rel_resid == st0[0].rel_resid
        assert np.array_equal(host(v), host(v0)), nt
    ref = orc.poisson_solve(cl, tol=1e-13, max_cycles=200)
    err = np.abs(host(v0) - ref["vlm"]).max() / np.abs(ref["vlm"]).max()
    assert err <= 1e-8, err


def test_split_choice_applies_only_where_the_level_is_finest():
    """A batch where 65^3 is the finest level of one cluster and the second level of another
    (129^3): the split choice for 65^3 is taken by the first and read as natural in-place
    sweeps by the second; the whole batch, with the learned guess, equals the natural one."""
    B = need_gpu()
    cls = [synth.pd13_small(n=65), synth.pd13_small(n=129)]
    rest = "129 129 129 4 0 128 0 0 0 0 0\n33 33 33 4 0 256 0 0 0 0 0\n"
    v0, st0, _ = _solve(B, cls, "65 65 65 4 0 256 0 0 0 0 0\n" + rest, 129, guess=True)
    v1, st1, _ = _solve(B, cls, "65 65 65 4 3 256 0 0 0 0 0\n" + rest, 129, guess=True)
    v2, st2, _ = _solve(B, cls, "65 65 65 4 3 256 0 0 0 0 0\n129 129 129 4 3 128 0 0 0 0 0\n"
                        "33 33 33 4 0 256 0 0 0 0 0\n", 129, guess=True)
    for v, st in ((v1, st1), (v2, st2)):
        assert [s.status for s in st] == [0, 0]
        assert [s.cycles for s in st] == [s.cycles for s in st0]
        assert np.array_equal(host(v), host(v0))


def test_tuner_offers_split_storage_on_the_finest_level():
    """The tuner times the split candidates on the finest FP32 level only; whatever it picks,
    the table round-trips and an FP64 entry with the split choice is refused."""
    B = need_gpu()
    cl = synth.pd13_small(n=97)
    v, st, tab = _solve(B, [cl], None, 97)
    assert st[0].status == 0 and st[0].rel_resid <= 1e-10
    rows = {tuple(int(a) for a in line.split()[:4]): line.split()[4:6] for line in tab.strip().splitlines()}
    assert (97, 97, 97, 4) in rows
    assert all(r[0] != "3" for k, r in rows.items() if k[:3] != (97, 97, 97))
    solver = B.Poisson(n_max=97, max_atoms=13, precision=B.LASTO_PREC_MIXED)
    solver.set_tune_table(tab)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        solver.set_tune_table("97 97 97 8 3 256 0 0 0 0 0\n")
    solver.close()


def _batch_solve(B, cls, launch, guess=True, table=None):
    import torch
    solver = B.Poisson(n_max=max(c.n for c in cls), max_atoms=max(c.n_atoms for c in cls), max_batch=len(cls),
                       precision=B.LASTO_PREC_MIXED, launch=launch)
    if guess:
        solver.set_guess()
    if table is not None:
        solver.set_tune_table(table)
    dcs = [B.DeviceCluster(c) for c in cls]
    v = torch.empty((sum(c.n_atoms for c in cls), 25), dtype=torch.float64, device="cuda")
    pot = torch.empty(sum(c.n ** 3 for c in cls), dtype=torch.float64, device="cuda")
    out = []
    for rep in range(2):                      # capture, then replay
        st = solver.solve(dcs, v, potential=pot)
        torch.cuda.synchronize()
        out.append((host(v).copy(), host(pot).copy(), [(s.status, s.cycles, s.outer, s.rel_resid) for s in st]))
    solver.close()
    return out


def test_lockstep_batch_equals_branches():
    """launch = 2: clusters of the same grid shape run their iterations in lockstep (each kernel
    launched once for the group, members that have converged skip it); a mixed batch of two
    groups (three Pd13 65^3 with different densities, two Pd13 33^3) and a cluster alone in its
    shape (97^3) gives bitwise the V_LM, potentials and stats of the branch graph (itself
    checked against the oracle elsewhere), on the capture and on the replay."""
    B = need_gpu()
    cls = [synth.pd13_small(n=65, seed=1), synth.pd13_small(n=33, seed=2), synth.pd13_small(n=65, seed=3),
           synth.pd13_small(n=97, seed=4), synth.pd13_small(n=33, seed=5), synth.pd13_small(n=65, seed=6)]
    ref = _batch_solve(B, cls, 0)
    got = _batch_solve(B, cls, 2)
    for (v0, p0, s0), (v1, p1, s1) in zip(ref, got):
        assert all(s[0] == 0 and s[3] <= 1e-10 for s in s1)
        assert s0 == s1
        assert np.array_equal(v0, v1) and np.array_equal(p0, p1)


def test_lockstep_batch_of_eight_pd55():
    """The benchmarked batch (8 Pd55 densities on the graded 129^3 mesh, learned guess) in
    lockstep: bitwise the branch graph's results."""
    B = need_gpu()
    cls = [synth.pd55_graded129(seed=1 + k) for k in range(8)]
    ref = _batch_solve(B, cls, 0)
    got = _batch_solve(B, cls, 2)
    for (v0, p0, s0), (v1, p1, s1) in zip(ref, got):
        assert s0 == s1
        assert np.array_equal(v0, v1) and np.array_equal(p0, p1)


def test_lockstep_in_split_storage_equals_branches_in_natural_storage():
    """The finest level's storage order and the launch form are independent choices: branches
    over natural storage and lockstep batches over colour-split storage (row-per-warp and
    plane-staged half sweeps) give bitwise the same V_LM, potentials and stats -- every
    reduction is formed in an order that depends on the grid shape alone."""
    B = need_gpu()
    cls = [synth.pd13_small(n=65, seed=11 + k) for k in range(4)]
    rest = "33 33 33 4 0 256 0 0 0 0 0\n"
    ref = _batch_solve(B, cls, 0, table="65 65 65 4 0 256 0 0 0 0 0\n" + rest)
    for nt in (0, 1):
        got = _batch_solve(B, cls, 2, table=f"65 65 65 4 3 {nt} 0 0 0 0 0\n" + rest)
        for (v0, p0, s0), (v1, p1, s1) in zip(ref, got):
            assert s0 == s1, nt
            assert np.array_equal(v0, v1) and np.array_equal(p0, p1), nt
