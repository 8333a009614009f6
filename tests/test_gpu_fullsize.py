"""Full-size parity of every workload against the FP64 oracle, in the forms that are timed.

The oracle's answers (V_LM of Eq. 3.6, solved to its 1e-13 floor) are stored by
tests/golden/make_oracle_vlm.py, an oracle-only script, because the largest ones take the
oracle minutes to hours.  Each test rebuilds the same seeded clusters, checks that the stored
answer belongs to them (input fingerprint), solves them on the GPU through the C ABI in the
benchmarked form, and requires every cluster's coefficients within 1e-8 of the oracle
relative to its largest |V_LM| (and the GPU's own residual <= 1e-10):

  * the benchmarked batch: 8 Pd55 densities on the graded 129^3 mesh in one graph launch,
    learned initial guess, FP64 defect correction around FP32 multigrid-preconditioned CG;
  * the uneven batch: all 64 Pd13/Pd55/Pd147 clusters on 65^3..193^3 meshes in one launch;
  * the learned-guess solves: held-out clusters started from the network's guess, computed
    outside the solve and inside its graph (including a 97^3 mesh);
  * Pd561 on the graded 385^3 mesh (57 M nodes): the chosen form on the 8 SCF-like densities
    back to back, the later ones warm-started from the previous potential, and the plain
    FP64 form on the first.
"""
import os

import numpy as np
import pytest

import synth
from gpu_common import host, need_gpu
from golden.make_oracle_vlm import guess_eval_clusters, path as golden_path, stored_vlm

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0806_1723_gb300", "weights",
                       "unet_pd_33.npz")
TOL = 1e-8


def _check(group, clusters, vlm, stats, first=0):
    """Every cluster of a concatenated V_LM against its stored oracle answer (the clusters
    are positions first, first + 1, ... of their group)."""
    off, worst = 0, 0.0
    for q, (cl, st) in enumerate(zip(clusters, stats)):
        ref = stored_vlm(group, cl, first + q)
        got = vlm[off:off + cl.n_atoms]
        off += cl.n_atoms
        assert st.status == 0 and st.rel_resid <= 1e-10, (cl.name, st.status, st.rel_resid)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL, (cl.name, err)
        worst = max(worst, err)
    assert off == vlm.shape[0]
    return worst


def _need(group, count):
    from golden.make_oracle_vlm import load
    if not os.path.exists(golden_path(group)) or len(load(group)) < count:
        pytest.skip(f"stored oracle answers for {group} not generated")


def test_benchmarked_batch_of_eight_pd55():
    import torch
    B = need_gpu()
    _need("pd55x8", 8)
    cls = [synth.pd55_graded129(seed=1 + k) for k in range(8)]
    solver = B.Poisson(n_max=129, max_atoms=55, max_batch=8, precision=B.LASTO_PREC_MIXED)
    solver.set_guess()
    dcs = [B.DeviceCluster(c) for c in cls]
    vlm = torch.empty((8 * 55, 25), dtype=torch.float64, device="cuda")
    for rep in range(2):                                 # capture, then replay
        st = solver.solve(dcs, vlm)
        torch.cuda.synchronize()
        assert [s.guess for s in st] == [1] * 8
        _check("pd55x8", cls, host(vlm), st)


def test_uneven_batch_of_64():
    import torch
    B = need_gpu()
    _need("batch64", 64)
    cls = synth.batch64()
    solver = B.Poisson(n_max=max(c.n for c in cls), max_atoms=max(c.n_atoms for c in cls), max_batch=len(cls),
                       precision=B.LASTO_PREC_MIXED)
    solver.set_guess()
    dcs = [B.DeviceCluster(c) for c in cls]
    vlm = torch.empty((sum(c.n_atoms for c in cls), 25), dtype=torch.float64, device="cuda")
    st = solver.solve(dcs, vlm)
    torch.cuda.synchronize()
    _check("batch64", cls, host(vlm), st)
    assert {(c.n_atoms, c.n) for c in cls} >= {(147, 193), (147, 161), (55, 193), (13, 65)}
    solver.close()
    del dcs, vlm
    torch.cuda.empty_cache()


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="trained weights not shipped")
def test_learned_guess_solves_match_the_oracle():
    import torch
    B = need_gpu()
    _need("guess_eval", 12)
    from paper_0806_1723_gb300 import unet as U
    cls = guess_eval_clusters()
    # guess computed outside the solve (held-out seed 77)
    net = U.UNet.load(WEIGHTS, nb=1)
    single = B.Poisson(n_max=129, max_atoms=147, precision=B.LASTO_PREC_MIXED)
    for i, c in enumerate(cls[:8]):
        dc = B.DeviceCluster(c)
        v = torch.empty((c.n_atoms, 25), dtype=torch.float64, device="cuda")
        st = single.solve(dc, v, guess=U.learned_guess(net, dc))
        torch.cuda.synchronize()
        _check("guess_eval", [c], host(v), st, first=i)
    # the network inside the solve's graph (seed 78 and the 97^3 mesh)
    batch = cls[8:]
    inside = B.Poisson(n_max=129, max_atoms=147, max_batch=len(batch), precision=B.LASTO_PREC_MIXED)
    inside.set_guess(WEIGHTS)
    dcs = [B.DeviceCluster(c) for c in batch]
    v = torch.empty((sum(c.n_atoms for c in batch), 25), dtype=torch.float64, device="cuda")
    st = inside.solve(dcs, v)
    torch.cuda.synchronize()
    assert [s.guess for s in st] == [1] * len(batch)
    _check("guess_eval", batch, host(v), st, first=8)


def test_pd561_chosen_form_sequence_and_plain_form():
    import torch
    B = need_gpu()
    _need("pd561", 1)
    from golden.make_oracle_vlm import load
    seq = synth.pd561_graded385()[:len(load("pd561"))]     # the densities the oracle has solved
    first = B.Poisson(n_max=385, max_atoms=561, precision=B.LASTO_PREC_MIXED)
    first.set_guess()
    warm = B.Poisson(n_max=385, max_atoms=561, precision=B.LASTO_PREC_MIXED)
    v = torch.empty((561, 25), dtype=torch.float64, device="cuda")
    pot = torch.empty(385 ** 3, dtype=torch.float64, device="cuda")
    for s, cl in enumerate(seq):
        dc = B.DeviceCluster(cl)
        # the first density from the learned guess, each later one from the previous potential
        st = warm.solve(dc, v, potential=pot, guess=pot) if s else first.solve(dc, v, potential=pot)
        torch.cuda.synchronize()
        assert st[0].guess == (0 if s else 1)
        _check("pd561", [cl], host(v), st, first=s)
    first.close()
    warm.close()
    plain = B.Poisson(n_max=385, max_atoms=561, precision=B.LASTO_PREC_FP64)
    st = plain.solve(B.DeviceCluster(seq[0]), v)
    torch.cuda.synchronize()
    _check("pd561", seq[:1], host(v), st)
    plain.close()
    del v, pot
    torch.cuda.empty_cache()
