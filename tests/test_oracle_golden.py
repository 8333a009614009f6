"""The stored oracle answers (tests/golden/oracle_vlm_*.npz) belong to the clusters the
tests rebuild, were solved to the oracle's floor, and are what the oracle gives today.

They are written by tests/golden/make_oracle_vlm.py, which calls only the oracle; this test
re-solves the cheapest stored cluster of each group and compares, so a stale or hand-edited
file fails here, on the CPU, before any GPU comparison uses it."""
import os

import numpy as np
import pytest

from golden.make_oracle_vlm import GROUPS, TOL, fingerprint, load, path


@pytest.mark.parametrize("group", sorted(GROUPS))
def test_stored_answers_match_inputs_and_floor(group):
    if not os.path.exists(path(group)):
        pytest.skip(f"{group} not generated")
    stored = load(group)
    clusters = GROUPS[group]()
    if len(stored) < len(clusters):
        pytest.skip(f"{group}: {len(stored)} of {len(clusters)} clusters generated so far")
    assert [s[0] for s in stored] == [c.name for c in clusters]
    for cl, (name, vlm, stats, fp) in zip(clusters, stored):
        assert vlm.shape == (cl.n_atoms, 25) and np.all(np.isfinite(vlm))
        assert stats[0] == 0 and stats[2] <= TOL, (cl.name, stats)
        assert np.allclose(fp, fingerprint(cl), rtol=1e-12, atol=0.0), cl.name


@pytest.mark.parametrize("group", ["pd55x8", "batch64", "guess_eval"])
def test_stored_answer_is_reproduced_by_the_oracle(orc, group):
    if not os.path.exists(path(group)):
        pytest.skip(f"{group} not generated")
    clusters = GROUPS[group]()
    i = min(range(len(clusters)), key=lambda q: clusters[q].n ** 3 * clusters[q].n_atoms)
    cl = clusters[i]
    out = orc.poisson_solve(cl, tol=TOL, max_cycles=600)
    ref = load(group)[i][1]
    assert out["status"] == 0
    assert np.abs(out["vlm"] - ref).max() <= 1e-12 * np.abs(ref).max()
