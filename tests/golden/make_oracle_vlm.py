#!/usr/bin/env python3
"""Writes the stored oracle answers the full-size parity tests and the bench compare with.

Every value here comes from the FP64 CPU oracle (``oracle/``) solving the same seeded
synthetic clusters the GPU tests build (``synth/``), to the oracle's floor (relative
residual 1e-13, stationary V(2,2) cycles, l <= 4 multipole faces).  Nothing here touches
the CUDA library.  One ``.npz`` per workload group, keyed by the cluster's position in the
group (names repeat across seeds):

  NNN/name         the cluster's name
  NNN/vlm          V_LM on every sphere [n_atoms][25] (Eq. 3.6)
  NNN/stats        oracle status, cycles, final relative residual
  NNN/hist         the oracle's relative residual after each cycle (cycle 0 = the start)
  NNN/fingerprint  a few sums of the cluster's inputs, so a test can tell that the
                   stored answer belongs to the cluster it rebuilt

A group is written after every cluster, so an interrupted run keeps what it finished and
the next run resumes after it.

Groups (the workloads are synth's):
  pd55x8      Pd55 graded 129^3, density seeds 1..8 (the 8-cluster batch)
  batch64     the 64 uneven clusters Pd13/55/147 on 65^3..193^3
  guess_eval  held-out clusters of the learned guess (seeds 77, 78; Pd13 on 97^3, seed 79)
  pd561       Pd561 graded 385^3, the 8 SCF-like densities

Usage: python tests/golden/make_oracle_vlm.py [group ...]   (default: all; pd561 takes hours)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

TOL = 1e-13
MAX_CYCLES = 600


def fingerprint(cl) -> np.ndarray:
    """Sums of the inputs that fix a cluster (compared with a relative tolerance)."""
    return np.array([cl.n, cl.n_atoms, cl.half_width, cl.h_min, cl.h_max, cl.p_max,
                     float(np.sum(cl.pos * np.array([1.0, 2.0, 3.0]))), float(np.sum(cl.slater_w)),
                     float(np.sum(cl.slater_w * cl.slater_zeta)), float(np.sum(cl.c_lm * np.arange(1, 25))),
                     float(np.sum(np.abs(cl.c_lm)))])


def guess_eval_clusters():
    out = list(synth.workloads.guess_training_set(8, seed=77)) + list(synth.workloads.guess_training_set(3, seed=78))
    pos = synth.clusters.cuboctahedron13()
    out.append(synth.workloads.make_cluster("Pd13-graded-97", pos, np.random.default_rng(79), n=97,
                                            half_width=synth.workloads.graded_box(pos), h_min=0.12, h_max=0.6))
    return out


GROUPS = {
    "pd55x8": lambda: [synth.pd55_graded129(seed=1 + k) for k in range(8)],
    "batch64": lambda: synth.batch64(),
    "guess_eval": guess_eval_clusters,
    "pd561": lambda: synth.pd561_graded385(),
}


def path(group: str) -> str:
    return os.path.join(HERE, f"oracle_vlm_{group}.npz")


def make(group: str) -> None:
    clusters = GROUPS[group]()
    data = {}
    if os.path.exists(path(group)):                   # resume: keep the clusters already solved
        z = np.load(path(group))
        data = {k: z[k] for k in z.files}
    for i, cl in enumerate(clusters):
        key = f"{i:03d}"
        if f"{key}/hist" in data and str(data[f"{key}/name"]) == cl.name and np.allclose(
                data[f"{key}/fingerprint"], fingerprint(cl), rtol=1e-12, atol=0.0):
            continue
        t0 = time.perf_counter()
        out = oracle.poisson_solve(cl, tol=TOL, max_cycles=MAX_CYCLES)
        dt = time.perf_counter() - t0
        if out["status"] != 0:
            raise SystemExit(f"{cl.name}: oracle status {out['status']} after {out['cycles']} cycles "
                             f"(residual {out['rel_resid']:.2e})")
        data[f"{key}/name"] = np.array(cl.name)
        data[f"{key}/vlm"] = out["vlm"]
        data[f"{key}/stats"] = np.array([out["status"], out["cycles"], out["rel_resid"]])
        data[f"{key}/hist"] = np.asarray(out["hist"], dtype=np.float64)
        data[f"{key}/fingerprint"] = fingerprint(cl)
        tmp = path(group) + ".tmp.npz"
        np.savez_compressed(tmp, **data)
        os.replace(tmp, path(group))
        print(f"{group}: {i} {cl.name} cycles={out['cycles']} rel_resid={out['rel_resid']:.2e} {dt:.1f} s",
              flush=True)


def load(group: str) -> list:
    """[(name, vlm, stats, fingerprint)] of a stored group, in group order (FileNotFoundError if absent)."""
    z = np.load(path(group))
    keys = sorted({k.split("/", 1)[0] for k in z.files})
    return [(str(z[f"{k}/name"]), z[f"{k}/vlm"], z[f"{k}/stats"], z[f"{k}/fingerprint"]) for k in keys]


def history(group: str, index: int) -> np.ndarray:
    """The oracle's relative residual after each cycle for cluster `index` of a stored group."""
    return np.load(path(group))[f"{index:03d}/hist"]


def stored_vlm(group: str, cl, index: int) -> np.ndarray:
    """The stored oracle V_LM of cluster cl, position `index` of its group, after checking that
    the stored answer was made for cl's inputs."""
    name, vlm, stats, fp = load(group)[index]
    if name != cl.name or not np.allclose(fp, fingerprint(cl), rtol=1e-12, atol=0.0):
        raise ValueError(f"{cl.name}: stored oracle answer {index} of {group} was made for other inputs")
    return vlm


if __name__ == "__main__":
    for g in (sys.argv[1:] or list(GROUPS)):
        make(g)
