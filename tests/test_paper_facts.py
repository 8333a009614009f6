"""The numbers the paper prints that this step uses (tests/golden/paper_facts.json)."""
import json
import os

import numpy as np

import synth
from synth import clusters

FACTS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def test_small_cluster_geometries_follow_the_paper():
    assert abs(np.linalg.norm(np.diff(clusters.dimer(), axis=0)) - FACTS["pd2_bond_au"]["value"]) < 1e-12
    assert abs(clusters.min_pair_distance(clusters.square4()) - FACTS["pd4_edge_au"]["value"]) < 1e-12
    assert abs(clusters.min_pair_distance(clusters.cube8()) - FACTS["pd8_edge_au"]["value"]) < 1e-12


def test_harmonic_count_matches_lmax(orc):
    assert len(orc.solid_harmonics(0.3, 0.2, 0.1)) == (FACTS["l_max_density_potential"]["value"] + 1) ** 2


def test_pseudo_density_sign_at_origin(orc):
    for cl in (synth.pd2_dimer(), synth.pd13_uniform65()):
        q, rhoR, drhoR, coef = orc.sphere_params(cl)
        assert np.all(np.sign(coef[:, 0]) == FACTS["pseudo_density_at_origin_sign"]["value"])
