"""The interface defaults of the steps built here against the values the
paper prints for its configuration fields (tests/golden/paper_config_defaults.txt,
each line with its source in the paper's configuration reference)."""
import inspect
import os

import pytest

import oracle
from paper_2606_26089_b300 import binding as B

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_config_defaults.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, value, src = line.split(" ", 2)
        assert src.startswith("App. C"), line
        out[key] = value
    return out


def test_pileup_defaults():
    g = _golden()
    sig = inspect.signature(B.make_pileup).parameters
    assert sig["sigma_z"].default == float(g["pileup.sigma_z"])
    assert sig["max_z"].default == float(g["pileup.max_z_spread"])
    assert sig["sigma_t"].default == float(g["pileup.sigma_t"])
    assert sig["max_t"].default == float(g["pileup.max_t_spread"])
    assert sig["smear_hs"].default is (g["pileup.smear_hs_vertex"] == "true")
    # the oracle's merge uses the same time defaults
    osig = inspect.signature(oracle.pileup_merge).parameters
    assert osig["sigma_t"].default == float(g["pileup.sigma_t"]) and osig["max_t"].default == float(g["pileup.max_t_spread"])


def test_cluster_defaults():
    g = _golden()
    p = B.make_jet_params()
    assert p.collection == B.COLLECTIONS.get(g["cluster.collection"], 0) == 0
    assert p.p == B.JET_ALGORITHMS[g["cluster.algorithm"]]
    assert p.R == pytest.approx(float(g["cluster.dr"]))
    assert p.pt_min == float(g["cluster.pt_min"])
    assert p.nconst_min == int(g["cluster.nconst_min"])


def test_filter_defaults():
    g = _golden()
    f = B.make_filter({"conditions": [{"field": "pt", "op": ">", "value": 1.0}]})
    assert f.collection == B.COLLECTIONS[g["filter.collection"]]
    assert f.combine == {"all": 0, "any": 1}[g["filter.combine"]]
    assert f.update_features == (g["filter.update_event_features"] == "true")
