"""The oracle against the paper's printed constants and its own committed fixtures.

``oracle_bump_200.json`` is written by ``tests/golden/make_golden.py``, which
calls only the oracle; it guards against unintended changes of the oracle's
arithmetic (such a change must cite the passage that justifies it).
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import scenario

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_fb_weights_are_the_papers():
    c = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    assert tuple(c["fb_weights"]["value"]) == oracle.BETA


@pytest.mark.parametrize("two_level", [False, True])
def test_bump_regression(two_level):
    gold = json.load(open(os.path.join(GOLD, "oracle_bump_200.json")))
    s = scenario.gaussian_bump_case(two_level=two_level)
    g = gold[s.name]
    m = oracle.Mesh.from_scenario(s)
    h, u = oracle.run_scenario(s, g["steps"])
    mass, av = oracle.diagnostics(m, h, u)
    assert mass == pytest.approx(g["mass"], rel=1e-14)
    assert av == pytest.approx(g["abs_vorticity"], rel=1e-13)
    for i, v in g["h"].items():
        assert h[int(i)] == pytest.approx(v, rel=1e-13)
    umax = max(abs(v) for v in g["u"].values())
    for e, v in g["u"].items():
        assert abs(u[int(e)] - v) <= 1e-11 * umax
