"""Write the oracle regression fixtures under tests/golden/ (calls only oracle/ and synth/).

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from synth import scenario  # noqa: E402

SAMPLE_CELLS = [0, 17, 333, 512, 777, 1023]
SAMPLE_EDGES = [0, 5, 1000, 1536, 2500, 3071]


def main():
    out = {}
    for two_level in (False, True):
        s = scenario.gaussian_bump_case(two_level=two_level)
        m = oracle.Mesh.from_scenario(s)
        h, u = oracle.run_scenario(s, 200)
        mass, av = oracle.diagnostics(m, h, u)
        out[s.name] = {
            "steps": 200, "dt": s.dt, "M": s.M,
            "mass": mass, "abs_vorticity": av,
            "h": {str(i): float(h[i]) for i in SAMPLE_CELLS},
            "u": {str(e): float(u[e]) for e in SAMPLE_EDGES},
        }
    with open(os.path.join(HERE, "oracle_bump_200.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
