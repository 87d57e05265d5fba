"""Writes oracle_trajectory.json: the FP64 oracle's L2 trajectories and final
parameter norms on one seeded mixture, for each update of P.  A regression
fixture (not a pin: the values come from the oracle itself, which the pins
check against the paper and the mathematics); it flags any later change of
the oracle's arithmetic.  Calls only oracle/ and the seeded generator.

    python tests/golden/make_oracle_trajectory.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import fastfca_as as ffa  # noqa: E402
from oracle.fastfca_as import OpCounter  # noqa: E402
from paper_1805_09498_gb300.synth import make_problem  # noqa: E402

CASE = dict(I=3, J=3, F=3, N=64, seed=123, iters=5, K=1)
UPDATES = [("fpi", 0.0), ("gradient", 0.05), ("natural_gradient", 0.2), ("newton", 1.0), ("em", 0.0)]


def trajectories():
    c = CASE
    p = make_problem(c["I"], c["J"], c["F"], c["N"], seed=c["seed"])
    out = {}
    for name, mu in UPDATES:
        v, lam, P, tr = ffa.iterate(p.y, p.v0, p.lam0, p.P0, c["iters"], K=c["K"], counter=OpCounter(),
                                   p_update=name, mu=mu)
        out[name] = {"mu": mu, "trace": [float(t) for t in tr],
                     "norm_v": float(np.linalg.norm(v)), "norm_lam": float(np.linalg.norm(lam)),
                     "norm_P": float(np.linalg.norm(P))}
    return out


if __name__ == "__main__":
    doc = {"_source": "written by tests/golden/make_oracle_trajectory.py from oracle/ (regression "
                      "fixture of the oracle's own values, not a pin)",
           "case": CASE, "updates": trajectories()}
    with open(os.path.join(HERE, "oracle_trajectory.json"), "w") as fh:
        json.dump(doc, fh, indent=1)
    print("written")
