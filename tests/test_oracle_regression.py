"""The oracle reproduces its committed trajectories (tests/golden/
oracle_trajectory.json, written by make_oracle_trajectory.py): a change of
its arithmetic shows here and must name the passage that justifies it."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_oracle_reproduces_its_committed_trajectories():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mot", os.path.join(GOLDEN, "make_oracle_trajectory.py"))
    mot = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mot)
    with open(os.path.join(GOLDEN, "oracle_trajectory.json")) as fh:
        ref = json.load(fh)
    assert ref["case"] == mot.CASE
    got = mot.trajectories()
    for name, r in ref["updates"].items():
        g = got[name]
        np.testing.assert_allclose(g["trace"], r["trace"], rtol=1e-10, err_msg=name)
        for k in ("norm_v", "norm_lam", "norm_P"):
            np.testing.assert_allclose(g[k], r[k], rtol=1e-10, err_msg=f"{name} {k}")
