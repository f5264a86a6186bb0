"""The oracle reproduces its stored results (tests/golden/, written by
tests/golden/make_golden.py). A change of the oracle's arithmetic shows up here and
must cite, in its commit, the passage of the paper that justifies it."""
import json
import os

import numpy as np

from paper_1204_2586_gb300.inputs import kuhn_mesh

HERE = os.path.dirname(os.path.abspath(__file__))


def test_p2_n8_golden(oracle_mod):
    g = json.load(open(os.path.join(HERE, "golden", "p2_n8_oracle.json")))
    xyz, t = kuhn_mesh(8, 0.2, 0)
    P = oracle_mod.Problem(xyz, t, 2)
    assert (P.nh, P.nH, P.nnz_h, P.nnz_H) == (g["n_h"], g["n_H"], g["nnz_h"], g["nnz_H"])
    P.setup(theta=0.25, mode=0)
    out = P.solve()
    assert out["iters"] == g["iters"] and out["status"] == g["status"]
    assert np.allclose(out["hist"], g["hist"], rtol=1e-12, atol=0)
    assert [P.level(l)["A"].shape[0] for l in range(P.levels())] == g["level_rows"]
