"""Writes the stored oracle results under tests/golden/ (calls only the oracle and the
seeded input generators). Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1204_2586_gb300.inputs import kuhn_mesh  # noqa: E402


def p2_n8():
    """P2 Poisson, kappa = 1, 8^3 Kuhn cubes, 0.2h jitter (seed 0), sine source,
    additive preconditioner (1 SGS sweep + one P1 AMG V-cycle, theta = 0.25)."""
    xyz, t = kuhn_mesh(8, 0.2, 0)
    P = oracle.Problem(xyz, t, 2)
    P.setup(theta=0.25, mode=0)
    out = P.solve()
    levels = [P.level(l) for l in range(P.levels())]
    return dict(
        workload="P2 Poisson, 8^3 jittered Kuhn cubes (3072 tets), kappa=1, sine source",
        n_h=P.nh, n_H=P.nH, nnz_h=P.nnz_h, nnz_H=P.nnz_H, nnz_pi=P.nnz_pi,
        level_rows=[int(L["A"].shape[0]) for L in levels],
        level_nnz=[int(L["A"].nnz) for L in levels],
        level_colours=[int(L["ncolour"]) for L in levels],
        fine_colours=int(P.fine_colour().max() + 1),
        iters=out["iters"], status=out["status"],
        hist=[float(v) for v in out["hist"]],
        true_rel=out["true_rel"],
        rhs_norm=float((P.rhs() ** 2).sum() ** 0.5),
    )


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "p2_n8_oracle.json"), "w") as f:
        json.dump(p2_n8(), f, indent=1)
        f.write("\n")
