"""Writes tests/golden/oracle_small_problems.json from the FP64 oracle only
(oracle/ and the seeded generators in gen/): regression values of small
problems that the CPU tests re-check. Run from the repository root:

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.abspath(os.path.join(HERE, "..", "..")))

import gen  # noqa: E402
import oracle  # noqa: E402
from oracle import nlp as ON  # noqa: E402


def values():
    out = {}
    lp = gen.random_lp(2000, 1000, 5, seed=0)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, gen.lp_ordering(lp))
    r = oracle.ipm_lp(S, lp, tol=1e-8)
    out["random_lp_2000x1000_seed0"] = {"objective": r["objective"], "iterations": r["iterations"],
                                        "nnz_l": int(S.nnz_l), "nsuper": int(S.nsuper)}
    lp = gen.grid_lp(8, seed=1)
    S = oracle.analyze(lp.n, lp.m, lp.rowptr, lp.col, gen.nd_order_grid3d(8))
    r = oracle.ipm_lp(S, lp, tol=1e-8)
    out["grid_lp_8_seed1"] = {"objective": r["objective"], "iterations": r["iterations"],
                              "nnz_l": int(S.nnz_l), "nsuper": int(S.nsuper), "flops": S.flops}
    P = gen.grid_nlp(12, seed=6)
    S = oracle.analyze(P.n, P.m, P.rowptr, P.col, gen.nd_order_grid_nlp(12), P.wp, P.wi)
    r = ON.ipm_grid_nlp(S, P, tol=1e-8)
    out["grid_nlp_12_seed6"] = {"objective": r["objective"], "iterations": r["iterations"]}
    return out


if __name__ == "__main__":
    v = values()
    with open(os.path.join(HERE, "oracle_small_problems.json"), "w") as f:
        json.dump(v, f, indent=1, sort_keys=True)
    print(json.dumps(v, indent=1))
