"""Writes tests/golden/replication_oracle_256.json: the FP64 oracle on the Sec. 4.1 analytic
problems (Tables 2-3 settings) -- iterations (applications of T, per-step stopping test), restart
cycles and final residual of GMRES(10) to ||b - A p|| <= 1e-8 for every partition and setting.

Calls only oracle/ and the input generators.  Run from the repository root:
    python tests/golden/make_replication.py
"""

import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2606_08883_gb300 import workloads as W  # noqa: E402


def main():
    paper = json.load(open(os.path.join(HERE, "paper_tables_2_3.json")))
    out = {"generator": "tests/golden/make_replication.py (FP64 oracle, per-step Givens check, absolute tol 1e-8, "
                        "GMRES(10), alpha 10, max_iter 400)", "N": 256, "results": {}}
    for variable, key in ((False, "constant"), (True, "variable")):
        prob, _exact = W.analytic(256, variable)
        for name, (l, s) in paper["settings"].items():
            for part in paper["partitions"]:
                m = int(part.split("x")[0])
                sub = 256 // m
                p, info, _ = oracle.solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=(sub, sub, 1), l=l,
                                          smooth_steps=s, alpha=10.0, tol=1e-8, tol_relative=False, restart=10,
                                          max_iter=400)
                it = info["iterations"]
                out["results"][f"{key}|{name}|{part}"] = {
                    "iterations": it, "cycles": math.ceil(it / 10), "abs_res": info["abs_res"],
                    "converged": info["status"] == 0, "sub": sub, "l": l, "s": s}
                print(key, name, part, it, f"{info['abs_res']:.2e}", flush=True)
    with open(os.path.join(HERE, "replication_oracle_256.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
