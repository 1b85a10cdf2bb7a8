"""The paper's analytic experiments (Sec. 4.1, Tables 2-3) on the GPU path: iteration counts equal
the FP64 oracle's (stored by tests/golden/make_replication.py).  The paper's own counts are kept in
tests/golden/paper_tables_2_3.json for the side-by-side report; they depend on interface-space and
smoothing details the paper leaves to its references, so they are context, not a parity target."""

import json
import os

import pytest

from paper_2606_08883_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    gold = json.load(open(os.path.join(HERE, "golden", "replication_oracle_256.json")))["results"]
    out = []
    for key, r in gold.items():
        if r["sub"] + 2 * r["l"] <= 64:   # box width the GPU path implements
            out.append((key, r))
    return out


def test_replication_iterations_match_oracle():
    from paper_2606_08883_gb300 import mrcm
    cases = _cases()
    assert len(cases) >= 29
    probs = {False: W.analytic(256, False)[0], True: W.analytic(256, True)[0]}
    exact = 0
    for key, r in cases:
        kind, name, part = key.split("|")
        prob = probs[kind == "variable"]
        q = W.Params(sub=(r["sub"], r["sub"], 1), oversample=r["l"], smooth_steps=r["s"], alpha=10.0, tol=1e-8,
                     tol_relative=0, restart=10, max_iter=400)
        s = mrcm.Solver(prob, q)
        s.factor()
        p, info = s.solve(allow_not_converged=True)
        s.close()
        assert abs(info["iterations"] - r["iterations"]) <= 1, (key, info["iterations"], r["iterations"])
        assert (info["status"] == 0) == r["converged"], key
        exact += info["iterations"] == r["iterations"]
    # a difference of one is only allowed where the residual estimate sits at the tolerance
    assert exact >= len(cases) - 2
