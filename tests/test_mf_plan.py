"""Host checks of the nested-dissection plan of the multifrontal coupling factorisation (no GPU).

The plan (plan.cpp) orders the coupling unknowns of Eq. 13-14 by a recursive bisection of the
subdomain grid.  Pinned here against the FP64 oracle's coupling matrix G:
* every unknown is eliminated by exactly one front, a front's update unknowns are eliminated by its
  ancestors, and a child's update set lies inside its parent's front;
* every structural nonzero of G is assembled exactly once, by a front that holds its row and column;
* a multifrontal LU written here in numpy on the plan's fronts (Schur complements added into the
  parent, explicit inverses of the pivot blocks) solves the oracle's G to rounding.
"""

import numpy as np
import pytest

from oracle.mrcm import MRCMOS
from paper_2606_08883_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_2606_08883_gb300 import build
    build.build()
    from paper_2606_08883_gb300 import mrcm
    return mrcm


CASES = {
    # cells, subdomain size, oversampling, interface degree
    "grid-16x16": ((64, 64, 1), (4, 4, 1), 1, 0),
    "ragged-12x9": ((58, 35, 1), (5, 4, 1), 1, 0),
    "strip-16x1": ((128, 8, 1), (8, 8, 1), 2, 0),
    "degree1-8x8": ((48, 48, 1), (6, 6, 1), 2, 1),
}


def _home_ordered_G(pre):
    """The oracle's G with row i the row homed at unknown i (the flux row of interface e at the
    lower subdomain's +a side, the pressure row at the upper one's -a side), as the library orders it."""
    P, nq = pre.part, pre.nq
    G = np.zeros_like(pre.G)
    for e, (a, s, s2) in enumerate(P.interfaces):
        for q in range(nq):
            cf = pre.coff[s] + pre.subs[s].funcs.index((2 * a + 1, q))
            cp = pre.coff[s2] + pre.subs[s2].funcs.index((2 * a, q))
            G[cf] = pre.G[2 * nq * e + q]
            G[cp] = pre.G[2 * nq * e + nq + q]
    return G


def _setup(name):
    n, sub, l, deg = CASES[name]
    prob = W.random_problem(n, seed=5, contrast=1e2)
    q = W.Params(sub=sub, oversample=l, smooth_steps=1, iface_degree=deg)
    pre = MRCMOS(prob.K, prob.h, prob.dim, prob.bc_kind, q.sub, q.oversample, q.smooth_steps, q.alpha, deg)
    return prob, q, pre


@pytest.mark.parametrize("name", list(CASES))
def test_plan_eliminates_every_unknown_once_and_assembles_every_entry_once(lib, name):
    prob, q, pre = _setup(name)
    plan = lib.plan_mf_export(prob, q)
    assert plan["used"] and plan["NC"] == pre.n_coarse
    fr = plan["fronts"]
    piv = np.concatenate([f["unknowns"][:f["np"]] for f in fr])
    assert np.array_equal(np.sort(piv), np.arange(plan["NC"]))
    owner = np.empty(plan["NC"], dtype=int)
    for i, f in enumerate(fr):
        owner[f["unknowns"][:f["np"]]] = i
    for i, f in enumerate(fr):
        for c in f["children"]:
            assert fr[c]["parent"] == i and fr[c]["level"] < f["level"]
            assert set(fr[c]["unknowns"][fr[c]["np"]:]) <= set(f["unknowns"])
        # update unknowns belong to ancestors
        anc, p = set(), f["parent"]
        while p >= 0:
            anc.add(p)
            p = fr[p]["parent"]
        assert all(owner[u] in anc for u in f["unknowns"][f["np"]:])
    G = _home_ordered_G(pre)
    rows, cols = np.nonzero(G)
    want = set(zip(rows.tolist(), cols.tolist()))
    got = [tuple(e) for f in fr for e in f["entries"].tolist()]
    assert len(got) == len(set(got))          # each entry once
    assert want <= set(got)                   # every nonzero (the rest are structural zeros)
    for f in fr:
        us = set(f["unknowns"].tolist())
        assert all(r in us and c in us for r, c in f["entries"].tolist())


@pytest.mark.parametrize("name", list(CASES))
def test_multifrontal_elimination_on_the_plan_solves_the_oracle_G(lib, name):
    prob, q, pre = _setup(name)
    plan = lib.plan_mf_export(prob, q)
    G = _home_ordered_G(pre)
    fr = plan["fronts"]
    S = {}
    fac = []
    for i, f in enumerate(fr):
        idx = f["unknowns"]
        npv = f["np"]
        pos = {u: k for k, u in enumerate(idx.tolist())}
        F = np.zeros((len(idx), len(idx)))
        for r, c in f["entries"].tolist():
            F[pos[r], pos[c]] = G[r, c]
        for c in f["children"]:
            uc, Sc = S.pop(c)
            m = [pos[u] for u in uc]
            F[np.ix_(m, m)] += Sc
        A11inv = np.linalg.inv(F[:npv, :npv])
        D = A11inv @ F[:npv, npv:]
        B = F[npv:, :npv] @ A11inv
        S[i] = (idx[npv:].tolist(), F[npv:, npv:] - F[npv:, :npv] @ D)
        fac.append((idx, npv, A11inv, B, D))
    rhs = np.random.default_rng(3).standard_normal(plan["NC"])
    keep, w = {}, {}
    for i, (idx, npv, A11inv, B, D) in enumerate(fac):
        v = np.zeros(len(idx))
        v[:npv] = rhs[idx[:npv]]
        pos = {u: k for k, u in enumerate(idx.tolist())}
        for c in fr[i]["children"]:
            uc, wc = w.pop(c)
            for u, val in zip(uc, wc):
                v[pos[u]] += val
        keep[i] = v[:npv]
        w[i] = (idx[npv:].tolist(), v[npv:] - B @ v[:npv])
    x = np.zeros(plan["NC"])
    for i in reversed(range(len(fac))):
        idx, npv, A11inv, B, D = fac[i]
        x[idx[:npv]] = A11inv @ keep[i] - D @ x[idx[npv:]]
    ref = np.linalg.solve(G, rhs)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-11


def test_band_factorisation_reports_no_plan(lib):
    prob, q, pre = _setup("grid-16x16")
    q.coarse_solver = 1
    assert not lib.plan_mf_export(prob, q)["used"]
