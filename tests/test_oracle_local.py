"""Pins of the oracle's local Robin / Dirichlet operators (Eq. 5-6, Eq. 11-12, Eq. 15)."""

import numpy as np
import pytest

from oracle import grid
from oracle.local import BoxOperator, robin_face
from paper_2606_08883_gb300 import workloads as W


def _setup(dim=2, seed=0):
    n = (12, 10, 1) if dim == 2 else (6, 6, 4)
    prob = W.random_problem(n, dim=dim, seed=seed, contrast=1e3)
    T = grid.transmissibilities(prob.K, prob.h, dim, prob.bc_kind)
    return prob, T


@pytest.mark.parametrize("dim", [2, 3])
def test_dirichlet_restriction_is_submatrix_of_A(dim):
    prob, T = _setup(dim)
    A = grid.dense_matrix(T, dim, prob.K.shape)
    n = [prob.K.shape[2], prob.K.shape[1], prob.K.shape[0]]
    lo, hi = ((1, 2, 0), (5, 7, 1)) if dim == 2 else ((1, 1, 1), (4, 5, 3))
    op = BoxOperator(prob.K, T, prob.h, dim, n, lo, hi, False, 10.0, (4, 5, 2))
    cells = [i + n[0] * (j + n[1] * k) for k in range(lo[2], hi[2]) for j in range(lo[1], hi[1]) for i in range(lo[0], hi[0])]
    assert np.allclose(op.dense(), A[np.ix_(cells, cells)], rtol=0, atol=1e-13 * np.abs(A).max())


def test_robin_coefficient_satisfies_robin_condition_and_limits():
    prob, T = _setup()
    a, inside, outside = 0, (4, 3, 0), (5, 3, 0)
    tau, beta, t_r, area = robin_face(prob.K, prob.h, a, inside, outside, 10.0, (4, 5, 1))
    # Eq. 6: beta = alpha H / K_H with K_H the harmonic mean, H the subdomain edge along the normal
    k1, k2 = prob.K[0, 3, 4], prob.K[0, 3, 5]
    assert np.isclose(beta, 10.0 * 4 * prob.h[0] * (k1 + k2) / (2 * k1 * k2), rtol=1e-14)
    # Eq. 5: with F = t_R (p_c - lambda), the face pressure p_c - F/tau and velocity F/|f| obey
    # -beta u + p = lambda
    p_c, lam = 0.37, -1.2
    F = t_r * (p_c - lam)
    assert np.isclose(-beta * F / area + (p_c - F / tau), lam, rtol=1e-13)
    # alpha -> 0: Dirichlet data at the face (t_R -> tau); alpha -> inf: no flow (t_R -> 0)
    _, _, t0, _ = robin_face(prob.K, prob.h, a, inside, outside, 1e-14, (4, 5, 1))
    _, _, t8, _ = robin_face(prob.K, prob.h, a, inside, outside, 1e14, (4, 5, 1))
    assert np.isclose(t0, tau, rtol=1e-10) and t8 < 1e-10 * tau


def test_robin_box_solution_mass_balance_and_dense_solve():
    prob, T = _setup(seed=4)
    n = [12, 10, 1]
    lo, hi = (2, 1, 0), (9, 10, 1)   # touches the +y (Neumann) boundary, Robin elsewhere
    op = BoxOperator(prob.K, T, prob.h, 2, n, lo, hi, True, 10.0, (4, 5, 1))
    rng = np.random.default_rng(1)
    src = rng.standard_normal(op.n_loc)
    lam = {i: rng.standard_normal() for i in range(len(op.robin_faces))}
    rhs = src.copy()
    for i, (side, li, tau, beta, t_r, area, t_f) in enumerate(op.robin_faces):
        rhs[li] += t_r * lam[i]
    x = op.solve(rhs)
    assert np.allclose(x, np.linalg.solve(op.dense(), rhs), rtol=1e-11, atol=1e-11)
    # per-cell mass balance: net outflow through every face equals the source
    w = op.w
    X = x.reshape(w[2], w[1], w[0])
    out = np.zeros_like(X)
    for a in range(2):
        Ta = T[a][:, lo[1]:hi[1] + (a == 1), lo[0]:hi[0] + (a == 0)]
        ax = grid.np_axis(a)
        Xp = np.concatenate([np.zeros_like(grid.take(X, a, slice(0, 1))), X,
                             np.zeros_like(grid.take(X, a, slice(0, 1)))], axis=ax)
        F = Ta * (grid.take(Xp, a, slice(0, w[a] + 1)) - grid.take(Xp, a, slice(1, w[a] + 2)))
        out += grid.take(F, a, slice(1, w[a] + 1)) - grid.take(F, a, slice(0, w[a]))
    out = out.ravel()
    # replace the flux through Robin faces (computed above as T_f x_c) by t_R (x_c - lambda)
    for i, (side, li, tau, beta, t_r, area, t_f) in enumerate(op.robin_faces):
        out[li] += t_r * (x[li] - lam[i]) - t_f * x[li]
    assert np.allclose(out, src, rtol=0, atol=1e-10 * np.abs(src).max())
