"""Pins of the oracle's restarted right-preconditioned GMRES (Algorithm 1) and of the
approximate-inverse framework of Appendix A."""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import grid
from oracle.gmres import fgmres, NOT_CONVERGED
from oracle.mrcm import MRCMOS
from oracle.solve import solve
from paper_2606_08883_gb300 import workloads as W


def _tiny(seed=1, l=1, smooth=0, contrast=1e3, n=(12, 12, 1), sub=(4, 4, 1)):
    prob = W.random_problem(n, seed=seed, contrast=contrast)
    pre = MRCMOS(prob.K, prob.h, 2, prob.bc_kind, sub, l, smooth, 10.0)
    A = grid.dense_matrix(pre.T, 2, pre.shape)
    N = A.shape[0]
    Tm = np.column_stack([pre.apply(np.eye(N)[:, j].reshape(pre.shape)).ravel() for j in range(N)])
    b = grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f).ravel()
    return prob, pre, A, Tm, b


def test_history_matches_textbook_gmres_on_explicit_AT():
    prob, pre, A, Tm, b = _tiny()
    AT = A @ Tm
    m = 5
    p, info = fgmres(lambda v: A @ v, lambda v: Tm @ v, b, tol=1e-10, m=m, max_iter=m, check_every_step=False)
    ref = []
    spla.gmres(AT, b, rtol=1e-30, atol=0.0, restart=m, maxiter=1, callback=lambda r: ref.append(r),
               callback_type="pr_norm")
    ours = np.array(info["history"][1:m + 1]) / np.linalg.norm(b)
    assert len(ref) >= m
    assert np.allclose(ours, ref[:m], rtol=1e-7, atol=1e-14)


def test_minimal_residual_property_within_a_cycle():
    prob, pre, A, Tm, b = _tiny(seed=3, l=2, smooth=1)
    E = np.eye(A.shape[0]) - A @ Tm
    hist = []
    for j in range(1, 6):
        p, info = fgmres(lambda v: A @ v, lambda v: Tm @ v, b, tol=1e-30, m=j, max_iter=j)
        hist.append(np.linalg.norm(b - A @ p))
        # GMRES minimises over all degree-j polynomials, including (1 - z)^j
        assert hist[-1] <= np.linalg.norm(np.linalg.matrix_power(E, j) @ b) * (1 + 1e-10) + 1e-14
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


def test_converged_solution_matches_direct_solve():
    prob = W.random_problem((16, 16, 1), seed=5, contrast=1e4)
    p, info, pre = solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=(4, 4, 1), l=2,
                         smooth_steps=1, alpha=10.0, tol=1e-10, restart=10)
    A = grid.dense_matrix(pre.T, 2, pre.shape)
    b = info["b"].ravel()
    x = np.linalg.solve(A, b)
    assert info["status"] == 0 and info["rel_res"] <= 1e-10
    assert np.isclose(info["abs_res"], np.linalg.norm(b - A @ p.ravel()), rtol=1e-6)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(p.ravel() - x) <= cond * 1e-10 * np.linalg.norm(x)


def test_single_subdomain_converges_in_one_iteration():
    prob = W.random_problem((10, 10, 1), seed=6, contrast=1e3)
    p, info, pre = solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=(10, 10, 1), l=0,
                         smooth_steps=0, tol=1e-12, restart=10)
    assert info["iterations"] == 1 and info["restarts"] == 0 and info["rel_res"] <= 1e-12


def test_not_converged_and_zero_rhs():
    prob, pre, A, Tm, b = _tiny(seed=7)
    p, info = fgmres(lambda v: A @ v, lambda v: Tm @ v, b, tol=1e-14, m=10, max_iter=1)
    assert info["status"] == NOT_CONVERGED and info["iterations"] == 1
    assert np.linalg.norm(b - A @ p) < np.linalg.norm(b)
    p0, info0 = fgmres(lambda v: A @ v, lambda v: Tm @ v, np.zeros_like(b), tol=1e-8)
    assert info0["iterations"] == 0 and not p0.any()


def test_restart_reuses_iterate():
    prob, pre, A, Tm, b = _tiny(seed=8, l=0, smooth=0)
    p_full, info_full = fgmres(lambda v: A @ v, lambda v: Tm @ v, b, tol=1e-9, m=3, max_iter=200)
    assert info_full["status"] == 0 and info_full["restarts"] >= 1
    # resuming from a saved iterate is a restart: the first cycle of the resumed run starts there
    p_half, info_half = fgmres(lambda v: A @ v, lambda v: Tm @ v, b, tol=1e-9, m=3, max_iter=3)
    p_res, info_res = fgmres(lambda v: A @ v, lambda v: Tm @ v, b, p0=p_half, tol=1e-9, m=3, max_iter=200)
    assert info_res["iterations"] + 3 == info_full["iterations"]
    assert np.allclose(p_res, p_full, rtol=1e-10, atol=1e-12)


def _energy_eps(A, Tm):
    w, U = np.linalg.eigh(A)
    Ah = (U * np.sqrt(w)) @ U.T
    Aih = (U / np.sqrt(w)) @ U.T
    return np.linalg.norm(np.eye(A.shape[0]) - Ah @ (A @ Tm) @ Aih, 2)


def test_oversampling_brings_the_energy_contraction_below_one():
    # Appendix A's assumption ||I - A T||_A < 1 holds for MRCM-OS with one sweep on this field,
    # and it is the oversampling that gives it: the same sweep after the non-overlapping MRCM
    # (l = 0), or the oversampled MRCM without a sweep, leave ||I - A T||_A above one
    assert _energy_eps(*_tiny(seed=9, l=2, smooth=1, contrast=10.0)[2:4]) < 0.6
    assert _energy_eps(*_tiny(seed=9, l=0, smooth=1, contrast=10.0)[2:4]) > 1.0
    assert _energy_eps(*_tiny(seed=9, l=2, smooth=0, contrast=10.0)[2:4]) > 1.0


@pytest.mark.parametrize("smooth", [1, 2])
def test_appendix_a_energy_norm_bound(smooth):
    # Appendix A: if ||I - A T||_A = eps < 1, GMRES on the transformed system reduces its residual
    # at least by eps per step.  Checked with a textbook GMRES on B = A^1/2 (A T) A^-1/2.
    prob, pre, A, Tm, b = _tiny(seed=9, l=2, smooth=smooth, contrast=10.0)
    w, U = np.linalg.eigh(A)
    Ah = (U * np.sqrt(w)) @ U.T
    Aih = (U / np.sqrt(w)) @ U.T
    B = Ah @ (A @ Tm) @ Aih
    eps = np.linalg.norm(np.eye(len(b)) - B, 2)
    assert eps < 1.0
    bt = Ah @ b
    res = [np.linalg.norm(bt)]
    spla.gmres(B, bt, rtol=1e-30, atol=0.0, restart=6, maxiter=1,
               callback=lambda r: res.append(r * np.linalg.norm(bt)), callback_type="pr_norm")
    for m in range(1, 6):
        assert res[m] <= eps ** m * res[0] * (1 + 1e-8)
    # the same eps bounds the similar matrix's spectrum: |lambda - 1| <= eps
    lam = sla.eigvals(A @ Tm)
    assert np.abs(lam - 1.0).max() <= eps * (1 + 1e-8)
