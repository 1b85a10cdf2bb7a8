"""GPU parity: every stage of the CUDA path against the FP64 oracle on the same seeded inputs,
called through the C ABI.

Tolerances (FP64 path): transmissibilities and b are the same closed formulas evaluated in a
different association order, so they agree to a few ulps (1e-14 relative).  The local solves,
coupling solve and Krylov recurrences use different (but backward-stable) elimination orders
(block-line Cholesky and band LU on the GPU, LAPACK band Cholesky and dense LU in the oracle), so
agreement is bounded by eps times the condition numbers involved: 1e-10 relative L2 on the
moderate-contrast fields (K spread 1e3) used here, with iteration counts equal.
"""

import numpy as np
import pytest
import torch

from oracle import grid
from oracle.mrcm import MRCMOS
from oracle.solve import solve as oracle_solve
from paper_2606_08883_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrcm():
    from paper_2606_08883_gb300 import mrcm as m
    return m


def _rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _oracle(prob, q):
    return MRCMOS(prob.K, prob.h, prob.dim, prob.bc_kind, q.sub, q.oversample, q.smooth_steps, q.alpha,
                  q.iface_degree)


CASES = {
    "mrcm-48x40": (dict(n=(48, 40, 1), seed=1), dict(sub=(8, 8, 1), oversample=0, smooth_steps=0)),
    "os-48x40": (dict(n=(48, 40, 1), seed=2), dict(sub=(8, 8, 1), oversample=2, smooth_steps=1)),
    "os-96x64-l4s2": (dict(n=(96, 64, 1), seed=3), dict(sub=(16, 16, 1), oversample=4, smooth_steps=2)),
    "ragged-60x36": (dict(n=(60, 36, 1), seed=4), dict(sub=(12, 9, 1), oversample=3, smooth_steps=1)),
    "single-32": (dict(n=(32, 32, 1), seed=5), dict(sub=(32, 32, 1), oversample=0, smooth_steps=1)),
    "widest-64": (dict(n=(64, 64, 1), seed=6), dict(sub=(32, 32, 1), oversample=16, smooth_steps=1)),
    "stripes-128x64": (dict(n=(128, 64, 1), seed=7), dict(sub=(4, 32, 1), oversample=3, smooth_steps=1)),
    "dirichlet-all": (dict(n=(48, 48, 1), seed=8, bc_kind=[0, 0, 0, 0, 1, 1]),
                      dict(sub=(16, 12, 1), oversample=2, smooth_steps=2)),
    "neumann-data": (dict(n=(40, 40, 1), seed=9, bc_kind=[0, 1, 1, 0, 1, 1]),
                     dict(sub=(10, 8, 1), oversample=1, smooth_steps=1)),
    # grids the subdomain size does not divide: the last subdomain of each row / column is shorter
    "uneven-61x45": (dict(n=(61, 45, 1), seed=10), dict(sub=(16, 12, 1), oversample=3, smooth_steps=1)),
    "uneven-50x37-l0": (dict(n=(50, 37, 1), seed=11, bc_kind=[0, 1, 0, 1, 1, 1]),
                        dict(sub=(16, 12, 1), oversample=0, smooth_steps=1)),
    "uneven-40x20-tall": (dict(n=(40, 20, 1), seed=12), dict(sub=(16, 32, 1), oversample=2, smooth_steps=2)),
    # one row / one column of subdomains (interfaces along one axis only), the largest oversampling
    # a subdomain allows (l = sub - 1), and boxes of a few cells
    "strip-96x12": (dict(n=(96, 12, 1), seed=13), dict(sub=(12, 12, 1), oversample=3, smooth_steps=1)),
    "column-12x96": (dict(n=(12, 96, 1), seed=16, bc_kind=[1, 1, 0, 0, 1, 1]),
                     dict(sub=(12, 16, 1), oversample=2, smooth_steps=1)),
    "max-oversample-48": (dict(n=(48, 48, 1), seed=14), dict(sub=(8, 8, 1), oversample=7, smooth_steps=1)),
    "tiny-boxes-8x8": (dict(n=(8, 8, 1), seed=15, bc_kind=[0, 0, 0, 0, 1, 1]),
                       dict(sub=(4, 4, 1), oversample=1, smooth_steps=2)),
}


def _case(name):
    pk, qk = CASES[name]
    prob = W.random_problem(pk["n"], seed=pk["seed"], contrast=1e3, bc_kind=pk.get("bc_kind"))
    q = W.Params(**qk)
    q.tol = 1e-10
    return prob, q


@pytest.mark.parametrize("name", ["os-48x40", "ragged-60x36", "dirichlet-all", "neumann-data", "uneven-61x45"])
def test_transmissibilities_rhs_operator(mrcm, name):
    prob, q = _case(name)
    s = mrcm.Solver(prob, q)
    s.factor()
    T = grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind)
    tr = s.debug(mrcm.MRCM_DBG_TRANS)
    nx, ny = prob.n[0], prob.n[1]
    assert _rel(tr[:(nx + 1) * ny], T[0]) < 1e-14
    assert _rel(tr[(nx + 1) * ny:], T[1]) < 1e-14
    b = grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f)
    assert _rel(s.rhs().cpu().numpy(), b) < 1e-14
    v = np.random.default_rng(0).standard_normal(prob.K.shape)
    w = s.apply_operator(torch.as_tensor(v.ravel(), device="cuda")).cpu().numpy()
    assert _rel(w, grid.matvec(T, v, 2)) < 1e-13


def _phi_gpu_layout(pre, s_idx, smax):
    """Oracle phi of subdomain s in the library layout [4 nq functions][4 sides][smax], function
    r nq + q the degree-q function of side r."""
    d = pre.subs[s_idx]
    nq = pre.nq
    out = np.zeros((4 * nq, 4, smax))
    for jj, (r, qd) in enumerate(d.funcs):
        off = 0
        for k in d.sides:
            ln = int((d.gamma_side == k).sum())
            out[r * nq + qd, k, :ln] = d.phi[jj, off:off + ln]
            off += ln
    return out


# degree 1: piecewise-linear multiplier and test spaces on every Robin side (two functions a side)
@pytest.mark.parametrize("name,degree", [("os-48x40", 0), ("os-96x64-l4s2", 0), ("ragged-60x36", 0),
                                         ("mrcm-48x40", 0), ("stripes-128x64", 0), ("uneven-61x45", 0),
                                         ("uneven-50x37-l0", 0), ("os-48x40", 1), ("ragged-60x36", 1),
                                         ("mrcm-48x40", 1), ("uneven-61x45", 1)])
def test_informed_spaces_basis_moments_and_coupling_matrix(mrcm, name, degree):
    prob, q = _case(name)
    q.iface_degree = degree
    s = mrcm.Solver(prob, q)
    s.factor()
    pre = _oracle(prob, q)
    P = pre.part
    nq = pre.nq
    assert nq == 1 + degree
    smax = max(q.sub[0], q.sub[1])
    phi = s.debug(mrcm.MRCM_DBG_PHI).reshape(P.S, 4 * nq, 4, smax)
    psi = s.debug(mrcm.MRCM_DBG_PSI).reshape(4 * nq, -1)
    mom = s.debug(mrcm.MRCM_DBG_MOMENTS).reshape(P.S, 4, 4 * nq, nq, 2)
    ref_phi = np.stack([_phi_gpu_layout(pre, i, smax) for i in range(P.S)])
    assert _rel(phi, ref_phi) < 1e-11
    nx = prob.n[0]
    for d in pre.subs:
        lo, hi = P.box[d.s, 0], P.box[d.s, 1]
        cells = (np.arange(lo[1], hi[1])[:, None] * nx + np.arange(lo[0], hi[0])[None, :]).ravel()
        for jj, (r, qd) in enumerate(d.funcs):
            fn = r * nq + qd
            assert _rel(psi[fn, cells], d.psi[:, jj]) < 1e-10
            for k in d.sides:
                for qt in range(nq):
                    assert np.isclose(mom[d.s, k, fn, qt, 0], d.Fbar[k, qt, jj], rtol=1e-9,
                                      atol=1e-12 * np.abs(d.Fbar).max())
                    assert np.isclose(mom[d.s, k, fn, qt, 1], d.Pbar[k, qt, jj], rtol=1e-9,
                                      atol=1e-12 * np.abs(d.Pbar).max())
    G = s.debug(mrcm.MRCM_DBG_G).reshape(P.E2 * nq, P.E2 * nq)
    assert _rel(G, pre.G) < 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_apply_precond_matches_oracle(mrcm, name):
    prob, q = _case(name)
    s = mrcm.Solver(prob, q)
    s.factor()
    s.debug(mrcm.MRCM_DBG_ZMRCM, enable_only=True)
    pre = _oracle(prob, q)
    rng = np.random.default_rng(11)
    for trial in range(2):
        r = rng.standard_normal(prob.K.shape)
        z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
        parts = pre.apply_parts(r)
        assert _rel(s.debug(mrcm.MRCM_DBG_COARSE), parts["c"]) < 1e-9 if pre.part.E2 else True
        assert _rel(s.debug(mrcm.MRCM_DBG_ZMRCM), parts["z_mrcm"]) < 1e-10
        assert _rel(z, parts["z"]) < 1e-10, (name, trial, _rel(z, parts["z"]))


@pytest.mark.parametrize("name", ["os-48x40", "os-96x64-l4s2", "ragged-60x36", "dirichlet-all", "uneven-61x45"])
def test_multiplicative_smoothing_matches_oracle(mrcm, name):
    # the multicolour sweep: one launch per colour over that colour's boxes, z updated in place
    prob, q = _case(name)
    q.smooth_kind = 1
    s = mrcm.Solver(prob, q)
    s.factor()
    pre = MRCMOS(prob.K, prob.h, prob.dim, prob.bc_kind, q.sub, q.oversample, q.smooth_steps, q.alpha, 0, 1)
    add = MRCMOS(prob.K, prob.h, prob.dim, prob.bc_kind, q.sub, q.oversample, q.smooth_steps, q.alpha, 0, 0)
    rng = np.random.default_rng(31)
    for trial in range(2):
        r = rng.standard_normal(prob.K.shape)
        z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
        ref = pre.apply(r)
        assert _rel(z, ref) < 1e-10, (name, trial, _rel(z, ref))
        assert _rel(add.apply(r), ref) > 1e-6  # the two sweeps really differ on this case
    s.close()


def test_multiplicative_smoothing_gmres_matches_oracle(mrcm):
    prob, q = _case("os-96x64-l4s2")
    q.smooth_kind, q.tol, q.restart = 1, 1e-9, 30
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve()
    p_ref, info_ref, _ = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                      l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                      tol_relative=True, restart=q.restart, max_iter=q.max_iter, smooth_kind=1)
    assert info["status"] == 0 and info["iterations"] == info_ref["iterations"]
    assert _rel(p.cpu().numpy(), p_ref) < 1e-10
    s.close()


# Short restarts (4, 8) cover the restart path; GMRES(30) is the workloads' setting.  The last case
# is the non-overlapping MRCM followed by a sweep: without oversampling the sweep does not make
# I - A T a contraction (Appendix A), GMRES(30) stagnates there, and it takes a Krylov dimension
# it never reaches.
@pytest.mark.parametrize("name,restart", [("os-96x64-l4s2", 4), ("mrcm-48x40", 8), ("dirichlet-all", 4),
                                          ("os-48x40", 30), ("ragged-60x36", 30), ("uneven-61x45", 30),
                                          ("uneven-50x37-l0", 100)])
def test_gmres_matches_oracle(mrcm, name, restart):
    prob, q = _case(name)
    q.tol = 1e-9
    q.restart = restart
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve(fluxes=True)
    p_ref, info_ref, pre = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                        l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                        tol_relative=True, restart=q.restart, max_iter=q.max_iter)
    assert info["status"] == 0 and info["rel_res"] <= q.tol
    assert info["iterations"] == info_ref["iterations"]
    assert info["restarts"] == info_ref["restarts"]
    if restart < 30:
        assert info["restarts"] > 0
    assert _rel(p.cpu().numpy(), p_ref) < 1e-10
    hist_ref = np.array(info_ref["history"])
    assert len(info["history"]) == len(hist_ref)
    assert np.allclose(info["history"], hist_ref, rtol=1e-6, atol=1e-12 * hist_ref[0])
    ux, uy = info["u"]
    assert _rel(ux.cpu().numpy(), info_ref["u"][0]) < 1e-10
    assert _rel(uy.cpu().numpy(), info_ref["u"][1]) < 1e-10


def test_fp32_local_solves_reach_fp64_tolerance(mrcm):
    prob, q = _case("os-96x64-l4s2")
    q.tol = 1e-8
    q.restart = 30
    p_ref, info_ref, _ = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                      l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                      restart=q.restart)
    q.local_prec = W.PREC_FP32
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve()
    assert info["status"] == 0 and info["rel_res"] <= 1e-8
    assert info["iterations"] <= info_ref["iterations"] + 1
    assert _rel(p.cpu().numpy(), p_ref) < 1e-6


def test_edge_cases(mrcm):
    prob, q = _case("single-32")
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve()
    assert info["iterations"] == 1 and info["rel_res"] <= q.tol
    zero = torch.zeros(prob.cells, dtype=torch.float64, device="cuda")
    p0, info0 = s.solve(b=zero)
    assert info0["iterations"] == 0 and float(p0.abs().max()) == 0.0
    prob, q = _case("os-48x40")
    q.max_iter = 1
    q.tol = 1e-14
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve(allow_not_converged=True)
    assert info["status"] == mrcm.MRCM_ERR_NOT_CONVERGED and info["iterations"] == 1
    with pytest.raises(mrcm.MRCMError) as ei:
        s.solve()
    assert ei.value.status == mrcm.MRCM_ERR_NOT_CONVERGED
    bad = W.random_problem((48, 40, 1), seed=3)
    bad.K = bad.K.copy()
    bad.K[0, 3, 5] = -1.0
    s = mrcm.Solver(bad, q)
    with pytest.raises(mrcm.MRCMError) as ei:
        s.factor()
    assert ei.value.status == mrcm.MRCM_ERR_INVALID_ARG
    with pytest.raises(mrcm.MRCMError) as ei:
        s.apply_precond(torch.zeros(bad.cells, dtype=torch.float64, device="cuda"))
    assert ei.value.status == mrcm.MRCM_ERR_INVALID_ARG


def test_workspace_too_small_and_deterministic(mrcm):
    import ctypes as C
    prob, q = _case("os-48x40")
    need = mrcm.footprint(prob, q)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    K = torch.as_tensor(prob.K.ravel(), device="cuda")
    p = mrcm.make_problem(prob, K.data_ptr())
    pq = mrcm.make_params(q)
    h = C.c_void_p()
    rc = mrcm.mrcm_setup(C.byref(p), C.byref(pq), C.c_void_p(ws.data_ptr()), need - 256, None, C.byref(h))
    assert rc == mrcm.MRCM_ERR_OOM
    s = mrcm.Solver(prob, q)
    s.factor()
    a, _ = s.solve()
    b, _ = s.solve()
    assert torch.equal(a, b)


def test_profile_records_only_the_selected_phases(mrcm):
    """Per-phase event timing restricted to one phase: that phase alone carries launches and time,
    and the solution is the unprofiled one."""
    prob, q = _case("os-48x40")
    s = mrcm.Solver(prob, q)
    s.factor()
    ref, _ = s.solve()
    s.profile(True, phases=["schwarz"])
    s.factor()
    got, _ = s.solve()
    prof = s.profile_read(reset=True)
    assert torch.equal(got, ref)
    assert prof["schwarz"][1] > 0 and prof["schwarz"][0] > 0.0
    assert all(v == (0.0, 0) for k, v in prof.items() if k != "schwarz"), prof
    n_all = prof["schwarz"][1]
    s.profile(True, phases=["schwarz"], every=4)   # occurrences 0, 4, 8, ... of the phase
    s.factor()
    s.solve()
    prof = s.profile_read(reset=True)
    assert prof["schwarz"][1] == (n_all + 3) // 4   # one launch per additive sweep
    s.profile(True)
    s.factor()
    s.solve()
    prof = s.profile_read(reset=True)
    s.profile(False)
    for k in ("factor_ohat_robin", "factor_omega", "informed", "basis", "particular", "schwarz", "krylov"):
        assert prof[k][1] > 0, k


def test_full_size_channels_512_matches_oracle(mrcm):
    """The 512 x 512 channelised workload (contrast 1e6, 16 x 16 subdomains of 32 x 32, l = 4, two
    sweeps, FP64, GMRES(30)) in the configuration the benchmark times, against a full oracle solve:
    iterations equal, p and the face velocities to 1e-10, and one application of T."""
    prob, q = W.channels(512, seed=1)
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve(fluxes=True)
    p_ref, info_ref, pre = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                        l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                        tol_relative=True, restart=q.restart, max_iter=q.max_iter)
    assert info["status"] == 0 and info["rel_res"] <= 1e-8
    assert info["iterations"] == info_ref["iterations"]
    assert _rel(p.cpu().numpy(), p_ref) < 1e-10
    assert _rel(info["u"][0].cpu().numpy(), info_ref["u"][0]) < 1e-10
    assert _rel(info["u"][1].cpu().numpy(), info_ref["u"][1]) < 1e-10
    # T on a random vector: the local Robin and Dirichlet problems of a contrast-1e6 field have
    # condition numbers near 1e9, so two backward-stable elimination orders agree to about
    # eps * 1e9 ~ 1e-7 at worst; measured about 2e-11
    r = np.random.default_rng(5).standard_normal(prob.K.shape)
    z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
    assert _rel(z, pre.apply(r)) < 1e-9
    s.close()


# a diagonal permeability tensor, components drawn independently: every face takes the component
# along its normal (transmissibilities, Dirichlet and Robin half transmissibilities, coarse K_H)
TENSOR_CASES = {
    "tensor-os-48x40": (dict(n=(48, 40, 1), seed=21), dict(sub=(8, 8, 1), oversample=2, smooth_steps=1)),
    "tensor-ragged-60x36": (dict(n=(60, 36, 1), seed=22, bc_kind=[0, 1, 0, 1, 1, 1]),
                            dict(sub=(12, 9, 1), oversample=3, smooth_steps=1)),
    "tensor-mrcm-48x48": (dict(n=(48, 48, 1), seed=23, bc_kind=[0, 0, 0, 0, 1, 1]),
                          dict(sub=(16, 12, 1), oversample=0, smooth_steps=0)),
}


def _tensor_case(name):
    pk, qk = TENSOR_CASES[name]
    prob = W.random_problem(pk["n"], seed=pk["seed"], contrast=1e3, bc_kind=pk.get("bc_kind"), tensor=True)
    q = W.Params(**qk)
    q.tol, q.restart = 1e-10, 30
    return prob, q


@pytest.mark.parametrize("name", list(TENSOR_CASES))
def test_diagonal_tensor_matches_oracle(mrcm, name):
    prob, q = _tensor_case(name)
    s = mrcm.Solver(prob, q)
    s.factor()
    T = grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind)
    tr = s.debug(mrcm.MRCM_DBG_TRANS)
    nx, ny = prob.n[0], prob.n[1]
    assert _rel(tr[:(nx + 1) * ny], T[0]) < 1e-14
    assert _rel(tr[(nx + 1) * ny:], T[1]) < 1e-14
    b = grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f)
    assert _rel(s.rhs().cpu().numpy(), b) < 1e-14
    pre = _oracle(prob, q)
    # the scalar field of the x component alone gives a different preconditioner on this case
    scalar = MRCMOS(prob.K[0], prob.h, prob.dim, prob.bc_kind, q.sub, q.oversample, q.smooth_steps, q.alpha)
    rng = np.random.default_rng(41)
    for trial in range(2):
        r = rng.standard_normal(grid.cell_shape(prob.K))
        z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
        ref = pre.apply(r)
        assert _rel(z, ref) < 1e-10, (name, trial, _rel(z, ref))
        assert _rel(scalar.apply(r), ref) > 1e-3
    p, info = s.solve()
    p_ref, info_ref, _ = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                      l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=1e-10,
                                      tol_relative=True, restart=q.restart, max_iter=q.max_iter)
    assert info["status"] == 0 and info["iterations"] == info_ref["iterations"]
    assert _rel(p.cpu().numpy(), p_ref) < 1e-10
    s.close()


def test_diagonal_tensor_with_equal_components_is_the_scalar_path(mrcm):
    prob, q = _case("os-48x40")
    tprob = W.Problem(prob.dim, prob.n, prob.h, np.stack([prob.K, prob.K]), prob.bc_kind, prob.bc_val, prob.f)
    a, b = mrcm.Solver(prob, q), mrcm.Solver(tprob, q)
    a.factor()
    b.factor()
    r = torch.as_tensor(np.random.default_rng(5).standard_normal(prob.K.size), device="cuda")
    assert torch.equal(a.apply_precond(r), b.apply_precond(r))
    a.close()
    b.close()


def test_banded_coupling_solve_above_the_dense_limit(mrcm):
    # 44 x 44 subdomains: 2E = 7,568 coupling unknowns, above the explicit-inverse limit, so every
    # apply runs the band LU solve (the path of the 2048 x 2048 workload's 16,128 unknowns)
    prob = W.random_problem((264, 264, 1), seed=13, contrast=1e3)
    q = W.Params(sub=(6, 6, 1), oversample=2, smooth_steps=2, tol=1e-9, restart=30, max_iter=300)
    s = mrcm.Solver(prob, q)
    s.factor()
    s.debug(mrcm.MRCM_DBG_ZMRCM, enable_only=True)
    pre = _oracle(prob, q)
    assert pre.part.E2 == 7568
    r = np.random.default_rng(17).standard_normal(prob.K.shape)
    z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
    parts = pre.apply_parts(r)
    assert _rel(s.debug(mrcm.MRCM_DBG_COARSE), parts["c"]) < 1e-9
    assert _rel(z, parts["z"]) < 1e-10
    p, info = s.solve()
    p_ref, info_ref, _ = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                      l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                      tol_relative=True, restart=q.restart, max_iter=q.max_iter)
    assert info["status"] == 0 and info["iterations"] == info_ref["iterations"]
    assert _rel(p.cpu().numpy(), p_ref) < 1e-10
    s.close()


@pytest.mark.parametrize("name", ["os-48x40", "os-96x64-l4s2", "ragged-60x36", "mrcm-48x40", "dirichlet-all",
                                  "uneven-61x45", "uneven-40x20-tall", "single-32"])
def test_piecewise_linear_interface_spaces_match_oracle(mrcm, name):
    prob, q = _case(name)
    q.iface_degree = 1
    s = mrcm.Solver(prob, q)
    s.factor()
    s.debug(mrcm.MRCM_DBG_ZMRCM, enable_only=True)
    pre = _oracle(prob, q)
    rng = np.random.default_rng(51)
    for trial in range(2):
        r = rng.standard_normal(prob.K.shape)
        z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
        parts = pre.apply_parts(r)
        if pre.part.E2:
            assert _rel(s.debug(mrcm.MRCM_DBG_COARSE), parts["c"]) < 1e-9
        assert _rel(s.debug(mrcm.MRCM_DBG_ZMRCM), parts["z_mrcm"]) < 1e-10
        assert _rel(z, parts["z"]) < 1e-10, (name, trial, _rel(z, parts["z"]))
    s.close()


@pytest.mark.parametrize("name", ["os-96x64-l4s2", "uneven-61x45"])
def test_piecewise_linear_gmres_matches_oracle(mrcm, name):
    prob, q = _case(name)
    q.iface_degree, q.tol, q.restart = 1, 1e-9, 30
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve()
    p_ref, info_ref, _ = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                      l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                      tol_relative=True, restart=q.restart, max_iter=q.max_iter, iface_degree=1)
    assert info["status"] == 0 and info["iterations"] == info_ref["iterations"]
    assert _rel(p.cpu().numpy(), p_ref) < 1e-10
    s.close()


# the Robin parameter alpha of Eq. 6 enters beta = alpha H / K_H on every interface face
@pytest.mark.parametrize("alpha,degree", [(0.5, 0), (3.0, 0), (100.0, 0), (3.0, 1)])
def test_alpha_sweep_matches_oracle(mrcm, alpha, degree):
    prob, q = _case("os-96x64-l4s2")
    q.alpha, q.iface_degree = alpha, degree
    s = mrcm.Solver(prob, q)
    s.factor()
    pre = _oracle(prob, q)
    r = np.random.default_rng(61).standard_normal(prob.K.shape)
    z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
    assert _rel(z, pre.apply(r)) < 1e-10
    s.close()


def test_autotuned_launch_shapes_give_identical_results(mrcm):
    # the tuned variants (line-block ring depth of the local solves, cluster size of the coupling
    # factorisation) change how data is staged, never the arithmetic
    prob, q = _case("os-96x64-l4s2")
    q.coarse_pivoting = 1   # the pivoted coupling LU is the autotuned one (its variants give identical factors)
    r = torch.as_tensor(np.random.default_rng(71).standard_normal(prob.cells), device="cuda")
    out = {}
    try:
        for mode in (0, 2):  # built-in choices, then freshly tuned shapes
            mrcm.autotune(mode)
            s = mrcm.Solver(prob, q)
            s.factor()
            z = s.apply_precond(r)
            p, info = s.solve()
            out[mode] = (z.clone(), p.clone(), info["iterations"])
            s.close()
    finally:
        mrcm.autotune(1)
    assert torch.equal(out[0][0], out[2][0]) and torch.equal(out[0][1], out[2][1]) and out[0][2] == out[2][2]
    table = mrcm.autotune_table()
    kinds = {e["kind"] for e in table}
    assert {0, 1} <= kinds, table
    for e in table:
        assert 0 <= e["choice"] < e["ncand"] and e["ncand"] >= 2 and e["best_us"] > 0.0, e


def test_full_size_quarter_five_spot_64_matches_oracle(mrcm):
    """The 64 x 64 quarter-five-spot workload (log-normal field, 4 x 4 subdomains of 16 x 16, l = 2,
    one sweep, FP64, GMRES(30)) at its full size against the oracle: iterations equal, p and u to 1e-10."""
    prob, q = W.quarter_five_spot(64, seed=1)
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve(fluxes=True)
    p_ref, info_ref, _ = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                      l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                      tol_relative=True, restart=q.restart, max_iter=q.max_iter)
    assert info["status"] == 0 and info["iterations"] == info_ref["iterations"]
    assert _rel(p.cpu().numpy(), p_ref) < 1e-10
    assert _rel(info["u"][0].cpu().numpy(), info_ref["u"][0]) < 1e-10
    assert _rel(info["u"][1].cpu().numpy(), info_ref["u"][1]) < 1e-10
    s.close()


def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads_oracle.json")
    return json.load(open(path))["results"][name]


def test_full_size_lognormal_2048_matches_oracle(mrcm):
    """The 2048 x 2048 log-normal workload (variance 4, correlation length 0.05, 64 x 64 subdomains
    of 32 x 32, l = 2, one sweep, GMRES(30); 16,128 coupling unknowns on the blocked band path) at
    full size.  FP64: iterations equal to the oracle's stored count and p equal to its stored
    pressure at 1024 sampled cells to 1e-10; one application of T against the oracle's.  Mixed
    (FP32 local factors and solves, FP64 GMRES): the true FP64 residual meets 1e-8 and p is within
    1e-6 of the oracle's (the FP32 solves make T a different operator; the outer residual bounds
    the error through the conditioning of A)."""
    gold = _golden("lognormal-2048")
    idx, ps = np.asarray(gold["sample_cells"]), np.asarray(gold["p_sample"])
    prob, q = W.lognormal(2048, seed=1)
    T = grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind)
    b = grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f)
    its = {}
    for prec in (W.PREC_FP64, W.PREC_FP32):
        q.local_prec = prec
        s = mrcm.Solver(prob, q)
        s.factor()
        p, info = s.solve()
        assert info["status"] == 0, (prec, info)
        pn = p.cpu().numpy()
        r = b - grid.matvec(T, pn.reshape(prob.K.shape), 2)
        assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(b), prec
        err = np.linalg.norm(pn[idx] - ps) / np.linalg.norm(ps)
        its[prec] = info["iterations"]
        if prec == W.PREC_FP64:
            assert info["iterations"] == gold["iterations"]
            assert err < 1e-10, err
            pre = MRCMOS(prob.K, prob.h, 2, prob.bc_kind, q.sub, q.oversample, q.smooth_steps, q.alpha)
            rv = np.random.default_rng(7).standard_normal(prob.K.shape)
            z = s.apply_precond(torch.as_tensor(rv.ravel(), device="cuda")).cpu().numpy()
            assert _rel(z, pre.apply(rv)) < 1e-10
            del pre
        else:
            assert err < 1e-6, err
        s.close()
    assert its[W.PREC_FP32] <= its[W.PREC_FP64] + 2, its
    # the set-up solves refined once in FP64: the count of the FP64 form
    q.local_prec, q.refine_setup = W.PREC_FP32, 1
    s = mrcm.Solver(prob, q)
    s.factor()
    p, info = s.solve()
    pn = p.cpu().numpy()
    r = b - grid.matvec(T, pn.reshape(prob.K.shape), 2)
    assert info["status"] == 0 and np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(b)
    assert info["iterations"] <= its[W.PREC_FP64] + 1, (info["iterations"], its)
    assert np.linalg.norm(pn[idx] - ps) / np.linalg.norm(ps) < 1e-6
    s.close()


@pytest.mark.parametrize("name,degree", [("lognormal-128", 0), ("lognormal-128", 1), ("os-96x64-l4s2", 0),
                                         ("uneven-61x45", 0), ("ragged-60x36", 1), ("column-12x96", 0)])
def test_refined_fp32_setup_solves(mrcm, name, degree):
    # refine_setup: the FP32 informed and basis solves (1), or the basis solves alone (2), take one
    # FP64 residual and a second solve.
    # One step contracts the solve error by about cond(box) eps_32: on a smooth field (the
    # log-normal workloads) that is small and the side moments come much closer to the FP64 path's;
    # on the contrast-1e3 white-noise boxes it is near one and the step changes little.  On every
    # case the true residual meets the tolerance and GMRES needs at most one iteration more than FP64.
    if name == "lognormal-128":
        prob, q = W.lognormal(128, seed=5, variance=2.0, corr=0.1, sub=16, oversample=2, smooth_steps=1)
    else:
        prob, q = _case(name)
    q.iface_degree, q.tol = degree, 1e-8
    T = grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind)
    b = grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f)
    res = {}
    for prec, ref in ((W.PREC_FP64, 0), (W.PREC_FP32, 0), (W.PREC_FP32, 1), (W.PREC_FP32, 2)):
        q.local_prec, q.refine_setup = prec, ref
        s = mrcm.Solver(prob, q)
        s.factor()
        p, info = s.solve()
        assert info["status"] == 0
        r = b - grid.matvec(T, p.cpu().numpy().reshape(prob.K.shape), 2)
        assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(b)
        res[(prec, ref)] = (s.debug(mrcm.MRCM_DBG_MOMENTS), info["iterations"])
        s.close()
    m64, it64 = res[(W.PREC_FP64, 0)]
    (m_plain, it_plain), (m_ref, it_ref) = res[(W.PREC_FP32, 0)], res[(W.PREC_FP32, 1)]
    if name == "lognormal-128":
        assert _rel(m_ref, m64) < 0.25 * _rel(m_plain, m64), (_rel(m_ref, m64), _rel(m_plain, m64))
    assert it_ref <= it64 + 1, (it64, it_plain, it_ref)
    # refine_setup = 2: the basis solves alone refined
    assert res[(W.PREC_FP32, 2)][1] <= it64 + 1, (it64, res[(W.PREC_FP32, 2)][1])


@pytest.mark.parametrize("contrast", [1e6, 1e9])
def test_high_contrast_matches_oracle_within_conditioning(mrcm, contrast):
    # K spread over 6 and 9 decades: local condition numbers reach about contrast * (box size)^2,
    # so the two elimination orders agree to eps times that, not to 1e-10
    prob = W.random_problem((48, 40, 1), seed=17, contrast=contrast)
    q = W.Params(sub=(8, 8, 1), oversample=2, smooth_steps=1, tol=1e-9, restart=30)
    s = mrcm.Solver(prob, q)
    s.factor()
    pre = _oracle(prob, q)
    r = np.random.default_rng(18).standard_normal(prob.K.shape)
    z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
    assert _rel(z, pre.apply(r)) < 1e-16 * contrast * 64 ** 2
    p, info = s.solve()
    T = grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind)
    b = grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f)
    resid = b - grid.matvec(T, p.cpu().numpy().reshape(prob.K.shape), 2)
    assert info["status"] == 0 and np.linalg.norm(resid) <= 1.0001e-9 * np.linalg.norm(b)
    s.close()


# the mixed form on the variants: FP32 local factors and solves, FP64 GMRES and true residual;
# the criterion is the FP64 tolerance reached in at most one iteration more than the FP64 form
@pytest.mark.parametrize("variant", ["uneven", "degree1", "tensor", "multiplicative", "alpha3"])
def test_mixed_precision_variants_reach_fp64_tolerance(mrcm, variant):
    if variant == "tensor":
        prob, q = _tensor_case("tensor-ragged-60x36")
    else:
        prob, q = _case("uneven-61x45" if variant == "uneven" else "os-96x64-l4s2")
    q.tol = 1e-8
    if variant == "degree1":
        q.iface_degree = 1
    if variant == "multiplicative":
        q.smooth_kind = 1
    if variant == "alpha3":
        q.alpha = 3.0
    T = grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind)
    b = grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f)
    its = {}
    for prec in (W.PREC_FP64, W.PREC_FP32):
        q.local_prec = prec
        s = mrcm.Solver(prob, q)
        s.factor()
        p, info = s.solve()
        assert info["status"] == 0, (variant, prec)
        r = b - grid.matvec(T, p.cpu().numpy().reshape(grid.cell_shape(prob.K)), 2)
        assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(b), (variant, prec)
        its[prec] = info["iterations"]
        s.close()
    assert its[W.PREC_FP32] <= its[W.PREC_FP64] + 1, (variant, its)


def test_banded_coupling_solve_degree1_above_the_dense_limit(mrcm):
    # piecewise-linear spaces on the 44 x 44 partition: 15,136 coupling unknowns with twice the band
    # width, so the blocked substitution carries about 700 rows from block to block
    prob = W.random_problem((264, 264, 1), seed=13, contrast=1e3)
    q = W.Params(sub=(6, 6, 1), oversample=2, smooth_steps=2, tol=1e-9, restart=30, max_iter=300, iface_degree=1)
    s = mrcm.Solver(prob, q)
    s.factor()
    s.debug(mrcm.MRCM_DBG_ZMRCM, enable_only=True)
    pre = _oracle(prob, q)
    assert pre.n_coarse == 15136
    r = np.random.default_rng(17).standard_normal(prob.K.shape)
    z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
    parts = pre.apply_parts(r)
    assert _rel(s.debug(mrcm.MRCM_DBG_COARSE), parts["c"]) < 1e-9
    assert _rel(z, parts["z"]) < 1e-10
    s.close()


@pytest.mark.parametrize("name,degree", [("os-96x64-l4s2", 0), ("uneven-61x45", 0), ("mrcm-48x40", 1),
                                         ("dirichlet-all", 1)])
def test_coupling_lu_without_pivoting_matches_the_pivoted_one(mrcm, name, degree):
    # the coupling matrix is factored without row interchanges over the whole GPU unless a pivot is
    # zero or an entry grows; the coefficients c and T agree with the partially pivoted factors and
    # with the oracle's (LAPACK getrf) to rounding
    prob, q = _case(name)
    q.iface_degree = degree
    pre = _oracle(prob, q)
    r = np.random.default_rng(81).standard_normal(prob.K.shape)
    parts = pre.apply_parts(r)
    out = {}
    for piv in (0, 1):
        q.coarse_pivoting = piv
        s = mrcm.Solver(prob, q)
        s.factor()
        s.debug(mrcm.MRCM_DBG_ZMRCM, enable_only=True)
        z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
        out[piv] = (s.debug(mrcm.MRCM_DBG_COARSE), z)
        assert _rel(out[piv][0], parts["c"]) < 1e-9
        assert _rel(z, parts["z"]) < 1e-10
        s.close()
    assert _rel(out[0][0], out[1][0]) < 1e-11


@pytest.mark.parametrize("kind", ["random-256", "lognormal-512"])
def test_multifrontal_coupling_matches_the_band_lu_and_the_oracle(mrcm, kind):
    # 64 x 64 subdomains (16,128 coupling unknowns): the nested-dissection multifrontal LU
    # (coarse_solver = 0) against the band LU (coarse_solver = 1) and the oracle (SuperLU with
    # threshold pivoting on the same G): coefficients c and T(r) to rounding
    if kind == "random-256":
        prob = W.random_problem((256, 256, 1), seed=23, contrast=1e3)
        q = W.Params(sub=(4, 4, 1), oversample=2, smooth_steps=1, tol=1e-10, restart=30, max_iter=300)
    else:
        prob, q = W.lognormal(512, seed=3, sub=8, oversample=2, smooth_steps=1, prec=W.PREC_FP64)
    pre = _oracle(prob, q)
    assert pre.n_coarse == 16128
    r = np.random.default_rng(29).standard_normal(prob.K.shape)
    parts = pre.apply_parts(r)
    out = {}
    for solver, method in ((0, "multifrontal"), (1, "band")):
        q.coarse_solver = solver
        s = mrcm.Solver(prob, q)
        s.factor()
        assert s.coarse_method() == method
        s.debug(mrcm.MRCM_DBG_ZMRCM, enable_only=True)
        z = s.apply_precond(torch.as_tensor(r.ravel(), device="cuda")).cpu().numpy()
        out[solver] = (s.debug(mrcm.MRCM_DBG_COARSE), z)
        assert _rel(out[solver][0], parts["c"]) < 1e-9
        assert _rel(z, parts["z"]) < 1e-10
        s.close()
    assert _rel(out[0][0], out[1][0]) < 1e-11


# FP32 local solves on boxes of every kind the two-warp steps handle: exact widths 32 and 36 (the
# 36-wide ones with the corner rows), narrower and intermediate widths (per-column width tests),
# and 40 (the one-CTA kernels); informed spaces and basis (four right-hand sides, refined) and
# particular solves and sweeps (one).  The refined set-up solves (phi, psi) against the FP64 oracle
# at the FP32-with-one-refinement level (measured 1.0e-5 to 1.5e-5 on these contrast-1e2 white-noise
# fields); z at the FP32 level: the FP32 particular solves' rounding is
# magnified by the coupling system (measured on these fields: G to 5e-6 but c to 4e-4 and z to
# 5e-4 to 8e-4 relative, the same for the one-CTA kernels of the 40-wide boxes, while the FP64 path
# agrees to 1e-13); and the GMRES solution and iteration count against a full oracle solve.
@pytest.mark.parametrize("n,sub,l", [((128, 96, 1), (32, 32, 1), 2),    # boxes 36 (hat) and 32
                                     ((120, 90, 1), (30, 30, 1), 2),    # 34 and 30
                                     ((96, 72, 1), (24, 24, 1), 2),     # 28 and 24
                                     ((64, 48, 1), (16, 16, 1), 2),     # 20 and 16
                                     ((144, 108, 1), (36, 36, 1), 2)])  # 40 and 36
def test_fp32_two_warp_line_solves_match_the_oracle(mrcm, n, sub, l):
    prob = W.random_problem(n, seed=17, contrast=1e2)
    q = W.Params(sub=sub, oversample=l, smooth_steps=1, tol=1e-9, restart=30, max_iter=200,
                 local_prec=W.PREC_FP32, refine_setup=1)
    pre = _oracle(prob, q)
    s = mrcm.Solver(prob, q)
    s.factor()
    P = pre.part
    smax = max(q.sub[0], q.sub[1])
    phi = s.debug(mrcm.MRCM_DBG_PHI).reshape(P.S, 4, 4, smax)
    ref_phi = np.stack([_phi_gpu_layout(pre, i, smax) for i in range(P.S)])
    assert _rel(phi, ref_phi) < 5e-5
    psi = s.debug(mrcm.MRCM_DBG_PSI).reshape(4, -1)
    nx = prob.n[0]
    for d in pre.subs:
        lo, hi = P.box[d.s, 0], P.box[d.s, 1]
        cells = (np.arange(lo[1], hi[1])[:, None] * nx + np.arange(lo[0], hi[0])[None, :]).ravel()
        for jj, (r, qd) in enumerate(d.funcs):
            assert _rel(psi[r, cells], d.psi[:, jj]) < 5e-5
    rr = np.random.default_rng(19).standard_normal(prob.K.shape)
    z = s.apply_precond(torch.as_tensor(rr.ravel(), device="cuda")).cpu().numpy()
    assert _rel(z, pre.apply_parts(rr)["z"]) < 2e-3
    p_ref, info_ref, _ = oracle_solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub,
                                      l=q.oversample, smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol,
                                      restart=q.restart)
    p, info = s.solve()
    assert info["status"] == 0 and info["rel_res"] <= 1e-9
    assert info["iterations"] <= info_ref["iterations"] + 1
    assert _rel(p.cpu().numpy(), p_ref) < 1e-6


def test_multifrontal_coupling_solve_is_repeatable(mrcm):
    # the dataflow solve (completion flags stamped with an epoch kept in device memory) gives the
    # same bits on every application, and after a second factorisation
    prob = W.random_problem((256, 256, 1), seed=23, contrast=1e3)
    q = W.Params(sub=(4, 4, 1), oversample=2, smooth_steps=1, tol=1e-10, restart=30, max_iter=300)
    s = mrcm.Solver(prob, q)
    s.factor()
    assert s.coarse_method() == "multifrontal"
    r = torch.as_tensor(np.random.default_rng(31).standard_normal(prob.cells), device="cuda")
    s.debug(mrcm.MRCM_DBG_ZMRCM, enable_only=True)
    z1 = s.apply_precond(r).cpu().numpy()
    c1 = s.debug(mrcm.MRCM_DBG_COARSE)
    for _ in range(3):
        z2 = s.apply_precond(r).cpu().numpy()
        assert np.array_equal(z1, z2)
    s.factor()
    z3 = s.apply_precond(r).cpu().numpy()
    assert np.array_equal(z1, z3) and np.array_equal(c1, s.debug(mrcm.MRCM_DBG_COARSE))
