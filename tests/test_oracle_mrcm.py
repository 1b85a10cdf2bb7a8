"""Pins of the oracle's MRCM-OS preconditioner T (Sec. 2.1, Sec. 3, Eq. 11-15)."""

import numpy as np
import pytest

from oracle import grid
from oracle.local import BoxOperator, robin_face
from oracle.mrcm import MRCMOS
from paper_2606_08883_gb300 import workloads as W


def _pre(prob, sub, l, s, degree=0, alpha=10.0):
    return MRCMOS(prob.K, prob.h, prob.dim, prob.bc_kind, sub, l, s, alpha, degree)


def _dense_A(pre):
    return grid.dense_matrix(pre.T, pre.dim, pre.shape)


@pytest.mark.parametrize("smooth", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_single_subdomain_is_exact_inverse(dim, smooth):
    n = (10, 8, 1) if dim == 2 else (6, 5, 4)
    prob = W.random_problem(n, dim=dim, seed=2, contrast=1e4)
    pre = _pre(prob, n, 0, smooth)
    r = np.random.default_rng(0).standard_normal(prob.K.shape)
    z = pre.apply(r)
    assert pre.part.E2 == 0
    ref = np.linalg.solve(_dense_A(pre), r.ravel()).reshape(r.shape)
    assert np.linalg.norm(z - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("degree", [0, 1])
def test_zero_oversampling_gives_side_polynomials(degree):
    prob = W.random_problem((12, 12, 1), seed=5, contrast=1e3)
    pre = _pre(prob, (4, 4, 1), 0, 0, degree)
    for d in pre.subs:
        for j, (k, q) in enumerate(d.funcs):
            on = d.gamma_side == k
            assert np.array_equal(d.phi[j, ~on], np.zeros((~on).sum()))
            assert np.array_equal(d.phi[j, on], d.test[q, on])
            if q == 0:
                assert (d.phi[j, on] == 1.0).all()


def _monolithic(pre, r):
    """Solve Eq. 11-14 (homogeneous data, source r) as one dense system: every subdomain's local
    pressures plus the multiplier coefficients, with the flux and pressure continuity rows."""
    P = pre.part
    offs = np.concatenate([[0], np.cumsum([d.op.n_loc for d in pre.subs])])
    nz = offs[-1]
    nc = pre.n_coarse
    M = np.zeros((nz + nc, nz + nc))
    rhs = np.zeros(nz + nc)
    for d in pre.subs:
        o = offs[d.s]
        M[o:o + d.op.n_loc, o:o + d.op.n_loc] = d.op.dense()
        rhs[o:o + d.op.n_loc] = d.op.restrict(r)
        for j in range(len(d.funcs)):
            col = nz + pre.coff[d.s] + j
            np.add.at(M[:, col], o + d.gamma_li, -d.t_r * d.phi[j])
    nq = pre.nq

    def face_terms(d, side):
        """Rows expressing F(f) and |f| P(f) on the faces of ``side`` as linear forms."""
        m = d.gamma_side == side
        idx = np.nonzero(m)[0]
        o = offs[d.s]
        Fz = np.zeros((len(idx), nz + nc))
        for t, i in enumerate(idx):
            Fz[t, o + d.gamma_li[i]] += d.t_r[i]
            for j in range(len(d.funcs)):
                Fz[t, nz + pre.coff[d.s] + j] -= d.t_r[i] * d.phi[j, i]
        lam = np.zeros((len(idx), nz + nc))
        for t, i in enumerate(idx):
            for j in range(len(d.funcs)):
                lam[t, nz + pre.coff[d.s] + j] += d.phi[j, i]
        Pw = d.area[idx, None] * lam + d.beta[idx, None] * Fz
        return Fz, Pw, d.test[:, m]

    for e, (a, s, s2) in enumerate(P.interfaces):
        F1, P1, t1 = face_terms(pre.subs[s], 2 * a + 1)
        F2, P2, t2 = face_terms(pre.subs[s2], 2 * a)
        assert np.array_equal(t1, t2)
        for q in range(nq):
            M[nz + 2 * nq * e + q] = t1[q] @ (F1 + F2)
            M[nz + 2 * nq * e + nq + q] = t1[q] @ (P1 - P2)
    x = np.linalg.solve(M, rhs)
    z = np.zeros(pre.shape)
    for d in pre.subs:
        z[d.op.sl] = x[offs[d.s]:offs[d.s] + d.op.n_loc].reshape(d.op.w[2], d.op.w[1], d.op.w[0])
    return z, x[nz:]


def _monolithic_oversampled(pre, r):
    """The same coupled system written on the extended regions (l > 0): unknowns are the
    pressures of every hat-Omega_s (source r on hat-Omega_s, Robin data sum_k c_sk lambda^k on the
    boundary of hat-Omega_s, Eq. 15) and the coefficients c; the flux and pressure continuity rows
    (Eq. 13-14) take the discrete flux F = T_f (q_c - q_c') and the face pressure q_c - F / tau_c of
    the extended solutions on the Gamma faces.  No informed trace and no Omega_s problem appear:
    their agreement with this system is what the test checks."""
    P = pre.part
    K, T, h = pre.K, pre.T, pre.h
    ops = [BoxOperator(K, T, h, pre.dim, pre.n, P.obox[d.s, 0], P.obox[d.s, 1], True, pre.alpha, pre.sub)
           for d in pre.subs]
    offs = np.concatenate([[0], np.cumsum([o.n_loc for o in ops])])
    nz = offs[-1]
    nc = pre.n_coarse
    M = np.zeros((nz + nc, nz + nc))
    rhs = np.zeros(nz + nc)
    for d, op in zip(pre.subs, ops):
        o = offs[d.s]
        M[o:o + op.n_loc, o:o + op.n_loc] = op.dense()
        rhs[o:o + op.n_loc] = op.restrict(r)
        olo, ohi = P.obox[d.s, 0], P.obox[d.s, 1]
        for j, (k, q) in enumerate(d.funcs):
            col = nz + pre.coff[d.s] + j
            for (pos, inside, outside) in P.side_faces(olo, ohi, k):
                _tau, _beta, t_r, _area = robin_face(K, h, k // 2, inside, outside, pre.alpha, pre.sub)
                M[o + op.local_index(inside), col] -= t_r * pre.side_poly(q, pos, k, olo, ohi)
    nq = pre.nq

    def face_terms(d, side):
        op, o = ops[d.s], offs[d.s]
        faces = P.gamma_faces(d.s, side)
        Fz = np.zeros((len(faces), nz + nc))
        Pw = np.zeros((len(faces), nz + nc))
        test = np.zeros((nq, len(faces)))
        for t, (pos, inside, outside) in enumerate(faces):
            a = side // 2
            tau, _beta, _tr, area = robin_face(K, h, a, inside, outside, pre.alpha, pre.sub)
            tf = T[a][pos[2], pos[1], pos[0]]
            ci, co = o + op.local_index(inside), o + op.local_index(outside)
            Fz[t, ci] += tf
            Fz[t, co] -= tf
            Pw[t, ci] += area
            Pw[t] -= area / tau * Fz[t]
            for q in range(nq):
                test[q, t] = pre.side_poly(q, pos, side, P.box[d.s, 0], P.box[d.s, 1])
        return Fz, Pw, test

    for e, (a, s, s2) in enumerate(P.interfaces):
        F1, P1, t1 = face_terms(pre.subs[s], 2 * a + 1)
        F2, P2, t2 = face_terms(pre.subs[s2], 2 * a)
        for q in range(nq):
            M[nz + 2 * nq * e + q] = t1[q] @ F1 + t2[q] @ F2
            M[nz + 2 * nq * e + nq + q] = t1[q] @ P1 - t2[q] @ P2
    x = np.linalg.solve(M, rhs)
    z = np.zeros(pre.shape)
    for d, op in zip(pre.subs, ops):
        zz = x[offs[d.s]:offs[d.s] + op.n_loc].reshape(op.w[2], op.w[1], op.w[0])
        inner = tuple(slice(int(P.box[d.s, 0, a] - P.obox[d.s, 0, a]), int(P.box[d.s, 1, a] - P.obox[d.s, 0, a]))
                      for a in (2, 1, 0))
        z[d.op.sl] = zz[inner]
    return z, x[nz:]


# n2: the 2-D grid; (14, 11) is not divisible by the 4 x 4 subdomains (last sizes 2 and 3)
@pytest.mark.parametrize("l,degree,dim,n2", [(0, 0, 2, (12, 12)), (1, 0, 2, (12, 12)), (2, 0, 2, (12, 12)),
                                             (2, 1, 2, (12, 12)), (1, 0, 3, None), (0, 0, 2, (14, 11)),
                                             (1, 0, 2, (14, 11)), (1, 1, 2, (14, 11))])
def test_superposition_equals_monolithic_dense_solve(l, degree, dim, n2):
    if dim == 2:
        prob = W.random_problem(n2 + (1,), seed=11, contrast=1e3)
        sub = (4, 4, 1)
    else:
        prob = W.random_problem((6, 6, 4), dim=3, seed=11, contrast=1e3, bc_kind=[0, 0, 1, 1, 1, 1])
        sub = (3, 3, 2)
    pre = _pre(prob, sub, l, 0, degree)
    if dim == 2:
        assert tuple(pre.part.m[:2]) == tuple(-(-v // 4) for v in n2)
    r = np.random.default_rng(3).standard_normal(prob.K.shape)
    parts = pre.apply_parts(r)
    z_ref, c_ref = (_monolithic if l == 0 else _monolithic_oversampled)(pre, r)
    assert np.linalg.norm(parts["z_mrcm"] - z_ref) <= 1e-10 * np.linalg.norm(z_ref)
    assert np.linalg.norm(parts["c"] - c_ref) <= 1e-9 * np.linalg.norm(c_ref)


@pytest.mark.parametrize("l", [0, 2])
def test_diagonal_tensor_superposition_and_single_subdomain(l):
    # anisotropic K: the superposition still equals the monolithic coupled solve, and one subdomain
    # still gives T = A^-1 for the tensor operator
    prob = W.random_problem((12, 12, 1), seed=31, contrast=1e3, tensor=True)
    pre = _pre(prob, (4, 4, 1), l, 0)
    r = np.random.default_rng(32).standard_normal(pre.shape)
    parts = pre.apply_parts(r)
    z_ref, c_ref = (_monolithic if l == 0 else _monolithic_oversampled)(pre, r)
    assert np.linalg.norm(parts["z_mrcm"] - z_ref) <= 1e-10 * np.linalg.norm(z_ref)
    one = _pre(prob, (12, 12, 1), 0, 1)
    ref = np.linalg.solve(_dense_A(one), r.ravel()).reshape(r.shape)
    assert np.linalg.norm(one.apply(r) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("tensor,n", [(False, (16, 12, 1)), (True, (16, 12, 1)), (False, (19, 15, 1))])
def test_mass_balance_and_weak_continuity(tensor, n):
    prob = W.random_problem(n, seed=8, contrast=1e4, tensor=tensor)
    pre = _pre(prob, (4, 4, 1), 2, 0)
    r = np.random.default_rng(9).standard_normal(pre.shape)
    parts = pre.apply_parts(r)
    z, c = parts["z_mrcm"], parts["c"]
    P = pre.part
    Fside, Pside = {}, {}
    for d in pre.subs:
        zs = d.op.restrict(z)
        lam = parts["phi0"][d.s] + d.phi.T @ c[pre.coff[d.s]:pre.coff[d.s] + len(d.funcs)]
        # per-cell mass balance inside the subdomain: A^R z_s - t_R lambda = r
        res = d.op.dense() @ zs
        np.add.at(res, d.gamma_li, -d.t_r * lam)
        assert np.allclose(res, d.op.restrict(r), rtol=0, atol=1e-10 * np.abs(r).max())
        F = d.t_r * (zs[d.gamma_li] - lam)
        Pw = d.area * lam + d.beta * F
        for k in d.sides:
            m = d.gamma_side == k
            Fside[(d.s, k)] = F[m].sum()
            Pside[(d.s, k)] = Pw[m].sum()
    scale = max(abs(v) for v in Fside.values())
    pscale = max(abs(v) for v in Pside.values())
    for (a, s, s2) in P.interfaces:
        assert abs(Fside[(s, 2 * a + 1)] + Fside[(s2, 2 * a)]) <= 1e-10 * scale      # Eq. 13
        assert abs(Pside[(s, 2 * a + 1)] - Pside[(s2, 2 * a)]) <= 1e-10 * pscale     # Eq. 14


@pytest.mark.parametrize("l,smooth,nx", [(0, 0, 20), (1, 0, 20), (2, 1, 20), (3, 2, 20), (2, 1, 23)])
def test_exact_on_fields_constant_along_interfaces(l, smooth, nx):
    # stripes along x spanning the whole y range; K and the target pressure depend on x only, so
    # the true Robin data is constant on every interface and lies in the P0 multiplier space
    rng = np.random.default_rng(21)
    ny = 6
    kx = 10.0 ** rng.uniform(-2, 2, size=nx)
    prob = W.Problem(2, (nx, ny, 1), (1.0 / nx, 1.0 / ny, 1.0), np.tile(kx, (ny, 1))[None],
                     [0, 0, 1, 1, 1, 1])
    pre = _pre(prob, (4, ny, 1), l, smooth)
    p_star = np.tile(rng.standard_normal(nx), (ny, 1))[None]
    r = pre.Av(p_star)
    z = pre.apply(r)
    assert np.linalg.norm(z - p_star) <= 1e-10 * np.linalg.norm(p_star)


def test_linearity():
    prob = W.random_problem((16, 16, 1), seed=12, contrast=1e5)
    pre = _pre(prob, (4, 4, 1), 2, 2)
    rng = np.random.default_rng(13)
    r1, r2 = rng.standard_normal(prob.K.shape), rng.standard_normal(prob.K.shape)
    lhs = pre.apply(2.0 * r1 - 3.0 * r2)
    rhs = 2.0 * pre.apply(r1) - 3.0 * pre.apply(r2)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(rhs)


@pytest.mark.parametrize("n", [(12, 10, 1), (15, 13, 1)])
def test_schwarz_sweep_matches_dense_restricted_additive_schwarz(n):
    prob = W.random_problem(n, seed=14, contrast=1e3)
    pre = _pre(prob, (4, 5, 1), 2, 1)
    A = _dense_A(pre)
    rng = np.random.default_rng(15)
    r, z = rng.standard_normal(prob.K.shape), rng.standard_normal(prob.K.shape)
    n = np.array(pre.n)
    rho = r.ravel() - A @ z.ravel()
    z_ref = z.ravel().copy()
    for s in range(pre.part.S):
        lo, hi = pre.part.box[s, 0], pre.part.box[s, 1]
        olo = np.maximum(lo - 2, 0)
        ohi = np.minimum(hi + 2, n)
        ohi[2], olo[2] = 1, 0
        cells = [i + n[0] * j for j in range(olo[1], ohi[1]) for i in range(olo[0], ohi[0])]
        delta = np.linalg.solve(A[np.ix_(cells, cells)], rho[cells])
        for t, c in enumerate(cells):
            i, j = c % n[0], c // n[0]
            if lo[0] <= i < hi[0] and lo[1] <= j < hi[1]:
                z_ref[c] += delta[t]
    z_new = pre.sweep(r, z)
    assert np.allclose(z_new.ravel(), z_ref, rtol=1e-11, atol=1e-11)
    # a fixed point of the sweep: the exact solution is left unchanged
    z_star = np.linalg.solve(A, r.ravel()).reshape(r.shape)
    assert np.linalg.norm(pre.sweep(r, z_star) - z_star) <= 1e-11 * np.linalg.norm(z_star)


def _colour_blocks(pre):
    """Cells of each colour (independent of the oracle's colouring code: parity of the subdomain
    coordinates of the cell itself)."""
    nz, ny, nx = pre.shape
    out = {}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = ((i // pre.sub[0]) % 2) | (((j // pre.sub[1]) % 2) << 1) | (((k // pre.sub[2]) % 2) << 2)
                out.setdefault(c, []).append(i + nx * (j + ny * k))
    return [out[c] for c in sorted(out)]


@pytest.mark.parametrize("dim,ragged", [(2, False), (3, False), (2, True)])
def test_multiplicative_sweep_without_overlap_is_block_gauss_seidel(dim, ragged):
    # l = 0: each colour's subdomains are pairwise uncoupled, so one multiplicative sweep is the
    # textbook block Gauss-Seidel step z + M^-1 (r - A z), M the block lower triangle of A in colour
    # order; the additive sweep is block Jacobi z + D^-1 (r - A z).
    n, sub = ((16, 12, 1), (4, 3, 1)) if dim == 2 else ((8, 6, 4), (2, 3, 2))
    if ragged:
        n = (17, 13, 1)
    prob = W.random_problem(n, dim=dim, seed=21, contrast=1e3)
    A = None
    for kind in (0, 1):
        pre = MRCMOS(prob.K, prob.h, prob.dim, prob.bc_kind, sub, 0, 1, 10.0, 0, kind)
        if A is None:
            A = _dense_A(pre)
        blocks = _colour_blocks(pre)
        order = np.concatenate(blocks)
        Ap = A[np.ix_(order, order)]
        M = np.zeros_like(Ap)
        o = 0
        for bl in blocks:
            o2 = o + len(bl)
            if kind == 1:
                M[o:o2, :o2] = Ap[o:o2, :o2]
            else:
                M[o:o2, o:o2] = Ap[o:o2, o:o2]
            o = o2
        rng = np.random.default_rng(22 + kind)
        r, z = rng.standard_normal(prob.K.shape), rng.standard_normal(prob.K.shape)
        res = (r.ravel() - A @ z.ravel())[order]
        z_ref = z.ravel().copy()
        z_ref[order] += np.linalg.solve(M, res)
        assert np.allclose(pre.sweep(r, z).ravel(), z_ref, rtol=1e-11, atol=1e-11), kind


def test_multiplicative_sweep_fixed_point_and_energy_decrease():
    prob = W.random_problem((16, 16, 1), seed=23, contrast=1e3)
    pre = MRCMOS(prob.K, prob.h, prob.dim, prob.bc_kind, (4, 4, 1), 2, 1, 10.0, 0, 1)
    A = _dense_A(pre)
    r = np.random.default_rng(24).standard_normal(prob.K.shape)
    z_star = np.linalg.solve(A, r.ravel()).reshape(r.shape)
    assert np.linalg.norm(pre.sweep(r, z_star) - z_star) <= 1e-11 * np.linalg.norm(z_star)
    # repeated sweeps from z = 0 converge to A^-1 r
    z = np.zeros_like(r)
    errs = []
    for _ in range(40):
        z = pre.sweep(r, z)
        e = (z - z_star).ravel()
        errs.append(np.sqrt(e @ A @ e))
    assert errs[-1] < 1e-3 * errs[0]


@pytest.mark.parametrize("l,degree,dim,n2", [(1, 0, 2, (16, 12)), (3, 0, 2, (16, 12)), (2, 1, 2, (16, 12)),
                                             (1, 0, 3, None), (1, 0, 2, (18, 14)), (1, 1, 2, (18, 14))])
def test_basis_equals_restricted_oversampled_solution(l, degree, dim, n2):
    # Eq. 15 and the Robin condition: phi_s^k is the Robin trace of q^k on Gamma_s, so the local
    # Robin solve with data phi_s^k reproduces q^k on Omega_s exactly.
    from oracle.local import BoxOperator, robin_face
    if dim == 2:
        prob = W.random_problem(n2 + (1,), seed=31, contrast=1e4)
        sub = (4, 4, 1)
    else:
        prob = W.random_problem((6, 6, 4), dim=3, seed=31, contrast=1e3, bc_kind=[0, 0, 1, 1, 1, 1])
        sub = (3, 3, 2)
    pre = _pre(prob, sub, l, 0, degree)
    P = pre.part
    for d in pre.subs:
        olo, ohi = P.obox[d.s, 0], P.obox[d.s, 1]
        oop = BoxOperator(prob.K, pre.T, prob.h, dim, pre.n, olo, ohi, True, 10.0, sub)
        M = oop.dense()
        for j, (k, q) in enumerate(d.funcs):
            rhs = np.zeros(oop.n_loc)
            for (pos, inside, outside) in P.side_faces(olo, ohi, k):
                _tau, _beta, t_r, _area = robin_face(prob.K, prob.h, k // 2, inside, outside, 10.0, sub)
                rhs[oop.local_index(inside)] += t_r * pre.side_poly(q, pos, k, olo, ohi)
            qk = np.linalg.solve(M, rhs).reshape(oop.w[2], oop.w[1], oop.w[0])
            inner = tuple(slice(int(P.box[d.s, 0, a] - olo[a]), int(P.box[d.s, 1, a] - olo[a])) for a in (2, 1, 0))
            ref = qk[inner].ravel()
            assert np.allclose(d.psi[:, j], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("l,dim,n2", [(1, 2, (16, 12)), (3, 2, (16, 12)), (1, 3, None), (2, 2, (19, 15))])
def test_particular_equals_restricted_oversampled_solution(l, dim, n2):
    # the source term's basis function is built on the extended region: psi_s0, the local Robin
    # solve on Omega_s with source r and the informed particular trace phi_s0 as data, equals the
    # dense solve of the hat-Omega_s Robin problem with source r (zero data) restricted to Omega_s
    if dim == 2:
        prob = W.random_problem(n2 + (1,), seed=41, contrast=1e4)
        sub = (4, 4, 1)
    else:
        prob = W.random_problem((6, 6, 4), dim=3, seed=41, contrast=1e3, bc_kind=[0, 0, 1, 1, 1, 1])
        sub = (3, 3, 2)
    pre = _pre(prob, sub, l, 0)
    r = np.random.default_rng(42).standard_normal(pre.shape)
    psi0 = pre.apply_parts(r)["psi0"]
    P = pre.part
    for d in pre.subs:
        olo, ohi = P.obox[d.s, 0], P.obox[d.s, 1]
        oop = BoxOperator(prob.K, pre.T, prob.h, dim, pre.n, olo, ohi, True, 10.0, sub)
        q0 = np.linalg.solve(oop.dense(), oop.restrict(r)).reshape(oop.w[2], oop.w[1], oop.w[0])
        inner = tuple(slice(int(P.box[d.s, 0, a] - olo[a]), int(P.box[d.s, 1, a] - olo[a])) for a in (2, 1, 0))
        ref = q0[inner].ravel()
        assert np.allclose(psi0[d.s], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_zero_oversampling_has_no_particular_trace():
    # l = 0: hat-Omega = Omega, the source problem has zero Robin data on Gamma, so phi_s0 = 0 and T
    # is the plain MRCM of Eq. 11-14 (the monolithic l = 0 pin above covers its value)
    prob = W.random_problem((12, 12, 1), seed=43, contrast=1e3)
    pre = _pre(prob, (4, 4, 1), 0, 0)
    parts = pre.apply_parts(np.random.default_rng(44).standard_normal(pre.shape))
    assert all(np.array_equal(ph, np.zeros_like(ph)) for ph in parts["phi0"])


@pytest.mark.parametrize("variable", [False, True])
def test_oversampling_alone_cuts_iterations(variable):
    # Sec. 4.1 and Tables 2-3: with oversampling and no smoothing (MRCM-O) GMRES(10) needs far fewer
    # iterations than with the non-overlapping MRCM, and more oversampling needs fewer still.  The
    # Sec. 4.1 problems on a 64 x 64 grid, 4 x 4 and 8 x 8 subdomains, absolute tolerance 1e-8.
    from oracle.solve import solve
    prob, _exact = W.analytic(64, variable)
    for m in (4, 8):
        it = []
        for l in (0, 2, 4):
            _p, info, _pre_ = solve(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f, sub=(64 // m, 64 // m, 1), l=l,
                                    smooth_steps=0, alpha=10.0, tol=1e-8, tol_relative=False, restart=10, max_iter=400)
            assert info["status"] == 0
            it.append(info["iterations"])
        assert it[1] <= 0.6 * it[0] and it[2] <= 0.45 * it[0] and it[2] < it[1], it


def test_piecewise_linear_sides_need_two_faces():
    # 13 = 3 * 4 + 1: the last row of subdomains is one cell high, so its -x / +x Robin sides have a
    # single face, on which the linear side function vanishes (2 (0 + 1/2) / 1 - 1 = 0)
    prob = W.random_problem((12, 13, 1), seed=4)
    _pre(prob, (4, 4, 1), 0, 0, 0)
    with pytest.raises(ValueError):
        _pre(prob, (4, 4, 1), 0, 0, 1)
    # a one-cell-high grid: the -x / +x sides have one face each
    with pytest.raises(ValueError):
        _pre(W.random_problem((12, 1, 1), seed=4), (4, 1, 1), 0, 0, 1)
    # a single row of subdomains two cells high has no -y / +y Robin sides and two faces on the others
    pre = _pre(W.random_problem((12, 2, 1), seed=4), (4, 2, 1), 0, 0, 1)
    assert pre.nq == 2 and pre.n_coarse == 2 * pre.part.E2 == 8
    with pytest.raises(ValueError):
        _pre(prob, (4, 4, 1), 0, 0, 2)
