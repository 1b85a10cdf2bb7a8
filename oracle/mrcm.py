"""MRCM-OS as a preconditioner T (Sec. 2.1 and Sec. 3).

Set-up (MRCM-OS steps 1-3, with the preconditioner's homogeneous boundary conditions):

1. Informed multiplier spaces (Eq. 15, definition of phi_i^k):
   for every Robin side k of the oversampled region hat-Omega_s solve the homogeneous Robin problem
   with Robin data lambda^k = 1 on the faces of side k and 0 elsewhere.  On each face f of Gamma_s
   (inside cell c in Omega_s, outside cell c' in hat-Omega_s) take the discrete normal flux
   F = T_f (q_c - q_c'), the velocity u = F/|f|, the face pressure pi = q_c - F/tau_c and
   phi_s^k(f) = -beta_f u + pi (the informed trace of q).  With l = 0 the faces of Gamma_s lie on
   the Robin boundary, the Robin trace identity gives phi_s^k = lambda^k exactly, and that value is
   used.
2. Multiscale basis functions (MBF): psi_sk = (A^R_{Omega_s})^-1 (t_R phi_s^k on Gamma_s), with
   Robin traces F_sk(f) = t_R (psi_sk,c - phi_s^k(f)) and |f| P_sk(f) = |f| phi_s^k(f) + beta F_sk(f).
3. Coupling system (Eq. 13-14) with piecewise-constant M_H, V_H on each interface Gamma_{s,s'}
   (s the lower, s' the upper subdomain along axis a):
     flux row     sum_f F_s(f) + F_s'(f) = 0,
     pressure row sum_f |f| (P_s(f) - P_s'(f)) = 0,
   with F_s = F_s0 + sum_k c_sk F_sk and likewise P_s.  The matrix G is square (2E x 2E) and is
   factored by LU with partial pivoting (dense LAPACK getrf; SuperLU beyond 4096 unknowns).
4. Dirichlet restrictions A[hat-Omega_s, hat-Omega_s] for the smoothing sweeps.

Apply z = T r (the modified MRCM-O of Sec. 3: homogeneous conditions, source r).  The source
term's basis function is built on the extended region like the others (Sec. 1: oversampling lets
each MBF be constructed in an extended region while the coupling stays on the non-overlapping
partition):
  q_s0 = (A^R_{hat-Omega_s})^-1 r|hat-Omega_s (zero Robin data on the boundary of hat-Omega_s),
  phi_s0 = informed trace of q_s0 on Gamma_s (the formula of step 1; phi_s0 = 0 when l = 0),
  psi_s0 = (A^R_{Omega_s})^-1 (r|Omega_s + t_R phi_s0) with traces F_s0 = t_R (psi_s0,c - phi_s0),
  |f| P_s0 = |f| phi_s0 + beta F_s0, so that the Robin data of subdomain s is
  lambda_s = phi_s0 + sum_k c_sk phi_s^k;
  G c = -g0 where g0 collects the particular traces row by row;
  z|Omega_s = psi_s0 + sum_k c_sk psi_sk;
  then ``smooth_steps`` restricted Schwarz sweeps (the smoothing of MRCM-OS step 4, Sec. 2.1):
  additive (smooth_kind 0): rho = r - A z, delta_s = A[hat-Omega_s, hat-Omega_s]^-1 rho|hat-Omega_s,
  z|Omega_s += delta_s|Omega_s for all s at once; multiplicative multicolour (smooth_kind 1): the
  subdomains are coloured by the parities of their grid coordinates (2^dim colours) and the
  additive step is taken one colour after the other, each colour with the residual left by the
  colours before it.

Pinned by (tests/test_oracle_mrcm.py): one subdomain gives T = A^-1; l = 0 gives indicator phi and
phi_s0 = 0 (the MRCM of Eq. 11-14); a monolithic dense solve of the whole coupled system equals
the superposition; basis and particular solutions equal the restrictions of the oversampled
solutions; per-cell mass balance and weak flux / pressure continuity of the reconstruction;
exactness on a field that is constant along the interfaces; linearity of T; the smoothing sweep
leaves A^-1 r unchanged; the additive sweep equals a dense restricted additive Schwarz step; with
l = 0 the multiplicative sweep equals block Gauss-Seidel over the colour-ordered subdomain blocks;
oversampling alone cuts the GMRES iterations of the Sec. 4.1 problems well below plain MRCM, as
Sec. 4.1 and Tables 2-3 state; with one sweep the preconditioned operator satisfies Appendix A's
energy-norm contraction on a heterogeneous field.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import cell_shape, transmissibilities, matvec
from .local import BoxOperator, robin_face
from .partition import Partition


class _Sub:
    pass


class MRCMOS:
    def __init__(self, K, h, dim, bc_kind, sub, l, smooth_steps, alpha, iface_degree=0, smooth_kind=0):
        K = np.asarray(K, dtype=np.float64)  # scalar field, or diagonal tensor components stacked first
        self.K, self.h, self.dim = K, [float(v) for v in h], dim
        self.shape = cell_shape(K)
        n = [self.shape[2], self.shape[1], self.shape[0]]
        self.n = n
        self.sub = [int(v) for v in sub]
        self.l = int(l)
        self.smooth_steps = int(smooth_steps)
        if smooth_kind not in (0, 1):
            raise ValueError("smooth_kind must be 0 (additive) or 1 (multiplicative multicolour)")
        self.smooth_kind = int(smooth_kind)
        self.alpha = float(alpha)
        self.degree = int(iface_degree)
        self.nq = 1 + self.degree * (dim - 1)  # polynomial functions per side
        if self.degree not in (0, 1):
            raise ValueError("iface_degree must be 0 or 1")
        self.T = transmissibilities(K, self.h, dim, bc_kind)
        self.part = P = Partition(dim, n, self.sub, self.l)
        if self.degree == 1:
            # a linear function along a side needs two faces there, else it vanishes and the
            # coupling matrix loses a column and a row (a side of one face carries only constants)
            for s in range(P.S):
                for side in range(2 * dim):
                    if P.robin[s, side]:
                        for b in range(dim):
                            if b != side // 2 and P.box[s, 1, b] - P.box[s, 0, b] < 2:
                                raise ValueError("iface_degree 1 needs at least two faces on every Robin side")
        self.subs = []
        for s in range(P.S):
            self.subs.append(self._setup_subdomain(s))
        self._assemble_coarse()

    # ---------------------------------------------------------------- polynomial side functions
    def side_poly(self, q, pos, side, lo, hi):
        """Value at the face ``pos`` of polynomial function q on ``side`` of the box [lo, hi):
        q = 0 is the constant, q = 1 (and q = 2 in 3-D) the linear function of the first (second)
        in-plane axis, scaled to [-1, 1] over the box side."""
        if q == 0:
            return 1.0
        a = side // 2
        b = [x for x in range(3) if x != a][q - 1]
        return 2.0 * (pos[b] + 0.5 - lo[b]) / (hi[b] - lo[b]) - 1.0

    def informed_trace(self, d, q):
        """phi(f) = -beta_f u + pi on every Gamma_s face for oversampled solutions q (columns):
        F = T_f (q_c - q_c'), u = F/|f|, pi = q_c - F/tau_c (the definition of phi_i^k, Sec. 2.1)."""
        qc = q[d.g_in]
        F = (d.g_tf * (qc - q[d.g_out]).T).T
        pi = qc - (F.T / d.tau).T
        return (-(d.beta / d.area) * F.T).T + pi

    # ---------------------------------------------------------------- set-up, per subdomain
    def _setup_subdomain(self, s):
        P, K, T, h, dim, nq = self.part, self.K, self.T, self.h, self.dim, self.nq
        d = _Sub()
        d.s = s
        d.op = BoxOperator(K, T, h, dim, self.n, P.box[s, 0], P.box[s, 1], True, self.alpha, self.sub)
        # Gamma_s faces, in side order (identical to the Robin faces of the Omega_s operator)
        d.gamma = d.op.robin_faces
        d.gamma_side = np.array([f[0] for f in d.gamma], dtype=np.int64)
        d.gamma_li = np.array([f[1] for f in d.gamma], dtype=np.int64)
        d.tau = np.array([f[2] for f in d.gamma])
        d.beta = np.array([f[3] for f in d.gamma])
        d.t_r = np.array([f[4] for f in d.gamma])
        d.area = np.array([f[5] for f in d.gamma])
        d.t_f = np.array([f[6] for f in d.gamma])
        sides = [k for k in range(6) if P.robin[s, k]]
        d.sides = sides
        funcs = [(k, q) for k in sides for q in range(nq)]  # basis of Lambda_H^s, side-major
        d.funcs = funcs
        N = len(funcs)
        ng = len(d.gamma)
        gpos = [f[0] for k in sides for f in P.gamma_faces(s, k)]
        blo, bhi = P.box[s, 0], P.box[s, 1]
        # test-function values of M_H, V_H on every Gamma_s face: (nq, ng)
        d.test = np.array([[self.side_poly(q, gpos[i], int(d.gamma_side[i]), blo, bhi)
                            for i in range(ng)] for q in range(nq)]).reshape(nq, ng)
        # the oversampled Robin operator and, for every Gamma_s face, its inside / outside cells
        # in hat-Omega_s (used by the informed traces of step 1 and of the particular solve)
        d.oop = None
        if self.l > 0 and N > 0:
            olo, ohi = P.obox[s, 0], P.obox[s, 1]
            d.oop = BoxOperator(K, T, h, dim, self.n, olo, ohi, True, self.alpha, self.sub)
            g_in, g_out, g_tf = [], [], []
            for k in sides:
                for (pos, inside, outside) in P.gamma_faces(s, k):
                    g_in.append(d.oop.local_index(inside))
                    g_out.append(d.oop.local_index(outside))
                    g_tf.append(self.T[k // 2][pos[2], pos[1], pos[0]])
            d.g_in = np.array(g_in, dtype=np.int64)
            d.g_out = np.array(g_out, dtype=np.int64)
            d.g_tf = np.array(g_tf)
        # step 1: informed multiplier space
        phi = np.zeros((N, ng))
        if N > 0:
            if self.l == 0:
                for j, (k, q) in enumerate(funcs):
                    m = d.gamma_side == k
                    phi[j, m] = d.test[q, m]
            else:
                olo, ohi = P.obox[s, 0], P.obox[s, 1]
                ofaces = {k: P.side_faces(olo, ohi, k) for k in sides}
                rhs = np.zeros((d.oop.n_loc, N))
                for j, (k, q) in enumerate(funcs):
                    for (pos, inside, outside) in ofaces[k]:
                        a = k // 2
                        _tau, _beta, t_r, _area = robin_face(K, h, a, inside, outside, self.alpha, self.sub)
                        rhs[d.oop.local_index(inside), j] += t_r * self.side_poly(q, pos, k, olo, ohi)
                phi = self.informed_trace(d, d.oop.solve(rhs)).T
        d.phi = phi
        # step 2: multiscale basis functions and their side moments
        rhs = np.zeros((d.op.n_loc, N))
        for j in range(N):
            np.add.at(rhs[:, j], d.gamma_li, d.t_r * phi[j])
        d.psi = d.op.solve(rhs) if N > 0 else np.zeros((d.op.n_loc, 0))
        F = d.t_r[None, :] * (d.psi[d.gamma_li, :].T - phi)           # (N, ng)
        Pw = d.area[None, :] * phi + d.beta[None, :] * F              # |f| P
        # Fbar[side, q, j] = sum over faces of side of test_q F_j ; Pbar likewise with |f| P
        d.Fbar = np.zeros((6, nq, N))
        d.Pbar = np.zeros((6, nq, N))
        for k in sides:
            m = d.gamma_side == k
            d.Fbar[k] = d.test[:, m] @ F[:, m].T
            d.Pbar[k] = d.test[:, m] @ Pw[:, m].T
        # step 4 (set-up part): Dirichlet restriction on the oversampled region
        d.schwarz = None
        if self.smooth_steps > 0:
            d.schwarz = BoxOperator(K, T, h, dim, self.n, P.obox[s, 0], P.obox[s, 1], False, self.alpha, self.sub)
            inner = []
            for a in range(3):
                inner.append(slice(int(P.box[s, 0, a] - P.obox[s, 0, a]), int(P.box[s, 1, a] - P.obox[s, 0, a])))
            d.inner = (inner[2], inner[1], inner[0])
        return d

    # ---------------------------------------------------------------- set-up, coupling system
    def _assemble_coarse(self):
        P, nq = self.part, self.nq
        n_rows = P.E2 * nq
        self.n_coarse = n_rows
        self.coff = P.off * nq  # first coarse unknown of each subdomain
        G = np.zeros((n_rows, n_rows))
        for e, (a, s, s2) in enumerate(P.interfaces):
            lo_side, hi_side = 2 * a + 1, 2 * a  # +a side of s, -a side of s'
            d, d2 = self.subs[s], self.subs[s2]
            cs = self.coff[s] + np.arange(len(d.funcs))
            cs2 = self.coff[s2] + np.arange(len(d2.funcs))
            for q in range(nq):
                rf = 2 * nq * e + q          # flux rows of interface e
                rp = 2 * nq * e + nq + q     # pressure rows of interface e
                G[rf, cs] += d.Fbar[lo_side, q]
                G[rf, cs2] += d2.Fbar[hi_side, q]
                G[rp, cs] += d.Pbar[lo_side, q]
                G[rp, cs2] -= d2.Pbar[hi_side, q]
        self.G = G
        self._lu = None
        self._splu = None
        if n_rows == 0:
            return
        if n_rows <= 4096:
            self._lu = sla.lu_factor(G)
        else:
            self._splu = spla.splu(sp.csc_matrix(G), permc_spec="COLAMD", diag_pivot_thresh=1.0)

    def coarse_solve(self, rhs):
        if self.n_coarse == 0:
            return np.zeros(0)
        if self._lu is not None:
            return sla.lu_solve(self._lu, rhs)
        return self._splu.solve(rhs)

    # ---------------------------------------------------------------- apply
    def particular(self, r):
        """psi_s0 for every subdomain, the informed particular traces phi_s0 and the coarse
        right-hand side g0."""
        P, nq = self.part, self.nq
        psi0, phi0 = [], []
        F0 = np.zeros((P.S, 6, nq))
        P0 = np.zeros((P.S, 6, nq))
        for d in self.subs:
            rs = d.op.restrict(r).copy()
            ph = np.zeros(len(d.gamma))
            if d.oop is not None:
                # the source problem on the extended region, zero Robin data on its boundary
                ph = self.informed_trace(d, d.oop.solve(d.oop.restrict(r)))
                np.add.at(rs, d.gamma_li, d.t_r * ph)
            x = d.op.solve(rs)
            psi0.append(x)
            phi0.append(ph)
            F = d.t_r * (x[d.gamma_li] - ph)
            Pw = d.area * ph + d.beta * F
            for k in d.sides:
                m = d.gamma_side == k
                F0[d.s, k] = d.test[:, m] @ F[m]
                P0[d.s, k] = d.test[:, m] @ Pw[m]
        g0 = np.zeros(self.n_coarse)
        for e, (a, s, s2) in enumerate(P.interfaces):
            for q in range(nq):
                g0[2 * nq * e + q] = F0[s, 2 * a + 1, q] + F0[s2, 2 * a, q]
                g0[2 * nq * e + nq + q] = P0[s, 2 * a + 1, q] - P0[s2, 2 * a, q]
        self._phi0 = phi0
        return psi0, g0

    def reconstruct(self, psi0, c):
        z = np.zeros(self.shape)
        for d in self.subs:
            o = self.coff[d.s]
            zs = psi0[d.s] + d.psi @ c[o:o + len(d.funcs)]
            z[d.op.sl] = zs.reshape(d.op.w[2], d.op.w[1], d.op.w[0])
        return z

    def colour(self, s):
        """Colour of subdomain s: the parities of its grid coordinates, x in bit 0, y in bit 1, z in bit 2."""
        c = 0
        for a in range(self.dim):
            c |= (int(self.part.box[s, 0, a] // self.sub[a]) % 2) << a
        return c

    def sweep(self, r, z):
        """One restricted Schwarz sweep on A z = r: additive (all subdomains from one residual) or
        multiplicative multicolour (the additive step per colour, colours in order 0 .. 2^dim - 1,
        each from the residual after the previous colours)."""
        groups = [list(self.subs)] if self.smooth_kind == 0 else \
            [[d for d in self.subs if self.colour(d.s) == c] for c in range(2 ** self.dim)]
        z_new = z.copy()
        for group in groups:
            rho = r - matvec(self.T, z_new, self.dim)
            for d in group:
                w = d.schwarz.w
                delta = d.schwarz.solve(d.schwarz.restrict(rho)).reshape(w[2], w[1], w[0])
                z_new[d.op.sl] += delta[d.inner]
        return z_new

    def apply_parts(self, r):
        r = np.asarray(r, dtype=np.float64).reshape(self.shape)
        psi0, g0 = self.particular(r)
        c = self.coarse_solve(-g0)
        z = self.reconstruct(psi0, c)
        out = {"psi0": psi0, "phi0": self._phi0, "g0": g0, "c": c, "z_mrcm": z.copy()}
        for _ in range(self.smooth_steps):
            z = self.sweep(r, z)
        out["z"] = z
        return out

    def apply(self, r):
        return self.apply_parts(r)["z"]

    def Av(self, v):
        return matvec(self.T, np.asarray(v, dtype=np.float64).reshape(self.shape), self.dim)
