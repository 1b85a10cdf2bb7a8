"""Local operators on boxes: Robin problems (Eq. 5-6, Eq. 11-12, Eq. 15) and the Dirichlet
restriction A[D, D] used by the overlapping-Schwarz sweeps.

Robin condition on a face f of the box boundary that is interior to the domain (Eq. 5):
-beta u.n + p = lambda, u the outward velocity, with beta = alpha H / K_H (Eq. 6), K_H the
harmonic mean of the two cells touching f and H the subdomain edge length along the face normal.
With the half transmissibility tau_c of the inside cell, the face pressure pi_f and the outward
flux F = tau_c (p_c - pi_f), the condition pi_f = lambda + beta F / |f| gives

    F = t_R (p_c - lambda),   t_R = (1/tau_c + beta/|f|)^-1.

So the Robin operator of a box D is A[D, D] with, for every such face, T_f replaced by t_R on the
diagonal, and Robin data lambda enters the right-hand side as t_R lambda.  Faces on the domain
boundary keep their entries of A with zero data (homogeneous conditions, Sec. 3).

Local unknowns are ordered x fastest; the operator is stored in LAPACK lower band form and
factored / solved with LAPACK's band Cholesky (scipy.linalg.cholesky_banded / cho_solve_banded).

Pinned by: dense solves of the same operator built independently, per-cell mass balance of the
local solution including the Robin boundary fluxes (tests/test_oracle_local.py).
"""

import numpy as np
import scipy.linalg as sla

from .grid import face_area, k_axis, np_axis


def robin_face(K, h, a, inside, outside, alpha, sub):
    """(tau_in, beta, t_R, |f|) of the face between cell ``inside`` and cell ``outside`` (x,y,z)."""
    area = face_area(h, a)
    Ka = k_axis(K, a)  # the component across the face for a diagonal tensor
    k_in = Ka[inside[2], inside[1], inside[0]]
    k_out = Ka[outside[2], outside[1], outside[0]]
    tau = 2.0 * k_in * area / h[a]
    k_h = 2.0 * k_in * k_out / (k_in + k_out)
    beta = alpha * (sub[a] * h[a]) / k_h
    t_r = 1.0 / (1.0 / tau + beta / area)
    return tau, beta, t_r, area


def face_T(T, a, pos):
    return T[a][pos[2], pos[1], pos[0]]


class BoxOperator:
    """Robin (``robin=True``) or Dirichlet-restriction (``robin=False``) operator on [lo, hi)."""

    def __init__(self, K, T, h, dim, n, lo, hi, robin, alpha, sub):
        self.lo = [int(v) for v in lo]
        self.hi = [int(v) for v in hi]
        w = [self.hi[a] - self.lo[a] for a in range(3)]
        self.w = w
        self.n_loc = w[0] * w[1] * w[2]
        sl = (slice(self.lo[2], self.hi[2]), slice(self.lo[1], self.hi[1]), slice(self.lo[0], self.hi[0]))
        self.sl = sl
        strides = (1, w[0], w[0] * w[1])
        self.strides = strides
        bw = 0
        for a in range(dim):
            if w[a] > 1:
                bw = max(bw, strides[a])
        self.bw = bw
        # diagonal: every face of every cell of the box, as in A
        diag = np.zeros((w[2], w[1], w[0]))
        for a in range(dim):
            Ta = T[a]
            ax = np_axis(a)
            lo_faces = [slice(self.lo[2], self.hi[2]), slice(self.lo[1], self.hi[1]), slice(self.lo[0], self.hi[0])]
            hi_faces = list(lo_faces)
            hi_faces[ax] = slice(self.lo[a] + 1, self.hi[a] + 1)
            diag += Ta[tuple(lo_faces)] + Ta[tuple(hi_faces)]
        ab = np.zeros((bw + 1, self.n_loc))
        # couplings between box cells
        for a in range(dim):
            if w[a] < 2:
                continue
            ax = np_axis(a)
            inner = [slice(self.lo[2], self.hi[2]), slice(self.lo[1], self.hi[1]), slice(self.lo[0], self.hi[0])]
            inner[ax] = slice(self.lo[a] + 1, self.hi[a])  # faces strictly inside the box along a
            t_in = T[a][tuple(inner)]  # shape: w with w[a] - 1 along ax
            band = np.zeros((w[2], w[1], w[0]))
            dst = [slice(None)] * 3
            dst[ax] = slice(0, w[a] - 1)  # coupling stored at the lower cell: A[c + e_a, c]
            band[tuple(dst)] = -t_in
            ab[strides[a]] = band.ravel()
        # Robin faces: boundary faces of the box interior to the domain
        self.robin_faces = []  # (side, local inside index, tau, beta, t_R, area, T_f)
        for a in range(dim):
            for d in (0, 1):
                plane = self.lo[a] if d == 0 else self.hi[a]
                if plane == 0 or plane == n[a]:
                    continue
                others = [b for b in range(3) if b != a]
                b1, b2 = others
                for t2 in range(self.lo[b2], self.hi[b2]):
                    for t1 in range(self.lo[b1], self.hi[b1]):
                        pos = [0, 0, 0]
                        pos[a], pos[b1], pos[b2] = plane, t1, t2
                        inside, outside = list(pos), list(pos)
                        if d == 0:
                            outside[a] = plane - 1
                        else:
                            inside[a] = plane - 1
                        tau, beta, t_r, area = robin_face(K, h, a, inside, outside, alpha, sub)
                        t_f = face_T(T, a, pos)
                        li = self.local_index(inside)
                        if robin:
                            diag.ravel()[li] += t_r - t_f
                        self.robin_faces.append((2 * a + d, li, tau, beta, t_r, area, t_f))
        ab[0] = diag.ravel()
        self.ab = ab
        self.chol = sla.cholesky_banded(ab, lower=True)

    def local_index(self, c):
        return (c[0] - self.lo[0]) + self.w[0] * ((c[1] - self.lo[1]) + self.w[1] * (c[2] - self.lo[2]))

    def solve(self, rhs):
        """x = D^-1 rhs for one right-hand side (1-D) or several (columns of a 2-D array)."""
        return sla.cho_solve_banded((self.chol, True), rhs)

    def restrict(self, v):
        """Values of a global cell field on the box, local ordering."""
        return v[self.sl].ravel()

    def dense(self):
        """The operator as a dense matrix (tests on tiny boxes)."""
        n = self.n_loc
        M = np.zeros((n, n))
        for t in range(self.bw + 1):
            for j in range(n - t):
                M[j + t, j] = self.ab[t, j]
                M[j, j + t] = self.ab[t, j]
        return M
