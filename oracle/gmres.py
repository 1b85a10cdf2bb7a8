"""Restarted right-preconditioned GMRES storing Z = [z_1..z_m] (Algorithm 1, Sec. 3).

Per cycle: r0 = b - A p0, beta = ||r0||, v1 = r0/beta; for j = 1..m: z_j = T v_j, w = A z_j,
modified Gram-Schmidt h_ij = (w, v_i), w -= h_ij v_i (i = 1..j), h_{j+1,j} = ||w||,
v_{j+1} = w / h_{j+1,j}.  The least-squares problem min ||beta e1 - H y|| is reduced with Givens
rotations as the cycle goes, so |g_{j+1}| is the residual norm of the iterate p0 + Z_j y_j.

Readings where Algorithm 1 is silent: the estimate |g_{j+1}| is checked after every inner step
(the paper's tables report one or two iterations with Krylov dimension 10); when it meets the
tolerance, or at j = m, or on a lucky breakdown (h_{j+1,j} <= 1e-14 ||A z_j||), the iterate
p = p0 + Z y is formed and the true residual ||b - A p|| decides whether to stop or restart.
``iterations`` counts applications of T.  Tolerance: ||b - A p|| <= tol * ||b|| (relative) or
<= tol (absolute, as in the paper's tables); b = 0 with a relative tolerance returns p = 0.

Pinned by: a textbook GMRES (scipy.sparse.linalg.gmres) on the explicit matrix A T giving the
same residual history, and the converged p matching a direct solve (tests/test_oracle_gmres.py).
"""

import numpy as np

CONVERGED, NOT_CONVERGED = 0, 4


def _givens(a, b):
    if b == 0.0:
        return 1.0, 0.0, a
    t = float(np.hypot(a, b))
    return a / t, b / t, t


def fgmres(apply_A, apply_T, b, p0=None, tol=1e-8, tol_relative=True, m=30, max_iter=1000,
           check_every_step=True):
    b = np.asarray(b, dtype=np.float64).ravel()
    n = b.size
    p = np.zeros(n) if p0 is None else np.array(p0, dtype=np.float64).ravel().copy()
    info = {"iterations": 0, "restarts": 0, "cycles": 0, "history": [], "status": CONVERGED}
    bnorm = float(np.linalg.norm(b))
    if tol_relative and bnorm == 0.0:
        p[:] = 0.0
        info.update(abs_res=0.0, rel_res=0.0)
        return p, info
    tol_abs = tol * bnorm if tol_relative else tol
    r = b - apply_A(p)
    beta = float(np.linalg.norm(r))
    info["history"].append(beta)
    it = 0
    while True:
        if beta <= tol_abs:
            break
        if it >= max_iter:
            info["status"] = NOT_CONVERGED
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = apply_T(V[j])
            Z.append(z)
            it += 1
            w = apply_A(z)
            w_norm0 = float(np.linalg.norm(w))
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            hnext = H[j + 1, j]
            for i in range(j):
                t0 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                t1 = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j], H[i + 1, j] = t0, t1
            cs[j], sn[j], H[j, j] = _givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            info["history"].append(abs(g[j + 1]))
            k = j + 1
            breakdown = hnext <= 1e-14 * w_norm0
            if breakdown or it >= max_iter or (check_every_step and abs(g[j + 1]) <= tol_abs):
                break
            V.append(w / hnext)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            p = p + y[i] * Z[i]
        info["cycles"] += 1
        r = b - apply_A(p)
        beta = float(np.linalg.norm(r))
        info["history"].append(beta)
        if beta <= tol_abs:
            break
        if it >= max_iter:
            info["status"] = NOT_CONVERGED
            break
        info["restarts"] += 1
    info["iterations"] = it
    info["abs_res"] = beta
    info["rel_res"] = beta / bnorm if bnorm > 0 else 0.0
    return p, info
