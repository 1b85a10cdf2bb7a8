"""Whole-problem driver: assemble A and b, build T, run GMRES (Sec. 3 and Algorithm 1).

Arguments mirror the library's problem / parameter structs, as plain numpy data:
K (nz, ny, nx) > 0, or a diagonal tensor (d, nz, ny, nx) with its x, y (, z) components; h = (hx, hy, hz); dim 2 or 3; bc_kind[6] (0 Dirichlet, 1 Neumann) for the sides
-x, +x, -y, +y, -z, +z; bc_val[6] (None or the per-face data of that side); f (cell-integrated
source or None); sub[3]; l; smooth_steps; alpha; tol; tol_relative; restart; max_iter;
smooth_kind (0 additive, 1 multiplicative multicolour Schwarz sweeps).
"""

import numpy as np

from .grid import cell_shape, rhs, fluxes
from .mrcm import MRCMOS
from .gmres import fgmres


def build(K, h, dim, bc_kind, sub, l, smooth_steps, alpha, iface_degree=0, smooth_kind=0):
    return MRCMOS(K, h, dim, bc_kind, sub, l, smooth_steps, alpha, iface_degree, smooth_kind)


def solve(K, h, dim, bc_kind, bc_val=None, f=None, sub=(16, 16, 1), l=2, smooth_steps=1,
          alpha=10.0, tol=1e-8, tol_relative=True, restart=30, max_iter=1000, p0=None, pre=None, check_every_step=True,
          iface_degree=0, smooth_kind=0):
    K = np.asarray(K, dtype=np.float64)
    if pre is None:
        pre = build(K, h, dim, bc_kind, sub, l, smooth_steps, alpha, iface_degree, smooth_kind)
    b = rhs(K, h, dim, bc_kind, bc_val, f)
    shape = cell_shape(K)

    def apply_A(v):
        return pre.Av(v.reshape(shape)).ravel()

    def apply_T(v):
        return pre.apply(v.reshape(shape)).ravel()

    p, info = fgmres(apply_A, apply_T, b.ravel(), None if p0 is None else np.ravel(p0), tol,
                     tol_relative, restart, max_iter, check_every_step)
    p = p.reshape(shape)
    info["b"] = b
    info["u"] = fluxes(pre.T, p, h, dim, bc_kind, bc_val)
    return p, info, pre


def apply_precond(K, h, dim, bc_kind, sub, l, smooth_steps, alpha, r, smooth_kind=0):
    pre = build(K, h, dim, bc_kind, sub, l, smooth_steps, alpha, smooth_kind=smooth_kind)
    return pre.apply(np.asarray(r, dtype=np.float64).reshape(cell_shape(K)))
