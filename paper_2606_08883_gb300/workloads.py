"""Seeded synthetic inputs: permeability fields, boundary data and sources.

This module only generates problem data; it holds none of the method's arithmetic and is shared
by the tests, the benchmark and (as plain numpy arrays) the FP64 oracle.

Fields stand in for the paper's data sets, which are not available here: the analytic problems of
Sec. 4 case (i) are reproduced exactly; the SPE10 layers (case (ii)) and the thin-inclusion fields
(case (iii)) are replaced by seeded synthetic fields of the same character (sinuous high-contrast
channels, log-normal Gaussian random fields).

Array layout: (nz, ny, nx), x fastest.  Sides: -x, +x, -y, +y, -z, +z.  ``f`` is the source
integrated over each cell (midpoint rule for analytic densities).
"""

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

DIRICHLET, NEUMANN = 0, 1
PREC_FP64, PREC_FP32 = 0, 1


@dataclass
class Problem:
    dim: int
    n: tuple                      # cells per axis (nx, ny, nz)
    h: tuple                      # cell size per axis (hz = slab thickness in 2-D)
    K: np.ndarray                 # (nz, ny, nx) > 0
    bc_kind: List[int]            # 6 sides
    bc_val: List[Optional[np.ndarray]] = field(default_factory=lambda: [None] * 6)
    f: Optional[np.ndarray] = None
    name: str = ""

    @property
    def cells(self):
        return int(self.n[0] * self.n[1] * self.n[2])


@dataclass
class Params:
    sub: tuple = (16, 16, 1)
    oversample: int = 2
    smooth_steps: int = 1
    alpha: float = 10.0
    tol: float = 1e-8
    tol_relative: int = 1
    restart: int = 30
    max_iter: int = 500
    local_prec: int = PREC_FP64
    smooth_kind: int = 0          # 0 additive, 1 multiplicative multicolour Schwarz sweeps
    iface_degree: int = 0         # 0 piecewise-constant, 1 piecewise-linear side functions
    coarse_pivoting: int = 0      # 0 no-pivot coupling LU with a pivoted fallback, 1 always pivoted
    refine_setup: int = 0         # FP32 set-up solves refined once against the FP64 box operators: 1 all, 2 basis only
    coarse_solver: int = 0        # 0: nested-dissection multifrontal G (large 2-D systems); 1: band LU


# ---------------------------------------------------------------------------------------------
# Sec. 4 case (i): closed-form solutions on the unit square, Dirichlet x = 0, 1; Neumann y = 0, 1
# ---------------------------------------------------------------------------------------------

def analytic(N, variable=False):
    """(problem, exact cell-centre pressure).  Constant case: kappa = 1, p = cos 2pi x cos 2pi y.
    Variable case: kappa = 1 + sin pi x sin pi y, p = cos pi x cos pi y; its Dirichlet data are taken
    from the exact solution (cos pi y at x = 0, -cos pi y at x = 1)."""
    h = (1.0 / N, 1.0 / N, 1.0)
    xc = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    if variable:
        K = 1.0 + np.sin(np.pi * X) * np.sin(np.pi * Y)
        fd = 2 * np.pi ** 2 * np.cos(np.pi * X) * np.cos(np.pi * Y) * (1 + 2 * np.sin(np.pi * X) * np.sin(np.pi * Y))
        gl, gr = np.cos(np.pi * xc), -np.cos(np.pi * xc)
        exact = np.cos(np.pi * X) * np.cos(np.pi * Y)
    else:
        K = np.ones((N, N))
        fd = 8 * np.pi ** 2 * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)
        gl = gr = np.cos(2 * np.pi * xc)
        exact = np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    prob = Problem(2, (N, N, 1), h, K[None].copy(), [DIRICHLET, DIRICHLET, NEUMANN, NEUMANN, NEUMANN, NEUMANN],
                   [gl[None, :].copy(), gr[None, :].copy(), None, None, None, None],
                   (fd * h[0] * h[1])[None].copy(), name=f"analytic-{'variable' if variable else 'constant'}-{N}")
    return prob, exact[None]


# ---------------------------------------------------------------------------------------------
# Gaussian random fields by circulant embedding (Dietrich and Newsam, 1997)
# ---------------------------------------------------------------------------------------------

def grf(shape, h, corr, variance, seed, max_pad=8):
    """Zero-mean stationary Gaussian field with covariance variance * exp(-|d/corr|), d the
    separation vector scaled per axis by ``corr`` (a length per axis, (z, y, x) order like
    ``shape``).  Negative embedding eigenvalues below 1e-10 of the largest are clipped."""
    shape = tuple(int(s) for s in shape)
    corr = np.broadcast_to(np.asarray(corr, dtype=np.float64), (len(shape),))
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (len(shape),))
    rng = np.random.default_rng(seed)
    for pad in range(2, max_pad + 1):
        M = tuple(max(pad * s, 2) for s in shape)
        grids = np.meshgrid(*[np.minimum(np.arange(m), m - np.arange(m)) * h[i] / corr[i]
                              for i, m in enumerate(M)], indexing="ij")
        dist = np.sqrt(sum(g * g for g in grids))
        c = variance * np.exp(-dist)
        lam = np.fft.fftn(c).real
        if lam.min() >= -1e-10 * lam.max():
            break
    lam = np.maximum(lam, 0.0)
    xi = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    y = np.fft.fftn(np.sqrt(lam / lam.size) * xi)
    return np.ascontiguousarray(y.real[tuple(slice(0, s) for s in shape)])


def lognormal_field(n, h, corr, variance, seed):
    """K = exp(G) on a (nz, ny, nx) grid; corr is a length or (z, y, x) lengths."""
    shape = (n[2], n[1], n[0])
    hh = (h[2], h[1], h[0])
    return np.exp(grf(shape, hh, corr, variance, seed))


def channel_field(N, fill=0.30, contrast=1e6, seed=1):
    """Binary channelised field on the unit square: background 1, sinuous x-aligned channels of
    permeability ``contrast`` added until the channel fraction reaches ``fill``."""
    rng = np.random.default_rng(seed)
    xc = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    mask = np.zeros((N, N), dtype=bool)
    while mask.mean() < fill:
        y0 = rng.uniform(0.0, 1.0)
        amp = rng.uniform(0.02, 0.10)
        lam = rng.uniform(0.2, 0.6)
        ph = rng.uniform(0.0, 2 * np.pi)
        width = rng.uniform(0.01, 0.03)
        centre = y0 + amp * np.sin(2 * np.pi * X / lam + ph)
        mask |= np.abs(Y - centre) < 0.5 * width
    K = np.where(mask, contrast, 1.0)
    return K[None].copy()


def _flow_problem(dim, n, h, K, name):
    """p = 1 at x = 0, p = 0 at x = 1, no-flow elsewhere, no source (Sec. 4 cases (ii), (iii))."""
    if dim == 2:
        left = np.ones((1, n[1]))
        right = np.zeros((1, n[1]))
    else:
        left = np.ones((n[2], n[1]))
        right = np.zeros((n[2], n[1]))
    return Problem(dim, tuple(n), tuple(h), K, [DIRICHLET, DIRICHLET, NEUMANN, NEUMANN, NEUMANN, NEUMANN],
                   [left, right, None, None, None, None], None, name=name)


def flow_window(K, h, name="window"):
    """The flow problem of ``_flow_problem`` (p = 1 / 0 on the first / last x face, no flow across
    the others, no source) on a block of cells cut from a larger field: K (nz, ny, nx) is the block,
    h the cell size of the field it came from."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    n = (K.shape[2], K.shape[1], K.shape[0])
    dim = 2 if K.shape[0] == 1 else 3
    return _flow_problem(dim, n, tuple(h), K, name)


# ---------------------------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------------------------

def quarter_five_spot(N=64, seed=1):
    """2-D N x N, log-permeability GRF (exponential covariance, correlation length 0.1, variance
    2), Dirichlet 0 at x = 0 and x = 1, no-flow top and bottom, source +1 in cell (0, 0) and -1 in
    cell (N-1, N-1); 4 x 4 subdomains, oversampling 2, 1 smoothing step, GMRES(30) to 1e-8."""
    h = (1.0 / N, 1.0 / N, 1.0)
    K = lognormal_field((N, N, 1), h, 0.1, 2.0, seed)
    f = np.zeros((1, N, N))
    f[0, 0, 0] = 1.0
    f[0, N - 1, N - 1] = -1.0
    prob = Problem(2, (N, N, 1), h, K, [DIRICHLET, DIRICHLET, NEUMANN, NEUMANN, NEUMANN, NEUMANN],
                   [np.zeros((1, N)), np.zeros((1, N)), None, None, None, None], f,
                   name=f"qfs-grf-{N}x{N}-seed{seed}")
    params = Params(sub=(N // 4, N // 4, 1), oversample=2, smooth_steps=1, alpha=10.0, tol=1e-8,
                    tol_relative=1, restart=30, max_iter=500, local_prec=PREC_FP64)
    return prob, params


def channels(N=512, seed=1, sub=32, oversample=4, smooth_steps=2, prec=PREC_FP64):
    """2-D N x N binary channelised field (30 % fill, contrast 1e6), p = 1 / 0 on x = 0 / 1,
    16 x 16 subdomains of 32 x 32 at N = 512, oversampling 4, 2 smoothing steps, FP64, GMRES(30)
    (the workload fixes no restart length; 30 is the one the 64 x 64 workload states)."""
    h = (1.0 / N, 1.0 / N, 1.0)
    K = channel_field(N, 0.30, 1e6, seed)
    prob = _flow_problem(2, (N, N, 1), h, K, f"channels-{N}x{N}-seed{seed}")
    params = Params(sub=(sub, sub, 1), oversample=oversample, smooth_steps=smooth_steps, alpha=10.0, tol=1e-8,
                    tol_relative=1, restart=30, max_iter=600, local_prec=prec)
    return prob, params


def lognormal(N=2048, seed=1, variance=4.0, corr=0.05, sub=32, oversample=2, smooth_steps=1, prec=PREC_FP32):
    """2-D N x N log-normal field (variance 4, correlation length 0.05), p = 1 / 0 on x = 0 / 1,
    subdomains of 32 x 32, oversampling 2, 1 smoothing step, FP32 local solves with the basis
    solves refined once against the FP64 box operators (which keeps the GMRES count at the FP64
    one; refining the informed-space solves too changes no count on this field)."""
    h = (1.0 / N, 1.0 / N, 1.0)
    K = lognormal_field((N, N, 1), h, corr, variance, seed)
    prob = _flow_problem(2, (N, N, 1), h, K, f"lognormal-{N}x{N}-var{variance}-seed{seed}")
    params = Params(sub=(sub, sub, 1), oversample=oversample, smooth_steps=smooth_steps, alpha=10.0, tol=1e-8,
                    tol_relative=1, restart=30, max_iter=500, local_prec=prec,
                    refine_setup=2 if prec == PREC_FP32 else 0)
    return prob, params


def random_problem(n, dim=2, seed=0, contrast=10.0, bc_kind=None, source=True, dirichlet_data=True, tensor=False):
    """Small random test problem: K = contrast ** U(0, 1) per cell, random boundary data and source.
    tensor=True: a diagonal tensor, each of its dim components drawn independently (stacked first,
    x, y, z order)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    shape = (nz, ny, nx)
    K = contrast ** rng.uniform(0.0, 1.0, size=((dim,) + shape) if tensor else shape)
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz if dim == 3 else 1.0)
    if bc_kind is None:
        bc_kind = [DIRICHLET, DIRICHLET, NEUMANN, NEUMANN, NEUMANN, NEUMANN]
    layers = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
    bc_val = []
    for side in range(6):
        if side // 2 >= dim or not dirichlet_data:
            bc_val.append(None)
        else:
            bc_val.append(rng.uniform(-1.0, 1.0, size=layers[side]))
    f = rng.uniform(-1.0, 1.0, size=shape) * (h[0] * h[1] * h[2]) if source else None
    return Problem(dim, tuple(n), h, K, list(bc_kind), bc_val, f, name=f"random-{nx}x{ny}x{nz}-seed{seed}")
