"""Pins of the oracle's fine operator A, right-hand side b and fluxes against closed forms.

* Sec. 4 case (i): both analytic solutions are reached at second order in h (the discrete problem
  is solved with scipy's conjugate gradients, not with any oracle solver).
* One-dimensional layered media: the two-point flux scheme with harmonic transmissibilities is
  exact at cell centres; the closed form is the series-resistance formula.
* A diagonal permeability tensor: second order on a manufactured solution whose source is not
  symmetric in the two components; equal components reproduce the scalar field exactly.
* Structural facts of a TPFA matrix: symmetric, positive definite, non-positive off-diagonals,
  A 1 equal to the Dirichlet half transmissibilities.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle import grid
from paper_2606_08883_gb300 import workloads as W


def _cg_solve(prob):
    T = grid.transmissibilities(prob.K, prob.h, prob.dim, prob.bc_kind)
    b = grid.rhs(prob.K, prob.h, prob.dim, prob.bc_kind, prob.bc_val, prob.f)
    shape = grid.cell_shape(prob.K)
    op = spla.LinearOperator((b.size, b.size), matvec=lambda v: grid.matvec(T, v.reshape(shape), prob.dim).ravel())
    x, info = spla.cg(op, b.ravel(), rtol=1e-13, maxiter=20000)
    assert info == 0
    return x.reshape(shape)


@pytest.mark.parametrize("variable", [False, True])
def test_second_order_convergence(variable):
    errs = []
    for N in (16, 32, 64):
        prob, exact = W.analytic(N, variable)
        p = _cg_solve(prob)
        errs.append(np.sqrt(np.mean((p - exact) ** 2)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > 1.8, (errs, rates)
    assert errs[-1] < 2e-3


def _anisotropic(N, kx, ky):
    """Diagonal K = diag(kx, ky) on the unit square, p = cos(pi x) cos(2 pi y): -div(K grad p) =
    (kx + 4 ky) pi^2 p, Dirichlet data from p on x = 0, 1, no flow on y = 0, 1 (dp/dy = 0 there).
    The source is not symmetric in kx and ky, so a swapped axis shows."""
    h = (1.0 / N, 1.0 / N, 1.0)
    xc = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    exact = np.cos(np.pi * X) * np.cos(2 * np.pi * Y)
    K = np.stack([np.full((1, N, N), kx), np.full((1, N, N), ky)])
    f = ((kx + 4 * ky) * np.pi ** 2 * exact * h[0] * h[1])[None]
    yv = (np.arange(N) + 0.5) / N
    bc_val = [np.cos(2 * np.pi * yv)[None], -np.cos(2 * np.pi * yv)[None], None, None, None, None]
    prob = W.Problem(2, (N, N, 1), h, K, [0, 0, 1, 1, 1, 1], bc_val, f, name="anisotropic")
    return prob, exact[None]


def test_diagonal_tensor_second_order_convergence():
    for kx, ky in ((1.0, 25.0), (25.0, 1.0)):
        errs = []
        for N in (16, 32, 64):
            prob, exact = _anisotropic(N, kx, ky)
            errs.append(np.sqrt(np.mean((_cg_solve(prob) - exact) ** 2)))
        rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
        assert min(rates) > 1.8, (kx, ky, errs, rates)
        assert errs[-1] < 2e-3


def test_diagonal_tensor_with_equal_components_is_the_scalar_field():
    prob = W.random_problem((9, 7, 1), seed=3, contrast=1e3)
    Kt = np.stack([prob.K, prob.K])
    for a, (T1, T2) in enumerate(zip(grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind),
                                     grid.transmissibilities(Kt, prob.h, 2, prob.bc_kind))):
        assert np.array_equal(T1, T2), a
    assert np.array_equal(grid.rhs(prob.K, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f),
                          grid.rhs(Kt, prob.h, 2, prob.bc_kind, prob.bc_val, prob.f))


def test_layered_series_resistance_exact():
    rng = np.random.default_rng(3)
    nx, ny = 24, 5
    kx = 10.0 ** rng.uniform(-3, 3, size=nx)           # K depends on x only
    K = np.tile(kx, (ny, 1))[None]
    h = (1.0 / nx, 0.3 / ny, 1.0)
    gl, gr = 2.5, -0.75
    prob = W.Problem(2, (nx, ny, 1), h, K, [0, 0, 1, 1, 1, 1],
                     [np.full((1, ny), gl), np.full((1, ny), gr), None, None, None, None], None)
    p = _cg_solve(prob)
    # series resistances per unit area: each cell contributes h_x / K_c, split in two halves
    half = 0.5 * h[0] / kx
    R = 2.0 * half.sum()
    q = (gl - gr) / R                                 # Darcy velocity along +x
    centre = gl - q * (np.cumsum(2.0 * half) - half)  # drop from the left face to each centre
    assert np.allclose(p[0], centre[None, :], rtol=0, atol=1e-10 * abs(gl - gr))
    u = grid.fluxes(grid.transmissibilities(K, h, 2, prob.bc_kind), p, h, 2, prob.bc_kind, prob.bc_val)
    assert np.allclose(u[0], q, rtol=1e-9)
    assert np.allclose(u[1], 0.0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_matrix_structure(dim):
    n = (5, 4, 3) if dim == 3 else (6, 5, 1)
    prob = W.random_problem(n, dim=dim, seed=7, contrast=1e3,
                            bc_kind=[0, 1, 0, 1, 1, 1] if dim == 2 else [0, 1, 1, 0, 1, 1])
    T = grid.transmissibilities(prob.K, prob.h, dim, prob.bc_kind)
    A = grid.dense_matrix(T, dim, prob.K.shape)
    assert np.allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    off = A - np.diag(np.diag(A))
    assert off.max() <= 0
    # row sums: only Dirichlet faces leave a net diagonal term (half transmissibility of the cell)
    rs = A.sum(axis=1).reshape(prob.K.shape)
    expect = np.zeros_like(rs)
    for a in range(dim):
        tau = grid.half_transmissibility(prob.K, prob.h, a)
        for d, cell in ((0, 0), (1, prob.K.shape[grid.np_axis(a)] - 1)):
            if prob.bc_kind[2 * a + d] == 0:
                sl = [slice(None)] * 3
                sl[grid.np_axis(a)] = cell
                expect[tuple(sl)] += tau[tuple(sl)]
    assert np.allclose(rs, expect, rtol=1e-12, atol=1e-12 * np.abs(A).max())


def test_neumann_data_enters_with_outward_sign():
    # unit square, K = 1, p = 0 at x = 0, prescribed outward velocity z at x = 1: u = z everywhere
    N, z = 8, 0.7
    prob = W.Problem(2, (N, N, 1), (1.0 / N, 1.0 / N, 1.0), np.ones((1, N, N)), [0, 1, 1, 1, 1, 1],
                     [None, np.full((1, N), z), None, None, None, None], None)
    p = _cg_solve(prob)
    # u = -dp/dx = z  =>  p = -z x at cell centres (exact for a linear field)
    xc = (np.arange(N) + 0.5) / N
    assert np.allclose(p[0], -z * xc[None, :], atol=1e-10)
    u = grid.fluxes(grid.transmissibilities(prob.K, prob.h, 2, prob.bc_kind), p, prob.h, 2, prob.bc_kind, prob.bc_val)
    assert np.allclose(u[0], z, atol=1e-9)


def test_oracle_package_exports():
    assert oracle.SIDES[0] == "-x" and oracle.DIRICHLET == 0 and oracle.NEUMANN == 1
