"""Fine-grid operator A, right-hand side b and face fluxes (Sec. 3, Eq. 1a-1d).

The paper discretises the Darcy system u = -K grad p, div u = f with lowest-order Raviart-Thomas
elements and statically condenses it to A p = b in cell pressures.  Reading used here: on a
Cartesian mesh with the trapezoidal rule for the velocity mass matrix that condensation is the
two-point flux scheme with harmonic transmissibilities:

* half transmissibility of cell c toward a face normal to axis a: tau = 2 K_c |f| / h_a,
* interior face: T_f = (1/tau_c + 1/tau_c')^-1,
* Dirichlet face (p = g): T_f = tau_c and b_c += tau_c g_f,
* Neumann face (u.n = z): T_f = 0 and b_c -= |f| z_f,
* (A p)_c = sum_f T_f (p_c - p_nb(f)) with p_nb = 0 outside the domain,
* b_c += f_c, the cell-integrated source.

Arrays are numpy float64 with shape (nz, ny, nx): x is the fastest axis.  Physical axis a
(0 = x, 1 = y, 2 = z) is numpy axis 2 - a.  The face array of axis a has one more entry along that
axis: entry i separates cells i-1 and i.  A 2-D problem has nz = 1 and h[2] is the slab thickness.

Pinned by: second-order convergence to the paper's two closed-form solutions (Sec. 4, constant and
variable permeability), symmetry / zero row sums / positive definiteness of the assembled matrix,
and exact reproduction of a linear pressure field (tests/test_oracle_grid.py).
"""

import numpy as np

SIDES = ("-x", "+x", "-y", "+y", "-z", "+z")
DIRICHLET, NEUMANN = 0, 1


def np_axis(a):
    """numpy axis holding physical axis a (0 = x, 1 = y, 2 = z)."""
    return 2 - a


def take(arr, a, idx):
    """arr indexed along physical axis a by ``idx`` (an int or a slice)."""
    sl = [slice(None)] * arr.ndim
    sl[np_axis(a)] = idx
    return arr[tuple(sl)]


def put(arr, a, idx, value):
    sl = [slice(None)] * arr.ndim
    sl[np_axis(a)] = idx
    arr[tuple(sl)] = value


def face_area(h, a):
    """|f| of a face normal to axis a."""
    out = 1.0
    for b in range(3):
        if b != a:
            out *= h[b]
    return out


def cell_shape(K):
    """(nz, ny, nx) of a permeability given as a scalar field (nz, ny, nx) or as the diagonal of a
    tensor, components stacked first (d, nz, ny, nx) in x, y, z order."""
    return np.shape(K)[-3:]


def k_axis(K, a):
    """The permeability that acts across faces normal to axis a: the scalar field, or the a-th
    diagonal component of the tensor."""
    K = np.asarray(K, dtype=np.float64)
    return K[a] if K.ndim == 4 else K


def half_transmissibility(K, h, a):
    """tau_{c,f} = 2 K_c |f| / h_a for the faces of every cell normal to axis a (K_c the component
    along a for a diagonal tensor)."""
    return 2.0 * k_axis(K, a) * face_area(h, a) / h[a]


def transmissibilities(K, h, dim, bc_kind):
    """Face transmissibilities [Tx, Ty, Tz]; axes at or beyond ``dim`` carry no flow (all zero)."""
    T = []
    for a in range(3):
        shape = list(cell_shape(K))
        shape[np_axis(a)] += 1
        Ta = np.zeros(shape)
        if a < dim:
            n_a = cell_shape(K)[np_axis(a)]
            tau = half_transmissibility(K, h, a)
            if n_a > 1:
                t_lo = take(tau, a, slice(0, n_a - 1))
                t_hi = take(tau, a, slice(1, n_a))
                put(Ta, a, slice(1, n_a), 1.0 / (1.0 / t_lo + 1.0 / t_hi))
            if bc_kind[2 * a] == DIRICHLET:
                put(Ta, a, 0, take(tau, a, 0))
            if bc_kind[2 * a + 1] == DIRICHLET:
                put(Ta, a, n_a, take(tau, a, n_a - 1))
        T.append(Ta)
    return T


def rhs(K, h, dim, bc_kind, bc_val=None, f=None):
    """b = f + Dirichlet terms - Neumann terms.

    ``bc_val[side]`` is None (zero data) or an array shaped like the layer of cells touching that
    side: (nz, ny) for +-x, (nz, nx) for +-y, (ny, nx) for +-z.  Dirichlet data is the face
    pressure g, Neumann data the outward normal velocity z.
    """
    b = np.zeros(cell_shape(K)) if f is None else np.array(f, dtype=np.float64, copy=True)
    for a in range(dim):
        n_a = cell_shape(K)[np_axis(a)]
        tau = half_transmissibility(K, h, a)
        for d, cell in ((0, 0), (1, n_a - 1)):
            side = 2 * a + d
            if bc_val is None or bc_val[side] is None:
                continue
            val = np.asarray(bc_val[side], dtype=np.float64)
            layer = take(b, a, slice(cell, cell + 1))
            if bc_kind[side] == DIRICHLET:
                layer += np.expand_dims(take(tau, a, cell) * val, np_axis(a))
            else:
                layer -= face_area(h, a) * np.expand_dims(val, np_axis(a))
            put(b, a, slice(cell, cell + 1), layer)
    return b


def _face_flow(Ta, v, a, bc_side_values=(0.0, 0.0)):
    """Flow T_f (v_left - v_right) through every face of axis a (positive along +a).

    Outside the domain v takes the given boundary values (zero for the homogeneous operator).
    """
    lo_pad, hi_pad = bc_side_values
    lo = np.broadcast_to(np.expand_dims(np.asarray(lo_pad, dtype=np.float64), np_axis(a))
                         if np.ndim(lo_pad) else lo_pad, take(v, a, slice(0, 1)).shape)
    hi = np.broadcast_to(np.expand_dims(np.asarray(hi_pad, dtype=np.float64), np_axis(a))
                         if np.ndim(hi_pad) else hi_pad, take(v, a, slice(0, 1)).shape)
    vpad = np.concatenate([lo, v, hi], axis=np_axis(a))
    n_a = v.shape[np_axis(a)]
    left = take(vpad, a, slice(0, n_a + 1))
    right = take(vpad, a, slice(1, n_a + 2))
    return Ta * (left - right)


def matvec(T, v, dim):
    """(A v)_c = sum over faces of c of T_f (v_c - v_nb), v_nb = 0 outside the domain."""
    w = np.zeros_like(v)
    for a in range(dim):
        n_a = v.shape[np_axis(a)]
        F = _face_flow(T[a], v, a)
        w += take(F, a, slice(1, n_a + 1)) - take(F, a, slice(0, n_a))
    return w


def fluxes(T, p, h, dim, bc_kind, bc_val=None):
    """Darcy normal velocity u_f (positive along +a) on every face, per axis.

    Interior faces: T_f (p_c - p_c') / |f|; Dirichlet faces use the boundary pressure g;
    Neumann faces carry the prescribed velocity (outward z: +z on a + side, -z on a - side).
    """
    out = []
    for a in range(3):
        if a >= dim:
            out.append(np.zeros_like(T[a]))
            continue
        n_a = p.shape[np_axis(a)]
        vals = []
        for d in (0, 1):
            side = 2 * a + d
            g = 0.0
            if bc_kind[side] == DIRICHLET and bc_val is not None and bc_val[side] is not None:
                g = np.asarray(bc_val[side], dtype=np.float64)
            vals.append(g)
        F = _face_flow(T[a], p, a, (vals[0], vals[1]))
        u = F / face_area(h, a)
        for d, face in ((0, 0), (1, n_a)):
            side = 2 * a + d
            if bc_kind[side] == NEUMANN:
                z = 0.0
                if bc_val is not None and bc_val[side] is not None:
                    z = np.expand_dims(np.asarray(bc_val[side], dtype=np.float64), np_axis(a))
                put(u, a, slice(face, face + 1), (z if d == 1 else -z) + 0.0 * take(u, a, slice(face, face + 1)))
        out.append(u)
    return out


def dense_matrix(T, dim, shape):
    """A as a dense matrix (tiny grids only), built column by column from ``matvec``."""
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = matvec(T, e.reshape(shape), dim).ravel()
        e[j] = 0.0
    return A
