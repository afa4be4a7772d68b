"""Brute-force periodic linear finite elements, assembled as dense matrices.

An independent check of the oracle's Fourier-space formulation: nodal
displacements on voxel corners, one bilinear/trilinear element per voxel,
strain evaluated at the element centre (one quadrature point, weight 1).
The strain-displacement matrix is built from the shape-function derivatives
directly (no Fourier symbol), the stiffness K = sum_e B_e^T C_e B_e is
assembled node by node, and the periodic problem is solved by least squares
(K is singular through rigid translations and hourglass modes; the strain
field is unique).
"""
import itertools

import numpy as np

SQ2 = np.sqrt(2.0)


def _corners(d):
    return list(itertools.product((0, 1), repeat=d))  # (a_x, a_y[, a_z])


def shape_grad_centre(d):
    """dN/dx_alpha at the element centre for each corner, shape (2^d, d)."""
    out = []
    for c in _corners(d):
        g = []
        for alpha in range(d):
            val = 1.0 if c[alpha] == 1 else -1.0
            for beta in range(d):
                if beta != alpha:
                    val *= 0.5
            g.append(val)
        out.append(g)
    return np.array(out)


def mandel_pairs(d):
    return [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def strain_matrix(dims):
    """Global B: nodal displacement (d * nnode) -> Mandel strain per voxel
    (ncomp * nvox), in the (comp, z, y, x) layout of the oracle fields."""
    d = len(dims)
    pairs = mandel_pairs(d)
    ncomp = len(pairs)
    nvox = int(np.prod(dims))
    shape = tuple(reversed(dims))
    grads = shape_grad_centre(d)
    B = np.zeros((ncomp * nvox, d * nvox))
    for vox in itertools.product(*[range(n) for n in dims]):  # (ix, iy[, iz])
        vflat = np.ravel_multi_index(tuple(reversed(vox)), shape)
        for ci, c in enumerate(_corners(d)):
            node = tuple((vox[a] + c[a]) % dims[a] for a in range(d))
            nflat = np.ravel_multi_index(tuple(reversed(node)), shape)
            for m, (i, j) in enumerate(mandel_pairs(d)):
                row = m * nvox + vflat
                if i == j:
                    B[row, i * nvox + nflat] += grads[ci, i]
                else:
                    # sqrt2 * 1/2 (du_i/dx_j + du_j/dx_i)
                    B[row, i * nvox + nflat] += SQ2 * 0.5 * grads[ci, j]
                    B[row, j * nvox + nflat] += SQ2 * 0.5 * grads[ci, i]
    return B


def stiffness_blocks(lam, mu, d):
    """Per-voxel Mandel stiffness matrices, shape (nvox, ncomp, ncomp)."""
    ncomp = 3 if d == 2 else 6
    lam = np.ravel(lam)
    mu = np.ravel(mu)
    C = np.zeros((lam.size, ncomp, ncomp))
    for a in range(d):
        for b in range(d):
            C[:, a, b] = lam
    for a in range(ncomp):
        C[:, a, a] += 2.0 * mu
    return C


def block_diag_fields(Cv, nvox, ncomp):
    """Dense operator acting on (comp, vox)-ordered Mandel fields."""
    M = np.zeros((ncomp * nvox, ncomp * nvox))
    for a in range(ncomp):
        for b in range(ncomp):
            M[a * nvox:(a + 1) * nvox, b * nvox:(b + 1) * nvox] = np.diag(Cv[:, a, b])
    return M


def solve_elastic(dims, lam, mu, E_fixed, free_mask=None):
    """Minimise sum_e 1/2 eps_e : C_e : eps_e with eps = E + B u, E having
    the ``free_mask`` components free (zero mean stress).  Returns the Mandel
    strain field (ncomp, *shape)."""
    d = len(dims)
    ncomp = 3 if d == 2 else 6
    nvox = int(np.prod(dims))
    B = strain_matrix(dims)
    Cm = block_diag_fields(stiffness_blocks(lam, mu, d), nvox, ncomp)
    free = np.zeros(ncomp, bool) if free_mask is None else np.asarray(free_mask, bool)
    fidx = np.flatnonzero(free)
    # uniform-strain columns for the free mean components
    U = np.zeros((ncomp * nvox, len(fidx)))
    for col, c in enumerate(fidx):
        U[c * nvox:(c + 1) * nvox, col] = 1.0
    A = np.hstack([B, U])
    e0 = np.repeat(np.asarray(E_fixed, float), nvox)
    K = A.T @ Cm @ A
    rhs = -A.T @ Cm @ e0
    x, *_ = np.linalg.lstsq(K, rhs, rcond=1e-13)
    eps = e0 + A @ x
    return eps.reshape((ncomp,) + tuple(reversed(dims))), B
