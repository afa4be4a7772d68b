"""Brute-force periodic FE on linear simplices (test helper, no Fourier
symbol): every voxel split into the d! Kuhn simplices along its main
diagonal, the gradient of the linear interpolant on a simplex from the
general formula grad u = X^-1 [u(v_j) - u(v_0)]_j (X: rows v_j - v_0), the
global strain operator assembled from it, and the elastic cell problem
solved as one dense linear system."""
import itertools

import numpy as np

SQ2 = np.sqrt(2.0)


def _pairs(d):
    return [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def strain_matrix(dims):
    """Global B: nodal displacements (d * nnode, component-major) -> Mandel
    strain of every simplex, rows in the (comp, simplex, z, y, x) order of
    the oracle's simplex fields."""
    d = len(dims)
    perms = list(itertools.permutations(range(d)))
    nq = len(perms)
    pairs = _pairs(d)
    nc = len(pairs)
    shape = tuple(reversed(dims))
    nvox = int(np.prod(dims))
    B = np.zeros((nc * nq * nvox, d * nvox))
    for vox in itertools.product(*[range(n) for n in dims]):
        vflat = np.ravel_multi_index(tuple(reversed(vox)), shape)
        for q, pi in enumerate(perms):
            verts = [np.zeros(d, int)]
            for a in pi:
                v = verts[-1].copy()
                v[a] += 1
                verts.append(v)
            X = np.array([verts[j] - verts[0] for j in range(1, d + 1)], dtype=float)
            Xi = np.linalg.inv(X)  # grad = Xi @ [u(v_j) - u(v_0)]
            nodes = []
            for v in verts:
                node = tuple((vox[a] + v[a]) % dims[a] for a in range(d))
                nodes.append(np.ravel_multi_index(tuple(reversed(node)), shape))
            # dgrad[j][m] = d(du/dx_j) / d u(vertex m)
            dgrad = np.zeros((d, d + 1))
            for jj in range(d):
                dgrad[:, jj + 1] += Xi[:, jj]
                dgrad[:, 0] -= Xi[:, jj]
            for c, (i, j) in enumerate(pairs):
                row = (c * nq + q) * nvox + vflat
                for m, node in enumerate(nodes):
                    if i == j:
                        B[row, i * nvox + node] += dgrad[i, m]
                    else:
                        B[row, i * nvox + node] += dgrad[j, m] / SQ2
                        B[row, j * nvox + node] += dgrad[i, m] / SQ2
    return B


def solve_elastic(dims, lam, mu, E, free_mask=None):
    """Minimise sum over simplices of 1/2 eps:C:eps, eps = E + B u, the
    free_mask mean components free; lam / mu per voxel (shared by its
    simplices).  Returns the simplex strain field (ncomp, d!, *grid)."""
    d = len(dims)
    nq = len(list(itertools.permutations(range(d))))
    pairs = _pairs(d)
    nc = len(pairs)
    nvox = int(np.prod(dims))
    B = strain_matrix(dims)
    lamq = np.tile(np.ravel(lam), nq)
    muq = np.tile(np.ravel(mu), nq)
    n = nq * nvox
    C = np.zeros((nc * n, nc * n))
    for a in range(nc):
        C[a * n + np.arange(n), a * n + np.arange(n)] += 2 * muq
        for b in range(d):
            if a < d:
                C[a * n + np.arange(n), b * n + np.arange(n)] += lamq
    free = np.zeros(nc, bool) if free_mask is None else np.asarray(free_mask, bool)
    fidx = np.flatnonzero(free)
    U = np.zeros((nc * n, len(fidx)))
    for col, c in enumerate(fidx):
        U[c * n:(c + 1) * n, col] = 1.0
    A = np.hstack([B, U])
    e0 = np.repeat(np.asarray(E, float) * (1 - free), n)
    K = A.T @ C @ A
    x, *_ = np.linalg.lstsq(K, -A.T @ C @ e0, rcond=1e-13)
    eps = e0 + A @ x
    return eps.reshape((nc, nq) + tuple(reversed(dims))), B
