"""The cell problem on linear simplex elements with one quadrature point per
simplex (oracle).  TEST INFRASTRUCTURE ONLY, like the rest of this package.

Sec. 2.1 derives the projection from the gradient operator of a chosen
finite-element discretisation (Leute et al. 2022): any element type gives a
ringing-free projection through its shape-function derivatives, evaluated at
its quadrature points.  The solver of this repository uses one
bilinear / trilinear element per voxel with one quadrature point (reading
R1); this module provides the multi-quadrature-point alternative with linear
triangles / tetrahedra.

Reading (the paper gives no decomposition): every voxel is split into d!
simplices along its main diagonal (Kuhn / Freudenthal decomposition).  The
simplex of axis permutation pi has vertices v_0 = 0, v_j = v_{j-1} + e_{pi_j};
the linear interpolant's derivative along pi_j is u(v_j) - u(v_{j-1}), whose
Fourier symbol for the node grid at voxel corners is

    Dhat_{pi_j}(k) = exp(i sum_{l<j} th_{pi_l}) (e^{i th_{pi_j}} - 1).

Fields carry one strain (Mandel) per simplex: shape (ncomp, d!, *grid).  At
a frequency k the compatible strains are B(k) a, a in C^d, with B stacking
sym(Dhat_q (x) a) over the simplices q; the projector is the orthogonal one,
Ghat = B (B^H B)^+ B^H (all simplices have the same volume, so the
Euclidean inner product is the energy one).  At k = 0 a compatible field is
the same mean strain at every simplex: Ghat(0) averages the stress-controlled
components over the simplices and drops the strain-controlled ones.
Material, energy and the two algorithms are the voxel ones applied per
simplex (every simplex of a voxel has the voxel's phase).
"""
import itertools

import numpy as np

from .material import PhaseParams, evaluate, tangent_apply
from .tensors import SQ2, ncomp_of


def kuhn_permutations(d):
    return list(itertools.permutations(range(d)))


def simplex_symbols(grid):
    """Dhat, shape (d!, d, *grid) complex: derivative symbol of every simplex
    (factors e^{i th} - 1 exactly zero at k = 0)."""
    d = len(grid)
    e, diff = [], []
    for a in range(d):  # tensor axis a = array axis d-1-a
        n = grid[d - 1 - a]
        k = np.arange(n)
        ea = np.exp(2j * np.pi * k / n)
        da = np.where(k == 0, 0.0, ea - 1.0)
        view = [1] * d
        view[d - 1 - a] = n
        e.append(ea.reshape(view))
        diff.append(da.reshape(view))
    perms = kuhn_permutations(d)
    D = np.zeros((len(perms), d) + tuple(grid), dtype=np.complex128)
    for q, pi in enumerate(perms):
        prefix = np.ones(tuple(grid), dtype=np.complex128)
        for a in pi:
            D[q, a] = prefix * diff[a]
            prefix = prefix * e[a]
    return D


def _b_matrix(D):
    """B(k): (ncomp, nq, d, *grid), strain of simplex q from amplitude a."""
    nq, d = D.shape[:2]
    nc = ncomp_of(d)
    pairs = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    B = np.zeros((nc, nq, d) + D.shape[2:], dtype=np.complex128)
    for c, (i, j) in enumerate(pairs):
        if i == j:
            B[c, :, i] = D[:, i]
        else:
            B[c, :, j] += D[:, i] / SQ2
            B[c, :, i] += D[:, j] / SQ2
    return B


def project_hat(zh, D, free_mask):
    """Ghat applied per frequency to zh (ncomp, nq, *grid) complex."""
    nc, nq = zh.shape[:2]
    grid = zh.shape[2:]
    d = D.shape[1]
    B = _b_matrix(D)
    # move the frequency axes first: Bk (K, nc*nq, d), zk (K, nc*nq)
    K = int(np.prod(grid))
    Bk = np.moveaxis(B.reshape(nc * nq, d, K), -1, 0)
    zk = np.moveaxis(zh.reshape(nc * nq, K), -1, 0)
    M = np.einsum("kpi,kpj->kij", Bk.conj(), Bk)
    Mp = np.linalg.pinv(M, rcond=1e-12, hermitian=True)
    a = np.einsum("kij,kj->ki", Mp, np.einsum("kpi,kp->ki", Bk.conj(), zk))
    out = np.einsum("kpi,ki->kp", Bk, a)
    out = np.moveaxis(out, 0, -1).reshape(zh.shape)
    # k = 0: the same mean strain at every simplex on the free components
    idx0 = (slice(None), slice(None)) + (0,) * len(grid)
    out[idx0] = 0.0
    fm = np.asarray(free_mask, dtype=bool)
    for c in range(nc):
        if fm[c]:
            out[(c, slice(None)) + (0,) * len(grid)] = zh[(c, slice(None)) + (0,) * len(grid)].mean()
    return out


class SimplexRVE:
    """The cell problem of the oracle's RVE on Kuhn simplices (fields
    (ncomp, d!, *grid)); same interface for the solvers of ``solver.py``."""

    def __init__(self, phase_map, phases, free_mask=None):
        self.phase_map = np.asarray(phase_map)
        self.grid = self.phase_map.shape
        self.dim = self.phase_map.ndim
        self.ncomp = ncomp_of(self.dim)
        self.nq = len(kuhn_permutations(self.dim))
        self.shape = (self.nq,) + self.grid      # per-component field shape
        self.ndim = len(self.shape)
        self.params = PhaseParams(self.phase_map, phases)
        self.free_mask = (np.zeros(self.ncomp, dtype=bool) if free_mask is None
                          else np.asarray(free_mask, dtype=bool))
        self.D = simplex_symbols(self.grid)

    @staticmethod
    def dot(a, b):
        return float(np.sum(a * b))

    def norm(self, a):
        return float(np.sqrt(self.dot(a, a)))

    def G(self, x):
        zh = np.fft.fftn(x, axes=tuple(range(2, x.ndim)))
        return np.real(np.fft.ifftn(project_hat(zh, self.D, self.free_mask), axes=tuple(range(2, x.ndim))))

    def stress(self, eps, kappa_hist):
        return evaluate(eps, self.params, kappa_hist)

    def tangent(self, D, v):
        return tangent_apply(v, D, self.params.lam, self.params.mu)

    def hessp(self, D, v):
        return self.G(self.tangent(D, v))

    def gradient(self, sigma):
        return self.G(sigma)

    def mean(self, field):
        return field.reshape(self.ncomp, -1).mean(axis=1)
