"""Mandel notation for symmetric strain/stress tensors (oracle copy).

Small-strain setting of Sec. 2: strain and stress are symmetric second-order
tensors.  They are stored as orthonormal Mandel vectors so that the
Euclidean dot product of two Mandel vectors equals the tensor double
contraction A:B:

* 3D: (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12)
* 2D plane strain: (11, 22, sqrt2*12), with eps_33 = eps_13 = eps_23 = 0.

Fields are arrays of shape (ncomp, *grid) with grid = (Ny, Nx) or
(Nz, Ny, Nx); tensor index 0 is x, 1 is y, 2 is z.
"""
import numpy as np

SQ2 = np.sqrt(2.0)

# (i, j) tensor index of each Mandel slot
_PAIRS = {
    2: [(0, 0), (1, 1), (0, 1)],
    3: [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)],
}


def ncomp_of(ndim):
    return 3 if ndim == 2 else 6


def ndim_of(ncomp):
    return 2 if ncomp == 3 else 3


def normal_comps(ndim):
    return list(range(ndim))


def mandel_to_tensor(m):
    """(ncomp, ...) Mandel -> (..., d, d) tensor (real or complex)."""
    ncomp = m.shape[0]
    d = ndim_of(ncomp)
    t = np.zeros(m.shape[1:] + (d, d), dtype=m.dtype)
    for a, (i, j) in enumerate(_PAIRS[d]):
        if i == j:
            t[..., i, i] = m[a]
        else:
            t[..., i, j] = m[a] / SQ2
            t[..., j, i] = m[a] / SQ2
    return t


def tensor_to_mandel(t):
    """(..., d, d) tensor -> (ncomp, ...) Mandel.  The off-diagonal slot
    takes the mean of (i,j) and (j,i), i.e. the symmetric part."""
    d = t.shape[-1]
    out = np.zeros((ncomp_of(d),) + t.shape[:-2], dtype=t.dtype)
    for a, (i, j) in enumerate(_PAIRS[d]):
        if i == j:
            out[a] = t[..., i, i]
        else:
            out[a] = SQ2 * 0.5 * (t[..., i, j] + t[..., j, i])
    return out
