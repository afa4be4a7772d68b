"""DFTs, the FE gradient symbol and the compatibility projection (oracle).

Sec. 2.1: the projection of an arbitrary field zeta onto its compatible part
is a convolution, applied in Fourier space as a per-frequency contraction
(Eqs. (4)-(5)).  The per-frequency operator is built from a discrete
derivative symbol Dhat(k) through ghat = Dhat (x) Dhat^* / (Dhat . Dhat^*)
(Eq. (9)); with the linear finite-element derivative (Sec. 2.1, the
ringing-free discretisation) instead of the spectral one i*k (Eq. (10)).

Readings where the paper defers to other work:

* FE gradient symbol.  One bilinear (2D) / trilinear (3D) element per voxel
  with nodal displacements at voxel corners and a single quadrature point at
  the voxel centre.  The derivative along alpha at the centre is the mean of
  the forward differences over the 2^(d-1) element edges along alpha, whose
  Fourier symbol is
      Dhat_alpha(k) = (e^{i th_alpha} - 1) * prod_{beta != alpha} (1 + e^{i th_beta}) / 2,
  th_alpha = 2 pi k_alpha / N_alpha.  Factors that vanish mathematically
  (th = 0 for the difference, th = pi for an average) are set to exact zeros.
* Small-strain projector.  Ghat(k) is the orthogonal (Hermitian) projector
  onto {sym(Dhat(k) (x) a) : a in C^d}.  With n = Dhat/|Dhat| and v = zeta n*:
      Ghat : zeta = n (x) v + v (x) n - (n*^T zeta n*) n (x) n.
  Ghat = 0 wherever Dhat(k) = 0 and k != 0 (no compatible strain there).
* Mixed (stress) control at k = 0 (Sec. 3.3 imposes mean stress by modifying
  the projection): Ghat(0) = P_free, the 0/1 diagonal mask of the
  stress-controlled Mandel components; with full strain control it is 0.
"""
import numpy as np

from .tensors import mandel_to_tensor, tensor_to_mandel


def _spatial_axes(a):
    return tuple(range(1, a.ndim))


def dft_naive(a, inverse=False):
    """Plain DFT over every spatial axis (axis 0 is the component axis).

    Forward: X(k) = sum_j x(j) exp(-2 pi i j k / N); inverse: the conjugate
    kernel divided by N.  Each axis is a dense N x N matrix product, so this
    is only for tiny grids (it pins the FFT used elsewhere)."""
    out = np.asarray(a, dtype=np.complex128)
    sign = 1.0 if inverse else -1.0
    for ax in _spatial_axes(out):
        n = out.shape[ax]
        j = np.arange(n)
        mat = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
        if inverse:
            mat = mat / n
        out = np.moveaxis(np.tensordot(mat, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def fft(a, naive=False):
    """Forward DFT over the spatial axes (numpy's FFT as a library step)."""
    if naive:
        return dft_naive(a)
    return np.fft.fftn(a, axes=_spatial_axes(a))


def ifft(a, naive=False):
    if naive:
        return dft_naive(a, inverse=True)
    return np.fft.ifftn(a, axes=_spatial_axes(a))


def _angles_exact(n):
    """e^{i th} for th = 2 pi k / n, k = 0..n-1, and exact-zero masks of
    (e^{i th} - 1) (k = 0) and (1 + e^{i th}) (2k = n)."""
    k = np.arange(n)
    e = np.exp(2j * np.pi * k / n)
    diff = np.where(k == 0, 0.0, e - 1.0)
    avg = np.where(2 * k == n, 0.0, (1.0 + e) / 2.0)
    return diff, avg


def gradient_symbol(shape):
    """Dhat(k) of the one-point-quadrature linear FE gradient.

    ``shape`` is the numpy grid shape (Ny, Nx) or (Nz, Ny, Nx).  Returns a
    complex array (d, *shape) whose entry [alpha] is Dhat_alpha with alpha =
    0 (x), 1 (y), 2 (z)."""
    d = len(shape)
    dims = tuple(reversed(shape))  # (Nx, Ny[, Nz])
    out = np.ones((d,) + tuple(shape), dtype=np.complex128)
    for alpha in range(d):
        for beta in range(d):
            diff, avg = _angles_exact(dims[beta])
            fac = diff if beta == alpha else avg
            view = [1] * d
            view[d - 1 - beta] = dims[beta]
            out[alpha] = out[alpha] * fac.reshape(view)
    return out


def gradient_symbol_at(k, dims):
    """Dhat at one frequency k = (kx, ky[, kz]) of a grid dims = (Nx, Ny[, Nz])."""
    d = len(dims)
    out = np.ones(d, dtype=np.complex128)
    for alpha in range(d):
        for beta in range(d):
            n, kb = dims[beta], int(k[beta]) % dims[beta]
            e = np.exp(2j * np.pi * kb / n)
            if beta == alpha:
                fac = 0.0 if kb == 0 else e - 1.0
            else:
                fac = 0.0 if 2 * kb == n else (1.0 + e) / 2.0
            out[alpha] *= fac
    return out


def project_one(zeta, dhat):
    """Ghat(k) : zeta for a single frequency k != 0 (Mandel vector zeta,
    symbol dhat); 0 where dhat = 0."""
    t = mandel_to_tensor(np.asarray(zeta, dtype=np.complex128).reshape(-1, 1))[0]
    nrm = np.sqrt(np.sum(np.abs(dhat) ** 2))
    if nrm == 0.0:
        return np.zeros(len(zeta), dtype=np.complex128)
    n = dhat / nrm
    v = t @ np.conj(n)
    s = np.conj(n) @ v
    out = np.outer(n, v) + np.outer(v, n) - s * np.outer(n, n)
    return tensor_to_mandel(out[None])[:, 0]


def project_hat(zeta_hat, dhat, free_mask):
    """Apply Ghat(k) at every frequency to a Mandel spectrum (ncomp, *shape).

    ``free_mask``: boolean (ncomp,) of stress-controlled mean components."""
    t = mandel_to_tensor(zeta_hat)  # (..., d, d)
    n = np.moveaxis(dhat, 0, -1)  # (..., d)
    norm2 = np.sum(np.abs(n) ** 2, axis=-1)
    valid = norm2 > 0.0
    safe = np.where(valid, np.sqrt(norm2), 1.0)
    n = n / safe[..., None]
    nbar = np.conj(n)
    v = np.einsum("...ij,...j->...i", t, nbar)
    s = np.einsum("...i,...i->...", nbar, v)
    out_t = (np.einsum("...i,...j->...ij", n, v)
             + np.einsum("...i,...j->...ij", v, n)
             - s[..., None, None] * np.einsum("...i,...j->...ij", n, n))
    out_t = np.where(valid[..., None, None], out_t, 0.0)
    out = tensor_to_mandel(out_t)
    zero = (0,) * (zeta_hat.ndim - 1)
    mask = np.asarray(free_mask, dtype=bool)
    out[(slice(None),) + zero] = np.where(mask, zeta_hat[(slice(None),) + zero], 0.0)
    return out


def project(field, free_mask=None, naive=False, return_imag=False):
    """Real-space projection G zeta = F^-1{ Ghat : F{zeta} } (Eq. (5))."""
    ncomp = field.shape[0]
    if free_mask is None:
        free_mask = np.zeros(ncomp, dtype=bool)
    dhat = gradient_symbol(field.shape[1:])
    out = ifft(project_hat(fft(field, naive), dhat, free_mask), naive)
    if return_imag:
        return out.real, out.imag
    return out.real
