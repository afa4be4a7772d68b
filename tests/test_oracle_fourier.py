"""Pins of the oracle's DFT, FE gradient symbol and projection (CPU only).

Each check compares against something other than the oracle's own formula:
a naive DFT, the real-space finite-element strain operator assembled from
shape-function derivatives, dense linear algebra, or an exact identity.
"""
import numpy as np
import pytest

import oracle
from synth import random_field
from tests import fe_bruteforce as fe

RNG = np.random.default_rng(1234)


@pytest.mark.parametrize("shape", [(4, 6), (3, 4, 5), (5, 5)])
def test_fft_matches_naive_dft(shape):
    a = RNG.standard_normal((2,) + shape)
    np.testing.assert_allclose(oracle.fft(a), oracle.dft_naive(a), atol=1e-12)
    np.testing.assert_allclose(oracle.ifft(oracle.fft(a)).real, a, atol=1e-13)
    # Parseval
    n = np.prod(shape)
    assert np.isclose(np.sum(a * a), np.sum(np.abs(oracle.fft(a)) ** 2) / n, rtol=1e-13)


def _nodal_to_strain_fourier(u, dims):
    """FFT of the FE strain B u, built in real space."""
    d = len(dims)
    B = fe.strain_matrix(dims)
    ncomp = 3 if d == 2 else 6
    eps = (B @ u.ravel()).reshape((ncomp,) + tuple(reversed(dims)))
    return eps


@pytest.mark.parametrize("dims", [(4, 6), (6, 4), (3, 4, 5), (4, 4, 2)])
def test_symbol_matches_real_space_fe_strain(dims):
    """FFT(B u) = sym(Dhat (x) uhat) at every k: pins the stencil, its sign,
    axis order and the Mandel placement."""
    d = len(dims)
    shape = tuple(reversed(dims))
    u = RNG.standard_normal((d,) + shape)
    eps = _nodal_to_strain_fourier(u, dims)
    eps_hat = oracle.fft(eps)
    uhat = oracle.fft(u)
    dh = oracle.gradient_symbol(shape)
    t = 0.5 * (np.einsum("i...,j...->...ij", dh, uhat) + np.einsum("j...,i...->...ij", dh, uhat))
    np.testing.assert_allclose(oracle.tensor_to_mandel(t), eps_hat, atol=1e-11)


@pytest.mark.parametrize("dims", [(4, 4), (4, 6), (3, 4, 4), (2, 4, 3)])
def test_projection_equals_dense_orthogonal_projector(dims):
    """G equals the orthogonal projector onto range(B) (plus the k=0 free
    block), computed by dense pseudo-inverse -- pins the Ghat formula,
    including Ghat = 0 on hourglass frequencies."""
    d = len(dims)
    shape = tuple(reversed(dims))
    ncomp = 3 if d == 2 else 6
    nvox = int(np.prod(dims))
    B = fe.strain_matrix(dims)
    free = np.zeros(ncomp, bool)
    free[-1] = True
    free[0] = True
    U = np.zeros((ncomp * nvox, int(free.sum())))
    for col, c in enumerate(np.flatnonzero(free)):
        U[c * nvox:(c + 1) * nvox, col] = 1.0
    A = np.hstack([B, U])
    P = A @ np.linalg.pinv(A, rcond=1e-10)
    for _ in range(3):
        z = RNG.standard_normal((ncomp,) + shape)
        gz, gzi = oracle.project(z, free, return_imag=True)
        np.testing.assert_allclose(gz.ravel(), P @ z.ravel(), atol=1e-11)
        assert np.max(np.abs(gzi)) < 1e-12


def test_projection_properties_and_hourglass():
    shape = (6, 8, 4)
    z = RNG.standard_normal((6,) + shape)
    y = RNG.standard_normal((6,) + shape)
    gz = oracle.project(z)
    np.testing.assert_allclose(oracle.project(gz), gz, atol=1e-12)  # idempotent
    assert abs(np.sum(gz * y) - np.sum(z * oracle.project(y))) < 1e-10  # symmetric
    assert abs(np.mean(gz)) < 1e-13  # zero mean with full strain control
    # content only on the hourglass line (th_y = th_z = pi) is annihilated
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    hour = ((-1.0) ** (yy + zz)) * np.cos(2 * np.pi * xx / nx)
    fld = np.stack([hour * c for c in RNG.standard_normal(6)])
    assert np.max(np.abs(oracle.project(fld))) < 1e-12


def test_projection_k0_is_free_mask():
    shape = (4, 4)
    free = np.array([False, True, False])
    uni = np.ones((3,) + shape) * np.array([1.0, 2.0, 3.0])[:, None, None]
    out = oracle.project(uni, free)
    np.testing.assert_allclose(out, uni * free[:, None, None], atol=1e-14)


def test_symbol_consistent_with_spectral_at_low_k():
    """For small th the FE derivative tends to i*th (Eq. (10)'s spectral
    derivative): first-order consistency of the stencil."""
    n = 4096
    dh = oracle.gradient_symbol((n, n))
    th = 2 * np.pi / n
    assert abs(dh[0, 0, 1] / (1j * th) - 1) < 1e-3
    assert abs(dh[1, 1, 0] / (1j * th) - 1) < 1e-3


def test_real_input_gives_real_projection_3d():
    z = random_field(6, (5, 4, 3), seed=7)
    gz, gzi = oracle.project(z, return_imag=True)
    assert np.max(np.abs(gzi)) < 1e-13


def _per_frequency_projector(dhat):
    """Dense orthogonal (Hermitian) projector onto {sym(Dhat (x) a), a in C^d}
    in Mandel coordinates, from a pseudo-inverse (reading R2 written as its
    definition, not as the closed form)."""
    d = len(dhat)
    cols = []
    for j in range(d):
        e = np.zeros(d, dtype=np.complex128)
        e[j] = 1.0
        t = 0.5 * (np.outer(dhat, e) + np.outer(e, dhat))
        cols.append(oracle.tensor_to_mandel(t[None])[:, 0])
    A = np.stack(cols, axis=1)
    return A @ np.linalg.pinv(A, rcond=1e-12)


@pytest.mark.parametrize("dims", [(4, 6), (5, 4), (4, 3, 6), (2, 4, 4)])
def test_single_frequency_symbol_and_projector(dims):
    """gradient_symbol_at / project_one (the per-frequency forms the 256^3
    plane-wave GPU test uses) agree at every k of a small grid with the
    full-grid symbol and with a dense per-frequency projector; project_one
    also equals project_hat at that k (project_hat is pinned against the
    dense real-space projector above)."""
    d = len(dims)
    ncomp = 3 if d == 2 else 6
    shape = tuple(reversed(dims))
    dh = oracle.gradient_symbol(shape)
    zhat = RNG.standard_normal((ncomp,) + shape) + 1j * RNG.standard_normal((ncomp,) + shape)
    ph = oracle.project_hat(zhat, dh, np.zeros(ncomp, bool))
    for idx in np.ndindex(*shape):
        k = tuple(reversed(idx))  # (kx, ky[, kz])
        dk = oracle.gradient_symbol_at(k, dims)
        np.testing.assert_allclose(dk, dh[(slice(None),) + idx], atol=1e-15)
        z = zhat[(slice(None),) + idx]
        got = oracle.project_one(z, dk)
        if all(kk == 0 for kk in k):
            continue  # k = 0 is the mean block, handled by project_hat alone
        np.testing.assert_allclose(got, _per_frequency_projector(dk) @ z, atol=1e-12)
        np.testing.assert_allclose(got, ph[(slice(None),) + idx], atol=1e-12)
    # negative / aliased frequencies: the symbol is periodic in k
    k = (1, -1) if d == 2 else (1, -1, 2)
    kp = tuple(kk % n for kk, n in zip(k, dims))
    np.testing.assert_allclose(oracle.gradient_symbol_at(k, dims), oracle.gradient_symbol_at(kp, dims), atol=0)
