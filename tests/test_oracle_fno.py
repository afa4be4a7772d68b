"""Pins of the oracle's spectral neural operator (CPU only): finite
differences of the loss for every parameter group and the input, and the
spectral convolution against a naive DFT sum on a tiny grid."""
import numpy as np
import pytest

from oracle import fno


def _tiny(seed=0):
    rng = np.random.default_rng(seed)
    p = fno.init_params(cin=5, width=3, cout=2, layers=2, modes=4, seed=seed)
    X = rng.standard_normal((2, 6, 8, 10, 5))
    T = rng.standard_normal((2, 6, 8, 10, 2))
    return p, X, T


def test_gradients_match_central_differences():
    p, X, T = _tiny()
    L, g = fno.backward(p, X, T, modes=4, layers=2)
    rng = np.random.default_rng(1)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = fno.loss(fno.forward(p, X, 4, 2), T)
            flat[idx] = old - h
            lm = fno.loss(fno.forward(p, X, 4, 2), T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, an)


def test_spectral_conv_matches_naive_dft():
    """K(h) with the identity per-mode map equals the naive low-pass sum
    (1/N) sum_kept w_kx Re(H_k e^{ik.x}) written out with explicit phases."""
    rng = np.random.default_rng(3)
    B, nz, ny, nx, C, m = 1, 4, 6, 8, 2, 4
    h = rng.standard_normal((B, nz, ny, nx, C))
    R = np.zeros((m, m, m, 2 * C, 2 * C))
    R[..., np.arange(2 * C), np.arange(2 * C)] = 1.0
    out, _ = fno.spectral_forward(h, R, m)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ref = np.zeros_like(h)
    N = nz * ny * nx
    for kz in fno.mode_index(nz, m, True):
        for ky in fno.mode_index(ny, m, True):
            for kx in range(m):
                ph = 2 * np.pi * (kz * z / nz + ky * y / ny + kx * x / nx)
                Hk = np.einsum("bzyxc,zyx->bc", h, np.exp(-1j * ph))
                w = 1.0 if kx == 0 else 2.0
                ref += w / N * np.real(Hk[:, None, None, None, :] * np.exp(1j * ph)[None, ..., None])
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_gelu_derivative():
    x = np.linspace(-4, 4, 101)
    h = 1e-6
    np.testing.assert_allclose(fno.gelu_grad(x), (fno.gelu(x + h) - fno.gelu(x - h)) / (2 * h), atol=1e-8)
