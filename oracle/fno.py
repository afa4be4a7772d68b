"""Spectral neural operator of the learned warm start (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper has no
learned part; the network is specified as a 4-layer spectral neural operator
of width 32 with 16 retained modes per axis that maps (phase field, damage
field, last two strain-fluctuation increments) to the next increment.
Readings:

* Channels in: phase one-hot (2), damage (1), previous two fluctuation
  increments (6 + 6) = 15, zero-padded to ``cin``.  Channels out: 6.
* Layer l: u = K_l(h) + h W_l^T + b_l, h <- GELU(u) except after the last
  layer (the standard Fourier-neural-operator block); lift h0 = X Wl^T + bl,
  output Y = h_L Wq^T + bq.
* K(h) (spectral convolution): forward DFT (e^{-i k x}) over the three
  axes, keep kx in [0, m) on the real-FFT axis and ky, kz in [-m/2, m/2), map
  each retained mode's (Re, Im) channel pairs through a real 2C x 2C matrix
  (a superset of complex C x C multiplication), then the real inverse
  transform of that half spectrum (kx > 0 modes counted twice, 1/N scaling).
* GELU is the tanh approximation: 0.5 x (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))).
* Loss: mean squared error over every output entry.

Arrays are channels-last: X (B, Nz, Ny, Nx, Cin).  Parameters (dict):
  Wl (C, Cin), bl (C,), per layer W{l} (C, C), b{l} (C,), R{l} (mz, my, mx,
  2C, 2C) with rows (s_out, o) and columns (s_in, c), s = 0 real, 1 imag;
  Wq (Cout, C), bq (Cout,).
"""
import numpy as np

SQ = np.sqrt(2.0 / np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(SQ * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(SQ * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * SQ * (1.0 + 3 * 0.044715 * x * x)


def mode_index(n, m, centred):
    """Retained frequencies of an axis of length n: [0, m) on the real-FFT
    axis, [-m/2, m/2) (as FFT indices mod n) otherwise."""
    if not centred:
        return np.arange(m)
    return np.mod(np.arange(m) - m // 2, n)


def spectral_forward(h, R, m):
    """K(h) for h (B, Nz, Ny, Nx, C); returns (out, S) with S the retained
    spectrum (B, mz, my, mx, 2C) = (Re, Im) of the kept modes."""
    B, nz, ny, nx, C = h.shape
    H = np.fft.fftn(h, axes=(1, 2, 3))
    iz, iy, ix = mode_index(nz, m, True), mode_index(ny, m, True), mode_index(nx, m, False)
    Hk = H[:, iz][:, :, iy][:, :, :, ix]  # (B, m, m, m, C)
    S = np.concatenate([Hk.real, Hk.imag], axis=-1)
    Sm = np.einsum("zyxoi,bzyxi->bzyxo", R, S)
    Z = Sm[..., :C] + 1j * Sm[..., C:]
    half = np.zeros((B, nz, ny, nx // 2 + 1, C), dtype=np.complex128)
    tmp = np.zeros((B, nz, ny, m, C), dtype=np.complex128)
    for a, zz in enumerate(iz):
        for b_, yy in enumerate(iy):
            tmp[:, zz, yy] = Z[:, a, b_]
    half[:, :, :, :m] = tmp
    out = np.fft.irfftn(half, s=(nz, ny, nx), axes=(1, 2, 3))
    return out, S


def spectral_adjoint(g, R, S, m):
    """Given dL/dout g, return (dL/dh, dL/dR)."""
    B, nz, ny, nx, C = g.shape
    iz, iy, ix = mode_index(nz, m, True), mode_index(ny, m, True), mode_index(nx, m, False)
    # out = irfftn(half) is linear in Z: out = sum_k w_k Re(Z_k e^{i k x}) / N, w = 1 (kx=0) or 2
    N = nz * ny * nx
    G = np.fft.fftn(g, axes=(1, 2, 3))  # sum_x g e^{-ikx}
    w = np.where(ix == 0, 1.0, 2.0)
    Gk = G[:, iz][:, :, iy][:, :, :, ix] * w[None, None, None, :, None] / N
    # d/dRe Z = Re(Gk) ... derivative of Re(Z e^{ikx}) wrt Re Z is cos, wrt Im Z is -sin:
    # sum_x g cos = Re(G), sum_x g (-sin) = Im(G) with G = sum g e^{-ikx}
    dSm = np.concatenate([Gk.real, Gk.imag], axis=-1)
    dR = np.einsum("bzyxo,bzyxi->zyxoi", dSm, S)
    dS = np.einsum("zyxoi,bzyxo->bzyxi", R, dSm)
    # S = (Re, Im) of sum_x h e^{-ikx}: d/dh = Re part cos, Im part -sin -> sum over kept modes
    # dS_re/dh(x) = cos(kx), dS_im/dh(x) = -sin(kx): dh(x) = Re(sum_k (dS_re + i dS_im) e^{ikx})
    spec = dS[..., :C] + 1j * dS[..., C:]
    full = np.zeros((B, nz, ny, nx, C), dtype=np.complex128)
    for a, zz in enumerate(iz):
        for b_, yy in enumerate(iy):
            for c_, xx in enumerate(ix):
                full[:, zz, yy, xx] += spec[:, a, b_, c_]
    dH = np.fft.ifftn(full, axes=(1, 2, 3)).real * N
    return dH, dR


def init_params(cin=16, width=32, cout=6, layers=4, modes=16, seed=0):
    rng = np.random.default_rng(seed)
    p = {"Wl": rng.standard_normal((width, cin)) / np.sqrt(cin), "bl": np.zeros(width),
         "Wq": rng.standard_normal((cout, width)) / np.sqrt(width), "bq": np.zeros(cout)}
    for l in range(layers):
        p[f"W{l}"] = rng.standard_normal((width, width)) / np.sqrt(width)
        p[f"b{l}"] = np.zeros(width)
        p[f"R{l}"] = rng.standard_normal((modes, modes, modes, 2 * width, 2 * width)) / (2 * width)
    return p


def forward(p, X, modes, layers=4, keep=False):
    h = X @ p["Wl"].T + p["bl"]
    cache = {"h": [h], "u": [], "S": []}
    for l in range(layers):
        k, S = spectral_forward(h, p[f"R{l}"], modes)
        u = k + h @ p[f"W{l}"].T + p[f"b{l}"]
        cache["u"].append(u)
        cache["S"].append(S)
        h = gelu(u) if l < layers - 1 else u
        cache["h"].append(h)
    Y = h @ p["Wq"].T + p["bq"]
    return (Y, cache) if keep else Y


def loss(Y, T):
    return float(np.mean((Y - T) ** 2))


def backward(p, X, T, modes, layers=4):
    """Loss and gradients (dict) of the MSE loss."""
    Y, cache = forward(p, X, modes, layers, keep=True)
    g = {}
    dY = 2.0 * (Y - T) / Y.size
    hL = cache["h"][-1]
    g["Wq"] = dY.reshape(-1, dY.shape[-1]).T @ hL.reshape(-1, hL.shape[-1])
    g["bq"] = dY.reshape(-1, dY.shape[-1]).sum(0)
    dh = dY @ p["Wq"]
    for l in reversed(range(layers)):
        u = cache["u"][l]
        du = dh * gelu_grad(u) if l < layers - 1 else dh
        hin = cache["h"][l]
        g[f"W{l}"] = du.reshape(-1, du.shape[-1]).T @ hin.reshape(-1, hin.shape[-1])
        g[f"b{l}"] = du.reshape(-1, du.shape[-1]).sum(0)
        dk, dR = spectral_adjoint(du, p[f"R{l}"], cache["S"][l], modes)
        g[f"R{l}"] = dR
        dh = du @ p[f"W{l}"] + dk
    g["Wl"] = dh.reshape(-1, dh.shape[-1]).T @ X.reshape(-1, X.shape[-1])
    g["bl"] = dh.reshape(-1, dh.shape[-1]).sum(0)
    return loss(Y, T), g
