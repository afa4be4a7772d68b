"""Learned warm start: a spectral neural operator (library kernels) that
proposes the next load step's strain-fluctuation increment.

The proposal only seeds the trust-region solve (``rve_solve_step``'s
``init_incr``, projected onto compatible fields by the library); the plain
solver still decides convergence, so accuracy is unchanged and only the
iteration count can drop.  Torch supplies device memory only.
"""
import numpy as np
import torch

from . import binding as B

CIN, WIDTH, COUT = 16, 32, 6


def pack_params(p, layers):
    """Oracle-layout parameter dict -> the library's packed FP32 vector
    (weights stored [in][out])."""
    parts = [p["Wl"].T.ravel(), p["bl"].ravel()]
    for l in range(layers):
        parts += [p[f"W{l}"].T.ravel(), p[f"b{l}"].ravel(), p[f"R{l}"].ravel()]
    parts += [p["Wq"].T.ravel(), p["bq"].ravel()]
    return np.concatenate(parts).astype(np.float32)


def unpack_grads(vec, cin, width, cout, layers, modes):
    """Packed vector -> dict in the oracle's layout."""
    out, off = {}, 0

    def take(n):
        nonlocal off
        v = vec[off:off + n]
        off += n
        return v
    out["Wl"] = take(cin * width).reshape(cin, width).T
    out["bl"] = take(width)
    for l in range(layers):
        out[f"W{l}"] = take(width * width).reshape(width, width).T
        out[f"b{l}"] = take(width)
        out[f"R{l}"] = take(modes ** 3 * 4 * width * width).reshape(modes, modes, modes, 2 * width, 2 * width)
    out["Wq"] = take(width * cout).reshape(width, cout).T
    out["bq"] = take(cout)
    return out


class SpectralOperator:
    """Handle on the library's network (forward, loss/gradient, Adam)."""

    def __init__(self, layers=4, modes=16, seed=0, cin=CIN, cout=COUT, stream=None):
        self.layers, self.modes, self.cin, self.cout = layers, modes, cin, cout
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = B.rve_fno_create(cin, WIDTH, cout, layers, modes, seed, self.stream.cuda_stream)
        self.nparam = B.rve_fno_param_count(self.h)

    def set_params(self, vec):
        v = np.ascontiguousarray(vec, dtype=np.float32)
        assert v.size == self.nparam
        B.rve_fno_set_params(self.h, v.ctypes.data)

    def get_params(self, want_grad=False):
        p = np.empty(self.nparam, np.float32)
        g = np.empty(self.nparam, np.float32) if want_grad else None
        B.rve_fno_get_params(self.h, p.ctypes.data, g.ctypes.data if g is not None else 0)
        return (p, g) if want_grad else p

    def forward(self, X, dims):
        Y = torch.empty(X.shape[:-1] + (self.cout,), dtype=torch.float32, device=X.device)
        B.rve_fno_forward(self.h, X.shape[0], dims, X.data_ptr(), Y.data_ptr())
        return Y

    def loss_grad(self, X, T, dims):
        return B.rve_fno_loss_grad(self.h, X.shape[0], dims, X.data_ptr(), T.data_ptr())

    def adam_step(self, lr):
        B.rve_fno_adam_step(self.h, lr)

    def features(self, dims, phase, damage, d1, d2, scale):
        nz, ny, nx = dims[2], dims[1], dims[0]
        X = torch.empty((1, nz, ny, nx, self.cin), dtype=torch.float32, device=phase.device)
        B.rve_fno_pack_features(self.h, dims, phase.data_ptr(), damage.data_ptr() if damage is not None else 0,
                                d1.data_ptr() if d1 is not None else 0, d2.data_ptr() if d2 is not None else 0,
                                scale, X.data_ptr())
        return X

    def to_field(self, Y, dims, scale):
        out = torch.empty((self.cout, dims[2], dims[1], dims[0]), dtype=torch.float32, device=Y.device)
        B.rve_fno_unpack_output(self.h, dims, Y.data_ptr(), scale, out.data_ptr())
        return out

    def close(self):
        if getattr(self, "h", None) is not None:
            B.rve_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
