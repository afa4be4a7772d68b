"""Spectral neural operator of the learned warm start: library kernels (BF16
tensor-core contractions, FP32 accumulation) against the FP64 oracle
(needs a GB300)."""
import numpy as np
import pytest

from oracle import fno as ofno

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# BF16 operands (8 significant bits) through about a dozen chained
# contractions: a few parts in 1e3 per product, compounded -> 3e-2 relative.
TOL_Y = 3e-2
TOL_G = 6e-2


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30))


def _setup(layers, modes, seed=0, cin=16, cout=6):
    from paper_2207_10657_gb300 import build
    from paper_2207_10657_gb300.learned import SpectralOperator, pack_params
    build.build()
    p = ofno.init_params(cin=cin, width=32, cout=cout, layers=layers, modes=modes, seed=seed)
    net = SpectralOperator(layers=layers, modes=modes, cin=cin, cout=cout)
    net.set_params(pack_params(p, layers))
    return p, net


@pytest.mark.parametrize("layers,modes,dims,batch", [(2, 8, (20, 12, 10), 2), (4, 6, (16, 9, 14), 3),
                                                     (1, 4, (9, 8, 5), 1)])
def test_forward_matches_oracle(layers, modes, dims, batch):
    p, net = _setup(layers, modes, seed=layers)
    nx, ny, nz = dims
    rng = np.random.default_rng(5)
    X = rng.standard_normal((batch, nz, ny, nx, 16))
    ref = ofno.forward(p, X, modes, layers)
    got = net.forward(torch.from_numpy(X.astype(np.float32)).cuda(), dims).cpu().numpy()
    assert got.shape == ref.shape
    assert _rel(got, ref) < TOL_Y, _rel(got, ref)
    net.close()


def test_loss_and_gradient_match_oracle():
    layers, modes, dims, batch = 2, 6, (14, 10, 8), 2
    p, net = _setup(layers, modes, seed=3)
    nx, ny, nz = dims
    rng = np.random.default_rng(9)
    X = rng.standard_normal((batch, nz, ny, nx, 16))
    T = rng.standard_normal((batch, nz, ny, nx, 6))
    L_ref, g_ref = ofno.backward(p, X, T, modes, layers)
    L = net.loss_grad(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T.astype(np.float32)).cuda(),
                      dims)
    assert abs(L - L_ref) <= 1e-2 * L_ref
    from paper_2207_10657_gb300.learned import unpack_grads
    _, gv = net.get_params(want_grad=True)
    g = unpack_grads(gv, 16, 32, 6, layers, modes)
    for k in g_ref:
        assert _rel(g[k], g_ref[k]) < TOL_G, (k, _rel(g[k], g_ref[k]))
    net.close()


def test_adam_first_step_and_training_reduces_loss():
    layers, modes, dims, batch = 2, 4, (8, 8, 8), 2
    p, net = _setup(layers, modes, seed=1)
    rng = np.random.default_rng(2)
    X = torch.from_numpy(rng.standard_normal((batch, 8, 8, 8, 16)).astype(np.float32)).cuda()
    # a smooth target the network can represent: a fixed linear map of the input
    A = rng.standard_normal((16, 6)).astype(np.float32) / 4
    T = (X @ torch.from_numpy(A).cuda()).contiguous()
    p0 = net.get_params()
    L0 = net.loss_grad(X, T, dims)
    _, g0 = net.get_params(want_grad=True)
    lr = 1e-3
    net.adam_step(lr)
    p1 = net.get_params()
    # first Adam step: bias-corrected moments are g and g^2, update -lr g / (|g| + eps)
    expect = p0 - lr * g0 / (np.abs(g0) + 1e-8)
    assert np.max(np.abs(p1 - expect)) <= 1e-6 + 1e-3 * lr
    for _ in range(60):
        net.loss_grad(X, T, dims)
        net.adam_step(3e-3)
    L1 = net.loss_grad(X, T, dims)
    assert L1 < 0.25 * L0, (L0, L1)
    net.close()


def test_feature_packing_and_unpacking():
    from paper_2207_10657_gb300 import build
    from paper_2207_10657_gb300.learned import SpectralOperator
    build.build()
    net = SpectralOperator(layers=1, modes=4)
    dims = (10, 7, 5)
    V = 350
    rng = np.random.default_rng(3)
    ph = rng.integers(0, 2, V).astype(np.uint8)
    dm = rng.random(V).astype(np.float32)
    d1 = rng.standard_normal((6, V)).astype(np.float32)
    d2 = rng.standard_normal((6, V)).astype(np.float32)
    kp = rng.random(V).astype(np.float32)
    X = net.features(dims, torch.from_numpy(ph).cuda(), torch.from_numpy(dm).cuda(), torch.from_numpy(d1).cuda(),
                     torch.from_numpy(d2).cuda(), 2.0, torch.from_numpy(kp).cuda(), 4.0).cpu().numpy().reshape(V, 16)
    ref = np.zeros((V, 16), np.float32)
    ref[:, 0] = ph == 0
    ref[:, 1] = ph == 1
    ref[:, 2] = dm
    ref[:, 3:9] = 2.0 * d1.T
    ref[:, 9:15] = 2.0 * d2.T
    ref[:, 15] = 4.0 * kp
    assert np.array_equal(X, ref)
    Y = rng.standard_normal((1, 5, 7, 10, 6)).astype(np.float32)
    out = net.to_field(torch.from_numpy(Y).cuda(), dims, 0.5).cpu().numpy()
    assert np.array_equal(out.reshape(6, V), 0.5 * Y.reshape(V, 6).T)
    base = torch.from_numpy(d1.reshape(6, 5, 7, 10)).cuda()
    out = net.to_field(torch.from_numpy(Y).cuda(), dims, 0.5, base).cpu().numpy()
    assert np.allclose(out.reshape(6, V), d1 + 0.5 * Y.reshape(V, 6).T, rtol=1e-6, atol=1e-6)
    # targets: the inverse map, with and without a base field
    from paper_2207_10657_gb300 import binding as B
    f = torch.from_numpy(d2.reshape(6, 5, 7, 10)).cuda()
    T = torch.empty((1, 5, 7, 10, 6), device="cuda")
    B.rve_fno_pack_target(net.h, dims, f.data_ptr(), 2.0, T.data_ptr())
    assert np.array_equal(T.cpu().numpy().reshape(V, 6), 2.0 * d2.T)
    B.rve_fno_pack_target(net.h, dims, f.data_ptr(), 2.0, T.data_ptr(), base.data_ptr())
    assert np.allclose(T.cpu().numpy().reshape(V, 6), 2.0 * (d2 - d1).T, rtol=1e-6, atol=1e-6)
    # fluctuation increment between two strain fields
    inc = torch.empty_like(f)
    B.rve_fno_increment(net.h, dims, f.data_ptr(), base.data_ptr(), [0, 0, 1e-3, 0, 0, 0], inc.data_ptr())
    ref = (d2 - d1).copy()
    ref[2] -= np.float32(1e-3)
    assert np.allclose(inc.cpu().numpy().reshape(6, V), ref, rtol=1e-6, atol=1e-6)
    net.close()


def test_rejects_bad_shapes():
    from paper_2207_10657_gb300 import build, binding as B
    from paper_2207_10657_gb300.learned import SpectralOperator
    build.build()
    net = SpectralOperator(layers=1, modes=8)
    X = torch.zeros((1, 8, 8, 8, 16), device="cuda")
    with pytest.raises(B.RveError):
        net.forward(X, (8, 8, 8))  # Nx < 2 modes
    with pytest.raises(B.RveError):
        B.rve_fno_create(16, 48, 6, 1, 8)  # width must be 32
    net.close()
