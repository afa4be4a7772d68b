"""GPU path vs the FP64 CPU oracle, element by element (needs a GB300).

Tolerances: FP64 fields agree to 1e-11 relative (rounding of different
summation orders over O(log N) FFT stages); FP32 fields to 2e-6 relative L2
for single products (about 10x the FP32 unit roundoff times the FFT depth).
"""
import numpy as np
import pytest

import oracle
from synth import random_spheres, circular_inclusion, damage_snapshot, random_field, laminate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
TOL = {32: 2e-6, 64: 1e-11}


def _solver(dims, pm, phases, precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, phases, precision=precision, **kw)


def _oracle_rve(pm, phases, free=None):
    return oracle.RVE(pm, [oracle.Phase(*p) if p[2] else oracle.Phase(p[0], p[1]) for p in phases], free_mask=free)


def _to_dev(a, precision):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if precision == 32 else np.float64)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# generic-engine sizes, the compile-time-specialised FP32 sizes (32..512,
# 96/192/384; in 3D with Nx <= 256 the x-forward stages its rows by bulk
# tensor copies) and mixtures of both, degenerate 2-point axes and a 1024 axis
GRIDS = [(32, 24), (30, 40), (2, 2), (1024, 8), (8, 12, 10), (16, 16, 16), (24, 20, 18), (2, 2, 2),
         (6, 4, 1024), (96, 64), (512, 32), (32, 32, 32), (64, 32, 96), (128, 192, 8), (384, 6, 4),
         (8, 10, 512), (256, 8, 128), (512, 4, 8), (8, 128, 256), (4, 512, 64), (64, 64, 64), (4, 6, 384),
         (6, 4, 192), (4, 384, 6), (6, 96, 96), (96, 10, 6), (192, 6, 4)]


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", GRIDS)
def test_project_matches_oracle(dims, precision):
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    pm = np.zeros(tuple(reversed(dims)), np.uint8)
    s = _solver(dims, pm, [MATRIX], precision)
    for free in (None, [1] + [0] * (nc - 2) + [1]):
        if free is not None:
            s.set_free_mask(free)
        v = random_field(nc, dims, seed=11)
        out = s.project(_to_dev(v, precision)).cpu().numpy()
        ref = oracle.project(v, None if free is None else np.array(free, bool))
        assert _rel(out, ref) < TOL[precision], (dims, free)
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", [(32, 24), (64, 30), (8, 12, 10), (16, 16, 16), (24, 20, 18), (40, 36, 12),
                                  (64, 64), (256, 96), (32, 32, 32), (64, 96, 32), (128, 64, 64),
                                  (256, 8, 128), (8, 128, 256), (512, 4, 64), (64, 64, 64), (96, 10, 6),
                                  (192, 6, 4)])
def test_hessp_matches_oracle(dims, precision):
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    if nd == 2:
        pm = circular_inclusion(dims, 0.3)
    else:
        pm = random_spheres(dims, count=5, rmin=1.5, rmax=3.5, seed=4)
    D = damage_snapshot(pm, dmax=0.9, seed=1)
    s = _solver(dims, pm, [MATRIX, STIFF], precision)
    s.set_damage(_to_dev(D, precision))
    v = random_field(nc, dims, seed=2)
    out = s.hessp(_to_dev(v, precision)).cpu().numpy()
    ref = _oracle_rve(pm, [MATRIX, STIFF]).hessp(D.astype(np.float64), v)
    assert _rel(out, ref) < 5 * TOL[precision]
    # in-place (aliased) call
    x = _to_dev(v, precision)
    s.hessp(x, out=x)
    assert _rel(x.cpu().numpy(), ref) < 5 * TOL[precision]
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", [(32, 32), (12, 16, 10), (32, 32, 32)])
def test_state_stress_damage_and_energy(dims, precision):
    """Constitutive update (Appendix A) and the first-order incremental energy
    (Eq. (18)) against the oracle."""
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    pm = circular_inclusion(dims, 0.3) if nd == 2 else random_spheres(dims, count=3, rmin=1.5, rmax=3.0, seed=5)
    rng = np.random.default_rng(3)
    eps = rng.standard_normal((nc,) + pm.shape) * 4e-4
    kh = rng.uniform(0, 6e-4, pm.shape)
    if precision == 32:
        kh = kh.astype(np.float32).astype(np.float64)
    s = _solver(dims, pm, [MATRIX, STIFF], precision)
    s.set_state(_to_dev(eps, precision), _to_dev(kh, precision))
    st = s.get_state()
    orv = _oracle_rve(pm, [MATRIX, STIFF])
    sig, D, kap = orv.stress(eps, kh)
    # damage: identical except within 1e-3 of the threshold kappa0
    near = np.abs(kap - 1e-4) <= 1e-3 * 1e-4
    dg = st["damage"].cpu().numpy()
    assert np.max(np.abs(dg - D)[~near]) < (1e-5 if precision == 32 else 1e-12)
    assert _rel(st["sigma"].cpu().numpy(), sig) < 20 * TOL[precision]
    p = rng.standard_normal((nc,) + pm.shape) * 2e-4
    dW, dm, grad = s.energy_grad(_to_dev(p, precision))
    sig_t, _, _ = orv.stress(eps + p, kh)
    dW_ref = 0.5 * (np.sum(sig * p) + np.sum(sig_t * p))
    dm_ref = np.sum(sig * p) + 0.5 * np.sum(p * orv.tangent(D, p))
    tol = 1e-5 if precision == 32 else 1e-11
    assert abs(dW - dW_ref) <= tol * abs(dW_ref)
    assert abs(dm - dm_ref) <= tol * abs(dm_ref)
    assert _rel(grad.cpu().numpy(), orv.gradient(sig_t)) < 20 * TOL[precision]
    s.close()


def _oracle_curve(pm, phases, incs, free, prm):
    from oracle.solver import load_path
    orv = _oracle_rve(pm, phases, free)
    return load_path(orv, incs, prm)


def test_load_path_2d_plane_strain_fp64():
    """32x32 plane strain, centred inclusion (vol. frac. 0.3), eps_xx ramped
    0 -> 2e-3 in 20 increments, other components free: the homogenised
    stress-strain curve matches the oracle along the softening branch."""
    from oracle.solver import TRParams
    dims = (32, 32)
    pm = circular_inclusion(dims, 0.3)
    phases = [MATRIX, (10.0, 0.3, False, 0.0, 0.0)]
    free = [0, 1, 1]
    incs = [np.array([1e-4, 0, 0])] * 20
    R0 = 10 * np.sqrt(32 * 32) * 1e-4
    # the secant Hessian makes Newton converge linearly once damage grows:
    # generous iteration caps on both sides
    prm = TRParams(eta_eq=1e-8, eta_cg=1e-10, R0=R0, Rmax=R0, max_nr=400, max_cg=500)
    ref = _oracle_curve(pm, phases, incs, np.array(free, bool), prm)
    s = _solver(dims, pm, phases, 64, eta_eq=1e-8, eta_cg=1e-10, R0=R0, Rmax=R0, max_nr=400, max_cg=500)
    sig_gpu = []
    for n, dE in enumerate(incs):
        rep = s.solve_step(dE, free_mask=free)
        assert rep["converged"], (n, rep)
        sig_gpu.append(rep["mean_stress"][:3])
    sig_gpu = np.array(sig_gpu)
    sref = ref["mean_stress"]
    scale = np.max(np.abs(sref[:, 0]))
    err = np.max(np.abs(sig_gpu[:, 0] - sref[:, 0])) / scale
    assert err < 1e-4, err
    st = s.get_state()
    kap_gpu = st["kappa"].cpu().numpy()
    dmg_ref = ref["kappa"] > 1e-4
    near = np.abs(ref["kappa"] - 1e-4) <= 1e-3 * 1e-4
    # The centred disc and the uniaxial load are symmetric under x and y
    # mirrors (voxel i <-> N-1-i), so a localised band may form on either
    # mirror side: the damaged set is unique only up to that group.
    dg = kap_gpu > 1e-4
    images = [dg, dg[:, ::-1], dg[::-1, :], dg[::-1, ::-1]]
    nimg = [near, near[:, ::-1], near[::-1, :], near[::-1, ::-1]]
    assert any(np.array_equal(im[~(nr | near)], dmg_ref[~(nr | near)]) for im, nr in zip(images, nimg)), \
        (int(dg.sum()), int(dmg_ref.sum()))
    s.close()


def test_load_path_3d_fp32_uniaxial():
    """16^3 spheres in a damaging matrix, uniaxial eps_zz with the other
    components free, FP32 fields with FP64 reductions, relative residual
    1e-6: the elastic increment and the onset of damage give homogenised
    stresses within 1e-5 / 1e-4 of the oracle's."""
    from oracle.solver import TRParams
    dims = (16, 16, 16)
    pm = random_spheres(dims, count=6, rmin=2.0, rmax=3.5, seed=7)
    phases = [MATRIX, STIFF]
    free = [1, 1, 0, 1, 1, 1]
    incs = [np.array([0, 0, 4e-5, 0, 0, 0])] * 2
    R0 = 10 * np.sqrt(16 ** 3) * 4e-5
    prm = TRParams(eta_eq=1e-6, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=300)
    ref = _oracle_curve(pm, phases, incs, np.array(free, bool), prm)
    s = _solver(dims, pm, phases, 32, eta_eq=1e-6, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=300)
    out = []
    for dE in incs:
        rep = s.solve_step(dE, free_mask=free)
        assert rep["converged"]
        out.append(rep["mean_stress"])
    out = np.array(out)
    sref = ref["mean_stress"]
    assert abs(out[0, 2] - sref[0, 2]) <= 1e-5 * abs(sref[0, 2])
    assert abs(out[1, 2] - sref[1, 2]) <= 1e-4 * abs(sref[1, 2])
    s.close()


def test_elastic_step_64cube_fp32_matches_oracle():
    """One elastic increment on a 64^3 sphere cell (power-of-two passes of
    every axis, CG dot products fused into the x-inverse pass): homogenised
    stress within 1e-5 and strain field within 1e-4 (relative L2) of the
    oracle's."""
    from oracle.solver import TRParams
    dims = (64, 64, 64)
    pm = random_spheres(dims, count=48, rmin=2.0, rmax=5.0, seed=3)
    phases = [MATRIX, STIFF]
    free = [1, 1, 0, 1, 1, 1]
    incs = [np.array([0, 0, 1e-5, 0, 0, 0])]
    R0 = 10 * np.sqrt(64 ** 3) * 1e-5
    prm = TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=100)
    ref = _oracle_curve(pm, phases, incs, np.array(free, bool), prm)
    s = _solver(dims, pm, phases, 32, eta_eq=1e-6, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=100)
    rep = s.solve_step(incs[0], free_mask=free)
    assert rep["converged"]
    sref = ref["mean_stress"][0]
    assert np.linalg.norm(np.array(rep["mean_stress"]) - sref) <= 1e-5 * np.linalg.norm(sref)
    if ref.get("eps") is not None:
        eps = s.get_state()["eps"].cpu().numpy().astype(np.float64)
        assert _rel(eps, ref["eps"]) < 1e-4
    s.close()


def test_laminate_closed_form_gpu():
    """Bilayer laminate normal to z (interfaces on voxel faces): the GPU
    solve reproduces the exact per-layer strains."""
    dims = (8, 8, 16)
    pm = laminate(dims, axis=2)
    phases = [(1.0, 0.0, False, 0.0, 0.0), (10.0, 0.0, False, 0.0, 0.0)]
    s = _solver(dims, pm, phases, 64, eta_eq=1e-12, eta_cg=1e-12, R0=1e3, Rmax=1e3)
    rep = s.solve_step([0, 0, 1e-3, 0, 0, 0])
    assert rep["converged"]
    eps = s.get_state()["eps"].cpu().numpy()
    # nu = 0: Reuss along z -> e_a E_a = e_b E_b, mean 1e-3
    ea = 2e-3 * 10.0 / 11.0
    eb = 2e-3 - ea
    np.testing.assert_allclose(eps[2, :8], ea, rtol=1e-10)
    np.testing.assert_allclose(eps[2, 8:], eb, rtol=1e-10)
    assert abs(rep["mean_stress"][2] - 1e-3 / (0.5 / 1.0 + 0.5 / 10.0)) < 1e-12
    s.close()


def _plane_wave(A, k, dims):
    """Re(A e^{i k.x}) in float32, phase index reduced exactly mod N."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij", sparse=True)
    n = nx
    assert nx == ny == nz
    idx = (k[0] * x + k[1] * y + k[2] * z) % n
    c = np.cos(2 * np.pi * np.arange(n) / n)[idx]
    s = np.sin(2 * np.pi * np.arange(n) / n)[idx]
    return np.stack([(a.real * c - a.imag * s).astype(np.float32) for a in A])


@pytest.mark.parametrize("n", [256, 384])
def test_full_size_plane_wave_and_symmetry(n):
    """At the benchmark size (256^3, FP32, the launch configuration the bench
    times) and at the largest cell of the full-size sphere configuration
    (384^3: the compiled x-forward without bulk tensor copies, the staged z
    pass): single Fourier modes are projected exactly as the oracle's
    per-frequency operator predicts, and the Hessian-vector product is
    symmetric, positive and compatible (G H v = H v) on a heterogeneous
    damage snapshot."""
    dims = (n, n, n)
    pm = random_spheres(dims, count=144, rmin=4.0, rmax=10.0, seed=0)
    D = damage_snapshot(pm, dmax=0.9, seed=1)
    s = _solver(dims, pm, [MATRIX, STIFF], 32)
    rng = np.random.default_rng(0)
    h = n // 2
    for k in [(3, n - 6, h + 1), (h, 0, 17), (0, h, h), (77, 1, n - 1)]:
        A = rng.standard_normal(6) + 1j * rng.standard_normal(6)
        field = _plane_wave(A, k, dims)
        out = s.project(_to_dev(field, 32)).cpu().numpy()
        GA = oracle.project_one(A, oracle.gradient_symbol_at(k, dims))
        # the Nyquist-x mode is its own conjugate: only Re(GA e^{ikx}) survives
        ref = _plane_wave(GA, k, dims)
        # 5e-6 of the projected mode, plus the FP32 rounding of the forward
        # and inverse transforms relative to the input (unit roundoff 6e-8
        # times a few stages; a mode the FE gradient annihilates, such as
        # (0, N/2, N/2), has an exact result of zero and keeps only that)
        tol = 5e-6 * np.linalg.norm(ref) + 1e-7 * np.linalg.norm(field)
        assert np.linalg.norm(out - ref) < tol, k
        del field, out, ref
    s.set_damage(_to_dev(D, 32))
    u = s.project(_to_dev(random_field(6, dims, seed=5, dtype=np.float32), 32))
    w = s.project(_to_dev(random_field(6, dims, seed=6, dtype=np.float32), 32))
    Hu, Hw = s.hessp(u), s.hessp(w)
    a = torch.sum(u.double() * Hw.double()).item()
    b = torch.sum(Hu.double() * w.double()).item()
    assert abs(a - b) <= 1e-5 * abs(a)
    GHu = s.project(Hu)
    assert (torch.linalg.vector_norm((GHu - Hu).double()) / torch.linalg.vector_norm(Hu.double())).item() < 1e-5
    assert torch.sum(u.double() * Hu.double()).item() > 0
    s.close()


@pytest.mark.parametrize("n", [256, 384])
def test_laminate_closed_form_full_size_fp32(n):
    """The bilayer laminate of the full-size configuration (256^3, and the
    configuration's largest cell edge 384), general strain-controlled load
    with Poisson coupling, FP32 fields: per-layer strains of the closed form
    (written out from the interface conditions) within 1e-4 of the largest
    strain (the strain-field bound)."""
    from tests.test_oracle_solver import _laminate_exact
    dims = (n, n, n)
    pm = laminate(dims, axis=2)
    pa, pb = (1.0, 0.3, False, 0.0, 0.0), (10.0, 0.2, False, 0.0, 0.0)
    E = np.array([2e-4, -1e-4, 1e-3, 3e-4, -2e-4, 1e-4])
    s = _solver(dims, pm, [pa, pb], 32, eta_eq=1e-6, eta_cg=1e-4)
    rep = s.solve_step(E)
    assert rep["converged"]
    ea, eb = _laminate_exact(oracle.Phase(1.0, 0.3), oracle.Phase(10.0, 0.2), E)
    eps = s.get_state()["eps"]
    scale = float(np.abs(np.concatenate([ea, eb])).max())
    ta = torch.tensor(ea, dtype=torch.float32, device=eps.device).view(6, 1, 1, 1)
    tb = torch.tensor(eb, dtype=torch.float32, device=eps.device).view(6, 1, 1, 1)
    assert float((eps[:, :n // 2] - ta).abs().max()) < 1e-4 * scale
    assert float((eps[:, n // 2:] - tb).abs().max()) < 1e-4 * scale
    s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_load_path_mixed_shear_uniaxial(precision):
    """Mixed load path: eps_zz and the shear eps_yz ramped together (the
    other components stress-free) on a ragged 12x10x8 sphere cell, through
    the elastic increment and three increments of growing damage before the
    peak: homogenised eps_zz and shear stresses against the oracle (1e-5
    elastic, 1e-4 damaged), same damaged voxels."""
    from oracle.solver import TRParams
    dims = (12, 10, 8)
    pm = random_spheres(dims, count=3, rmin=1.5, rmax=2.5, seed=11)
    phases = [MATRIX, STIFF]
    free = [1, 1, 0, 0, 1, 1]
    inc = np.array([0, 0, 2e-5, np.sqrt(2) * 1e-5, 0, 0])
    incs = [inc] * 4
    R0 = 10 * np.sqrt(pm.size) * np.linalg.norm(inc)
    ref = _oracle_curve(pm, phases, incs, np.array(free, bool),
                        TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=400))
    eta = 1e-8 if precision == 64 else 1e-6
    s = _solver(dims, pm, phases, precision, eta_eq=eta, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=400)
    out = []
    for dE in incs:
        rep = s.solve_step(dE, free_mask=free)
        assert rep["converged"]
        out.append(rep["mean_stress"])
    out = np.array(out)
    sref = ref["mean_stress"]
    for n in range(4):
        tol = 1e-5 if n == 0 else 1e-4
        for c in (2, 3):
            assert abs(out[n, c] - sref[n, c]) <= tol * abs(sref[n, c]), (n, c, out[n, c], sref[n, c])
    kap = s.get_state()["kappa"].cpu().numpy().astype(np.float64)
    near = np.abs(ref["kappa"] - 1e-4) <= 1e-3 * 1e-4
    assert (ref["kappa"] > 1e-4).any()
    assert np.array_equal((kap > 1e-4)[~near], (ref["kappa"] > 1e-4)[~near])
    s.close()
