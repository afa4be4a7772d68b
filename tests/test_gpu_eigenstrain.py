"""Eigenstrain loading on the GPU (needs a GB300): the material evaluated at
eps + eps_eig (Algorithm 2) with a per-phase eigenstrain, against the FP64
oracle and closed forms.

Workload of the load-path cases: ASR-like cells (Sec. 3.3) -- aggregate
discs / spheres in a cement paste, single gel voxels inside the aggregates
with a growing stress-free expansion (eigenstrain -n * 5e-4 on the normal
components at increment n, the paper's medium step), every mean component
stress-free (free expansion).  Elastic constants and tensile strengths of
Table 2 (E in GPa, kappa0 = f_t / E), softening to zero stiffness at
10 kappa0."""
import numpy as np
import pytest

import oracle
from synth import gel_sites, laminate, random_circles, random_spheres

from tests.test_oracle_eigenstrain import _laminate_expansion

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PASTE = (12.0, 0.3, True, 2.5e-4, 2.5e-3)
AGG = (59.0, 0.3, True, 10.0 / 59000.0, 100.0 / 59000.0)
GEL = (11.0, 0.18, False, 0.0, 0.0)
K0 = {0: PASTE[3], 1: AGG[3]}


def _solver(dims, pm, phases, precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, phases, precision=precision, **kw)


def _oracle_rve(pm, phases, free=None, eig=None):
    return oracle.RVE(pm, [oracle.Phase(*p) if p[2] else oracle.Phase(p[0], p[1]) for p in phases],
                      free_mask=free, eigenstrain=eig)


def _to_dev(a, precision):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if precision == 32 else np.float64)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gel_tables(nd, nstep, step=5e-4):
    nc = 3 if nd == 2 else 6
    out = []
    for n in range(1, nstep + 1):
        t = np.zeros((3, nc))
        t[2, :nd] = -n * step
        out.append(t)
    return out


def _kappa0_map(pm):
    return np.where(pm == 0, K0[0], np.where(pm == 1, K0[1], np.inf))


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", [(32, 24), (24, 20, 18), (12, 16, 10)])
def test_state_with_eigenstrain_matches_oracle(dims, precision):
    """Constitutive evaluation at eps + eps_eig(phase), element by element:
    stress, damage, kappa, and the first-order incremental energy."""
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    base = random_circles(dims, 0.4, rmin=2.0, rmax=4.0, seed=1) if nd == 2 else \
        random_spheres(dims, count=4, rmin=2.0, rmax=3.5, seed=2)
    pm = gel_sites(base, 5, seed=3)
    rng = np.random.default_rng(4)
    eig = rng.standard_normal((3, nc)) * 3e-4
    eps = rng.standard_normal((nc,) + pm.shape) * 2e-4
    kh = rng.uniform(0, 4e-4, pm.shape)
    if precision == 32:
        eig = eig.astype(np.float32).astype(np.float64)
        kh = kh.astype(np.float32).astype(np.float64)
        eps = eps.astype(np.float32).astype(np.float64)
    phases = [PASTE, AGG, GEL]
    s = _solver(dims, pm, phases, precision)
    s.set_state(_to_dev(eps, precision), _to_dev(kh, precision))
    s.set_eigenstrain(eig)
    st = s.get_state()
    orv = _oracle_rve(pm, phases, eig=eig)
    sig, D, kap = orv.stress(eps, kh)
    k0 = _kappa0_map(pm)
    near = np.abs(kap - k0) <= 1e-3 * np.where(np.isfinite(k0), k0, 1.0)
    tol = 2e-6 if precision == 32 else 1e-12
    assert np.max(np.abs(st["damage"].cpu().numpy() - D)[~near]) < (1e-5 if precision == 32 else 1e-12)
    assert _rel(st["sigma"].cpu().numpy(), sig) < 20 * tol
    # strain stays eps (the eigenstrain enters the evaluation only)
    assert np.array_equal(st["eps"].cpu().numpy(), eps.astype(st["eps"].cpu().numpy().dtype))
    p = rng.standard_normal((nc,) + pm.shape) * 1e-4
    dW, dm, grad = s.energy_grad(_to_dev(p, precision))
    sig_t, _, _ = orv.stress(eps + p, kh)
    dW_ref = 0.5 * (np.sum(sig * p) + np.sum(sig_t * p))
    dm_ref = np.sum(sig * p) + 0.5 * np.sum(p * orv.tangent(D, p))
    etol = 1e-5 if precision == 32 else 1e-11
    assert abs(dW - dW_ref) <= etol * abs(dW_ref)
    assert abs(dm - dm_ref) <= etol * abs(dm_ref)
    assert _rel(grad.cpu().numpy(), orv.gradient(sig_t)) < 20 * tol
    # removing it restores the plain evaluation
    s.set_eigenstrain(None)
    sig0, _, _ = _oracle_rve(pm, phases).stress(eps, kh)
    assert _rel(s.get_state()["sigma"].cpu().numpy(), sig0) < 20 * tol
    s.close()


def test_set_eigenstrain_rejects_bad_tables():
    from paper_2207_10657_gb300.binding import RveError
    dims = (8, 8)
    pm = np.zeros((8, 8), np.uint8)
    s = _solver(dims, pm, [PASTE], 32)
    with pytest.raises(ValueError):
        s.set_eigenstrain(np.zeros((2, 3)))
    with pytest.raises(RveError):
        s.set_eigenstrain([[np.nan, 0.0, 0.0]])
    s.set_eigenstrain([[1e-4, 0.0, 0.0]])
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", [(8, 16), (4, 6, 8), (32, 32, 64)])
def test_laminate_free_expansion_gpu(dims, precision):
    """Bilayer laminate, layer A with an isotropic eigenstrain, free
    expansion: the per-layer strains of the closed form."""
    pa, pb = (1.0, 0.3, False, 0.0, 0.0), (10.0, 0.2, False, 0.0, 0.0)
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    pm = laminate(dims, axis=nd - 1)
    a = 3e-4
    table = np.zeros((2, nc))
    table[0, :nd] = a
    s = _solver(dims, pm, [pa, pb], precision, eta_eq=1e-6 if precision == 32 else 1e-11, eta_cg=1e-8,
                R0=1.0, Rmax=1.0)
    s.set_eigenstrain(table)
    rep = s.solve_step(np.zeros(nc), free_mask=[1] * nc)
    assert rep["converged"]
    sx, za, zb = _laminate_expansion(oracle.Phase(*pa[:2]), oracle.Phase(*pb[:2]), a, 0.5, nd == 2)
    eps = s.get_state()["eps"].cpu().numpy().astype(np.float64)
    half = dims[-1] // 2
    ea = np.zeros(nc)
    eb = np.zeros(nc)
    ea[:nd - 1] = sx
    eb[:nd - 1] = sx
    ea[nd - 1], eb[nd - 1] = za, zb
    tol = 1e-4 * a if precision == 32 else 1e-12 * a
    np.testing.assert_allclose(eps[:, :half].reshape(nc, -1) - ea[:, None], 0.0, atol=tol)
    np.testing.assert_allclose(eps[:, half:].reshape(nc, -1) - eb[:, None], 0.0, atol=tol)
    np.testing.assert_allclose(rep["mean_stress"][:nc], 0.0, atol=1e-5 * a * 10.0)
    s.close()


def _gpu_path(dims, pm, tables, precision, **opts):
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    s = _solver(dims, pm, [PASTE, AGG, GEL], precision, **opts)
    reps = []
    for t in tables:
        s.set_eigenstrain(t)
        reps.append(s.solve_step(np.zeros(nc), free_mask=[1] * nc))
    st = s.get_state()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in st.items()}
    s.close()
    return reps, out


def _oracle_path(pm, tables, prm):
    from oracle.solver import load_path
    nc = tables[0].shape[1]
    orv = _oracle_rve(pm, [PASTE, AGG, GEL], free=np.ones(nc, bool))
    return load_path(orv, [np.zeros(nc)] * len(tables), prm, eigenstrains=tables)


def test_asr_load_path_2d_fp64():
    """32x32 ASR-like cell, three expansion increments (elastic, onset of
    cracking next to the gel pixels, growth): mean strain, strain field and
    damaged set against the oracle, mean stress zero."""
    from oracle.solver import TRParams
    dims = (32, 32)
    pm = gel_sites(random_circles(dims, 0.4, rmin=3.0, rmax=6.0, seed=6), 6, seed=7)
    tables = _gel_tables(2, 3)
    R0 = 10 * np.sqrt(pm.size) * 5e-4
    opts = dict(eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=300)
    ref = _oracle_path(pm, tables, TRParams(**opts))
    reps, st = _gpu_path(dims, pm, tables, 64, **opts)
    assert all(r["converged"] for r in reps)
    ms = np.array([r["mean_strain"][:3] for r in reps])
    assert _rel(ms, ref["mean_strain"]) < 1e-6
    np.testing.assert_allclose(np.array([r["mean_stress"][:3] for r in reps]), 0.0, atol=1e-9)
    assert _rel(st["eps"], ref["eps"]) < 1e-6
    k0 = _kappa0_map(pm)
    near = np.abs(ref["kappa"] - k0) <= 1e-3 * np.where(np.isfinite(k0), k0, 1.0)
    dref = ref["kappa"] > k0
    assert dref.any()
    assert np.array_equal((st["kappa"] > k0)[~near], dref[~near])


def test_asr_load_path_3d_fp32():
    """16x12x20 ASR-like cell (ragged sizes, generic FFT engine), three
    expansion increments in FP32 fields: mean strain and strain field within
    1e-4 of the oracle's, the same damaged voxels."""
    from oracle.solver import TRParams
    dims = (16, 12, 20)
    pm = gel_sites(random_spheres(dims, count=4, rmin=2.5, rmax=4.0, seed=8), 4, seed=9)
    tables = _gel_tables(3, 3)
    R0 = 10 * np.sqrt(pm.size) * 5e-4
    ref = _oracle_path(pm, tables, TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=300))
    reps, st = _gpu_path(dims, pm, tables, 32, eta_eq=1e-6, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=300)
    assert all(r["converged"] for r in reps)
    ms = np.array([r["mean_strain"][:6] for r in reps])
    assert _rel(ms, ref["mean_strain"]) < 1e-4
    assert _rel(st["eps"], ref["eps"]) < 1e-4
    k0 = _kappa0_map(pm)
    near = np.abs(ref["kappa"] - k0) <= 1e-3 * np.where(np.isfinite(k0), k0, 1.0)
    dref = ref["kappa"] > k0
    assert dref.any()
    assert np.array_equal((st["kappa"] > k0)[~near], dref[~near])


def test_uniform_eigenstrain_equals_shifted_load_128cube_fp32():
    """At 128^3 (the compiled FP32 passes and the fused CG product): an
    eigenstrain e on every phase under mean-strain control E converges to
    the strain field of the load E + e without eigenstrain, shifted by -e
    (no oracle: a property of Algorithm 2 at any size)."""
    dims = (128, 128, 128)
    pm = random_spheres(dims, count=48, rmin=4.0, rmax=10.0, seed=0)
    phases = [(1.0, 0.3, True, 1e-4, 1e-3), (10.0, 0.2, False, 0.0, 0.0)]
    # elastic magnitudes (kappa stays below kappa0 = 1e-4 at the sphere
    # interfaces), so both paths converge in a few Newton iterations
    e = np.array([6e-6, -3e-6, 9e-6, 1.5e-6, 0.0, -1.5e-6])
    E = np.array([3e-6, 1.5e-6, 6e-6, 0.0, 1.5e-6, 0.0])
    R0 = 10 * np.sqrt(pm.size) * np.linalg.norm(E + e)
    opts = dict(eta_eq=1e-6, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=100)
    sa = _solver(dims, pm, phases, 32, **opts)
    sa.set_eigenstrain(np.repeat(e[None, :], 2, 0))
    ra = sa.solve_step(E, free_mask=[0] * 6, raise_on_error=False)
    ea = sa.get_state()
    sb = _solver(dims, pm, phases, 32, **opts)
    rb = sb.solve_step(E + e, free_mask=[0] * 6, raise_on_error=False)
    eb = sb.get_state()
    assert ra["converged"] and rb["converged"], (ra, rb)
    assert float(ea["kappa"].max()) < 1e-4
    shift = torch.tensor(e, dtype=torch.float32, device=ea["eps"].device).view(6, 1, 1, 1)
    num = torch.linalg.vector_norm((ea["eps"] + shift - eb["eps"]).double())
    assert float(num / torch.linalg.vector_norm(eb["eps"].double())) < 1e-4
    num = torch.linalg.vector_norm((ea["sigma"] - eb["sigma"]).double())
    assert float(num / torch.linalg.vector_norm(eb["sigma"].double())) < 1e-4
    assert np.allclose(ra["mean_stress"], rb["mean_stress"], rtol=1e-4, atol=1e-12)
    sa.close()
    sb.close()
