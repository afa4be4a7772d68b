"""Effective secant stiffness on the GPU (needs a GB300): against the FP64
oracle on damage snapshots, the uniform-damage closed form, the stiffness
loss of the ASR-like cell after gel expansion (Sec. 3.3), and symmetry and
the Voigt / Reuss bounds at 128^3."""
import numpy as np
import pytest

import oracle
from oracle.homogenize import effective_stiffness
from synth import circular_inclusion, damage_snapshot, gel_sites, random_circles, random_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)


def _solver(dims, pm, phases, precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, phases, precision=precision, **kw)


def _oracle_rve(pm, phases, free=None):
    return oracle.RVE(pm, [oracle.Phase(*p) if p[2] else oracle.Phase(p[0], p[1]) for p in phases], free_mask=free)


def _mandel_C(lam, mu, nc):
    nd = 2 if nc == 3 else 3
    C = 2.0 * mu * np.eye(nc)
    C[:nd, :nd] += lam
    return C


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dims", [(32, 24), (12, 16, 10), (24, 20, 18)])
def test_effective_stiffness_matches_oracle(dims, precision):
    nd = len(dims)
    pm = circular_inclusion(dims, 0.3) if nd == 2 else random_spheres(dims, count=3, rmin=1.5, rmax=3.0, seed=5)
    D = damage_snapshot(pm, dmax=0.9, seed=2, dtype=np.float64)
    if precision == 32:
        D = D.astype(np.float32).astype(np.float64)
    ref = effective_stiffness(_oracle_rve(pm, [MATRIX, STIFF]), D)
    s = _solver(dims, pm, [MATRIX, STIFF], precision)
    s.set_damage(torch.from_numpy(D.astype(np.float32 if precision == 32 else np.float64)).cuda())
    C, its = s.effective_stiffness(tol=1e-11 if precision == 64 else 1e-6, max_cg=5000)
    C = np.array(C)
    assert its > 0
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < (1e-8 if precision == 64 else 1e-4), err
    s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_uniform_damage_closed_form_gpu(precision):
    dims = (8, 8, 8)
    pm = np.zeros((8, 8, 8), np.uint8)
    s = _solver(dims, pm, [(2.0, 0.25, True, 1e-4, 1e-3)], precision)
    d = 0.25
    s.set_damage(torch.full((8, 8, 8), d, dtype=torch.float32 if precision == 32 else torch.float64).cuda())
    C, _ = s.effective_stiffness()
    lam, mu = 2.0 * 0.25 / (1.25 * 0.5), 2.0 / 2.5
    np.testing.assert_allclose(np.array(C), (1 - d) * _mandel_C(lam, mu, 6), rtol=1e-6 if precision == 32 else 1e-12,
                               atol=1e-7)
    s.close()


def test_stiffness_call_leaves_the_solver_state():
    """A load step after the stiffness computation matches one on a fresh
    context (free mask, radius and options restored)."""
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    free = [1, 1, 0, 1, 1, 1]
    dE = [0, 0, 1e-5, 0, 0, 0]  # both increments elastic
    a = _solver(dims, pm, [MATRIX, STIFF], 64, eta_eq=1e-10, max_nr=200)
    b = _solver(dims, pm, [MATRIX, STIFF], 64, eta_eq=1e-10, max_nr=200)
    a.solve_step(dE, free_mask=free)
    b.solve_step(dE, free_mask=free)
    a.effective_stiffness()
    ra = a.solve_step(dE)
    rb = b.solve_step(dE)
    np.testing.assert_allclose(ra["mean_stress"], rb["mean_stress"], rtol=1e-9, atol=1e-15)
    assert ra["R"] == rb["R"]
    a.close()
    b.close()


def test_asr_stiffness_loss_2d_fp64():
    """||C_bar|| / ||C_bar_0|| of the ASR-like 2D cell after three gel
    expansion increments (damage next to the gel pixels), against the
    oracle's path and homogenisation."""
    from oracle.material import damage_of_kappa
    from oracle.solver import TRParams, load_path
    dims = (32, 32)
    pm = gel_sites(random_circles(dims, 0.4, rmin=3.0, rmax=6.0, seed=6), 6, seed=7)
    phases = [(12.0, 0.3, True, 2.5e-4, 2.5e-3), (59.0, 0.3, True, 10.0 / 59000.0, 100.0 / 59000.0),
              (11.0, 0.18, False, 0.0, 0.0)]
    tables = []
    for n in (1, 2, 3):
        t = np.zeros((3, 3))
        t[2, :2] = -n * 5e-4
        tables.append(t)
    R0 = 10 * np.sqrt(pm.size) * 5e-4
    orv = _oracle_rve(pm, phases, np.ones(3, bool))
    ref = load_path(orv, [np.zeros(3)] * 3, TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=300),
                    eigenstrains=tables)
    k0 = np.where(pm == 0, 2.5e-4, np.where(pm == 1, 10.0 / 59000.0, np.inf))
    kf = 10 * k0
    Dref = np.where(pm < 2, damage_of_kappa(ref["kappa"], k0, kf), 0.0)
    C0 = effective_stiffness(orv, np.zeros(pm.shape))
    C1 = effective_stiffness(orv, Dref)
    ratio_ref = np.linalg.norm(C1) / np.linalg.norm(C0)
    s = _solver(dims, pm, phases, 64, eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=300)
    C0g, _ = s.effective_stiffness(tol=1e-11)
    for t in tables:
        s.set_eigenstrain(t)
        assert s.solve_step(np.zeros(3), free_mask=[1, 1, 1])["converged"]
    C1g, _ = s.effective_stiffness(tol=1e-11)
    ratio = np.linalg.norm(np.array(C1g)) / np.linalg.norm(np.array(C0g))
    assert ratio < 1.0 and ratio_ref < 1.0
    assert abs(ratio - ratio_ref) < 1e-6 * ratio_ref, (ratio, ratio_ref)
    s.close()


def test_effective_stiffness_128cube_symmetric_and_bounded():
    dims = (128, 128, 128)
    pm = random_spheres(dims, count=48, rmin=4.0, rmax=10.0, seed=0)
    D = damage_snapshot(pm, dmax=0.9, seed=2, dtype=np.float32)
    s = _solver(dims, pm, [MATRIX, STIFF], 32)
    s.set_damage(torch.from_numpy(D).cuda())
    C, _ = s.effective_stiffness(tol=1e-6, max_cg=2000)
    C = np.array(C)
    assert np.abs(C - C.T).max() < 1e-4 * np.abs(C).max()
    Cs = 0.5 * (C + C.T)
    lm, mm = 1.0 * 0.3 / (1.3 * 0.4), 1.0 / 2.6
    ls, ms = 10.0 * 0.2 / (1.2 * 0.6), 10.0 / 2.4
    keep = 1.0 - D.astype(np.float64)
    Cv = np.zeros((6, 6))
    Sr = np.zeros((6, 6))
    for phase_id, (l, m) in enumerate([(lm, mm), (ls, ms)]):
        sel = pm == phase_id
        k = keep[sel]
        Cv += k.sum() * _mandel_C(l, m, 6)
        Sr += (1.0 / k).sum() * np.linalg.inv(_mandel_C(l, m, 6))
    Cv /= pm.size
    Cr = np.linalg.inv(Sr / pm.size)
    assert np.linalg.eigvalsh(Cv - Cs).min() > -1e-4 * np.abs(Cv).max()
    assert np.linalg.eigvalsh(Cs - Cr).min() > -1e-4 * np.abs(Cv).max()
    s.close()
