"""Pins of the oracle's consistent damage tangent (CPU only): central
differences of the stress, the secant on unloading and below the threshold,
the symmetric part against the transposed dense Jacobian, and the
trust-region solver with it reaching the secant solver's equilibrium."""
import numpy as np
import pytest

import oracle
from oracle.consistent import ConsistentRVE, consistent_tangent_apply, positive_part
from oracle.material import PhaseParams, evaluate
from oracle.solver import TRParams, load_path
from synth import random_spheres

K0, KF = 1e-4, 1e-3


def _params(shape, nd):
    pm = np.zeros(shape, np.uint8)
    return pm, PhaseParams(pm, [oracle.Phase(1.0, 0.3, True, K0, KF)])


@pytest.mark.parametrize("nd", [2, 3])
def test_matches_central_differences_of_the_stress(nd):
    """d sigma/d eps : v against (sigma(eps + h v) - sigma(eps - h v)) / 2h
    on loading voxels in the softening range (away from kappa0, kappaf, the
    history and sign changes of the eigenvalues)."""
    nc = 3 if nd == 2 else 6
    shape = (6, 5) if nd == 2 else (4, 5, 3)
    pm, prm = _params(shape, nd)
    rng = np.random.default_rng(0)
    eps = rng.standard_normal((nc,) + shape) * 2e-4
    eps[:nd] += 3e-4
    v = rng.standard_normal((nc,) + shape) * 1e-4
    kt = np.sqrt(np.sum(positive_part(eps) ** 2, axis=0))
    kh = 0.7 * kt  # loading everywhere
    h = 1e-7
    sp, _, _ = evaluate(eps + h * v, prm, kh)
    sm, _, _ = evaluate(eps - h * v, prm, kh)
    fd = (sp - sm) / (2 * h)
    j = consistent_tangent_apply(v, eps, kh, prm)
    w = np.linalg.eigvalsh(oracle.mandel_to_tensor(eps))
    ok = (kt > 1.2 * K0) & (kt < 0.8 * KF) & (np.min(np.abs(w), axis=-1) > 1e-5)
    assert ok.sum() >= 10
    err = np.abs(j - fd)[:, ok].max() / np.abs(fd[:, ok]).max()
    assert err < 1e-6, err
    # the rank-one term matters there
    sec = (1 - evaluate(eps, prm, kh)[1]) * oracle.elastic_stress(v, prm.lam, prm.mu)
    assert np.abs(j - sec)[:, ok].max() > 1e-2 * np.abs(sec[:, ok]).max()


def test_secant_on_unloading_and_below_threshold():
    shape = (4, 4, 4)
    pm, prm = _params(shape, 3)
    rng = np.random.default_rng(1)
    eps = rng.standard_normal((6,) + shape) * 2e-4
    v = rng.standard_normal((6,) + shape)
    kt = np.sqrt(np.sum(positive_part(eps) ** 2, axis=0))
    kh = kt + 1e-4  # unloading: the history exceeds the trial measure
    _, D, _ = evaluate(eps, prm, kh)
    np.testing.assert_allclose(consistent_tangent_apply(v, eps, kh, prm),
                               (1 - D) * oracle.elastic_stress(v, prm.lam, prm.mu), rtol=1e-14, atol=0)
    small = eps * (0.5 * K0 / kt.max())  # every kappa below kappa0
    np.testing.assert_allclose(consistent_tangent_apply(v, small, None, prm),
                               oracle.elastic_stress(v, prm.lam, prm.mu), rtol=1e-14, atol=0)


def test_symmetric_part_is_half_j_plus_jt():
    shape = (3, 2, 2)
    pm, prm = _params(shape, 3)
    rng = np.random.default_rng(2)
    eps = rng.standard_normal((6,) + shape) * 2e-4
    eps[:3] += 3e-4
    kh = np.zeros(shape)
    cols = []
    cols_s = []
    for k in range(6):
        e = np.zeros((6,) + shape)
        e[k] = 1.0
        cols.append(consistent_tangent_apply(e, eps, kh, prm))
        cols_s.append(consistent_tangent_apply(e, eps, kh, prm, sym=True))
    J = np.stack(cols, axis=1)      # (6, 6, *shape): J[:, k] = J e_k
    S = np.stack(cols_s, axis=1)
    np.testing.assert_allclose(S, 0.5 * (J + np.swapaxes(J, 0, 1)), rtol=1e-12, atol=1e-15)
    assert np.abs(J - np.swapaxes(J, 0, 1)).max() > 1e-3 * np.abs(J).max()  # J itself is not symmetric


def test_consistent_hessian_reaches_the_secant_equilibrium_with_fewer_iterations():
    """16x12x10 spheres, uniaxial eps_zz through the onset of damage: the
    trust-region solver with the symmetric consistent tangent ends at the
    secant solver's equilibrium in far fewer Newton iterations."""
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    phases = [oracle.Phase(1.0, 0.3, True, K0, KF), oracle.Phase(10.0, 0.2)]
    free = np.array([True, True, False, True, True, True])
    incs = [np.array([0, 0, 5e-5, 0, 0, 0]), np.array([0, 0, 2e-5, 0, 0, 0])]
    R0 = 10 * np.sqrt(pm.size) * 5e-5
    prm = TRParams(eta_eq=1e-9, eta_cg=1e-3, R0=R0, Rmax=R0, max_nr=500)
    sec = load_path(oracle.RVE(pm, phases, free_mask=free), incs, prm)
    con = load_path(ConsistentRVE(pm, phases, free_mask=free), incs, prm)
    assert all(r.converged for r in sec["reports"]) and all(r.converged for r in con["reports"])
    np.testing.assert_allclose(con["mean_stress"], sec["mean_stress"], rtol=1e-7, atol=1e-14)
    assert np.linalg.norm(con["eps"] - sec["eps"]) <= 1e-6 * np.linalg.norm(sec["eps"])
    n_sec = sum(r.nr_iters for r in sec["reports"])
    n_con = sum(r.nr_iters for r in con["reports"])
    assert n_con * 5 < n_sec, (n_con, n_sec)


def test_full_tangent_newton_gmres_reaches_the_same_equilibrium():
    """The full (non-symmetric) consistent tangent needs a non-symmetric inner
    solver: inexact Newton with restarted GMRES on compatible directions and
    a backtracking line search on the first-order energy of Eq. (18) reaches
    the trust-region solvers' equilibrium at the damage onset in a handful
    of Newton iterations."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    LinearOperator, gmres = sla.LinearOperator, sla.gmres
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    phases = [oracle.Phase(1.0, 0.3, True, K0, KF), oracle.Phase(10.0, 0.2)]
    free = np.array([True, True, False, True, True, True])
    incs = [np.array([0, 0, 5e-5, 0, 0, 0]), np.array([0, 0, 2e-5, 0, 0, 0])]
    rve = oracle.RVE(pm, phases, free_mask=free)
    shape = (6,) + pm.shape
    n = int(np.prod(shape))
    eps, hist = np.zeros(shape), np.zeros(pm.shape)
    newton = []
    for dE in incs:
        eps = eps + dE.reshape(6, 1, 1, 1)
        sig, _, kap = rve.stress(eps, hist)
        g = rve.G(sig)
        its = 0
        while rve.norm(g) > 1e-9 * rve.norm(sig) and its < 50:
            its += 1

            def mv(x, eps=eps):
                v = rve.G(x.reshape(shape))
                return rve.G(consistent_tangent_apply(v, eps, hist, rve.params)).reshape(-1) + (x - v.reshape(-1))

            p, _ = gmres(LinearOperator((n, n), matvec=mv), -g.reshape(-1), rtol=1e-3, restart=50, maxiter=20)
            p = rve.G(p.reshape(shape))
            a, s0 = 1.0, rve.dot(sig, p)
            for _ in range(30):
                st, _, _ = rve.stress(eps + a * p, hist)
                if 0.5 * (s0 + rve.dot(st, p)) * a <= 1e-4 * a * s0:
                    break
                a *= 0.5
            eps = eps + a * p
            sig, _, kap = rve.stress(eps, hist)
            g = rve.G(sig)
        newton.append(its)
        hist = np.maximum(hist, kap)
    R0 = 10 * np.sqrt(pm.size) * 5e-5
    ref = load_path(oracle.RVE(pm, phases, free_mask=free), incs,
                    TRParams(eta_eq=1e-9, eta_cg=1e-3, R0=R0, Rmax=R0, max_nr=500))
    np.testing.assert_allclose(rve.mean(sig), ref["mean_stress"][-1], rtol=1e-7, atol=1e-14)
    assert np.linalg.norm(eps - ref["eps"]) <= 1e-6 * np.linalg.norm(ref["eps"])
    assert sum(newton) < 20, newton
