"""Pins of the oracle's solvers (CPU only): brute-force FE, closed forms for
homogeneous media and laminates, the first-order incremental energy on
quadratic problems, finite differences, Steihaug on dense matrices and the
1D spring example of Sec. 3.1."""
import math

import numpy as np
import pytest

import oracle
from oracle.solver import steihaug_cg, trust_region_step, TRParams, load_path
from oracle.spring1d import Spring1D
from synth import circular_inclusion, random_spheres, laminate
from tests import fe_bruteforce as fe

MATRIX = oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3)
STIFF = oracle.Phase(10.0, 0.2)
TIGHT = dict(eta_eq=1e-12, eta_cg=1e-12, R0=1e9, Rmax=1e9, max_cg=5000)


def elastic_solve(phase_map, phases, E, free=None, **kw):
    rve = oracle.RVE(phase_map, phases, free_mask=free)
    prm = TRParams(**{**TIGHT, **kw})
    res = load_path(rve, [E], prm)
    return res, rve


@pytest.mark.parametrize("dims,free", [
    ((8, 8), None),
    ((8, 8), np.array([False, True, True])),
    ((4, 4, 4), None),
    ((4, 4, 4), np.array([True, True, False, True, True, True])),
])
def test_elastic_solve_matches_bruteforce_fe(dims, free):
    """Projection + trust-region CG converge to the same strain field as the
    directly assembled periodic FE problem (the equivalence of the
    projection and displacement formulations, Sec. 1)."""
    if len(dims) == 2:
        pm = circular_inclusion(dims, 0.3)
        E = np.array([1e-3, 0.0, 0.0]) if free is not None else np.array([1e-3, -2e-4, 3e-4])
    else:
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        pm[1:3, 1:3, 0:2] = 1
        pm[3, 0, 3] = 1
        E = np.array([0, 0, 1e-3, 0, 0, 0.0]) if free is not None else np.array([1e-3, -2e-4, 3e-4, 1e-4, 0, 2e-4])
    # elastic: damage never starts below kappa0 with these small strains
    phases = [oracle.Phase(1.0, 0.3), STIFF]
    res, rve = elastic_solve(pm, phases, E, free)
    eps = res["eps"]
    lam, mu = rve.params.lam, rve.params.mu
    ref, _ = fe.solve_elastic(dims, lam, mu, E * (1 - (free if free is not None else 0)), free)
    np.testing.assert_allclose(eps, ref, atol=1e-12 * 1e3, rtol=0)
    assert np.max(np.abs(eps - ref)) / np.max(np.abs(ref)) < 1e-9


def test_homogeneous_medium_zero_fluctuation_and_poisson():
    pm = np.zeros((4, 6, 5), np.uint8)
    E = np.array([1e-3, -2e-4, 3e-4, 1e-4, 0, 2e-4])
    res, _ = elastic_solve(pm, [oracle.Phase(1.0, 0.3)], E)
    np.testing.assert_allclose(res["eps"], np.broadcast_to(E.reshape(6, 1, 1, 1), res["eps"].shape), atol=1e-15)
    free = np.array([True, True, False, True, True, True])
    res, _ = elastic_solve(pm, [oracle.Phase(1.0, 0.3)], np.array([0, 0, 1e-3, 0, 0, 0.0]), free)
    np.testing.assert_allclose(res["mean_strain"][-1], [-3e-4, -3e-4, 1e-3, 0, 0, 0], atol=1e-15)
    np.testing.assert_allclose(res["mean_stress"][-1], [0, 0, 1e-3, 0, 0, 0], atol=1e-15)
    # plane strain, eps_xx controlled: eps_yy = -nu/(1-nu) eps_xx
    res, _ = elastic_solve(np.zeros((6, 6), np.uint8), [oracle.Phase(1.0, 0.3)],
                           np.array([1e-3, 0, 0]), np.array([False, True, True]))
    np.testing.assert_allclose(res["mean_strain"][-1], [1e-3, -0.3 / 0.7 * 1e-3, 0], atol=1e-15)


def _laminate_exact(pa, pb, E):
    """Bilayer normal to z, equal thickness: in-plane strain continuous,
    out-of-plane strain per layer from traction continuity and the mean."""
    la, ma = oracle.lame(pa.E, pa.nu)
    lb, mb = oracle.lame(pb.E, pb.nu)
    exx, eyy, ezz, eyz, exz, exy = E
    # zz: (l+2m) e_zz + l (exx+eyy) equal in both layers, mean e_zz = ezz
    s = exx + eyy
    A = np.array([[la + 2 * ma, -(lb + 2 * mb)], [0.5, 0.5]])
    b = np.array([(lb - la) * s, ezz])
    za, zb = np.linalg.solve(A, b)
    # shear yz / xz: mu_a e_a = mu_b e_b, mean = E
    def ser(e):
        ea = 2 * mb * e / (ma + mb)
        return ea, 2 * e - ea
    yza, yzb = ser(eyz)
    xza, xzb = ser(exz)
    ea = np.array([exx, eyy, za, yza, xza, exy])
    eb = np.array([exx, eyy, zb, yzb, xzb, exy])
    return ea, eb


@pytest.mark.parametrize("nu", [0.0, 0.3])
def test_laminate_closed_form(nu):
    pa, pb = oracle.Phase(1.0, nu), oracle.Phase(10.0, 0.2 if nu else 0.0)
    dims = (4, 4, 8)
    pm = laminate(dims, axis=2)
    E = np.array([2e-4, -1e-4, 1e-3, 3e-4, -2e-4, 1e-4])
    res, rve = elastic_solve(pm, [pa, pb], E)
    ea, eb = _laminate_exact(pa, pb, E)
    eps = res["eps"]
    np.testing.assert_allclose(eps[:, :4].reshape(6, -1), np.repeat(ea[:, None], 64, 1), atol=1e-15)
    np.testing.assert_allclose(eps[:, 4:].reshape(6, -1), np.repeat(eb[:, None], 64, 1), atol=1e-15)
    if nu == 0.0:
        # Reuss (series) along z, Voigt (parallel) along x
        sig = res["mean_stress"][-1]
        assert np.isclose(sig[2], E[2] / (0.5 / 1.0 + 0.5 / 10.0))
        assert np.isclose(sig[0], 0.5 * (1.0 + 10.0) * E[0])


def test_faief_exact_on_quadratic_energy():
    """Elastic (quadratic W): the first-order incremental energy equals the
    exact energy change, so rho_bar = 1 to rounding."""
    pm = circular_inclusion((16, 16), 0.3)
    rve = oracle.RVE(pm, [oracle.Phase(1.0, 0.3), STIFF])
    prm = TRParams(eta_eq=1e-10, eta_cg=1e-3, R0=1e-3, Rmax=1.0)
    eps = np.zeros((3, 16, 16)) + np.array([1e-3, 0, 0]).reshape(3, 1, 1)
    _, _, _, _, rep = trust_region_step(rve, eps, np.zeros((16, 16)), prm.R0, prm)
    assert rep.converged and len(rep.rhos) >= 2
    np.testing.assert_allclose(rep.rhos, 1.0, atol=1e-9)


def test_gradient_matches_finite_difference_frozen_damage():
    """With D frozen, W = sum 1/2 (1-D) eps:C:eps; its directional derivative
    along a compatible delta equals (G sigma) . delta."""
    rng = np.random.default_rng(5)
    pm = random_spheres((8, 8, 8), count=3, rmin=1.5, rmax=2.5, seed=3)
    rve = oracle.RVE(pm, [MATRIX, STIFF])
    eps = rng.standard_normal((6, 8, 8, 8)) * 1e-3
    D = np.where(pm == 0, rng.uniform(0, 0.9, pm.shape), 0.0)
    sigma = (1 - D) * oracle.elastic_stress(eps, rve.params.lam, rve.params.mu)
    delta = rve.G(rng.standard_normal(eps.shape))
    h = 1e-4
    fd = (rve.energy_frozen(eps + h * delta, D) - rve.energy_frozen(eps - h * delta, D)) / (2 * h)
    an = rve.dot(rve.gradient(sigma), delta)
    assert abs(fd - an) <= 1e-9 * abs(an)
    # Hessian: second difference along delta equals delta . H delta
    fd2 = (rve.energy_frozen(eps + h * delta, D) - 2 * rve.energy_frozen(eps, D)
           + rve.energy_frozen(eps - h * delta, D)) / h ** 2
    assert abs(fd2 - rve.dot(delta, rve.hessp(D, delta))) <= 1e-6 * abs(fd2)


def test_hessp_symmetric_psd_and_identity_medium():
    rng = np.random.default_rng(6)
    pm = random_spheres((8, 8, 8), count=3, rmin=1.5, rmax=2.5, seed=4)
    rve = oracle.RVE(pm, [MATRIX, STIFF])
    D = np.where(pm == 0, rng.uniform(0, 0.9, pm.shape), 0.0)
    u = rve.G(rng.standard_normal((6, 8, 8, 8)))
    v = rve.G(rng.standard_normal((6, 8, 8, 8)))
    a, b = rve.dot(u, rve.hessp(D, v)), rve.dot(rve.hessp(D, u), v)
    assert abs(a - b) <= 1e-12 * abs(a)
    assert rve.dot(u, rve.hessp(D, u)) > 0
    # lambda = 0, mu = 1/2 gives C = I, so H v = G v
    ident = oracle.RVE(np.zeros((4, 4, 4), np.uint8), [oracle.Phase(1.0, 0.0)])
    w = rng.standard_normal((6, 4, 4, 4))
    np.testing.assert_allclose(ident.hessp(np.zeros((4, 4, 4)), w), ident.G(w), atol=1e-14)


def _dot(a, b):
    return float(np.dot(a, b))


def test_steihaug_dense_cases():
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    H = Q @ np.diag(np.linspace(1, 5, 12)) @ Q.T
    g = rng.standard_normal(12)
    p, info = steihaug_cg(lambda v: H @ v, g, 1e6, 1e-13, 100, _dot, restart_thr=1.0)
    np.testing.assert_allclose(p, -np.linalg.solve(H, g), atol=1e-11)
    assert info["reason"] == "converged" and not info["on_boundary"]
    p, info = steihaug_cg(lambda v: H @ v, g, 0.05, 1e-13, 100, _dot)
    assert info["on_boundary"] and np.isclose(np.linalg.norm(p), 0.05)
    # indefinite: lands on the boundary with a model value below m(0) = 0
    Hn = Q @ np.diag(np.linspace(-2, 5, 12)) @ Q.T
    p, info = steihaug_cg(lambda v: Hn @ v, g, 1.0, 1e-13, 100, _dot)
    assert info["on_boundary"] and np.isclose(np.linalg.norm(p), 1.0)
    assert g @ p + 0.5 * p @ Hn @ p < 0.0


@pytest.mark.parametrize("alpha", [1.0, -0.5, -1.0])
def test_spring_stiffness_eigenvalues(alpha):
    """Eq. (21): post-peak nodal stiffness has eigenvalues 0, 3k, (2a+1)k."""
    s = Spring1D(k=1.0, gamma0=0.1, alpha=alpha)
    K = s.nodal_stiffness(np.array([0.0, 0.0, 0.15]))
    ref = np.array([[(1 + alpha), -1, -alpha], [-1, 2, -1], [-alpha, -1, (1 + alpha)]])
    np.testing.assert_allclose(K, ref, atol=1e-15)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(K)), np.sort([0, 3, 2 * alpha + 1]), atol=1e-12)


@pytest.mark.parametrize("alpha", [1.0, -0.5, -1.0])
def test_spring_modified_vs_standard_trust_region(alpha):
    """Sec. 3.1: the modified solver (first-order incremental energy) and the
    standard one (exact energy) reach the same equilibrium, a minimiser of
    the energy; on the quadratic (convex, alpha = 1) problem their iterates
    coincide."""
    s = Spring1D(k=1.0, gamma0=0.1, alpha=alpha)
    xbar = 0.11
    start = np.array([xbar + 0.02, xbar - 0.05, xbar + 0.03])  # sum = 3 xbar
    out = {}
    for exact in (False, True):
        # at the broken-spring equilibrium sigma = 0, so the relative residual is
        # undefined there; Algorithm 2's second criterion |d_eps|/|eps| ends it
        prm = TRParams(eta_eq=1e-12, eta_nr=1e-12, eta_cg=1e-12, R0=0.05, Rmax=0.2,
                       exact_rho=exact, max_nr=200)
        eps, sig, _, _, rep = trust_region_step(s, start.copy(), None, prm.R0, prm, record_iterates=True)
        out[exact] = (eps, rep)
        assert rep.converged
        assert np.isclose(eps.sum(), 3 * xbar)
        assert np.max(np.abs(sig - sig.mean())) < 1e-10  # equal forces
    (e0, r0), (e1, r1) = out[False], out[True]
    np.testing.assert_allclose(e0, e1, atol=1e-9)
    if alpha < 0:
        # broken damage spring: elastic springs unloaded, all stretch in k0
        np.testing.assert_allclose(e0, [0, 0, 3 * xbar], atol=1e-9)
        assert s.energy(e0) < s.energy(np.full(3, xbar))
    else:
        assert len(r0.iterates) == len(r1.iterates)
        for a, b in zip(r0.iterates, r1.iterates):
            np.testing.assert_allclose(a, b, atol=1e-14)


class _QuarticProblem:
    """Dense non-quadratic test problem for Algorithm 2's radius and
    acceptance rules: W(x) = 1/2 x.K x + g4 sum x^4 - c.x, gradient
    sigma = K x + 4 g4 x^3 - c, Hessian B = K + 12 g4 diag(x^2).  No
    projection (G = identity), no history."""

    def __init__(self, K, g4, c):
        self.K, self.g4, self.c = K, g4, c
        self.stress_calls = []

    def stress(self, x, hist):
        self.stress_calls.append(np.array(x, copy=True))
        return self.K @ x + 4.0 * self.g4 * x ** 3 - self.c, np.array(x, copy=True), np.zeros_like(x)

    def gradient(self, sigma):
        return sigma

    def tangent(self, x, v):
        return self.K @ v + 12.0 * self.g4 * x ** 2 * v

    def hessp(self, x, v):
        return self.tangent(x, v)

    dot = staticmethod(_dot)

    @staticmethod
    def norm(a):
        return float(np.sqrt(np.dot(a, a)))


def _radius_trace(monkeypatch, Rmax, seen):
    """Run Algorithm 2 on the quartic problem and check every iteration's
    radius and acceptance against the printed rules; record the branches."""
    import oracle.solver as S

    radii, bounds, grads = [], [], []
    real_cg = S.steihaug_cg

    def spy(hv, g, R, tol, max_iter, dot, restart_thr=0.2):
        p, info = real_cg(hv, g, R, tol, max_iter, dot, restart_thr)
        radii.append(R)
        grads.append(np.array(g, copy=True))
        bounds.append(info["on_boundary"])
        return p, info

    monkeypatch.setattr(S, "steihaug_cg", spy)
    rng = np.random.default_rng(28)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    K = Q @ np.diag([0.2, 0.5, 1.0, 2.0, 3.0, 4.0]) @ Q.T
    prob = _QuarticProblem(K, 0.2, 3.0 * rng.standard_normal(6))
    x0 = 2.0 * rng.standard_normal(6)
    R0, eta_up = 1.0, 0.1
    prm = TRParams(eta_eq=1e-12, eta_nr=1e-12, eta_cg=1e-10, R0=R0, Rmax=Rmax, eta_up=eta_up, max_nr=60,
                   max_cg=50)
    x, _, _, Rend, rep = S.trust_region_step(prob, x0.copy(), None, R0, prm)
    assert rep.converged

    def W(y):
        return 0.5 * y @ K @ y + prob.g4 * np.sum(y ** 4) - prob.c @ y

    def grad(y):
        return K @ y + 4.0 * prob.g4 * y ** 3 - prob.c

    # stress calls: the start, then one trial per Newton iteration
    trials = prob.stress_calls[1:]
    assert len(trials) == len(radii) == rep.nr_iters
    base = x0.copy()
    R = R0
    for it, (Rk, xt, onb, gk) in enumerate(zip(radii, trials, bounds, grads)):
        assert Rk == R, f"iteration {it}: radius {Rk} handed to CG, rules give {R}"
        # the CG of this iteration starts from the last accepted point
        np.testing.assert_allclose(gk, grad(base), rtol=0, atol=1e-13)
        p = xt - base
        Bp = K @ p + 12.0 * prob.g4 * base ** 2 * p
        dm = grad(base) @ p + 0.5 * p @ Bp
        dW = 0.5 * (grad(base) + grad(xt)) @ p
        rho = dW / dm
        if rho < 0.25:
            R = 0.25 * R
            seen.add("shrink" if rho <= eta_up else "accept_and_shrink")
        elif rho > 0.75 and onb:
            seen.add("cap" if 2.0 * R > Rmax else "grow")
            R = min(2.0 * R, Rmax)
        else:
            seen.add("keep_interior" if rho > 0.75 else "keep")
        if rho > eta_up:
            base = xt
            seen.add("accept")
        else:
            seen.add("reject" if rho <= 0.0 else "reject_positive")
    assert Rend == R
    np.testing.assert_allclose(x, base, atol=0)
    # the end point is a stationary point of the quartic energy below the start
    assert np.linalg.norm(grad(x)) < 1e-9
    assert W(x) < W(x0)


def test_trust_region_radius_and_acceptance_rules(monkeypatch):
    """Algorithm 2's printed rules, checked on scripted traces: R is
    quartered when rho < 1/4, doubled (capped at R_max) when rho > 3/4 and the
    step ended on the boundary, kept otherwise, and a step is accepted iff
    rho > eta_up.  The test records the radius and the gradient handed to
    every CG solve and the point of every constitutive evaluation, and
    recomputes rho from Eqs. (18)-(19) with its own quartic energy; the
    traces together exercise every branch (including 0 < rho <= eta_up and
    eta_up < rho < 1/4), so a wrong factor or threshold in the oracle fails."""
    seen = set()
    for Rmax in (3.5, 3.8):
        _radius_trace(monkeypatch, Rmax, seen)
    want = {"shrink", "accept_and_shrink", "grow", "cap", "keep", "keep_interior", "accept", "reject_positive"}
    assert want <= seen, want - seen


def _laminate_parallel_softening(pa, pb, E):
    """Closed form of a 50/50 bilayer normal to z under the mean strain
    eps_xx = E with the other mean components stress-free, layer a damaging
    (pa.kappa0, pa.kappaf), layer b elastic.  Each layer keeps a uniform
    strain: eps_xx = E and a common eps_yy = e (in-plane continuity),
    eps_zz of layer i from sigma_zz = 0, no shear.  The principal strains
    besides E are compressive, so kappa = E in layer a and its damage
    follows from E alone; with w_i = (1 - D_i) / 2 and the plane-stress
    modulus l_i* = 2 l_i m_i / (l_i + 2 m_i), sigma_yy,i = (1 - D_i) (l_i*
    (E + e) + 2 m_i e) and zero mean sigma_yy give
    e = -E sum w_i l_i* / sum w_i (l_i* + 2 m_i), and the mean
    sigma_xx = sum w_i (l_i* (E + e) + 2 m_i E)."""
    (la, ma), (lb, mb) = oracle.lame(pa.E, pa.nu), oracle.lame(pb.E, pb.nu)
    k0, kf = pa.kappa0, pa.kappaf
    Da = 0.0 if E <= k0 else (1.0 if E >= kf else kf * (E - k0) / (E * (kf - k0)))
    w = np.array([0.5 * (1.0 - Da), 0.5])
    lam, mu = np.array([la, lb]), np.array([ma, mb])
    ls = 2.0 * lam * mu / (lam + 2.0 * mu)
    e = -E * np.sum(w * ls) / np.sum(w * (ls + 2.0 * mu))
    return float(np.sum(w * (ls * (E + e) + 2.0 * mu * E))), e


def test_laminate_parallel_loading_softening_curve():
    """Sec. 3.3 loading of a bilayer along its layers through the whole
    softening branch of the damaging layer (D up to 0.99): every increment's
    mean stress equals the closed form, and the damaging layer carries one
    uniform damage value."""
    pa, pb = oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3), oracle.Phase(10.0, 0.2)
    dims = (4, 4, 8)
    pm = laminate(dims, axis=2)
    free = np.array([False, True, True, True, True, True])
    rve = oracle.RVE(pm, [pa, pb], free_mask=free)
    inc = 4.5e-5
    prm = TRParams(eta_eq=1e-10, eta_cg=1e-12, R0=1.0, Rmax=1.0, max_nr=200, max_cg=2000)
    res = load_path(rve, [np.array([inc, 0, 0, 0, 0, 0])] * 20, prm)
    assert all(r.converged for r in res["reports"])
    for n in range(20):
        sxx, e = _laminate_parallel_softening(pa, pb, (n + 1) * inc)
        assert abs(res["mean_stress"][n][0] - sxx) <= 1e-9 * abs(sxx), n
        assert abs(res["mean_strain"][n][1] - e) <= 1e-9 * abs(e), n
    k = res["kappa"][:4]
    assert np.allclose(k, 20 * inc, rtol=1e-12)  # layer a: kappa = E everywhere
    assert np.all(res["kappa"][4:] == 0.0)        # layer b: elastic
