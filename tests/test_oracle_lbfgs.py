"""Pins of the oracle's L-BFGS solver with the first-order approximate
energy in its line search (CPU only): the two-loop recursion against the
explicit BFGS inverse-Hessian recursion, a dense quadratic against a linear
solve, elastic cells against the assembled periodic FE solution, the
approximate-energy line search against the exact-energy one on quadratic
energies (where Eq. (18) is exact), and the trust-region solver's
equilibrium at the onset of damage."""
import numpy as np
import pytest

import oracle
from oracle.lbfgs import LBFGSParams, lbfgs_step, load_path_lbfgs, two_loop
from oracle.solver import TRParams, load_path
from synth import circular_inclusion, random_spheres
from tests import fe_bruteforce as fe

STIFF = oracle.Phase(10.0, 0.2)


def test_two_loop_equals_dense_bfgs_recursion():
    """H g from the two-loop recursion equals the product with the matrix of
    the BFGS inverse update H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T
    applied to gamma I, oldest pair first (N&W Eq. (6.17))."""
    rng = np.random.default_rng(0)
    n = 12
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    S = [rng.standard_normal(n) for _ in range(5)]
    Y = [A @ s for s in S]
    rho = [1.0 / float(s @ y) for s, y in zip(S, Y)]
    gamma = 0.37
    H = gamma * np.eye(n)
    for s, y, r in zip(S, Y, rho):
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    g = rng.standard_normal(n)
    np.testing.assert_allclose(two_loop(g, S, Y, rho, gamma, np.dot), H @ g, rtol=1e-12, atol=1e-14)


class _Quadratic:
    """W(x) = 1/2 x^T A x - b^T x on R^n; 'stress' is its gradient and the
    projection is the identity."""

    def __init__(self, A, b):
        self.A, self.b = A, b

    def stress(self, x, hist):
        return self.A @ x - self.b, None, np.zeros(1)

    def gradient(self, s):
        return s

    @staticmethod
    def dot(a, b):
        return float(np.dot(a, b))

    def norm(self, a):
        return float(np.linalg.norm(a))

    def energy(self, x, hist):
        return 0.5 * float(x @ self.A @ x) - float(self.b @ x)


@pytest.mark.parametrize("m", [1, 3, 8])
def test_dense_quadratic_reaches_linear_solve(m):
    rng = np.random.default_rng(1)
    n = 30
    M = rng.standard_normal((n, n))
    A = M @ M.T + 0.5 * np.eye(n)
    b = rng.standard_normal(n)
    prob = _Quadratic(A, b)
    # g = sigma here, so |g|/|sigma| = 1 and the run ends at the iteration
    # cap (eta_eq < 0); the iterate is compared with the solution
    x, _, _, rep = lbfgs_step(prob, np.zeros(n), None,
                              LBFGSParams(eta_eq=-1.0, m=m, max_iter=400, gamma0=1.0 / np.linalg.norm(A, 2)))
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("dims,free", [
    ((8, 8), None),
    ((8, 8), np.array([False, True, True])),
    ((4, 4, 4), None),
    ((4, 4, 4), np.array([True, True, False, True, True, True])),
])
def test_elastic_lbfgs_matches_bruteforce_fe(dims, free):
    if len(dims) == 2:
        pm = circular_inclusion(dims, 0.3)
        E = np.array([1e-3, 0.0, 0.0]) if free is not None else np.array([1e-3, -2e-4, 3e-4])
    else:
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        pm[1:3, 1:3, 0:2] = 1
        pm[3, 0, 3] = 1
        E = np.array([0, 0, 1e-3, 0, 0, 0.0]) if free is not None else np.array([1e-3, -2e-4, 3e-4, 1e-4, 0, 2e-4])
    rve = oracle.RVE(pm, [oracle.Phase(1.0, 0.3), STIFF], free_mask=free)
    res = load_path_lbfgs(rve, [E], LBFGSParams(eta_eq=1e-13, m=8, max_iter=2000))
    assert res["reports"][0].converged
    ref, _ = fe.solve_elastic(dims, rve.params.lam, rve.params.mu, E * (1 - (free if free is not None else 0)), free)
    assert np.max(np.abs(res["eps"] - ref)) / np.max(np.abs(ref)) < 1e-9


def test_approximate_energy_line_search_equals_exact_on_quadratic():
    """Eq. (18) is exact for a quadratic energy (the trapezoidal rule on a
    linear gradient), so the line search takes the same step lengths and
    the iterates coincide with those of the exact-energy search."""
    dims = (12, 10)
    pm = circular_inclusion(dims, 0.3)
    rve = oracle.RVE(pm, [oracle.Phase(1.0, 0.3), STIFF])
    lam, mu = rve.params.lam, rve.params.mu

    def W(eps, hist):
        tr = eps[0] + eps[1]
        return float(np.sum(0.5 * lam * tr * tr + mu * np.sum(eps * eps, axis=0)))

    E = np.array([1e-3, -2e-4, 3e-4])
    eps0 = np.broadcast_to(E.reshape(3, 1, 1), (3,) + pm.shape).copy()
    prm = dict(eta_eq=1e-6, m=4, max_iter=300)
    xa, _, _, ra = lbfgs_step(rve, eps0, None, LBFGSParams(**prm), record_iterates=True)
    xb, _, _, rb = lbfgs_step(rve, eps0, None, LBFGSParams(energy=W, **prm), record_iterates=True)
    assert ra.converged and rb.converged
    assert ra.backtracks > 0  # the line search is exercised
    assert ra.alphas == rb.alphas
    for a, b in zip(ra.iterates, rb.iterates):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.max(np.abs(b)))
    # Near equilibrium the exact difference W(eps + s) - W(eps) falls below
    # the rounding of W itself and the exact-energy search stalls, while
    # Eq. (18) (sums of stress times step) keeps its accuracy: the reason
    # the paper gives for the approximate energy.
    tight = dict(eta_eq=1e-12, m=4, max_iter=300)
    _, _, _, ra = lbfgs_step(rve, eps0, None, LBFGSParams(**tight))
    _, _, _, rb = lbfgs_step(rve, eps0, None, LBFGSParams(energy=W, **tight))
    assert ra.converged and not rb.converged


def test_lbfgs_reaches_trust_region_equilibrium_at_damage_onset():
    """16x12x10 spheres in a damaging matrix, uniaxial eps_zz (the rest
    free), an elastic increment and the onset of damage: the L-BFGS and the
    trust-region Newton-CG solvers reach the same equilibrium."""
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    phases = [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3), STIFF]
    free = np.array([True, True, False, True, True, True])
    # both increments damage the matrix; larger second increments reach
    # states with several equilibria, where the two solvers may settle in
    # different ones
    incs = [np.array([0, 0, 5e-5, 0, 0, 0]), np.array([0, 0, 2e-5, 0, 0, 0])]
    r_lb = load_path_lbfgs(oracle.RVE(pm, phases, free_mask=free), incs, LBFGSParams(eta_eq=1e-9, m=8, max_iter=3000))
    R0 = 10 * np.sqrt(pm.size) * 5e-5
    r_tr = load_path(oracle.RVE(pm, phases, free_mask=free), incs,
                     TRParams(eta_eq=1e-9, eta_cg=1e-3, R0=R0, Rmax=R0, max_nr=500))
    assert all(r.converged for r in r_lb["reports"]) and all(r.converged for r in r_tr["reports"])
    assert r_lb["kappa"].max() > 1e-4  # damage started
    np.testing.assert_allclose(r_lb["mean_stress"], r_tr["mean_stress"], rtol=1e-6, atol=1e-12)
    assert np.linalg.norm(r_lb["eps"] - r_tr["eps"]) <= 1e-6 * np.linalg.norm(r_tr["eps"])
