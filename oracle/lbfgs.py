"""L-BFGS on the incremental energy with the first-order approximate energy
in the line search (oracle).  TEST INFRASTRUCTURE ONLY, like the rest of
this package.

The paper (Sec. 2.2.1, after Eq. (20)) notes that quasi-Newton methods such
as L-BFGS need the objective itself, and that the first-order incremental
energy of Eq. (18) can stand in for it, but gives no algorithm.  Reading
(each step below follows Nocedal & Wright, Numerical Optimization, 2nd ed.,
the reference the paper cites for its solvers):

* L-BFGS (N&W Alg. 7.5) on the compatible strain fields: the gradient is
  g = G : sigma (Eqs. (12), (5)), the search direction p = -H g with H the
  L-BFGS inverse Hessian from the newest m pairs (s_i, y_i), applied by the
  two-loop recursion (N&W Alg. 7.4).  s = eps_new - eps, y = g_new - g; both
  compatible, so p is compatible.
* Initial matrix H0 = gamma I with gamma = s.y / y.y of the newest pair
  (N&W Eq. (7.20)); before the first pair gamma0 = 1 / max over phases of
  (3 lambda + 2 mu), the largest eigenvalue of C, so that the first step
  does not overshoot.
* Line search: backtracking from alpha = 1, halving, until the Armijo
  condition holds with the energy change replaced by Eq. (18):
  DW(alpha) = 1/2 (sigma(eps) + sigma(eps + alpha p)) : alpha p
            <= c1 alpha sigma(eps) : p,   c1 = 1e-4
  (sigma : p = g : p for a compatible p).  At most ``max_backtrack``
  halvings; the step fails after that.
* A pair is stored only if s.y > 1e-12 |s| |y| (positive curvature along s;
  the pair is skipped where softening makes it fail, N&W Sec. 7.2).
* Convergence: |G : sigma| / |sigma| <= eta_eq, tested at the start of the
  load step and after every accepted step; ``max_iter`` iterations.
* Damage history as in the trust-region solver: trial states use
  max(kappa_n, kappa_trial); the caller commits kappa after convergence.
"""
from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class LBFGSParams:
    eta_eq: float = 1e-6
    m: int = 5
    max_iter: int = 500
    c1: float = 1e-4
    max_backtrack: int = 40
    gamma0: float = None      # default: 1 / max_phase(3 lambda + 2 mu)
    energy: object = None     # exact energy W(eps, hist) instead of Eq. (18) (tests)


@dataclass
class LBFGSReport:
    iters: int = 0
    trials: int = 0
    backtracks: int = 0
    skipped_pairs: int = 0
    converged: bool = False
    rel_residual: float = float("nan")
    alphas: list = field(default_factory=list)
    iterates: list = field(default_factory=list)


def two_loop(g, S, Y, rho, gamma, dot):
    """r = H g by the two-loop recursion (N&W Alg. 7.4); S, Y, rho ordered
    oldest first."""
    q = g.copy()
    k = len(S)
    a = [0.0] * k
    for i in range(k - 1, -1, -1):
        a[i] = rho[i] * dot(S[i], q)
        q = q - a[i] * Y[i]
    r = gamma * q
    for i in range(k):
        b = rho[i] * dot(Y[i], r)
        r = r + S[i] * (a[i] - b)
    return r


def default_gamma0(prob):
    lam, mu = prob.params.lam, prob.params.mu
    return 1.0 / float(np.max(3.0 * lam + 2.0 * mu))


def lbfgs_step(prob, eps, hist, prm, record_iterates=False):
    """One load step by L-BFGS from the already incremented strain ``eps``
    (Algorithm 2's load loop with the inner Newton-CG replaced).  Returns
    (eps, sigma, kappa, report); the caller commits the history."""
    rep = LBFGSReport()
    dot = prob.dot
    gamma0 = prm.gamma0 if prm.gamma0 is not None else default_gamma0(prob)
    sigma, _, kappa = prob.stress(eps, hist)
    g = prob.gradient(sigma)
    S, Y, rho = [], [], []
    gamma = gamma0

    def rel_of(g, sigma):
        ns = prob.norm(sigma)
        return prob.norm(g) / ns if ns > 0.0 else 0.0

    rel = rel_of(g, sigma)
    while rel > prm.eta_eq and rep.iters < prm.max_iter:
        rep.iters += 1
        p = -two_loop(g, S, Y, rho, gamma, dot)
        slope = dot(sigma, p)  # = g . p for a compatible p
        if not slope < 0.0:
            # not a descent direction (rounding at the floor): restart from
            # the scaled gradient
            S, Y, rho = [], [], []
            gamma = gamma0
            p = -gamma * g
            slope = dot(sigma, p)
        alpha = 1.0
        ok = False
        for _ in range(prm.max_backtrack + 1):
            rep.trials += 1
            s = alpha * p
            sig_t, _, kap_t = prob.stress(eps + s, hist)
            if prm.energy is not None:
                dW = prm.energy(eps + s, hist) - prm.energy(eps, hist)
            else:
                dW = 0.5 * (dot(sigma, s) + dot(sig_t, s))
            if dW <= prm.c1 * alpha * slope:
                ok = True
                break
            alpha *= 0.5
            rep.backtracks += 1
        if not ok:
            break
        rep.alphas.append(alpha)
        eps = eps + s
        g_new = prob.gradient(sig_t)
        y = g_new - g
        sy = dot(s, y)
        if sy > 1e-12 * prob.norm(s) * prob.norm(y):
            S.append(s)
            Y.append(y)
            rho.append(1.0 / sy)
            if len(S) > prm.m:
                S.pop(0)
                Y.pop(0)
                rho.pop(0)
            gamma = sy / dot(y, y)
        else:
            rep.skipped_pairs += 1
        sigma, kappa, g = sig_t, kap_t, g_new
        if record_iterates:
            rep.iterates.append(np.array(eps, copy=True))
        rel = rel_of(g, sigma)
    rep.converged = rel <= prm.eta_eq
    rep.rel_residual = rel
    return eps, sigma, kappa, rep


def load_path_lbfgs(prob, increments, prm, eigenstrains=None):
    """Algorithm 2's load loop with every load step solved by lbfgs_step."""
    ncomp = prob.ncomp
    eps = np.zeros((ncomp,) + prob.shape)
    hist = np.zeros(prob.shape)
    out = dict(mean_stress=[], mean_strain=[], reports=[])
    sigma = None
    for n, dE in enumerate(increments):
        eps = eps + np.asarray(dE, dtype=np.float64).reshape((ncomp,) + (1,) * prob.ndim)
        if eigenstrains is not None and eigenstrains[n] is not None:
            prob.set_eigenstrain(eigenstrains[n])
        eps, sigma, kappa, rep = lbfgs_step(prob, eps, hist, prm)
        hist = np.maximum(hist, kappa)
        out["mean_stress"].append(prob.mean(sigma))
        out["mean_strain"].append(prob.mean(eps))
        out["reports"].append(rep)
    out["kappa"], out["eps"], out["sigma"] = hist, eps, sigma
    out["mean_stress"] = np.asarray(out["mean_stress"])
    out["mean_strain"] = np.asarray(out["mean_strain"])
    return out
