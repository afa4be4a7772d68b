"""Steihaug CG (Algorithm 1) and trust-region Newton-CG with the first-order
incremental approximate energy (Algorithm 2), oracle versions.

Both are generic over a *problem* object providing

* ``stress(eps, hist) -> (sigma, aux, kappa)``  constitutive evaluation,
* ``gradient(sigma)``                          G : sigma,
* ``hessp(aux, v)``                            G : (B(aux) : v),
* ``tangent(aux, v)``                          B(aux) : v (no projection),
* ``dot(a, b)``, ``norm(a)``,
* optionally ``energy(eps, hist)`` for the standard (exact-ratio) variant.

Readings of the printed algorithms (they are partly garbled):

* Algorithm 1 uses one symbol for the CG iterate and the residual.  It is
  read as Steihaug's method as given in Nocedal & Wright (Alg. 7.2): iterate
  z0 = 0, residual r0 = g (the model gradient at 0; g = -b = G : sigma),
  direction d0 = -r0.  Exits: d^T H d <= 0 (negative curvature: the root tau
  of |z + tau d| = R with the lower model value), |z + alpha d| >= R
  (boundary: the non-negative root), |r| <= tol (converged), max_iter.
* Restart (Eq. (20), Powell): if |r_{j+1} . r_j| / |r_{j+1}|^2 > 0.2, the
  residual is recomputed from the iterate, r_{j+1} = H z_{j+1} + g, and
  beta = 0 (steepest descent).  The absolute value and |r_{j+1}|^2 follow
  Eq. (20); Algorithm 1 omits the absolute value.
* CG tolerance: relative, |r| <= eta_CG |g| (inexact Newton).
* Algorithm 2: Delta m = sigma : p + 1/2 p : B : p (= m(p) - m(0)) and
  Delta W = 1/2 (sigma + sigma_trial) : p (Eq. (18)), rho = DW / Dm
  (Eq. (19)); shrink R by 1/4 if rho < 1/4, double it (capped at R_max) if
  rho > 3/4 and the step ended on the boundary, accept if rho > eta_up.
  "|d_eps| = R" is the CG's on-boundary flag.  If |Dm| is at the rounding
  floor (<= 1e-14 (|sigma:p| + 1/2 |p:B:p|)) the step is taken as rho = 1;
  the standard variant (exact W, Eq. (15)) also takes rho = 1 once |Dm| is
  below 1e-14 |W|, where W(eps + p) - W(eps) is pure cancellation.
* Convergence after an accepted interior step: relative residual
  |G : sigma| / |sigma| <= eta_eq, or |d_eps| / |eps| <= eta_NR.
* R is initialised once and carries over between load steps (Algorithm 2
  sets it before the load loop).
* History: kappa is committed (kappa_n <- kappa) only when a load step has
  converged; trial states use max(kappa_n, kappa_trial).
"""
from dataclasses import dataclass, field
import math

import numpy as np


def _boundary_taus(zz, zd, dd, R):
    """Both roots tau- <= tau+ of |z + tau d|^2 = R^2 (needs |z| <= R)."""
    a = dd
    b = 2.0 * zd
    c = zz - R * R
    disc = max(b * b - 4.0 * a * c, 0.0)
    sq = math.sqrt(disc)
    # stable pair of roots
    q = -0.5 * (b + math.copysign(sq, b)) if b != 0.0 else -0.5 * sq
    if q == 0.0:
        return 0.0, 0.0
    t1 = q / a
    t2 = c / q
    return min(t1, t2), max(t1, t2)


def steihaug_cg(hv, g, R, tol, max_iter, dot, restart_thr=0.2):
    """Minimise m(p) = g.p + 1/2 p.H p over |p| <= R (Algorithm 1 reading).

    ``tol`` is the absolute residual tolerance.  Returns (p, info) where info
    holds ``iters``, ``hv`` (products used), ``restarts``, ``on_boundary``,
    ``reason`` and ``pHp`` (p.Hp is not returned; callers recompute)."""
    info = dict(iters=0, hv=0, restarts=0, on_boundary=False, reason="")
    z = np.zeros_like(g)
    r = g.copy()
    d = -r
    rr = dot(r, r)
    if math.sqrt(rr) <= tol or rr == 0.0:
        info["reason"] = "zero_rhs"
        return z, info
    for j in range(max_iter):
        Hd = hv(d)
        info["hv"] += 1
        info["iters"] = j + 1
        dHd = dot(d, Hd)
        zz, zd, dd = dot(z, z), dot(z, d), dot(d, d)
        if dHd <= 0.0:
            tm, tp = _boundary_taus(zz, zd, dd, R)
            rd = dot(r, d)
            q = lambda t: t * rd + 0.5 * t * t * dHd  # noqa: E731
            tau = tm if q(tm) < q(tp) else tp
            info.update(on_boundary=True, reason="negative_curvature")
            return z + tau * d, info
        alpha = rr / dHd
        z_new = z + alpha * d
        if math.sqrt(dot(z_new, z_new)) >= R:
            _, tp = _boundary_taus(zz, zd, dd, R)
            info.update(on_boundary=True, reason="boundary")
            return z + tp * d, info
        r_new = r + alpha * Hd
        rr_new = dot(r_new, r_new)
        if math.sqrt(rr_new) <= tol:
            info["reason"] = "converged"
            return z_new, info
        if abs(dot(r_new, r)) / rr_new > restart_thr:
            r_new = hv(z_new) + g
            info["hv"] += 1
            info["restarts"] += 1
            rr_new = dot(r_new, r_new)
            beta = 0.0
        else:
            beta = rr_new / rr
        d = -r_new + beta * d
        z, r, rr = z_new, r_new, rr_new
    info["reason"] = "max_iter"
    return z, info


@dataclass
class TRParams:
    eta_eq: float = 1e-6      # relative residual |G sigma| / |sigma|
    eta_nr: float = 0.0       # |d_eps| / |eps| (0 disables)
    eta_cg: float = 1e-2      # relative CG tolerance
    eta_up: float = 0.1       # acceptance threshold on rho
    R0: float = 1.0
    Rmax: float = 1.0
    max_nr: int = 50
    max_cg: int = 1000
    restart_thr: float = 0.2
    exact_rho: bool = False   # standard TR (needs problem.energy)


@dataclass
class StepReport:
    nr_iters: int = 0
    cg_iters: int = 0
    hv: int = 0
    restarts: int = 0
    rejected: int = 0
    boundary_hits: int = 0
    converged: bool = False
    rel_residual: float = float("nan")
    R: float = float("nan")
    rhos: list = field(default_factory=list)
    iterates: list = field(default_factory=list)


def _rel_residual(prob, sigma):
    gs = prob.gradient(sigma)
    ns = prob.norm(sigma)
    return gs, (prob.norm(gs) / ns if ns > 0.0 else 0.0)


def trust_region_step(prob, eps, hist, R, prm, record_iterates=False):
    """One load step of Algorithm 2 from the already incremented strain.

    ``eps`` is the strain after adding the macroscopic increment (and the
    warm-start field, if any); ``hist`` the committed history.  Returns
    (eps, sigma, kappa, R, report); the caller commits the history."""
    rep = StepReport()
    sigma, aux, kappa = prob.stress(eps, hist)
    g, rel = _rel_residual(prob, sigma)
    if rel <= prm.eta_eq:
        rep.converged, rep.rel_residual, rep.R = True, rel, R
        return eps, sigma, kappa, R, rep
    for _ in range(prm.max_nr):
        rep.nr_iters += 1
        gnorm = prob.norm(g)
        p, info = steihaug_cg(lambda v: prob.hessp(aux, v), g, R,
                              prm.eta_cg * gnorm, prm.max_cg, prob.dot,
                              prm.restart_thr)
        rep.cg_iters += info["iters"]
        rep.hv += info["hv"]
        rep.restarts += info["restarts"]
        on_b = info["on_boundary"]
        rep.boundary_hits += int(on_b)
        s_p = prob.dot(sigma, p)
        pBp = prob.dot(p, prob.tangent(aux, p))
        dm = s_p + 0.5 * pBp
        sig_t, aux_t, kappa_t = prob.stress(eps + p, hist)
        floor = 1e-14 * (abs(s_p) + 0.5 * abs(pBp))
        if prm.exact_rho:
            W0 = prob.energy(eps, hist)
            dW = prob.energy(eps + p, hist) - W0
            # the exact difference cancels below ~1e-14 |W|
            floor = max(floor, 1e-14 * abs(W0))
        else:
            dW = 0.5 * (s_p + prob.dot(sig_t, p))
        if abs(dm) <= floor:
            rho = 1.0
        else:
            rho = dW / dm
        rep.rhos.append(rho)
        if rho < 0.25:
            R = 0.25 * R
        elif rho > 0.75 and on_b:
            R = min(2.0 * R, prm.Rmax)
        if rho > prm.eta_up:
            eps = eps + p
            pn, en = prob.norm(p), prob.norm(eps)
            r_nr = pn / en if en > 0.0 else 0.0
            sigma, aux, kappa = sig_t, aux_t, kappa_t
            g, rel = _rel_residual(prob, sigma)
            if record_iterates:
                rep.iterates.append(np.array(eps, copy=True))
            if not on_b and (rel <= prm.eta_eq or (prm.eta_nr > 0.0 and r_nr <= prm.eta_nr)):
                rep.converged = True
                break
        else:
            rep.rejected += 1
    rep.rel_residual = _rel_residual(prob, sigma)[1]
    rep.R = R
    return eps, sigma, kappa, R, rep


def load_path(prob, increments, prm, eps0=None, hist0=None, warm_start=None,
              on_step=None, eigenstrains=None):
    """Ramp the macroscopic strain through ``increments`` (Mandel vectors
    applied uniformly, Algorithm 2's load loop) and return per-step results.

    ``eigenstrains`` (optional, one entry per increment) holds the per-phase
    eigenstrain table in force during that load step (Algorithm 2 adds it to
    the strain before every constitutive evaluation; None keeps the
    previous one).

    ``warm_start(step, eps) -> field or None`` may add a compatible initial
    fluctuation increment.  Returns dict with mean stresses, mean strains,
    reports and the final fields."""
    ncomp = prob.ncomp
    eps = np.zeros((ncomp,) + prob.shape) if eps0 is None else np.array(eps0, copy=True)
    hist = np.zeros(prob.shape) if hist0 is None else np.array(hist0, copy=True)
    R = prm.R0
    out = dict(mean_stress=[], mean_strain=[], reports=[], kappa=None, eps=None, sigma=None)
    for n, dE in enumerate(increments):
        eps = eps + np.asarray(dE, dtype=np.float64).reshape((ncomp,) + (1,) * prob.ndim)
        if eigenstrains is not None and eigenstrains[n] is not None:
            prob.set_eigenstrain(eigenstrains[n])
        if warm_start is not None:
            w = warm_start(n, eps)
            if w is not None:
                eps = eps + w
        eps, sigma, kappa, R, rep = trust_region_step(prob, eps, hist, R, prm)
        hist = np.maximum(hist, kappa)
        out["mean_stress"].append(prob.mean(sigma))
        out["mean_strain"].append(prob.mean(eps))
        out["reports"].append(rep)
        if on_step is not None:
            on_step(n, eps, sigma, hist, rep)
    out["kappa"], out["eps"], out["sigma"] = hist, eps, sigma
    out["mean_stress"] = np.asarray(out["mean_stress"])
    out["mean_strain"] = np.asarray(out["mean_strain"])
    return out
