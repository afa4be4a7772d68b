"""Isotropic damage material, per voxel (oracle).

Sec. 3.3 and Appendix A.  Each phase is isotropic linear elastic with
Young's modulus scaled by (1 - D) (Eq. (22)); D is driven by the tension
strain measure kappa = |eps^(t)|, eps^(t) the positive spectral part of the
strain (Eq. (A.1)), and follows the bilinear law of Eq. (A.3).

Readings:

* Elasticity.  lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)); in
  Mandel form C = lambda 1 (x) 1 + 2 mu I.  2D is plane strain
  (eps_33 = 0), so eps^(t) includes the zero third eigenvalue.
* Bilinear law.  Eq. (A.3) writes D = (kappa - kappa0)(1 + alpha)/kappa
  with alpha the relative softening slope.  Parametrised by the strain
  kappa_f at which the stiffness reaches zero, alpha = kappa0 / (kappa_f -
  kappa0), i.e. D = kappa_f (kappa - kappa0) / (kappa (kappa_f - kappa0))
  for kappa0 < kappa < kappa_f, D = 0 below kappa0 and D = 1 from kappa_f on.
* History (loading/unloading, Eq. (A.2)).  kappa = max(kappa_n,
  kappa_trial(eps)) with kappa_n the value committed at the end of the last
  converged load step; trial states inside a step leave no history behind.
* Stress sigma = (1 - D) C : eps (secant).  The Hessian used by the solver is
  the secant (1 - D) C with D frozen at the current state.
"""
from dataclasses import dataclass

import numpy as np

from .tensors import mandel_to_tensor, ndim_of


@dataclass
class Phase:
    E: float
    nu: float
    damaging: bool = False
    kappa0: float = np.inf
    kappaf: float = np.inf


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


class PhaseParams:
    """Per-voxel material parameters gathered from a phase map."""

    def __init__(self, phase_map, phases):
        pm = np.asarray(phase_map)
        lam = np.zeros(pm.shape)
        mu = np.zeros(pm.shape)
        dam = np.zeros(pm.shape, dtype=bool)
        k0 = np.full(pm.shape, np.inf)
        kf = np.full(pm.shape, np.inf)
        for pid, ph in enumerate(phases):
            sel = pm == pid
            l, m = lame(ph.E, ph.nu)
            lam[sel] = l
            mu[sel] = m
            dam[sel] = bool(ph.damaging)
            if ph.damaging:
                k0[sel] = ph.kappa0
                kf[sel] = ph.kappaf
        self.lam, self.mu, self.damaging = lam, mu, dam
        self.kappa0, self.kappaf = k0, kf


def elastic_stress(eps, lam, mu):
    """C : eps in Mandel form: 2 mu eps + lambda tr(eps) on the normals."""
    d = ndim_of(eps.shape[0])
    tr = sum(eps[i] for i in range(d))
    sig = 2.0 * mu * eps
    for i in range(d):
        sig[i] = sig[i] + lam * tr
    return sig


def tangent_apply(v, D, lam, mu):
    """Secant tangent (1 - D) C applied to a Mandel field v (Eq. (13) with
    the secant reading)."""
    return (1.0 - D) * elastic_stress(v, lam, mu)


def principal_strains(eps):
    """Eigenvalues of the strain tensor at every voxel, shape (*grid, 3).
    Plane strain (2D) appends the zero out-of-plane eigenvalue."""
    t = mandel_to_tensor(eps)
    w = np.linalg.eigvalsh(t)
    if t.shape[-1] == 2:
        w = np.concatenate([w, np.zeros(w.shape[:-1] + (1,))], axis=-1)
    return w


def kappa_of_strain(eps):
    """Tension strain measure kappa = |eps^(t)| (Eq. (A.1)): the Frobenius
    norm of the positive spectral part, sqrt(sum_i max(eps_i, 0)^2)."""
    w = principal_strains(eps)
    return np.sqrt(np.sum(np.maximum(w, 0.0) ** 2, axis=-1))


def damage_of_kappa(kappa, kappa0, kappaf):
    """Bilinear damage variable (Eq. (A.3), reading above)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    kappa0 = np.broadcast_to(kappa0, kappa.shape)
    kappaf = np.broadcast_to(kappaf, kappa.shape)
    out = np.zeros(kappa.shape)
    soft = (kappa > kappa0) & (kappa < kappaf)
    out[soft] = kappaf[soft] * (kappa[soft] - kappa0[soft]) / (
        kappa[soft] * (kappaf[soft] - kappa0[soft]))
    out[kappa >= kappaf] = 1.0
    return out


def evaluate(eps, params, kappa_hist=None):
    """Stress, damage and kappa of a trial strain field.

    Returns (sigma, D, kappa) with kappa = max(kappa_hist, kappa_trial)
    on damaging voxels (0 elsewhere)."""
    kt = kappa_of_strain(eps)
    kh = np.zeros(kt.shape) if kappa_hist is None else np.asarray(kappa_hist, np.float64)
    kappa = np.where(params.damaging, np.maximum(kh, kt), 0.0)
    D = np.where(params.damaging, damage_of_kappa(kappa, params.kappa0, params.kappaf), 0.0)
    sigma = (1.0 - D) * elastic_stress(eps, params.lam, params.mu)
    return sigma, D, kappa
