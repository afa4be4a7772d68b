"""Consistent damage tangent (oracle).  TEST INFRASTRUCTURE ONLY, like the
rest of this package.

The solver's Hessian is the secant (1 - D) C (reading R6).  Appendix A,
after Eq. (A.3), discusses the consistent tangent: it needs d kappa / d eps,
which through the strain eigenvectors looks singular for repeated
eigenvalues, and the paper rewrites eps^(t) = M eps M with the masking
matrix M = sum_i H(eps_i) q_i (x) q_i to obtain it without that singularity.
kappa^2 = sum_i max(eps_i, 0)^2 is a spectral function of eps, so its
derivative is sum_i 2 max(eps_i, 0) q_i (x) q_i = 2 eps^(t) and

    d kappa / d eps = eps^(t) / kappa,

the same as the masked form gives.  With sigma = (1 - D(kappa)) C : eps and
kappa = max(kappa_n, kappa_trial):

    d sigma / d eps : v = (1 - D) C : v - D'(kappa) [kappa_trial > kappa_n]
                          (C : eps) (eps^(t) : v) / kappa,
    D'(kappa) = kappa_f kappa_0 / (kappa^2 (kappa_f - kappa_0)) on (kappa_0, kappa_f)

(bilinear law of Eq. (A.3) as read in R4, zero elsewhere).  The rank-one
term is not symmetric ((C:eps) (x) eps^(t) differs from its transpose unless
C is a multiple of the identity), so Steihaug CG cannot take it as it is;
``sym=True`` applies its symmetric part.

``ConsistentRVE`` is the cell problem with that symmetric consistent tangent
as the Hessian of Algorithm 2 (the secant stays the problem's default).
"""
import numpy as np

from .material import damage_of_kappa, elastic_stress
from .rve import RVE
from .tensors import mandel_to_tensor, tensor_to_mandel


def positive_part(eps):
    """eps^(t) = sum_i max(eps_i, 0) q_i (x) q_i as a Mandel field (Eq. (A.1));
    plane strain adds only a zero eigenvalue."""
    t = mandel_to_tensor(eps)
    w, q = np.linalg.eigh(t)
    wp = np.maximum(w, 0.0)
    tp = np.einsum("...ik,...k,...jk->...ij", q, wp, q)
    return tensor_to_mandel(tp)


def damage_slope(kappa, kappa0, kappaf):
    """D'(kappa) of the bilinear law: kappa_f kappa_0 / (kappa^2 (kappa_f -
    kappa_0)) strictly between kappa_0 and kappa_f, 0 elsewhere."""
    kappa = np.asarray(kappa, dtype=np.float64)
    k0 = np.broadcast_to(kappa0, kappa.shape)
    kf = np.broadcast_to(kappaf, kappa.shape)
    out = np.zeros(kappa.shape)
    soft = (kappa > k0) & (kappa < kf)
    out[soft] = kf[soft] * k0[soft] / (kappa[soft] ** 2 * (kf[soft] - k0[soft]))
    return out


def consistent_tangent_apply(v, eps, kappa_hist, params, sym=False):
    """d sigma / d eps : v at the trial strain eps with committed history
    kappa_hist (the formula above); ``sym`` applies the symmetric part."""
    ep = positive_part(eps)
    kt = np.sqrt(np.sum(ep * ep, axis=0))
    kh = np.zeros(kt.shape) if kappa_hist is None else np.asarray(kappa_hist, dtype=np.float64)
    k = np.where(params.damaging, np.maximum(kh, kt), 0.0)
    D = np.where(params.damaging, damage_of_kappa(k, params.kappa0, params.kappaf), 0.0)
    loading = params.damaging & (kt > kh)
    dp = np.where(loading, damage_slope(k, params.kappa0, params.kappaf), 0.0)
    Cv = elastic_stress(v, params.lam, params.mu)
    Ce = elastic_stress(eps, params.lam, params.mu)
    n = np.where(kt > 0.0, ep / np.where(kt > 0.0, kt, 1.0), 0.0)
    nv = np.sum(n * v, axis=0)
    out = (1.0 - D) * Cv
    if sym:
        cv = np.sum(Ce * v, axis=0)
        return out - 0.5 * dp * (Ce * nv + n * cv)
    return out - dp * Ce * nv


class ConsistentRVE(RVE):
    """The cell problem with the symmetric part of the consistent tangent as
    the Hessian of Algorithm 2 (stress, gradient and energy unchanged)."""

    def stress(self, eps, kappa_hist):
        sigma, D, kappa = super().stress(eps, kappa_hist)
        return sigma, (self.eval_strain(eps), kappa_hist), kappa

    def tangent(self, aux, v):
        e, kh = aux
        return consistent_tangent_apply(v, e, kh, self.params, sym=True)

    def hessp(self, aux, v):
        return self.G(self.tangent(aux, v))
