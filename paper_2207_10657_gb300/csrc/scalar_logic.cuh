// Scalar logic of Steihaug CG (Algorithm 1) and of the trust-region ratio
// test (Algorithm 2), and the pointwise damage law (Appendix A), as device
// functions shared by the single-grid and the batched kernels.
#pragma once

#include "solver_kernels.cuh"

namespace rve {

// Both roots t- <= t+ of |z + t d|^2 = R^2 given zz, zd, dd (|z| <= R).
__device__ __forceinline__ void boundary_roots(double zz, double zd, double dd, double R, double* tm, double* tp) {
  const double a = dd, b = 2.0 * zd, c = zz - R * R;
  const double disc = fmax(b * b - 4.0 * a * c, 0.0);
  const double sq = sqrt(disc);
  const double q = (b != 0.0) ? -0.5 * (b + copysign(sq, b)) : -0.5 * sq;
  if (q == 0.0 || a == 0.0) { *tm = 0.0; *tp = 0.0; return; }
  const double t1 = q / a, t2 = c / q;
  *tm = fmin(t1, t2);
  *tp = fmax(t1, t2);
}

// Tension strain measure kappa = |eps^(t)| = sqrt(sum_i max(eps_i, 0)^2)
// (Eq. (A.1)) from the principal strains.  3D: closed-form eigenvalues of
// a symmetric 3x3 matrix by the trigonometric method (Smith 1961); 2D plane
// strain: the in-plane pair plus the zero out-of-plane eigenvalue.
template <typename R>
__device__ __forceinline__ R kappa_tension(const R* e, int nd) {
  const R is2 = (R)0.70710678118654752440;
  if (nd == 2) {
    const R m = (R)0.5 * (e[0] + e[1]);
    const R h = (R)0.5 * (e[0] - e[1]);
    const R o = e[2] * is2;
    const R r = sqrt(h * h + o * o);
    const R l1 = fmax(m + r, (R)0), l2 = fmax(m - r, (R)0);
    return sqrt(l1 * l1 + l2 * l2);
  }
  const R a00 = e[0], a11 = e[1], a22 = e[2];
  const R a12 = e[3] * is2, a02 = e[4] * is2, a01 = e[5] * is2;
  const R m = (a00 + a11 + a22) / (R)3;
  const R b00 = a00 - m, b11 = a11 - m, b22 = a22 - m;
  const R p2 = (b00 * b00 + b11 * b11 + b22 * b22 + (R)2 * (a01 * a01 + a02 * a02 + a12 * a12)) / (R)6;
  R l1, l2, l3;
  if (p2 <= (R)0) {
    l1 = l2 = l3 = m;
  } else {
    const R p = sqrt(p2);
    const R det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) + a02 * (a01 * a12 - b11 * a02);
    R r = det / ((R)2 * p2 * p);
    r = fmin(fmax(r, (R)-1), (R)1);
    const R phi = acos(r) / (R)3;
    const R twopi3 = (R)2.09439510239319549231;  // 2 pi / 3
    l1 = m + (R)2 * p * cos(phi);
    l3 = m + (R)2 * p * cos(phi + twopi3);
    l2 = (R)3 * m - l1 - l3;
  }
  l1 = fmax(l1, (R)0);
  l2 = fmax(l2, (R)0);
  l3 = fmax(l3, (R)0);
  return sqrt(l1 * l1 + l2 * l2 + l3 * l3);
}

// Bilinear damage (Eq. (A.3)): D = kf (k - k0) / (k (kf - k0)) on (k0, kf).
template <typename R>
__device__ __forceinline__ R damage_of(R k, R k0, R kf) {
  if (k <= k0) return (R)0;
  if (k >= kf) return (R)1;
  return kf * (k - k0) / (k * (kf - k0));
}

__device__ __forceinline__ void cg_init_scalars(DevScalars* S) {
  const double rr = S->rr;
  S->dd = rr;
  S->zd = 0.0;
  S->rd = -rr;
  S->zz = 0.0;
  S->iters = 0;
  S->restarts = 0;
  S->restart = 0;
  S->tau = 0.0;
  S->alpha = 0.0;
  S->beta = 0.0;
  if (!isfinite(rr)) S->status = CG_NONFINITE;
  else if (rr == 0.0 || sqrt(rr) <= S->tol) S->status = CG_ZERO;
  else S->status = CG_RUN;
}

__device__ __forceinline__ void cg_alpha_scalars(DevScalars* S) {
  if (S->status != CG_RUN) return;
  S->iters += 1;
  const double dHd = S->dHd;
  if (!isfinite(dHd)) { S->status = CG_NONFINITE; return; }
  double tm, tp;
  if (dHd <= 0.0) {
    boundary_roots(S->zz, S->zd, S->dd, S->R, &tm, &tp);
    const double qm = tm * S->rd + 0.5 * tm * tm * dHd;
    const double qp = tp * S->rd + 0.5 * tp * tp * dHd;
    S->tau = (qm < qp) ? tm : tp;
    S->status = CG_NEGCURV;
    return;
  }
  const double alpha = S->rr / dHd;
  const double zzp = S->zz + 2.0 * alpha * S->zd + alpha * alpha * S->dd;
  if (sqrt(fmax(zzp, 0.0)) >= S->R) {
    boundary_roots(S->zz, S->zd, S->dd, S->R, &tm, &tp);
    S->tau = tp;
    S->status = CG_BOUNDARY;
    return;
  }
  S->alpha = alpha;
}

__device__ __forceinline__ void cg_beta_scalars(DevScalars* S) {
  if (S->status != CG_RUN) return;
  S->zz = S->zz_new;
  const double rn = S->rr_new;
  if (!isfinite(rn)) { S->status = CG_NONFINITE; return; }
  if (sqrt(rn) <= S->tol) { S->status = CG_CONVERGED; return; }
  if (fabs(S->rnr) / rn > S->thr) {
    S->restart = 1;
  } else {
    S->restart = 0;
    S->beta = rn / S->rr;
    S->rr = rn;
  }
  if (S->iters >= S->max_cg) S->status = CG_MAXITER;
}

__device__ __forceinline__ void cg_restart_scalars(DevScalars* S) {
  S->rr = S->rr_new;
  S->beta = 0.0;
  S->restart = 0;
  S->restarts += 1;
}

__device__ __forceinline__ void tr_decide_scalars(DevScalars* S) {
  const double sp = S->sp, stp = S->stp, pBp = S->pBp;
  const double dm = sp + 0.5 * pBp;       // m(p) - m(0)
  const double dW = 0.5 * (sp + stp);     // Eq. (18)
  const double floor_ = 1e-14 * (fabs(sp) + 0.5 * fabs(pBp));
  double rho = (fabs(dm) <= floor_) ? 1.0 : dW / dm;  // Eq. (19)
  S->nonfinite = !isfinite(rho) || !isfinite(S->sts);
  const int on_b = (S->status == CG_BOUNDARY || S->status == CG_NEGCURV);
  if (rho < 0.25) S->R = 0.25 * S->R;
  else if (rho > 0.75 && on_b) S->R = fmin(2.0 * S->R, S->Rmax);
  S->accept = (rho > S->eta_up) ? 1 : 0;
  S->on_boundary = on_b;
  S->rho = rho;
  S->dm = dm;
  S->dW = dW;
}

}  // namespace rve
