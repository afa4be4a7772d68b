// Pointwise constitutive update (Appendix A), CG vector updates with FP64
// reductions (Algorithm 1), and one-thread scalar controllers for Steihaug
// CG and the trust-region ratio test (Algorithm 2).
#include <cmath>

#include "solver_kernels.cuh"

namespace rve {

constexpr int kVThreads = 256;
constexpr int kVBlocks = 152 * 4;  // persistent-style grid, grid-stride loops

// ------------------------------------------------------------ helpers
template <typename R, int NS>
__device__ __forceinline__ void finish_sums(KSum<R> (&acc)[NS], double* part) {
  __shared__ double red[NS * 32];
  double v[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) v[s] = acc[s].value();
  block_sum<NS>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) part[(long long)blockIdx.x * NS + s] = v[s];
  }
}

// Both roots t- <= t+ of |z + t d|^2 = R^2 given zz, zd, dd (|z| <= R).
__device__ void boundary_roots(double zz, double zd, double dd, double R, double* tm, double* tp) {
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

// ------------------------------------------------------------ CG kernels
template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_init(long long n, const R* __restrict__ g, R* __restrict__ z, R* __restrict__ r, R* __restrict__ d,
              double* __restrict__ part) {
  KSum<R> acc[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const R gi = g[i];
    z[i] = 0;
    r[i] = gi;
    d[i] = -gi;
    acc[0].add(gi * gi);
  }
  finish_sums<R, 1>(acc, part);
}

__global__ void k_cg_init_s(DevScalars* S) {
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

__global__ void k_cg_alpha(DevScalars* S) {
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

template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_update(long long n, R* __restrict__ z, R* __restrict__ r, const R* __restrict__ d,
                const R* __restrict__ Hd, const DevScalars* __restrict__ S, double* __restrict__ part) {
  const int status = S->status;
  KSum<R> acc[3];
  if (status == CG_BOUNDARY || status == CG_NEGCURV) {
    const R tau = (R)S->tau;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      z[i] += tau * d[i];
  } else if (status == CG_RUN) {
    const R a = (R)S->alpha;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      const R zi = z[i] + a * d[i];
      const R ro = r[i];
      const R rn = ro + a * Hd[i];
      z[i] = zi;
      r[i] = rn;
      acc[0].add(rn * rn);
      acc[1].add(rn * ro);
      acc[2].add(zi * zi);
    }
  }
  finish_sums<R, 3>(acc, part);
}

__global__ void k_cg_beta(DevScalars* S) {
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

template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_restart(long long n, R* __restrict__ r, const R* __restrict__ Hz, const R* __restrict__ g,
                 double* __restrict__ part) {
  KSum<R> acc[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const R ri = Hz[i] + g[i];
    r[i] = ri;
    acc[0].add(ri * ri);
  }
  finish_sums<R, 1>(acc, part);
}

__global__ void k_cg_restart_s(DevScalars* S) {
  S->rr = S->rr_new;
  S->beta = 0.0;
  S->restart = 0;
  S->restarts += 1;
}

template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_dupdate(long long n, const R* __restrict__ z, const R* __restrict__ r, R* __restrict__ d,
                 const DevScalars* __restrict__ S, double* __restrict__ part) {
  const R beta = (R)S->beta;
  KSum<R> acc[3];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const R ri = r[i];
    const R di = -ri + beta * d[i];
    d[i] = di;
    acc[0].add(di * di);
    acc[1].add(z[i] * di);
    acc[2].add(ri * di);
  }
  finish_sums<R, 3>(acc, part);
}

// ------------------------------------------------------- constitutive
// sigma_t = (1 - D_t) C : (eps + p), kappa_t = max(kappa_n, kappa(eps + p))
// on damaging phases.  Sums (group T): sig0:p, sig_t:p, p:(1-D0)C:p,
// sig_t:sig_t, p:p, (eps+p):(eps+p).
template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_trial(const GridDesc g, const MatTable<R> mt, const uint8_t* __restrict__ phase, const R* __restrict__ eps,
            const R* __restrict__ p, const R* __restrict__ khist, const R* __restrict__ sig0,
            const R* __restrict__ D0, R* __restrict__ sig_t, R* __restrict__ D_t, R* __restrict__ kap_t,
            double* __restrict__ part) {
  const int nc = g.ncomp, nd = g.ndim;
  const long long nv = g.nvox;
  KSum<R> acc[6];
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    R e[6], pv[6];
    for (int c = 0; c < nc; ++c) {
      pv[c] = p ? p[c * nv + v] : (R)0;
      e[c] = eps[c * nv + v] + pv[c];
    }
    const int ph = phase[v];
    const R lam = mt.lam[ph], mu = mt.mu[ph];
    R D = 0;
    R kap = 0;
    if (mt.damaging[ph]) {
      const R kt = kappa_tension<R>(e, nd);
      const R kh = khist ? khist[v] : (R)0;
      const R k = fmax(kh, kt);
      kap = k;
      D = damage_of<R>(k, mt.kappa0[ph], mt.kappaf[ph]);
    }
    const R keep = (R)1 - D;
    R tr = 0, trp = 0;
    for (int i = 0; i < nd; ++i) { tr += e[i]; trp += pv[i]; }
    const R keep0 = D0 ? (R)1 - D0[v] : (R)1;
    for (int c = 0; c < nc; ++c) {
      const R s = keep * ((R)2 * mu * e[c] + (c < nd ? lam * tr : (R)0));
      sig_t[c * nv + v] = s;
      const R bp = keep0 * ((R)2 * mu * pv[c] + (c < nd ? lam * trp : (R)0));
      if (sig0) acc[0].add(sig0[c * nv + v] * pv[c]);
      acc[1].add(s * pv[c]);
      acc[2].add(pv[c] * bp);
      acc[3].add(s * s);
      acc[4].add(pv[c] * pv[c]);
      acc[5].add(e[c] * e[c]);
    }
    if (D_t) D_t[v] = D;
    if (kap_t) kap_t[v] = kap;
  }
  finish_sums<R, 6>(acc, part);
}

// Algorithm 2 ratio test with the first-order incremental energy.
__global__ void k_tr_decide(DevScalars* S) {
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

template <typename R>
__global__ void __launch_bounds__(kVThreads) k_axpy(long long n, R a, const R* __restrict__ x, R* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

struct Inc6 { double v[6]; };

template <typename R>
__global__ void __launch_bounds__(kVThreads) k_add_uniform(long long nv, int nc, R* __restrict__ eps, const Inc6 dE) {
  const long long n = nv * nc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    eps[i] += (R)dE.v[i / nv];
}

template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_means(long long nv, int nc, const R* __restrict__ sig, const R* __restrict__ eps, double* __restrict__ part) {
  KSum<R> acc[12];
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < nc; ++c) {
      acc[c].add(sig[c * nv + v]);
      acc[6 + c].add(eps[c * nv + v]);
    }
  }
  finish_sums<R, 12>(acc, part);
}

// ------------------------------------------------------------ launchers
#define RVE_TRY(x)                                  \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return e_;               \
  } while (0)

template <typename R>
cudaError_t cg_init(const GridDesc& g, const R* gvec, R* z, R* r, R* d, DevScalars* S, double* part,
                    cudaStream_t st, long long* nl) {
  const long long n = g.nvox * g.ncomp;
  k_cg_init<R><<<kVBlocks, kVThreads, 0, st>>>(n, gvec, z, r, d, part);
  RVE_TRY(cudaGetLastError());
  RVE_TRY(reduce_partials(part, kVBlocks, 1, &S->rr, st, nl));
  k_cg_init_s<<<1, 1, 0, st>>>(S);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t cg_alpha(DevScalars* S, cudaStream_t st, long long* nl) {
  k_cg_alpha<<<1, 1, 0, st>>>(S);
  *nl += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t cg_update(const GridDesc& g, R* z, R* r, const R* d, const R* Hd, DevScalars* S, double* part,
                      cudaStream_t st, long long* nl) {
  const long long n = g.nvox * g.ncomp;
  k_cg_update<R><<<kVBlocks, kVThreads, 0, st>>>(n, z, r, d, Hd, S, part);
  RVE_TRY(cudaGetLastError());
  *nl += 1;
  return reduce_partials(part, kVBlocks, 3, &S->rr_new, st, nl);
}

cudaError_t cg_beta(DevScalars* S, cudaStream_t st, long long* nl) {
  k_cg_beta<<<1, 1, 0, st>>>(S);
  *nl += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t cg_restart(const GridDesc& g, R* r, const R* Hz, const R* gvec, DevScalars* S, double* part,
                       cudaStream_t st, long long* nl) {
  const long long n = g.nvox * g.ncomp;
  k_cg_restart<R><<<kVBlocks, kVThreads, 0, st>>>(n, r, Hz, gvec, part);
  RVE_TRY(cudaGetLastError());
  RVE_TRY(reduce_partials(part, kVBlocks, 1, &S->rr_new, st, nl));
  k_cg_restart_s<<<1, 1, 0, st>>>(S);
  *nl += 2;
  return cudaGetLastError();
}

template <typename R>
cudaError_t cg_dupdate(const GridDesc& g, const R* z, const R* r, R* d, DevScalars* S, double* part,
                       cudaStream_t st, long long* nl) {
  const long long n = g.nvox * g.ncomp;
  k_cg_dupdate<R><<<kVBlocks, kVThreads, 0, st>>>(n, z, r, d, S, part);
  RVE_TRY(cudaGetLastError());
  *nl += 1;
  return reduce_partials(part, kVBlocks, 3, &S->dd, st, nl);
}

template <typename R>
cudaError_t trial_eval(const GridDesc& g, const MatTable<R>& mt, const uint8_t* phase, const R* eps, const R* p,
                       const R* khist, const R* sig0, const R* D0, R* sig_t, R* D_t, R* kap_t,
                       DevScalars* S, double* part, cudaStream_t st, long long* nl) {
  k_trial<R><<<kVBlocks, kVThreads, 0, st>>>(g, mt, phase, eps, p, khist, sig0, D0, sig_t, D_t, kap_t, part);
  RVE_TRY(cudaGetLastError());
  *nl += 1;
  return reduce_partials(part, kVBlocks, 6, &S->sp, st, nl);
}

cudaError_t tr_decide(DevScalars* S, cudaStream_t st, long long* nl) {
  k_tr_decide<<<1, 1, 0, st>>>(S);
  *nl += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t axpy(long long n, R a, const R* x, R* y, cudaStream_t st, long long* nl) {
  k_axpy<R><<<kVBlocks, kVThreads, 0, st>>>(n, a, x, y);
  *nl += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t add_uniform(const GridDesc& g, R* eps, const double dE[6], cudaStream_t st, long long* nl) {
  Inc6 inc;
  for (int c = 0; c < 6; ++c) inc.v[c] = c < g.ncomp ? dE[c] : 0.0;
  k_add_uniform<R><<<kVBlocks, kVThreads, 0, st>>>(g.nvox, g.ncomp, eps, inc);
  *nl += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t field_means(const GridDesc& g, const R* sig, const R* eps, DevScalars* S, double* part,
                        cudaStream_t st, long long* nl) {
  k_means<R><<<kVBlocks, kVThreads, 0, st>>>(g.nvox, g.ncomp, sig, eps, part);
  RVE_TRY(cudaGetLastError());
  *nl += 1;
  return reduce_partials(part, kVBlocks, 12, &S->msig[0], st, nl);
}

#define RVE_INST(R)                                                                                              \
  template cudaError_t cg_init<R>(const GridDesc&, const R*, R*, R*, R*, DevScalars*, double*, cudaStream_t,     \
                                  long long*);                                                                  \
  template cudaError_t cg_update<R>(const GridDesc&, R*, R*, const R*, const R*, DevScalars*, double*,         \
                                    cudaStream_t, long long*);                                                  \
  template cudaError_t cg_restart<R>(const GridDesc&, R*, const R*, const R*, DevScalars*, double*,            \
                                     cudaStream_t, long long*);                                                 \
  template cudaError_t cg_dupdate<R>(const GridDesc&, const R*, const R*, R*, DevScalars*, double*,            \
                                     cudaStream_t, long long*);                                                 \
  template cudaError_t trial_eval<R>(const GridDesc&, const MatTable<R>&, const uint8_t*, const R*, const R*,   \
                                     const R*, const R*, const R*, R*, R*, R*, DevScalars*,                     \
                                     double*, cudaStream_t, long long*);                                        \
  template cudaError_t axpy<R>(long long, R, const R*, R*, cudaStream_t, long long*);                          \
  template cudaError_t add_uniform<R>(const GridDesc&, R*, const double*, cudaStream_t, long long*);           \
  template cudaError_t field_means<R>(const GridDesc&, const R*, const R*, DevScalars*, double*, cudaStream_t, \
                                      long long*);

RVE_INST(float)
RVE_INST(double)

}  // namespace rve
