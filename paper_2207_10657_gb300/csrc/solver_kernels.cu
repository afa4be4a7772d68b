// Pointwise constitutive update (Appendix A), CG vector updates with FP64
// reductions (Algorithm 1), and one-thread scalar controllers for Steihaug
// CG and the trust-region ratio test (Algorithm 2).
#include <cmath>

#include "scalar_logic.cuh"
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

// ------------------------------------------------------------ CG kernels
// Vector kernels stream 4-wide vectors (n is a multiple of 4: every grid
// dimension is even), two per thread per iteration, to keep enough bytes
// in flight per SM.
template <typename R> struct V4T;
template <> struct V4T<float> { using T = float4; };
template <> struct V4T<double> { using T = double4_32a; };
template <typename R> using V4 = typename V4T<R>::T;
template <typename R> __device__ __forceinline__ R& el(V4<R>& v, int i) { return (&v.x)[i]; }
template <typename R> __device__ __forceinline__ R elc(const V4<R>& v, int i) { return (&v.x)[i]; }
template <typename R> __device__ __forceinline__ V4<R> ld4(const R* p, long long i) {
  return *reinterpret_cast<const V4<R>*>(p + 4 * i);
}
template <typename R> __device__ __forceinline__ void st4(R* p, long long i, const V4<R>& v) {
  *reinterpret_cast<V4<R>*>(p + 4 * i) = v;
}
template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_init(long long n, const R* __restrict__ g, R* __restrict__ z, R* __restrict__ r, R* __restrict__ d,
              double* __restrict__ part) {
  KSum<R> acc[1];
  const long long n4 = n / 4;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const V4<R> gi = ld4(g, i);
    V4<R> zero, neg;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el<R>(zero, e) = 0;
      el<R>(neg, e) = -elc<R>(gi, e);
      acc[0].add(elc<R>(gi, e) * elc<R>(gi, e));
    }
    st4(z, i, zero);
    st4(r, i, gi);
    st4(d, i, neg);
  }
  finish_sums<R, 1>(acc, part);
}

__global__ void k_cg_init_s(DevScalars* S) { cg_init_scalars(S); }

__global__ void k_cg_alpha(DevScalars* S) { cg_alpha_scalars(S); }

template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_update(long long n, R* __restrict__ z, R* __restrict__ r, const R* __restrict__ d,
                const R* __restrict__ Hd, const DevScalars* __restrict__ S, double* __restrict__ part) {
  const int status = S->status;
  KSum<R> acc[3];
  const long long n4 = n / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (status == CG_BOUNDARY || status == CG_NEGCURV) {
    const R tau = (R)S->tau;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      V4<R> zi = ld4(z, i);
      const V4<R> di = ld4(d, i);
#pragma unroll
      for (int e = 0; e < 4; ++e) el<R>(zi, e) += tau * elc<R>(di, e);
      st4(z, i, zi);
    }
  } else if (status == CG_RUN) {
    const R a = (R)S->alpha;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < n4; i += 2 * stride) {
      V4<R> zi[2], ro[2], di[2], hi[2];
      const bool two = i + stride < n4;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 0 || two) {
          zi[u] = ld4(z, i + u * stride);
          ro[u] = ld4(r, i + u * stride);
          di[u] = ld4(d, i + u * stride);
          hi[u] = ld4(Hd, i + u * stride);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 0 || two) {
          V4<R> zn, rn;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const R zz = el<R>(zi[u], e) + a * el<R>(di[u], e);
            const R ov = el<R>(ro[u], e);
            const R nv = ov + a * el<R>(hi[u], e);
            el<R>(zn, e) = zz;
            el<R>(rn, e) = nv;
            acc[0].add(nv * nv);
            acc[1].add(nv * ov);
            acc[2].add(zz * zz);
          }
          st4(z, i + u * stride, zn);
          st4(r, i + u * stride, rn);
        }
      }
    }
  }
  finish_sums<R, 3>(acc, part);
}

__global__ void k_cg_beta(DevScalars* S) { cg_beta_scalars(S); }

template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_restart(long long n, R* __restrict__ r, const R* __restrict__ Hz, const R* __restrict__ g,
                 double* __restrict__ part) {
  KSum<R> acc[1];
  const long long n4 = n / 4;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const V4<R> h = ld4(Hz, i), gg = ld4(g, i);
    V4<R> ri;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el<R>(ri, e) = elc<R>(h, e) + elc<R>(gg, e);
      acc[0].add(el<R>(ri, e) * el<R>(ri, e));
    }
    st4(r, i, ri);
  }
  finish_sums<R, 1>(acc, part);
}

__global__ void k_cg_restart_s(DevScalars* S) { cg_restart_scalars(S); }

template <typename R>
__global__ void __launch_bounds__(kVThreads)
    k_cg_dupdate(long long n, const R* __restrict__ z, const R* __restrict__ r, R* __restrict__ d,
                 DevScalars* __restrict__ S, double* __restrict__ part) {
  // Algorithm 1 continues only while running without a pending restart: a
  // device-side loop reaches this kernel after every iteration, the host
  // loop only in that case.  (Skipped, the sums of group D go stale; they
  // are recomputed by the update after the restart and unused on exit.)
  // Every block takes the same decision: nothing in the launch writes status
  // or restart.
  if (S->status != CG_RUN || S->restart) return;
  const R beta = (R)S->beta;
  KSum<R> acc[3];
  const long long n4 = n / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += 2 * stride) {
    V4<R> zi[2], ri[2], di[2];
    const bool two = i + stride < n4;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 0 || two) {
        zi[u] = ld4(z, i + u * stride);
        ri[u] = ld4(r, i + u * stride);
        di[u] = ld4(d, i + u * stride);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 0 || two) {
        V4<R> dn;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const R rv = el<R>(ri[u], e);
          const R dv = -rv + beta * el<R>(di[u], e);
          el<R>(dn, e) = dv;
          acc[0].add(dv * dv);
          acc[1].add(el<R>(zi[u], e) * dv);
          acc[2].add(rv * dv);
        }
        st4(d, i + u * stride, dn);
      }
    }
  }
  finish_sums<R, 3>(acc, part);
  // group D (dd, zd, rd) summed by the last block to finish
  __shared__ double rsh[3 * 32];
  reduce_in_last_block<3>(part, gridDim.x, &S->dd, &S->red_cnt[1], rsh);
}

// ------------------------------------------------------- constitutive
// With e = eps + p + eps_eig(phase): sigma_t = (1 - D_t) C : e,
// kappa_t = max(kappa_n, kappa(e)) on damaging phases.  Sums (group T):
// sig0:p, sig_t:p, p:B0:p, sig_t:sig_t, p:p, (eps+p):(eps+p), with B0 the
// Hessian of the state: the secant (1-D0) C, plus the rank-one part of the
// symmetric consistent tangent where `ct` is set.
template <typename R, int NC>
__global__ void __launch_bounds__(kVThreads)
    k_trial(const GridDesc g, const MatTable<R> mt, const EigTable<R> eg, const ConsTan<R> ct,
            const uint8_t* __restrict__ phase, const R* __restrict__ eps,
            const R* __restrict__ p, const R* __restrict__ khist, const R* __restrict__ sig0,
            const R* __restrict__ D0, R* __restrict__ sig_t, R* __restrict__ D_t, R* __restrict__ kap_t,
            double* __restrict__ part) {
  // four consecutive voxels per thread (nvox is a multiple of 4)
  constexpr int nc = NC, nd = NC == 6 ? 3 : 2;
  const long long nv = g.nvox, nv4 = nv / 4;
  KSum<R> acc[6];
  for (long long v4 = (long long)blockIdx.x * blockDim.x + threadIdx.x; v4 < nv4;
       v4 += (long long)gridDim.x * blockDim.x) {
    V4<R> e[6], pv[6], s0[6];
#pragma unroll
    for (int c = 0; c < nc; ++c) {
      e[c] = ld4(eps + c * nv, v4);
      if (p) pv[c] = ld4(p + c * nv, v4);
      else pv[c] = V4<R>{0, 0, 0, 0};
      if (sig0) s0[c] = ld4(sig0 + c * nv, v4);
    }
    const V4<R> kh4 = khist ? ld4(khist, v4) : V4<R>{0, 0, 0, 0};
    const V4<R> d04 = D0 ? ld4(D0, v4) : V4<R>{0, 0, 0, 0};
    const uchar4 ph4 = *reinterpret_cast<const uchar4*>(phase + 4 * v4);
    const int phs[4] = {ph4.x, ph4.y, ph4.z, ph4.w};
    V4<R> sg[6], Dq, kq;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ph = phs[q];
      R ev[6], pq[6], et[6];
#pragma unroll
      for (int c = 0; c < nc; ++c) {
        pq[c] = elc<R>(pv[c], q);
        et[c] = elc<R>(e[c], q) + pq[c];
        ev[c] = eg.on ? et[c] + eg.e[ph][c] : et[c];
      }
      const R lam = mt.lam[ph], mu = mt.mu[ph];
      R D = 0, kap = 0;
      if (mt.damaging[ph]) {
        const R kt = kappa_tension<R>(ev, nd);
        // max(kappa_n, kappa_t) that keeps a NaN history (fmax would drop
        // it): invalid input then reaches the sums and is reported
        const R khq = elc<R>(kh4, q);
        const R k = kt > khq ? kt : khq;
        kap = k;
        D = damage_of<R>(k, mt.kappa0[ph], mt.kappaf[ph]);
      }
      const R keep = (R)1 - D;
      R tr = 0, trp = 0;
#pragma unroll
      for (int i = 0; i < nd; ++i) { tr += ev[i]; trp += pq[i]; }
      const R keep0 = (R)1 - elc<R>(d04, q);
      const long long vq = 4 * v4 + q;
      const R hdp = (ct.dp && p) ? (R)0.5 * ct.dp[vq] : (R)0;
      R np_ = 0, ap_ = 0;
      if (hdp != (R)0) {
#pragma unroll
        for (int c = 0; c < nc; ++c) {
          np_ += ct.n[c * nv + vq] * pq[c];
          ap_ += ct.a[c * nv + vq] * pq[c];
        }
      }
#pragma unroll
      for (int c = 0; c < nc; ++c) {
        const R sv = keep * ((R)2 * mu * ev[c] + (c < nd ? lam * tr : (R)0));
        el<R>(sg[c], q) = sv;
        R bp = keep0 * ((R)2 * mu * pq[c] + (c < nd ? lam * trp : (R)0));
        if (hdp != (R)0) bp -= hdp * (ct.a[c * nv + vq] * np_ + ct.n[c * nv + vq] * ap_);
        if (sig0) acc[0].add(elc<R>(s0[c], q) * pq[c]);
        acc[1].add(sv * pq[c]);
        acc[2].add(pq[c] * bp);
        acc[3].add(sv * sv);
        acc[4].add(pq[c] * pq[c]);
        acc[5].add(et[c] * et[c]);
      }
      el<R>(Dq, q) = D;
      el<R>(kq, q) = kap;
    }
#pragma unroll
    for (int c = 0; c < nc; ++c) st4(sig_t + c * nv, v4, sg[c]);
    if (D_t) st4(D_t, v4, Dq);
    if (kap_t) st4(kap_t, v4, kq);
  }
  finish_sums<R, 6>(acc, part);
}

// Algorithm 2 ratio test with the first-order incremental energy.
__global__ void k_tr_decide(DevScalars* S) { tr_decide_scalars(S); }

template <typename R>
__global__ void __launch_bounds__(kVThreads) k_axpy(long long n, R a, const R* __restrict__ x, R* __restrict__ y) {
  const long long n4 = n / 4;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const V4<R> xi = ld4(x, i);
    V4<R> yi = ld4(y, i);
#pragma unroll
    for (int e = 0; e < 4; ++e) el<R>(yi, e) += a * elc<R>(xi, e);
    st4(y, i, yi);
  }
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
  *nl += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t trial_eval(const GridDesc& g, const MatTable<R>& mt, const EigTable<R>& eg, const uint8_t* phase,
                       const R* eps, const R* p, const R* khist, const R* sig0, const R* D0, R* sig_t, R* D_t,
                       R* kap_t, DevScalars* S, double* part, cudaStream_t st, long long* nl, const ConsTan<R>& ct) {
  if (g.ncomp == 6)
    k_trial<R, 6><<<kVBlocks, kVThreads, 0, st>>>(g, mt, eg, ct, phase, eps, p, khist, sig0, D0, sig_t, D_t, kap_t,
                                                  part);
  else
    k_trial<R, 3><<<kVBlocks, kVThreads, 0, st>>>(g, mt, eg, ct, phase, eps, p, khist, sig0, D0, sig_t, D_t, kap_t,
                                                  part);
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
  template cudaError_t trial_eval<R>(const GridDesc&, const MatTable<R>&, const EigTable<R>&, const uint8_t*, \
                                     const R*, const R*,                                                        \
                                     const R*, const R*, const R*, R*, R*, R*, DevScalars*,                     \
                                     double*, cudaStream_t, long long*, const ConsTan<R>&);                     \
  template cudaError_t axpy<R>(long long, R, const R*, R*, cudaStream_t, long long*);                          \
  template cudaError_t add_uniform<R>(const GridDesc&, R*, const double*, cudaStream_t, long long*);           \
  template cudaError_t field_means<R>(const GridDesc&, const R*, const R*, DevScalars*, double*, cudaStream_t, \
                                      long long*);

RVE_INST(float)
RVE_INST(double)

}  // namespace rve
