// L-BFGS vector kernels (Nocedal & Wright Alg. 7.5 with the compact
// representation of the inverse Hessian; the paper's remark after Eq. (20)
// that the first-order incremental energy makes quasi-Newton methods
// usable).  Each pass is a grid-stride stream over 4-wide vectors; sums are
// Neumaier-compensated per thread and FP64 across threads.
#include <algorithm>

#include "hv_passes.cuh"
#include "lbfgs.cuh"

namespace rve {

namespace {

constexpr int kLThreads = 256;
constexpr int kLBlocks = 152 * 4;

template <typename R> struct W4T;
template <> struct W4T<float> { using T = float4; };
template <> struct W4T<double> { using T = double4_32a; };
template <typename R> using W4 = typename W4T<R>::T;
template <typename R> __device__ __forceinline__ R& el(W4<R>& v, int i) { return (&v.x)[i]; }
template <typename R> __device__ __forceinline__ W4<R> ld4(const R* p, long long i) {
  return *reinterpret_cast<const W4<R>*>(p + 4 * i);
}
template <typename R> __device__ __forceinline__ void st4(R* p, long long i, const W4<R>& v) {
  *reinterpret_cast<W4<R>*>(p + 4 * i) = v;
}

template <typename R, int NS>
__device__ __forceinline__ void block_partials(KSum<R> (&acc)[NS], double* part) {
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

template <typename R>
struct LbGroup {
  const R* s[kLbGroup];
  const R* y[kLbGroup];
};

// Pass A over one group of G pairs: s_i . g, y_i . g and, with NEWP, s_i . yn
// and y_i . yn (yn the newest pair's y).
template <typename R, int G, bool NEWP>
__global__ void __launch_bounds__(kLThreads)
    k_lb_dots(long long n4, const R* __restrict__ g, const LbGroup<R> P, const R* __restrict__ yn,
              double* __restrict__ part) {
  KSum<R> acc[4 * G];
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x) {
    W4<R> g4 = ld4(g, k), n4v;
    if constexpr (NEWP) n4v = ld4(yn, k);
#pragma unroll
    for (int i = 0; i < G; ++i) {
      W4<R> s4 = ld4(P.s[i], k), y4 = ld4(P.y[i], k);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[i].add(el<R>(s4, e) * el<R>(g4, e));
        acc[G + i].add(el<R>(y4, e) * el<R>(g4, e));
        if constexpr (NEWP) {
          acc[2 * G + i].add(el<R>(s4, e) * el<R>(n4v, e));
          acc[3 * G + i].add(el<R>(y4, e) * el<R>(n4v, e));
        }
      }
    }
  }
  block_partials<R, 4 * G>(acc, part);
}

struct LbCoefArgs {
  int k, new_pair;
  int slot[kLbMaxMemory];
  double gamma;
};

// One thread: new entries of S^T Y and Y^T Y, then the two triangular solves
// of the compact representation and the coefficients of pass C.
__global__ void k_lb_coef(LbScalars* L, const LbCoefArgs A) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int k = A.k;
  double a[kLbMaxMemory], c[kLbMaxMemory], u[kLbMaxMemory], t[kLbMaxMemory], p[kLbMaxMemory];
  for (int j = 0; j < k; ++j) {
    const int q = j / kLbGroup, i = j % kLbGroup;
    const int G = min(kLbGroup, k - q * kLbGroup);
    a[j] = L->gsum[q][i];
    c[j] = L->gsum[q][G + i];
    if (A.new_pair) {
      const int sj = A.slot[j], sn = A.slot[k - 1];
      L->SY[sj][sn] = L->gsum[q][2 * G + i];
      L->YY[sj][sn] = L->gsum[q][3 * G + i];
      L->YY[sn][sj] = L->gsum[q][3 * G + i];
    }
  }
  // R_ij = s_i . y_j (i <= j) in ring order; u = R^-1 a
  for (int i = k - 1; i >= 0; --i) {
    double v = a[i];
    for (int j = i + 1; j < k; ++j) v -= L->SY[A.slot[i]][A.slot[j]] * u[j];
    u[i] = v / L->SY[A.slot[i]][A.slot[i]];
  }
  // t = (D + gamma Y^T Y) u - gamma c; p = R^-T t
  for (int i = 0; i < k; ++i) {
    double v = L->SY[A.slot[i]][A.slot[i]] * u[i] - A.gamma * c[i];
    for (int j = 0; j < k; ++j) v += A.gamma * L->YY[A.slot[i]][A.slot[j]] * u[j];
    t[i] = v;
  }
  for (int i = 0; i < k; ++i) {
    double v = t[i];
    for (int j = 0; j < i; ++j) v -= L->SY[A.slot[j]][A.slot[i]] * p[j];
    p[i] = v / L->SY[A.slot[i]][A.slot[i]];
  }
  for (int j = 0; j < k; ++j) {
    L->cS[j] = -p[j];
    L->cY[j] = A.gamma * u[j];
  }
}

// Pass C over one group: d = cg g + sum cS_i s_i + cY_i y_i (FIRST), or
// d += the group's terms.
template <typename R, int G, bool FIRST>
__global__ void __launch_bounds__(kLThreads)
    k_lb_combine(long long n4, const R* __restrict__ g, const LbGroup<R> P, const double* __restrict__ cS,
                 const double* __restrict__ cY, double cg, R* d) {
  R a[G], b[G];
#pragma unroll
  for (int i = 0; i < G; ++i) {
    a[i] = (R)cS[i];
    b[i] = (R)cY[i];
  }
  const R cgr = (R)cg;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x) {
    W4<R> v;
    if constexpr (FIRST) {
      v = ld4(g, k);
#pragma unroll
      for (int e = 0; e < 4; ++e) el<R>(v, e) *= cgr;
    } else {
      v = ld4(d, k);
    }
#pragma unroll
    for (int i = 0; i < G; ++i) {
      W4<R> s4 = ld4(P.s[i], k), y4 = ld4(P.y[i], k);
#pragma unroll
      for (int e = 0; e < 4; ++e) el<R>(v, e) += a[i] * el<R>(s4, e) + b[i] * el<R>(y4, e);
    }
    st4(d, k, v);
  }
}

template <typename R>
__global__ void __launch_bounds__(kLThreads) k_lb_scale(long long n4, const R* src, R* dst, R c) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x) {
    W4<R> v = ld4(src, k);
#pragma unroll
    for (int e = 0; e < 4; ++e) el<R>(v, e) *= c;
    st4(dst, k, v);
  }
}

template <typename R>
__global__ void __launch_bounds__(kLThreads)
    k_lb_pair(long long n4, const R* __restrict__ s, R* __restrict__ g, R* __restrict__ gnew,
              double* __restrict__ part) {
  KSum<R> acc[2];
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x) {
    W4<R> go = ld4(g, k), gn = ld4(gnew, k), ss = ld4(s, k), y;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el<R>(y, e) = el<R>(gn, e) - el<R>(go, e);
      acc[0].add(el<R>(ss, e) * el<R>(y, e));
      acc[1].add(el<R>(y, e) * el<R>(y, e));
    }
    st4(g, k, gn);
    st4(gnew, k, y);
  }
  block_partials<R, 2>(acc, part);
}

}  // namespace

// One full wave: the SM count times the blocks of `kernel` resident per SM
// (the pass kernels of large groups hold many accumulators, so fewer blocks
// fit than the default grid assumes and a second, partial wave would idle
// most of the GPU), capped so that ns partial sums per block fit the
// partial-sum buffer.
template <typename K>
static int full_wave(K kernel, int ns) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
      cudaSuccess || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kLThreads, 0) != cudaSuccess ||
      per < 1 || sms < 1)
    return kLBlocks;
  return std::max(1, std::min(sms * per, 32768 / std::max(ns, 1)));
}

template <typename R, int G>
static cudaError_t dots_g(long long n4, const R* g, const LbGroup<R>& P, const R* yn, double* part,
                          cudaStream_t st, int* nblocks) {
  static const int bt = full_wave(k_lb_dots<R, G, true>, 4 * G);
  static const int bf = full_wave(k_lb_dots<R, G, false>, 4 * G);
  if (yn) k_lb_dots<R, G, true><<<bt, kLThreads, 0, st>>>(n4, g, P, yn, part);
  else k_lb_dots<R, G, false><<<bf, kLThreads, 0, st>>>(n4, g, P, yn, part);
  *nblocks = yn ? bt : bf;
  return cudaGetLastError();
}

template <typename R, int G>
static cudaError_t combine_g(long long n4, const R* g, const LbGroup<R>& P, const double* cS, const double* cY,
                             double cg, bool first, R* d, cudaStream_t st) {
  static const int bt = full_wave(k_lb_combine<R, G, true>, 0);
  static const int bf = full_wave(k_lb_combine<R, G, false>, 0);
  if (first) k_lb_combine<R, G, true><<<bt, kLThreads, 0, st>>>(n4, g, P, cS, cY, cg, d);
  else k_lb_combine<R, G, false><<<bf, kLThreads, 0, st>>>(n4, g, P, cS, cY, cg, d);
  return cudaGetLastError();
}

#define RVE_LB_GSWITCH(G_, CALL) \
  switch (G_) {                  \
    case 1: e = CALL(1); break;  \
    case 2: e = CALL(2); break;  \
    case 3: e = CALL(3); break;  \
    case 4: e = CALL(4); break;  \
    case 5: e = CALL(5); break;  \
    case 6: e = CALL(6); break;  \
    case 7: e = CALL(7); break;  \
    default: e = CALL(8); break; \
  }

template <typename R>
cudaError_t lb_direction(long long n, const R* g, const LbRing<R>& ring, bool new_pair, double gamma, R* d,
                         LbScalars* L, double* part, cudaStream_t st, long long* nl) {
  const int k = ring.k;
  const long long n4 = n / 4;
  if (k < 1 || k > kLbMaxMemory) return cudaErrorInvalidValue;
  const int ngrp = (k + kLbGroup - 1) / kLbGroup;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < ngrp && e == cudaSuccess; ++q) {
    const int G = min(kLbGroup, k - q * kLbGroup);
    LbGroup<R> P{};
    for (int i = 0; i < G; ++i) {
      P.s[i] = ring.s[q * kLbGroup + i];
      P.y[i] = ring.y[q * kLbGroup + i];
    }
    const R* yn = new_pair ? ring.y[k - 1] : nullptr;
    int nb = kLBlocks;
#define RVE_LB_DOTS(G_) dots_g<R, G_>(n4, g, P, yn, part, st, &nb)
    RVE_LB_GSWITCH(G, RVE_LB_DOTS)
#undef RVE_LB_DOTS
    ++*nl;
    if (e == cudaSuccess) e = reduce_partials(part, nb, 4 * G, &L->gsum[q][0], st, nl);
  }
  if (e != cudaSuccess) return e;
  LbCoefArgs A{};
  A.k = k;
  A.new_pair = new_pair ? 1 : 0;
  A.gamma = gamma;
  for (int j = 0; j < k; ++j) A.slot[j] = ring.slot[j];
  k_lb_coef<<<1, 1, 0, st>>>(L, A);
  ++*nl;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int q = 0; q < ngrp && e == cudaSuccess; ++q) {
    const int G = min(kLbGroup, k - q * kLbGroup);
    LbGroup<R> P{};
    for (int i = 0; i < G; ++i) {
      P.s[i] = ring.s[q * kLbGroup + i];
      P.y[i] = ring.y[q * kLbGroup + i];
    }
    const double* cS = &L->cS[q * kLbGroup];
    const double* cY = &L->cY[q * kLbGroup];
#define RVE_LB_COMB(G_) combine_g<R, G_>(n4, g, P, cS, cY, -gamma, q == 0, d, st)
    RVE_LB_GSWITCH(G, RVE_LB_COMB)
#undef RVE_LB_COMB
    ++*nl;
  }
  return e;
}

template <typename R>
cudaError_t lb_scale(long long n, const R* src, R* dst, double c, cudaStream_t st, long long* nl) {
  k_lb_scale<R><<<kLBlocks, kLThreads, 0, st>>>(n / 4, src, dst, (R)c);
  ++*nl;
  return cudaGetLastError();
}

template <typename R>
cudaError_t lb_pair(long long n, const R* s, R* g, R* gnew, LbScalars* L, double* part, cudaStream_t st,
                    long long* nl) {
  k_lb_pair<R><<<kLBlocks, kLThreads, 0, st>>>(n / 4, s, g, gnew, part);
  ++*nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return reduce_partials(part, kLBlocks, 2, &L->sy, st, nl);
}

#define RVE_LB_INST(R)                                                                                         \
  template cudaError_t lb_direction<R>(long long, const R*, const LbRing<R>&, bool, double, R*, LbScalars*,   \
                                       double*, cudaStream_t, long long*);                                    \
  template cudaError_t lb_scale<R>(long long, const R*, R*, double, cudaStream_t, long long*);                \
  template cudaError_t lb_pair<R>(long long, const R*, R*, R*, LbScalars*, double*, cudaStream_t, long long*);

RVE_LB_INST(float)
RVE_LB_INST(double)

}  // namespace rve
