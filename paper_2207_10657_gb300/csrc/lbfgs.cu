// L-BFGS vector kernels (Nocedal & Wright Alg. 7.4 / 7.5; the paper's remark
// after Eq. (20) that the first-order incremental energy makes quasi-Newton
// methods usable).  Each pass is a grid-stride stream over 4-wide vectors;
// sums are Neumaier-compensated per thread and FP64 across threads.
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
__global__ void __launch_bounds__(kLThreads) k_lb_dot(long long n4, const R* __restrict__ x, const R* __restrict__ y,
                                                      double* __restrict__ part) {
  KSum<R> acc[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    W4<R> a = ld4(x, i), b = ld4(y, i);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[0].add(el<R>(a, e) * el<R>(b, e));
  }
  block_partials<R, 1>(acc, part);
}

template <typename R>
__global__ void __launch_bounds__(kLThreads)
    k_lb_loop1(long long n4, const R* src, R* q, const R* __restrict__ y, const R* __restrict__ w, double rho, int i,
               LbScalars* L, double* __restrict__ part) {
  const double a = rho * L->sum;
  const R ar = (R)a;
  KSum<R> acc[1];
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x) {
    W4<R> v = ld4(src, k), yy = ld4(y, k);
#pragma unroll
    for (int e = 0; e < 4; ++e) el<R>(v, e) -= ar * el<R>(yy, e);
    st4(q, k, v);
    if (w) {
      W4<R> ww = ld4(w, k);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[0].add(el<R>(ww, e) * el<R>(v, e));
    }
  }
  block_partials<R, 1>(acc, part);
  // every thread has read L->sum before any block can finish; the block that
  // stores a_i does so after its own reads
  if (blockIdx.x == 0 && threadIdx.x == 0) L->a[i] = a;
}

template <typename R>
__global__ void __launch_bounds__(kLThreads)
    k_lb_loop2(long long n4, const R* src, R* out, const R* __restrict__ s, const R* __restrict__ w, double rho,
               double f, double sgn, int i, const LbScalars* __restrict__ L, double* __restrict__ part) {
  const double b = rho * f * L->sum;
  const R c = (R)(L->a[i] - b), fr = (R)f, sr = (R)sgn;
  KSum<R> acc[1];
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x) {
    W4<R> v = ld4(src, k), ss = ld4(s, k), o;
#pragma unroll
    for (int e = 0; e < 4; ++e) el<R>(v, e) = fr * el<R>(v, e) + c * el<R>(ss, e);
    if (w) {
      W4<R> ww = ld4(w, k);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[0].add(el<R>(ww, e) * el<R>(v, e));
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) el<R>(o, e) = sr * el<R>(v, e);
    st4(out, k, o);
  }
  block_partials<R, 1>(acc, part);
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

template <typename R>
cudaError_t lb_dot(long long n, const R* x, const R* y, LbScalars* L, double* part, cudaStream_t st,
                   long long* nl) {
  k_lb_dot<R><<<kLBlocks, kLThreads, 0, st>>>(n / 4, x, y, part);
  ++*nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return reduce_partials(part, kLBlocks, 1, &L->sum, st, nl);
}

template <typename R>
cudaError_t lb_loop1(long long n, const R* src, R* q, const R* y, const R* w, double rho, int i, LbScalars* L,
                     double* part, cudaStream_t st, long long* nl) {
  k_lb_loop1<R><<<kLBlocks, kLThreads, 0, st>>>(n / 4, src, q, y, w, rho, i, L, part);
  ++*nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !w) return e;
  return reduce_partials(part, kLBlocks, 1, &L->sum, st, nl);
}

template <typename R>
cudaError_t lb_loop2(long long n, const R* src, R* out, const R* s, const R* w, double rho, double f, double sgn,
                     int i, LbScalars* L, double* part, cudaStream_t st, long long* nl) {
  k_lb_loop2<R><<<kLBlocks, kLThreads, 0, st>>>(n / 4, src, out, s, w, rho, f, sgn, i, L, part);
  ++*nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !w) return e;
  return reduce_partials(part, kLBlocks, 1, &L->sum, st, nl);
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

#define RVE_LB_INST(R)                                                                                           \
  template cudaError_t lb_dot<R>(long long, const R*, const R*, LbScalars*, double*, cudaStream_t, long long*); \
  template cudaError_t lb_loop1<R>(long long, const R*, R*, const R*, const R*, double, int, LbScalars*,       \
                                   double*, cudaStream_t, long long*);                                         \
  template cudaError_t lb_loop2<R>(long long, const R*, R*, const R*, const R*, double, double, double, int,   \
                                   LbScalars*, double*, cudaStream_t, long long*);                             \
  template cudaError_t lb_scale<R>(long long, const R*, R*, double, cudaStream_t, long long*);                 \
  template cudaError_t lb_pair<R>(long long, const R*, R*, R*, LbScalars*, double*, cudaStream_t, long long*);

RVE_LB_INST(float)
RVE_LB_INST(double)

}  // namespace rve
