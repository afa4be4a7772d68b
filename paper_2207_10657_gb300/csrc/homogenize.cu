// Sum of the secant stress (1 - D) C : v over the cell, per Mandel component.
#include "homogenize.cuh"
#include "hv_passes.cuh"

namespace rve {

namespace {

constexpr int kHThreads = 256;
constexpr int kHBlocks = 152 * 4;

template <typename R, int NC>
__global__ void __launch_bounds__(kHThreads)
    k_tangent_sum(const GridDesc g, const MatTable<R> mt, const uint8_t* __restrict__ phase,
                  const R* __restrict__ D, const R* __restrict__ v, double* __restrict__ part) {
  constexpr int nd = NC == 6 ? 3 : 2;
  const long long nv = g.nvox;
  KSum<R> acc[NC];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    const int ph = phase[i];
    const R keep = (R)1 - D[i];
    const R lam = mt.lam[ph], mu = mt.mu[ph];
    R x[NC], tr = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = v[c * nv + i];
#pragma unroll
    for (int c = 0; c < nd; ++c) tr += x[c];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c].add(keep * ((R)2 * mu * x[c] + (c < nd ? lam * tr : (R)0)));
  }
  __shared__ double red[NC * 32];
  double s[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) s[c] = acc[c].value();
  block_sum<NC>(s, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) part[(long long)blockIdx.x * NC + c] = s[c];
  }
}

}  // namespace

template <typename R>
cudaError_t tangent_sum(const GridDesc& g, const MatTable<R>& mt, const uint8_t* phase, const R* D, const R* v,
                        double* out, double* part, cudaStream_t st, long long* nl) {
  if (g.ncomp == 6) k_tangent_sum<R, 6><<<kHBlocks, kHThreads, 0, st>>>(g, mt, phase, D, v, part);
  else k_tangent_sum<R, 3><<<kHBlocks, kHThreads, 0, st>>>(g, mt, phase, D, v, part);
  ++*nl;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return reduce_partials(part, kHBlocks, g.ncomp, out, st, nl);
}

template cudaError_t tangent_sum<float>(const GridDesc&, const MatTable<float>&, const uint8_t*, const float*,
                                        const float*, double*, double*, cudaStream_t, long long*);
template cudaError_t tangent_sum<double>(const GridDesc&, const MatTable<double>&, const uint8_t*, const double*,
                                         const double*, double*, double*, cudaStream_t, long long*);

}  // namespace rve
