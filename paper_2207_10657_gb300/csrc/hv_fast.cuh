// Dispatch into the compile-time-specialised FP32 passes (hv_fast.cu).
// Each returns cudaErrorNotSupported when the axis length has no
// specialisation; the caller then uses the generic pass.
#pragma once

#include "hv_passes.cuh"

namespace rve {

bool fast_size(int n);
// With `partials` (tangent mode only) every block also writes its sum of
// in : (tangent : in) to partials[block]; *nblocks receives the block count.
// ct (may be NULL): with ct->dp set, the tangent mode applies the symmetric
// consistent tangent instead of the secant.
cudaError_t fast_xfwd(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                      const MatTable<float>& mt, float2* spec, const float2* tw, bool tangent, double* partials,
                      int* nblocks, cudaStream_t st, const ConsTan<float>* ct = nullptr);
cudaError_t fast_xinv(const GridDesc& g, const float2* spec, float* out, const float* dotw, double* partials,
                      const float2* tw, bool dot, bool self, int* nblocks, cudaStream_t st);
// x-inverse that applies the Steihaug-CG iterate / residual update with the
// product instead of storing it (status / alpha / tau: device scalars;
// partials: three sums per block, block-major).
cudaError_t fast_xinv_cg(const GridDesc& g, const float2* spec, float* z, float* r, const float* d, const int* status,
                         const double* alpha, const double* tau, double* partials, const float2* tw, int* nblocks,
                         cudaStream_t st);
cudaError_t fast_ycols(const GridDesc& g, float2* spec, const float2* tw, bool inv, cudaStream_t st);
cudaError_t fast_zproj(const GridDesc& g, float2* spec, const SpecWork<float>& w, cudaStream_t st);
cudaError_t fast_yproj2d(const GridDesc& g, float2* spec, const SpecWork<float>& w, cudaStream_t st);

}  // namespace rve
