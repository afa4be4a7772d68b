// Dispatch into the cluster x+y passes (hv_cluster.cu): 3D FP32 grids with
// Nx = Ny in {64, 96, 128, 192, 256}.  Each returns cudaErrorNotSupported
// (nothing launched) for other grids; the caller then runs the separate x
// and y passes.  twm: e^{-2 pi i t / M}, t < M = Nx / 4.
#pragma once

#include "hv_passes.cuh"

namespace rve {

bool cluster_size_ok(const GridDesc& g);
// blocks of one cluster pass (one partial sum each)
int cluster_blocks(const GridDesc& g);
// x and y forward transforms (tangent applied on load when `tangent`; with
// `partials`, every block's share of in : (tangent : in) in partials[block])
cudaError_t cluster_xyfwd(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                          const MatTable<float>& mt, float2* spec, const float2* twn, const float2* twm, bool tangent,
                          double* partials, cudaStream_t st);
// y and x inverse transforms, scaled by 1/Nvox, stored to `out` (with the
// dot product with dotw -- or with the output itself when `self` -- in
// partials[block] when `dot`)
cudaError_t cluster_yxinv(const GridDesc& g, const float2* spec, float* out, const float* dotw, double* partials,
                          const float2* twn, const float2* twm, bool dot, bool self, cudaStream_t st);
// y and x inverse transforms with the Steihaug-CG update of fast_xinv_cg
// (three sums per block, block-major)
cudaError_t cluster_yxinv_cg(const GridDesc& g, const float2* spec, float* z, float* r, const float* d,
                             const int* status, const double* alpha, const double* tau, double* partials,
                             const float2* twn, const float2* twm, cudaStream_t st);

}  // namespace rve
