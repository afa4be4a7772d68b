// The x-forward pass with bulk tensor copies (hv_tma.cu): 3D FP32 grids with
// six components per voxel, Nx in {32, 64, 96, 128, 192, 256}, plain or
// secant tangent.  Returns cudaErrorNotSupported (nothing launched) for
// other grids or when the tensor-map encoder is unavailable; the caller then
// runs the compiled x-forward pass.  With `partials` (tangent only) every
// block writes its share of in : (tangent : in) to partials[block];
// *nblocks receives the block count.  wait_err: set to 1 by a CTA whose
// copies did not arrive within the wait limit.  S (may be NULL; used with
// `partials` only): the last block to finish also sums the shares into
// S->dHd and takes the CG step-length decision of Algorithm 1 on S.
#pragma once

#include "hv_passes.cuh"

namespace rve {

cudaError_t tma_xfwd(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                     const MatTable<float>& mt, float2* spec, const float2* tw, bool tangent, double* partials,
                     int* nblocks, cudaStream_t st, int* wait_err, DevScalars* S = nullptr);

}  // namespace rve
