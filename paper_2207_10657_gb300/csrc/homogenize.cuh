// Volume average of the secant stress (1 - D) C : v of a field, the last step
// of the effective-stiffness computation (first-order homogenisation of the
// linearised cell problem; the stiffness-loss measure of Sec. 3.3).
#pragma once

#include "hv_passes.cuh"

namespace rve {

// out[c] <- sum over voxels of ((1 - D) C : v)_c, c < ncomp (FP64, device).
template <typename R>
cudaError_t tangent_sum(const GridDesc& g, const MatTable<R>& mt, const uint8_t* phase, const R* D, const R* v,
                        double* out, double* part, cudaStream_t st, long long* nl);

}  // namespace rve
