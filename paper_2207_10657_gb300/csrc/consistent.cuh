// Per-voxel data of the symmetric consistent damage tangent for the state
// (Appendix A): on loading voxels (kappa_trial > kappa_n, kappa0 < kappa <
// kappaf) dp = D'(kappa), a = C : eps and n = eps^(t) / kappa, from which the
// tangent passes form (1-D) C : v - dp/2 (a (n.v) + n (a.v)).  kappa^2 is a
// spectral function of the strain, so d kappa / d eps = eps^(t) / kappa.
#pragma once

#include "hv_passes.cuh"
#include "solver_kernels.cuh"

namespace rve {

// dp (Nvox) for every voxel; a, n (ncomp x Nvox) where dp != 0.  The
// material sees eps + eps_eig(phase), as the constitutive kernel does.
template <typename R>
cudaError_t cons_prep(const GridDesc& g, const MatTable<R>& mt, const EigTable<R>& eg, const uint8_t* phase,
                      const R* eps, const R* khist, R* dp, R* a, R* n, cudaStream_t st, long long* nl);

}  // namespace rve
