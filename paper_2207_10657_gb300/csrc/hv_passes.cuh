// Host-side description of the FFT / projection passes of one grid.
#pragma once

#include "common.cuh"
#include "pass_timer.cuh"

namespace rve {

struct GridDesc {
  int ndim;       // 2 or 3
  int nx, ny, nz; // nz = 1 in 2D
  int nxh;        // nx/2 + 1 (half spectrum along x)
  int ncomp;      // 3 or 6
  long long nvox;
  long long nrows;  // ny * nz voxel rows along x
  int nq = 1;       // strain points per voxel: 1 (one element per voxel), 2 (2D Kuhn
                    // triangles) or 6 (3D Kuhn tetrahedra); the spectral lines are then
                    // c * nq + q, ncomp = 6 or 36
};

// Rank-one part of the symmetric consistent damage tangent, per voxel: the
// tangent applied to v is (1-D) C : v - dp/2 (a (n.v) + n (a.v)) with
// a = C : eps, n = eps^(t) / kappa and dp = D'(kappa) on loading voxels
// (0 elsewhere; a and n are read only where dp != 0).  All NULL: secant.
template <typename R> struct ConsTan {
  const R* dp = nullptr;  // Nvox
  const R* a = nullptr;   // ncomp x Nvox
  const R* n = nullptr;   // ncomp x Nvox
};

// Tables and workspace for the spectral passes at precision R.
template <typename R> struct SpecWork {
  AxisPlan px, py, pz;
  Cx<R>* tw[3] = {nullptr, nullptr, nullptr};    // e^{-2 pi i t / n_axis}
  Cx<R>* gdiff[3] = {nullptr, nullptr, nullptr}; // e^{i th} - 1 (exact 0 at k=0)
  Cx<R>* gavg[3] = {nullptr, nullptr, nullptr};  // (1 + e^{i th})/2 (exact 0 at 2k=n)
  Cx<R>* spec = nullptr;                          // ncomp * nz * ny * nxh
  unsigned free_mask = 0;                         // bit c: Mandel comp c stress-controlled
  // tiling
  int qx;   // voxel rows per x-pass block
  int ty;   // kx columns per y-pass block
  int tz;   // kx columns per z-pass / 2D y-pass block
  double* partials = nullptr;  // per-block FP64 partial sums (epilogues)
  int max_partials = 0;
  PassTimer* timer = nullptr;  // optional per-pass event timing
  ConsTan<R> cons;             // set: tangent passes apply the consistent tangent
  bool generic = false;        // true: never take the compiled FP32 passes
  bool unfused = false;        // true: compiled passes, but CG scalars and updates as the generic path
  bool cluster = false;        // true: the cluster x+y passes where they apply (opt-in: slower, see hv_cluster.cu)
  Cx<R>* twq = nullptr;        // e^{-2 pi i t / (Nx/4)}: the cluster passes' y sub-transform
  int* wait_err = nullptr;     // device word a kernel sets when a bounded wait runs out (NULL: no TMA passes)
};

enum class XIn { Plain = 0, Tangent = 1 };

// Launch helpers (hv_passes.cu).  Every pass runs on `st`; the number of
// launches issued is added to *nlaunch.
template <typename R>
cudaError_t spectral_apply(const GridDesc& g, SpecWork<R>& w, const MatTable<R>& mt, const R* in,
                           const uint8_t* phase, const R* damage, XIn mode, R* out,
                           const R* dot_with, double* dot_out, cudaStream_t st, long long* nlaunch);

struct DevScalars;  // solver_kernels.cuh

// One Steihaug-CG iteration's product on the compiled FP32 x passes, on the
// device scalars S: the forward passes with d:H:d formed in the x-forward
// pass (into S->dHd), then Algorithm 1's step length, then the x-inverse
// applying z += alpha d, r += alpha Hd (or z += tau d on an exit) with
// r'.r', r'.r, z'.z into S->rr_new, S->rnr, S->zz_new, then the convergence
// / beta decision.  Hd is never stored.  The persistent x-forward pass
// reduces d:H:d and takes the step-length decision in its last block; else
// one single-block kernel does both, as one does after the x-inverse.
// Returns cudaErrorNotSupported (nothing launched) when Nx has no compiled
// pass.
cudaError_t spectral_hv_cg(const GridDesc& g, SpecWork<float>& w, const MatTable<float>& mt, const float* d,
                           const uint8_t* phase, const float* damage, float* z, float* r, DevScalars* S,
                           cudaStream_t st, long long* nlaunch);

template <typename R>
cudaError_t spectral_setup(const GridDesc& g, SpecWork<R>& w);
template <typename R>
void spectral_free(SpecWork<R>& w);
// Plans and tile sizes only, no device allocation (the caller provides
// the tables and the spectrum storage in SpecWork).
template <typename R>
cudaError_t spectral_plan(const GridDesc& g, SpecWork<R>& w);

// FP64 final reduction of per-block partials: out[s] = sum_b part[b*ns + s]
// (out: ns contiguous device doubles).  Fixed summation order.
cudaError_t reduce_partials(const double* part, int nblocks, int ns, double* out, cudaStream_t st,
                            long long* nlaunch);

}  // namespace rve
