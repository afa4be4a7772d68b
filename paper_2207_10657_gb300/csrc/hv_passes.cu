// Spectral passes of the Hessian-vector product and of the projection:
//   x-forward (tangent fused) -> y-forward -> z-forward + projection +
//   z-inverse -> y-inverse -> x-inverse (+ fused FP64 dot product).
// 2D: x-forward -> y-forward + projection + y-inverse -> x-inverse.
//
// Sec. 2.1: G : zeta = F^-1{ Ghat(k) : F{zeta} } (Eq. (5)), Ghat from the
// linear finite-element gradient symbol through Eq. (9); the Hessian-vector
// product of Eq. (8) applies the tangent first, then the projection.
#include <algorithm>
#include <cmath>
#include <vector>

#include <type_traits>

#include "hv_cluster.cuh"
#include "hv_fast.cuh"
#include "hv_passes.cuh"
#include "hv_tma.cuh"
#include "passes_generic.cuh"
#include "project.cuh"
#include "scalar_logic.cuh"
#include "solver_kernels.cuh"

namespace rve {


// ------------------------------------------------------------ reduction
__global__ void k_reduce_partials(const double* __restrict__ part, int nb, int ns, double* __restrict__ out) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(long long)b * ns + s];
  double v[1] = {acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) out[s] = v[0];
}

cudaError_t reduce_partials(const double* part, int nblocks, int ns, double* out, cudaStream_t st,
                            long long* nlaunch) {
  k_reduce_partials<<<ns, 256, 0, st>>>(part, nblocks, ns, out);
  if (nlaunch) ++*nlaunch;
  return cudaGetLastError();
}

// ================================================================ host side
static void make_plan(int n, AxisPlan& p) {
  p.n = n;
  p.nstages = 0;
  int m = n, twos = 0;
  while (m % 2 == 0) { m /= 2; ++twos; }
  // powers of two: radix 8 as far as possible, then 4 / 4x4 / 2
  int n8 = twos / 3, rem = twos % 3;
  int n4 = 0, n2 = 0;
  if (rem == 2) n4 = 1;
  else if (rem == 1) {
    if (n8 > 0) { --n8; n4 = 2; } else n2 = 1;
  }
  for (int i = 0; i < n8; ++i) p.radix[p.nstages++] = 8;
  for (int i = 0; i < n4; ++i) p.radix[p.nstages++] = 4;
  for (int i = 0; i < n2; ++i) p.radix[p.nstages++] = 2;
  while (m % 3 == 0) { m /= 3; p.radix[p.nstages++] = 3; }
  while (m % 5 == 0) { m /= 5; p.radix[p.nstages++] = 5; }
}

template <typename R>
static cudaError_t upload_tables(int n, Cx<R>** tw, Cx<R>** gdiff, Cx<R>** gavg) {
  std::vector<Cx<R>> t(n), d(n), a(n);
  for (int k = 0; k < n; ++k) {
    // angles from long double libm calls, rounded once to R
    const long double th = 2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)n;
    const long double c = cosl(th), s = sinl(th);
    t[k] = Cx<R>{(R)c, (R)(-s)};
    d[k] = (k == 0) ? Cx<R>{0, 0} : Cx<R>{(R)(c - 1.0L), (R)s};
    a[k] = (2 * k == n) ? Cx<R>{0, 0} : Cx<R>{(R)((1.0L + c) * 0.5L), (R)(s * 0.5L)};
  }
  cudaError_t e;
  if ((e = cudaMalloc(tw, n * sizeof(Cx<R>))) != cudaSuccess) return e;
  if ((e = cudaMalloc(gdiff, n * sizeof(Cx<R>))) != cudaSuccess) return e;
  if ((e = cudaMalloc(gavg, n * sizeof(Cx<R>))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(*tw, t.data(), n * sizeof(Cx<R>), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(*gdiff, d.data(), n * sizeof(Cx<R>), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  return cudaMemcpy(*gavg, a.data(), n * sizeof(Cx<R>), cudaMemcpyHostToDevice);
}

static int pow2_floor(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

template <typename R>
cudaError_t spectral_setup(const GridDesc& g, SpecWork<R>& w) {
  using C = Cx<R>;
  make_plan(g.nx, w.px);
  make_plan(g.ny, w.py);
  make_plan(g.ndim == 3 ? g.nz : 1, w.pz);
  cudaError_t e;
  const int ns[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < g.ndim; ++a)
    if ((e = upload_tables<R>(ns[a], &w.tw[a], &w.gdiff[a], &w.gavg[a])) != cudaSuccess) return e;
  const size_t nspec = (size_t)g.ncomp * g.nrows * g.nxh;
  if ((e = cudaMalloc(&w.spec, nspec * sizeof(C))) != cudaSuccess) return e;
  if (std::is_same<R, float>::value && cluster_size_ok(g)) {
    // twiddles of the cluster passes' M-point y sub-transform (M = Nx / 4)
    const int m = g.nx / 4;
    std::vector<C> t(m);
    for (int k = 0; k < m; ++k) {
      const long double th = 2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)m;
      t[k] = C{(R)cosl(th), (R)(-sinl(th))};
    }
    if ((e = cudaMalloc(&w.twq, m * sizeof(C))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(w.twq, t.data(), m * sizeof(C), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  // x passes: npair * nx <= kXThreads * kXEpt complex per block
  const int ex = kXThreads * kXEpt;
  int q = (2 * ex) / (g.ncomp * g.nx);
  if (g.ncomp & 1) q &= ~1;
  q = std::max(q, (g.ncomp & 1) ? 2 : 1);
  w.qx = (int)std::min<long long>(q, g.nrows + (g.nrows & 1));
  // y columns
  const int ey = kYThreads * kYEpt;
  w.ty = std::max(1, std::min(pow2_floor(std::max(1, ey / g.ny)), 64));
  // z + projection (3D) or y + projection (2D)
  if (g.ndim == 3) {
    const int ez = std::min(kZThreads * kZEpt, (int)(kSmemCap / sizeof(C)));
    w.tz = std::max(1, std::min(pow2_floor(std::max(1, ez / (g.ncomp * g.nz))), 16));
  } else {
    const int e2 = std::min(kYThreads * kYEpt, (int)(kSmemCap / sizeof(C)));
    w.tz = std::max(1, std::min(pow2_floor(std::max(1, e2 / (g.ncomp * g.ny))), 64));
  }
  // up to three partial sums per x block (the fused CG x-inverse), and the
  // compile-time x passes may take a single row per block (Nx = 512)
  w.max_partials = (int)std::max<long long>(3 * g.nrows + 8, 4096 * 8);
  if ((e = cudaMalloc(&w.partials, (size_t)w.max_partials * sizeof(double))) != cudaSuccess) return e;
  // opt in to large dynamic shared memory
  cudaFuncSetAttribute(k_xfwd<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_xfwd<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_ycols<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_ycols<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_zproj<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_yproj2d<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_xinv<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_xinv<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  return cudaGetLastError();
}

// Plans and tile sizes for a caller that brings its own tables and spectrum
// storage (no device allocation): the same choices as spectral_setup.
template <typename R>
cudaError_t spectral_plan(const GridDesc& g, SpecWork<R>& w) {
  using C = Cx<R>;
  make_plan(g.nx, w.px);
  make_plan(g.ny, w.py);
  make_plan(g.ndim == 3 ? g.nz : 1, w.pz);
  const int ex = kXThreads * kXEpt;
  int q = (2 * ex) / (g.ncomp * g.nx);
  if (g.ncomp & 1) q &= ~1;
  q = std::max(q, (g.ncomp & 1) ? 2 : 1);
  w.qx = (int)std::min<long long>(q, g.nrows + (g.nrows & 1));
  const int ey = kYThreads * kYEpt;
  w.ty = std::max(1, std::min(pow2_floor(std::max(1, ey / g.ny)), 64));
  if (g.ndim == 3) {
    const int ez = std::min(kZThreads * kZEpt, (int)(kSmemCap / sizeof(C)));
    w.tz = std::max(1, std::min(pow2_floor(std::max(1, ez / (g.ncomp * g.nz))), 16));
  } else {
    const int e2 = std::min(kYThreads * kYEpt, (int)(kSmemCap / sizeof(C)));
    w.tz = std::max(1, std::min(pow2_floor(std::max(1, e2 / (g.ncomp * g.ny))), 64));
  }
  cudaFuncSetAttribute(k_xfwd<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_ycols<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_ycols<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_zproj<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_yproj2d<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_xinv<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  return cudaGetLastError();
}

template <typename R>
void spectral_free(SpecWork<R>& w) {
  for (int a = 0; a < 3; ++a) {
    if (w.tw[a]) cudaFree(w.tw[a]);
    if (w.gdiff[a]) cudaFree(w.gdiff[a]);
    if (w.gavg[a]) cudaFree(w.gavg[a]);
    w.tw[a] = w.gdiff[a] = w.gavg[a] = nullptr;
  }
  if (w.spec) cudaFree(w.spec);
  if (w.partials) cudaFree(w.partials);
  if (w.twq) cudaFree(w.twq);
  w.spec = nullptr;
  w.partials = nullptr;
  w.twq = nullptr;
}

// y / z passes with the projection (3D) or the y pass with the projection
// (2D), between the x-forward and the x-inverse passes.
template <typename R>
static cudaError_t spectral_middle(const GridDesc& g, SpecWork<R>& w, cudaStream_t st, long long* nlp,
                                   bool skip_yfwd = false, bool skip_yinv = false) {
  using C = Cx<R>;
  constexpr bool F32 = std::is_same<R, float>::value;
  long long nl = 0;
  cudaError_t e;
  if (g.ndim == 3) {
    const dim3 yg((g.nxh + w.ty - 1) / w.ty, g.nz, g.ncomp);
    const size_t ysm = (size_t)w.ty * g.ny * sizeof(C);
    const dim3 zg((g.nxh + w.tz - 1) / w.tz, g.ny);
    const size_t zsm = (size_t)g.ncomp * w.tz * g.nz * sizeof(C);
    for (int pass = 0; pass < 3; ++pass) {
      if ((pass == 0 && skip_yfwd) || (pass == 2 && skip_yinv)) continue;  // done by the cluster x+y passes
      e = cudaErrorNotSupported;
      PassScope ps(w.timer, st, pass == 0 ? PASS_YFWD : (pass == 1 ? PASS_ZPROJ : PASS_YINV));
      if constexpr (F32) {
        if (!w.generic && pass != 1 && fast_size(g.ny)) e = fast_ycols(g, w.spec, w.tw[1], pass == 2, st);
        if (!w.generic && pass == 1 && fast_size(g.nz)) e = fast_zproj(g, w.spec, w, st);
      }
      if (e == cudaErrorNotSupported) {
        if (pass == 0) k_ycols<R, false><<<yg, kYThreads, ysm, st>>>(w.spec, g, w.ty, w.py, w.tw[1]);
        else if (pass == 2) k_ycols<R, true><<<yg, kYThreads, ysm, st>>>(w.spec, g, w.ty, w.py, w.tw[1]);
        else
          k_zproj<R><<<zg, kZThreads, zsm, st>>>(w.spec, g, w.tz, w.pz, w.tw[2], w.gdiff[0], w.gavg[0],
                                                 w.gdiff[1], w.gavg[1], w.gdiff[2], w.gavg[2], w.free_mask);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) return e;
      ++nl;
    }
  } else {
    e = cudaErrorNotSupported;
    PassScope ps(w.timer, st, PASS_YPROJ2D);
    if constexpr (F32) {
      if (!w.generic && fast_size(g.ny)) e = fast_yproj2d(g, w.spec, w, st);
    }
    if (e == cudaErrorNotSupported) {
      const dim3 pg((g.nxh + w.tz - 1) / w.tz);
      const size_t psm = (size_t)g.ncomp * w.tz * g.ny * sizeof(C);
      k_yproj2d<R><<<pg, kYThreads, psm, st>>>(w.spec, g, w.tz, w.py, w.tw[1], w.gdiff[0], w.gavg[0], w.gdiff[1],
                                               w.gavg[1], w.free_mask);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    ++nl;
  }
  *nlp += nl;
  return cudaSuccess;
}

// the cluster x+y passes were asked for and apply (3D FP32, Nx = Ny of a
// cluster length)
template <typename R>
static bool use_cluster(const GridDesc& g, const SpecWork<R>& w) {
  return std::is_same<R, float>::value && w.cluster && !w.generic && w.twq != nullptr && cluster_size_ok(g);
}

template <typename R>
cudaError_t spectral_apply(const GridDesc& g, SpecWork<R>& w, const MatTable<R>& mt, const R* in,
                           const uint8_t* phase, const R* damage, XIn mode, R* out,
                           const R* dot_with, double* dot_out, cudaStream_t st, long long* nlaunch) {
  using C = Cx<R>;
  constexpr bool F32 = std::is_same<R, float>::value;
  long long nl = 0;
  cudaError_t e;
  const int xblocks = (int)((g.nrows + w.qx - 1) / w.qx);
  const size_t xsm = (size_t)((g.ncomp * w.qx) / 2) * g.nx * sizeof(C);
  // dot(in, G:B:in) for a compatible input (in = G:in, as every CG direction
  // is) equals dot(in, B:in): the compiled x-forward pass forms it from the
  // tangent it already computes, so the x-inverse need not read `in` again
  bool fwd_dot = false;
  int fwd_blocks = 0;
  // the cluster passes take the x and y transforms together (not the
  // consistent tangent's forward pass)
  const bool cl = use_cluster(g, w);
  const bool cl_fwd = cl && !(mode == XIn::Tangent && w.cons.dp != nullptr);
  // x forward (tangent fused)
  e = cudaErrorNotSupported;
  {
  PassScope ps(w.timer, st, PASS_XFWD);
  if constexpr (F32) {
    if (cl_fwd) {
      const bool want = mode == XIn::Tangent && dot_with != nullptr && dot_with == in && !w.unfused;
      e = cluster_xyfwd(g, in, phase, damage, mt, w.spec, w.tw[0], w.twq, mode == XIn::Tangent,
                        want ? w.partials : nullptr, st);
      fwd_blocks = cluster_blocks(g);
      fwd_dot = want && e == cudaSuccess;
    } else if (!w.generic && fast_size(g.nx)) {
      const bool want = mode == XIn::Tangent && dot_with != nullptr && dot_with == in && !w.unfused;
      if (!(mode == XIn::Tangent && w.cons.dp != nullptr))
        e = tma_xfwd(g, in, phase, damage, mt, w.spec, w.tw[0], mode == XIn::Tangent, want ? w.partials : nullptr,
                     &fwd_blocks, st, w.wait_err);
      if (e == cudaErrorNotSupported)
        e = fast_xfwd(g, in, phase, damage, mt, w.spec, w.tw[0], mode == XIn::Tangent, want ? w.partials : nullptr,
                      &fwd_blocks, st, &w.cons);
      fwd_dot = want && e == cudaSuccess;
    }
  }
  if (e == cudaErrorNotSupported) {
    if (mode == XIn::Tangent)
      k_xfwd<R, 1><<<xblocks, kXThreads, xsm, st>>>(in, phase, damage, mt, w.spec, g, w.qx, w.px, w.tw[0], w.cons);
    else
      k_xfwd<R, 0><<<xblocks, kXThreads, xsm, st>>>(in, phase, damage, mt, w.spec, g, w.qx, w.px, w.tw[0],
                                                    ConsTan<R>{});
    e = cudaGetLastError();
  }
  }
  if (e != cudaSuccess) return e;
  ++nl;
  if ((e = spectral_middle<R>(g, w, st, &nl, cl_fwd, cl)) != cudaSuccess) return e;
  const R scale = (R)(1.0 / (double)g.nvox);
  const bool dot = dot_with != nullptr && !fwd_dot;
  const bool self = dot && (dot_with == out);
  int nblocks = xblocks;
  e = cudaErrorNotSupported;
  {
  PassScope ps(w.timer, st, PASS_XINV);
  if constexpr (F32) {
    if (cl) {
      e = cluster_yxinv(g, w.spec, out, self ? nullptr : dot_with, w.partials, w.tw[0], w.twq, dot, self, st);
      nblocks = cluster_blocks(g);
    } else if (!w.generic && fast_size(g.nx)) {
      e = fast_xinv(g, w.spec, out, self ? nullptr : dot_with, w.partials, w.tw[0], dot, self, &nblocks, st);
    }
  }
  if (e == cudaErrorNotSupported) {
    nblocks = xblocks;
    if (dot)
      k_xinv<R, true><<<xblocks, kXThreads, xsm, st>>>(w.spec, out, self ? nullptr : dot_with, w.partials, g, w.qx,
                                                       w.px, w.tw[0], scale, self);
    else
      k_xinv<R, false><<<xblocks, kXThreads, xsm, st>>>(w.spec, out, nullptr, nullptr, g, w.qx, w.px, w.tw[0],
                                                        scale, false);
    e = cudaGetLastError();
  }
  }
  if (e != cudaSuccess) return e;
  ++nl;
  if (dot || fwd_dot) {
    e = reduce_partials(w.partials, fwd_dot ? fwd_blocks : nblocks, 1, dot_out, st, &nl);
    if (e != cudaSuccess) return e;
  }
  if (nlaunch) *nlaunch += nl;
  return cudaSuccess;
}

// Single-block launches (256 threads): a CG pass's block sums reduced into
// the device scalars, then the scalar step of Algorithm 1 that needs them.
__global__ void __launch_bounds__(256) k_reduce_alpha(const double* __restrict__ part, int nb, DevScalars* S) {
  __shared__ double sh[32];
  block_reduce_partials<1>(part, nb, &S->dHd, sh);
  if (threadIdx.x == 0) cg_alpha_scalars(S);
}

__global__ void __launch_bounds__(256) k_reduce_beta(const double* __restrict__ part, int nb, DevScalars* S) {
  __shared__ double sh[3 * 32];
  block_reduce_partials<3>(part, nb, &S->rr_new, sh);
  if (threadIdx.x == 0) cg_beta_scalars(S);
}

cudaError_t spectral_hv_cg(const GridDesc& g, SpecWork<float>& w, const MatTable<float>& mt, const float* d,
                           const uint8_t* phase, const float* damage, float* z, float* r, DevScalars* S,
                           cudaStream_t st, long long* nlaunch) {
  if (w.generic || w.unfused || !fast_size(g.nx)) return cudaErrorNotSupported;
  long long nl = 0;
  cudaError_t e;
  int fb = 0, ib = 0;
  const bool cl = use_cluster(g, w), cl_fwd = cl && w.cons.dp == nullptr;
  bool fwd_reduced = false;  // d:H:d and the step length done by the x-forward launch
  {
    PassScope ps(w.timer, st, PASS_XFWD);
    if (cl_fwd) {
      e = cluster_xyfwd(g, d, phase, damage, mt, w.spec, w.tw[0], w.twq, true, w.partials, st);
      fb = cluster_blocks(g);
    } else {
      e = w.cons.dp == nullptr ? tma_xfwd(g, d, phase, damage, mt, w.spec, w.tw[0], true, w.partials, &fb, st,
                                          w.wait_err, S)
                               : cudaErrorNotSupported;
      fwd_reduced = e == cudaSuccess;
      if (e == cudaErrorNotSupported)
        e = fast_xfwd(g, d, phase, damage, mt, w.spec, w.tw[0], true, w.partials, &fb, st, &w.cons);
    }
  }
  if (e != cudaSuccess) return e;
  ++nl;
  if (!fwd_reduced) {
    k_reduce_alpha<<<1, 256, 0, st>>>(w.partials, fb, S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++nl;
  }
  if ((e = spectral_middle<float>(g, w, st, &nl, cl_fwd, cl)) != cudaSuccess) return e;
  {
    PassScope ps(w.timer, st, PASS_XINV);
    if (cl) {
      e = cluster_yxinv_cg(g, w.spec, z, r, d, &S->status, &S->alpha, &S->tau, w.partials, w.tw[0], w.twq, st);
      ib = cluster_blocks(g);
    } else {
      e = fast_xinv_cg(g, w.spec, z, r, d, &S->status, &S->alpha, &S->tau, w.partials, w.tw[0], &ib, st);
    }
  }
  if (e != cudaSuccess) return e;
  ++nl;
  k_reduce_beta<<<1, 256, 0, st>>>(w.partials, ib, S);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ++nl;
  if (nlaunch) *nlaunch += nl;
  return cudaSuccess;
}

template cudaError_t spectral_setup<float>(const GridDesc&, SpecWork<float>&);
template cudaError_t spectral_setup<double>(const GridDesc&, SpecWork<double>&);
template cudaError_t spectral_plan<float>(const GridDesc&, SpecWork<float>&);
template void spectral_free<float>(SpecWork<float>&);
template void spectral_free<double>(SpecWork<double>&);
template cudaError_t spectral_apply<float>(const GridDesc&, SpecWork<float>&, const MatTable<float>&, const float*,
                                           const uint8_t*, const float*, XIn, float*, const float*, double*,
                                           cudaStream_t, long long*);
template cudaError_t spectral_apply<double>(const GridDesc&, SpecWork<double>&, const MatTable<double>&,
                                            const double*, const uint8_t*, const double*, XIn, double*,
                                            const double*, double*, cudaStream_t, long long*);

}  // namespace rve
