// FP32 spectral passes specialised at compile time for the common axis
// lengths (powers of two from 32 to 512 and 3 * 2^k up to 384).  Same data
// layout and the same arithmetic as the generic passes in hv_passes.cu;
// only the FFT engine (fft_fast.cuh) and the staging differ: global loads
// are batched in registers before they are written to shared memory, and
// the x passes give consecutive threads consecutive x so that the
// line-interleaved shared-memory accesses stay (nearly) conflict free.
#include "hv_fast.cuh"
#include "hv_tiles.cuh"
#include "project.cuh"

namespace rve {

// MODE 0: plain; 1: secant tangent; 2: symmetric consistent tangent (the
// secant plus the rank-one correction of ConsTan on loading voxels).
template <int N, int NC, int MODE>
__global__ void __launch_bounds__(kFT)
    kf_xfwd(const float* __restrict__ in, const uint8_t* __restrict__ phase, const float* __restrict__ dmg,
            const MatTable<float> mt, float2* __restrict__ spec, const long long nrows, const long long nvox,
            const float2* __restrict__ tw, double* __restrict__ partials, const float* __restrict__ cdp = nullptr,
            const float* __restrict__ ca = nullptr, const float* __restrict__ cn = nullptr) {
  constexpr int Q = xq<N, NC>();
  __shared__ __align__(16) float2 buf[NC * Q / 2 * N];
  __shared__ double red[32];
  const long long row0 = (long long)blockIdx.x * Q;
  const float acc = xfwd_rows<N, NC, MODE>(buf, in, phase, dmg, mt, spec, nrows, nvox, tw, row0, nrows, cdp, ca, cn);
  if (MODE >= 1 && partials) {
    double val[1] = {(double)acc};
    block_sum<1>(val, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = val[0];
  }
}

template <int N, int NC, bool DOT, bool CG = false>
__global__ void __launch_bounds__(kFT, 4)
    kf_xinv(const float2* __restrict__ spec, float* __restrict__ out, const float* __restrict__ dotw,
            double* __restrict__ partials, const long long nrows, const long long nvox,
            const float2* __restrict__ tw, const float scale, const bool self_dot, float* __restrict__ cz = nullptr,
            float* __restrict__ cr = nullptr, const float* __restrict__ cd = nullptr,
            const int* __restrict__ cstatus = nullptr, const double* __restrict__ calpha = nullptr,
            const double* __restrict__ ctau = nullptr) {
  constexpr int Q = xq<N, NC>();
  __shared__ __align__(16) float2 buf[NC * Q / 2 * N];
  __shared__ double red[3 * 32];
  const long long row0 = (long long)blockIdx.x * Q;
  xinv_rows<N, NC, DOT, CG, false>(buf, red, spec, out, dotw, partials, nrows, nvox, tw, scale, self_dot, cz, cr, cd,
                                   cstatus, calpha, ctau, row0, nrows, blockIdx.x);
}

template <int N, bool INV>
__global__ void __launch_bounds__(kFT)
    kf_ycols(float2* __restrict__ spec, const int nz, const int nxh, const float2* __restrict__ tw) {
  constexpr int TX = ytx<N>();
  __shared__ __align__(16) float2 buf[TX * N];
  ycols_tile<N, INV, false>(buf, spec, ((long long)blockIdx.z * nz + blockIdx.y) * N, blockIdx.x * TX, nxh, tw);
}

// ------------------------------------------------- z + projection (3D)
template <int N>
__global__ void __launch_bounds__(zthreads<N>(), zminblocks<N>())
    kf_zproj(float2* __restrict__ spec, const int ny, const int nxh, const float2* __restrict__ tw,
             const float2* __restrict__ gdx, const float2* __restrict__ gax, const float2* __restrict__ gdy,
             const float2* __restrict__ gay, const float2* __restrict__ gdz, const float2* __restrict__ gaz,
             const unsigned free_mask) {
  constexpr int TX = ztx<N>();
  constexpr int NL = 6 * TX;
  constexpr int NT = zthreads<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const int kx0 = blockIdx.x * TX, ky = blockIdx.y;
  const int tv = min(TX, nxh - kx0);
  // line l = c * TX + t: component c, column kx0 + t
  auto load = [&](int l, int z) -> float2 {
    const int c = l / TX, t = l - (l / TX) * TX;
    return t < tv ? spec[(((long long)c * N + z) * ny + ky) * nxh + kx0 + t] : make_float2(0.f, 0.f);
  };
  auto store = [&](int l, int z, float2 v) {
    const int c = l / TX, t = l - (l / TX) * TX;
    if (t < tv) spec[(((long long)c * N + z) * ny + ky) * nxh + kx0 + t] = v;
  };
  // The first forward stage reads straight from global memory and the last
  // inverse stage writes straight back, where a thread's butterflies fit in
  // registers (at most 24 complex values); otherwise the tile is staged
  // through shared memory.
  constexpr int R0 = fft_radix(N, 0);
  constexpr bool DIRECT = ((NL * (N / R0) + NT - 1) / NT) * R0 <= 24;
  if constexpr (DIRECT) {
    fft_stage0_from<N, NL, NT, false>(buf, load);
    fft_ct_range<N, NL, NT, false, 1, fft_nstages(N)>(buf, tw);
  } else {
    constexpr int STEPS = (N * NL + NT - 1) / NT;
    constexpr int LB = STEPS < 8 ? STEPS : 8;
    for (int s0 = 0; s0 < STEPS; s0 += LB) {
      float2 tmp[LB];
#pragma unroll
      for (int b = 0; b < LB; ++b) {
        const int idx = threadIdx.x + (s0 + b) * NT;
        tmp[b] = (s0 + b < STEPS && idx < N * NL) ? load(idx - (idx / NL) * NL, idx / NL) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int b = 0; b < LB; ++b) {
        const int idx = threadIdx.x + (s0 + b) * NT;
        if (s0 + b < STEPS && idx < N * NL) buf[idx] = tmp[b];
      }
    }
    __syncthreads();
    fft_ct<N, NL, NT, false>(buf, tw);
  }
  // every point of a thread has the same column t (NT is a multiple of TX):
  // the x and y factors of the symbol are formed once
  static_assert(NT % TX == 0, "z-pass threads must be a multiple of its columns");
  const int t = threadIdx.x % TX, kx = kx0 + t;
  if (t < tv) {
    const float2 ay = gay[ky], dy = gdy[ky], ax = gax[kx], dx = gdx[kx];
    const float2 fx = cmul(dx, ay), fy = cmul(ax, dy), fz = cmul(ax, ay);
    const bool kxy0 = kx == 0 && ky == 0;
    for (int z = threadIdx.x / TX; z < N; z += NT / TX) {
      float2 m[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) m[c] = buf[z * NL + c * TX + t];
      const float2 az = gaz[z];
      project3<float>(m, cmul(fx, az), cmul(fy, az), cmul(fz, gdz[z]), kxy0 && z == 0, free_mask);
#pragma unroll
      for (int c = 0; c < 6; ++c) buf[z * NL + c * TX + t] = m[c];
    }
  }
  __syncthreads();
  // inverse z transform
  if constexpr (DIRECT) {
    fft_ct_range<N, NL, NT, true, 0, fft_nstages(N) - 1>(buf, tw);
    fft_stage_last_to<N, NL, NT, true>(buf, tw, store);
  } else {
    fft_ct<N, NL, NT, true>(buf, tw);
    for (int idx = threadIdx.x; idx < N * NL; idx += NT) store(idx - (idx / NL) * NL, idx / NL, buf[idx]);
  }
}

// ------------------------------------------------- y + projection (2D)
// NCL = 3: one element per pixel (Mandel components); NCL = 6: the two Kuhn
// triangles of every pixel (lines c * 2 + q).
template <int N, int NCL> constexpr int p2tx_l() {
  return (kFBudget / (NCL * N)) < 16 ? ((kFBudget / (NCL * N)) < 1 ? 1 : kFBudget / (NCL * N)) : 16;
}

template <int N, int NCL>
__global__ void __launch_bounds__(kFT)
    kf_yproj2d(float2* __restrict__ spec, const int nxh, const float2* __restrict__ tw,
               const float2* __restrict__ gdx, const float2* __restrict__ gax, const float2* __restrict__ gdy,
               const float2* __restrict__ gay, const unsigned free_mask) {
  constexpr int TX = p2tx_l<N, NCL>();
  constexpr int NL = NCL * TX;
  __shared__ __align__(16) float2 buf[N * NL];
  const int kx0 = blockIdx.x * TX;
  const int tv = min(TX, nxh - kx0);
  for (int idx = threadIdx.x; idx < N * NL; idx += kFT) {
    const int y = idx / NL, rem = idx - (idx / NL) * NL;
    const int c = rem / TX, t = rem - (rem / TX) * TX;
    buf[idx] = t < tv ? spec[((long long)c * N + y) * nxh + kx0 + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_ct<N, NL, kFT, false>(buf, tw);
  for (int pt = threadIdx.x; pt < N * TX; pt += kFT) {
    const int y = pt / TX, t = pt - (pt / TX) * TX;
    const int kx = kx0 + t;
    if (t >= tv) continue;
    float2 m[NCL];
#pragma unroll
    for (int c = 0; c < NCL; ++c) m[c] = buf[y * NL + c * TX + t];
    if constexpr (NCL == 3) {
      project2<float>(m, cmul(gdx[kx], gay[y]), cmul(gax[kx], gdy[y]), kx == 0 && y == 0, free_mask);
    } else {
      const float2 dx = gdx[kx], dy = gdy[y];
      project_simplex2<float>(m, make_float2(1.f + dx.x, dx.y), dx, make_float2(1.f + dy.x, dy.y), dy,
                              kx == 0 && y == 0, free_mask);
    }
#pragma unroll
    for (int c = 0; c < NCL; ++c) buf[y * NL + c * TX + t] = m[c];
  }
  __syncthreads();
  fft_ct<N, NL, kFT, true>(buf, tw);
  for (int idx = threadIdx.x; idx < N * NL; idx += kFT) {
    const int y = idx / NL, rem = idx - (idx / NL) * NL;
    const int c = rem / TX, t = rem - (rem / TX) * TX;
    if (t < tv) spec[((long long)c * N + y) * nxh + kx0 + t] = buf[idx];
  }
}

// ================================================================ dispatch
#define RVE_FAST_SIZES(X) X(32) X(64) X(128) X(256) X(512) X(96) X(192) X(384)

bool fast_size(int n) {
#define RVE_CASE(n_) if (n == n_) return true;
  RVE_FAST_SIZES(RVE_CASE)
#undef RVE_CASE
  return false;
}

template <int N>
static cudaError_t xfwd_n(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                          const MatTable<float>& mt, float2* spec, const float2* tw, bool tangent, double* partials,
                          int* nblocks, cudaStream_t st, const ConsTan<float>* ct) {
  double* pd = tangent ? partials : nullptr;
  const bool cons = tangent && ct && ct->dp;
  if (g.ncomp == 6) {
    constexpr int Q = xq<N, 6>();
    const int blocks = (int)((g.nrows + Q - 1) / Q);
    *nblocks = blocks;
    if (tangent && g.nq == 2)
      kf_xfwd<N, 6, 3><<<blocks, kFT, 0, st>>>(in, phase, dmg, mt, spec, g.nrows, g.nvox, tw, pd);
    else if (cons)
      kf_xfwd<N, 6, 2><<<blocks, kFT, 0, st>>>(in, phase, dmg, mt, spec, g.nrows, g.nvox, tw, pd, ct->dp, ct->a,
                                                ct->n);
    else if (tangent) kf_xfwd<N, 6, 1><<<blocks, kFT, 0, st>>>(in, phase, dmg, mt, spec, g.nrows, g.nvox, tw, pd);
    else kf_xfwd<N, 6, 0><<<blocks, kFT, 0, st>>>(in, phase, dmg, mt, spec, g.nrows, g.nvox, tw, nullptr);
  } else {
    constexpr int Q = xq<N, 3>();
    const int blocks = (int)((g.nrows + Q - 1) / Q);
    *nblocks = blocks;
    if (cons)
      kf_xfwd<N, 3, 2><<<blocks, kFT, 0, st>>>(in, phase, dmg, mt, spec, g.nrows, g.nvox, tw, pd, ct->dp, ct->a,
                                                ct->n);
    else if (tangent) kf_xfwd<N, 3, 1><<<blocks, kFT, 0, st>>>(in, phase, dmg, mt, spec, g.nrows, g.nvox, tw, pd);
    else kf_xfwd<N, 3, 0><<<blocks, kFT, 0, st>>>(in, phase, dmg, mt, spec, g.nrows, g.nvox, tw, nullptr);
  }
  return cudaGetLastError();
}

template <int N>
static cudaError_t xinv_n(const GridDesc& g, const float2* spec, float* out, const float* dotw, double* partials,
                          const float2* tw, bool dot, bool self, int* nblocks, cudaStream_t st) {
  const float scale = (float)(1.0 / (double)g.nvox);
  if (g.ncomp == 6) {
    constexpr int Q = xq<N, 6>();
    const int blocks = (int)((g.nrows + Q - 1) / Q);
    *nblocks = blocks;
    if (dot) kf_xinv<N, 6, true><<<blocks, kFT, 0, st>>>(spec, out, dotw, partials, g.nrows, g.nvox, tw, scale, self);
    else kf_xinv<N, 6, false><<<blocks, kFT, 0, st>>>(spec, out, dotw, partials, g.nrows, g.nvox, tw, scale, self);
  } else {
    constexpr int Q = xq<N, 3>();
    const int blocks = (int)((g.nrows + Q - 1) / Q);
    *nblocks = blocks;
    if (dot) kf_xinv<N, 3, true><<<blocks, kFT, 0, st>>>(spec, out, dotw, partials, g.nrows, g.nvox, tw, scale, self);
    else kf_xinv<N, 3, false><<<blocks, kFT, 0, st>>>(spec, out, dotw, partials, g.nrows, g.nvox, tw, scale, self);
  }
  return cudaGetLastError();
}

template <int N>
static cudaError_t ycols_n(const GridDesc& g, float2* spec, const float2* tw, bool inv, cudaStream_t st) {
  constexpr int TX = ytx<N>();
  const dim3 grid((g.nxh + TX - 1) / TX, g.nz, g.ncomp);
  if (inv) kf_ycols<N, true><<<grid, kFT, 0, st>>>(spec, g.nz, g.nxh, tw);
  else kf_ycols<N, false><<<grid, kFT, 0, st>>>(spec, g.nz, g.nxh, tw);
  return cudaGetLastError();
}

template <int N>
static cudaError_t zproj_n(const GridDesc& g, float2* spec, const SpecWork<float>& w, cudaStream_t st) {
  constexpr int TX = ztx<N>();
  const size_t smem = (size_t)N * 6 * TX * sizeof(float2);
  // the attribute is per device: set it once on every device that runs the pass
  constexpr int kDevs = 64;
  static bool attr[kDevs] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kDevs || !attr[dev]) {
    e = cudaFuncSetAttribute(kf_zproj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kDevs) attr[dev] = true;
  }
  const dim3 grid((g.nxh + TX - 1) / TX, g.ny);
  kf_zproj<N><<<grid, zthreads<N>(), smem, st>>>(spec, g.ny, g.nxh, w.tw[2], w.gdiff[0], w.gavg[0], w.gdiff[1],
                                                  w.gavg[1], w.gdiff[2], w.gavg[2], w.free_mask);
  return cudaGetLastError();
}

template <int N>
static cudaError_t yproj2d_n(const GridDesc& g, float2* spec, const SpecWork<float>& w, cudaStream_t st) {
  if (g.ncomp == 6) {
    constexpr int TX = p2tx_l<N, 6>();
    kf_yproj2d<N, 6><<<(g.nxh + TX - 1) / TX, kFT, 0, st>>>(spec, g.nxh, w.tw[1], w.gdiff[0], w.gavg[0],
                                                             w.gdiff[1], w.gavg[1], w.free_mask);
  } else {
    constexpr int TX = p2tx_l<N, 3>();
    kf_yproj2d<N, 3><<<(g.nxh + TX - 1) / TX, kFT, 0, st>>>(spec, g.nxh, w.tw[1], w.gdiff[0], w.gavg[0],
                                                             w.gdiff[1], w.gavg[1], w.free_mask);
  }
  return cudaGetLastError();
}

cudaError_t fast_xfwd(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                      const MatTable<float>& mt, float2* spec, const float2* tw, bool tangent, double* partials,
                      int* nblocks, cudaStream_t st, const ConsTan<float>* ct) {
#define RVE_CASE(n_) \
  if (g.nx == n_) return xfwd_n<n_>(g, in, phase, dmg, mt, spec, tw, tangent, partials, nblocks, st, ct);
  RVE_FAST_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

cudaError_t fast_xinv(const GridDesc& g, const float2* spec, float* out, const float* dotw, double* partials,
                      const float2* tw, bool dot, bool self, int* nblocks, cudaStream_t st) {
#define RVE_CASE(n_) \
  if (g.nx == n_) return xinv_n<n_>(g, spec, out, dotw, partials, tw, dot, self, nblocks, st);
  RVE_FAST_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

template <int N>
static cudaError_t xinv_cg_n(const GridDesc& g, const float2* spec, float* z, float* r, const float* d,
                             const int* status, const double* alpha, const double* tau, double* partials,
                             const float2* tw, int* nblocks, cudaStream_t st) {
  const float scale = (float)(1.0 / (double)g.nvox);
  if (g.ncomp == 6) {
    constexpr int Q = xq<N, 6>();
    const int blocks = (int)((g.nrows + Q - 1) / Q);
    *nblocks = blocks;
    kf_xinv<N, 6, false, true><<<blocks, kFT, 0, st>>>(spec, nullptr, nullptr, partials, g.nrows, g.nvox, tw, scale,
                                                       false, z, r, d, status, alpha, tau);
  } else {
    constexpr int Q = xq<N, 3>();
    const int blocks = (int)((g.nrows + Q - 1) / Q);
    *nblocks = blocks;
    kf_xinv<N, 3, false, true><<<blocks, kFT, 0, st>>>(spec, nullptr, nullptr, partials, g.nrows, g.nvox, tw, scale,
                                                       false, z, r, d, status, alpha, tau);
  }
  return cudaGetLastError();
}

cudaError_t fast_xinv_cg(const GridDesc& g, const float2* spec, float* z, float* r, const float* d, const int* status,
                         const double* alpha, const double* tau, double* partials, const float2* tw, int* nblocks,
                         cudaStream_t st) {
#define RVE_CASE(n_) \
  if (g.nx == n_) return xinv_cg_n<n_>(g, spec, z, r, d, status, alpha, tau, partials, tw, nblocks, st);
  RVE_FAST_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

cudaError_t fast_ycols(const GridDesc& g, float2* spec, const float2* tw, bool inv, cudaStream_t st) {
#define RVE_CASE(n_) \
  if (g.ny == n_) return ycols_n<n_>(g, spec, tw, inv, st);
  RVE_FAST_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

cudaError_t fast_zproj(const GridDesc& g, float2* spec, const SpecWork<float>& w, cudaStream_t st) {
#define RVE_CASE(n_) \
  if (g.nz == n_) return zproj_n<n_>(g, spec, w, st);
  RVE_FAST_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

cudaError_t fast_yproj2d(const GridDesc& g, float2* spec, const SpecWork<float>& w, cudaStream_t st) {
#define RVE_CASE(n_) \
  if (g.ny == n_) return yproj2d_n<n_>(g, spec, w, st);
  RVE_FAST_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

}  // namespace rve
