// The x and y transforms of the 3D product in one pass per direction,
// through thread-block clusters (FP32, Nx = Ny = N, compiled lengths up to
// 256).  The five-pass product (x, y, z + projection, y, x) writes and reads
// the spectrum between the x and y passes; here one cluster of kCR CTAs
// owns one component c of one z-plane -- its N x N real values forward, its
// N x (N/2 + 1) half spectrum backward -- and the y transform never leaves
// the chip:
//
//   forward  CTA r takes the rows y = r + kCR m (m < M = N / kCR): tangent
//            on load, x FFT of the rows (packed in pairs), then the M-point
//            FFT over m of every column kx (Y_r).  After a cluster barrier
//            CTA q reads Y_0..Y_{kCR-1} at its own quarter of k2 from the
//            other CTAs' shared memory and finishes the transform with one
//            kCR-point DFT:  X[k2 + M k1] = sum_r w_kCR^{r k1} w_N^{r k2} Y_r[k2]
//            (four-step split of the N-point DFT), stored to the spectrum.
//   inverse  CTA q reads the rows k2 + M k1 of its quarter of k2, takes
//            the inverse kCR-point DFT over k1, multiplies by w_N^{-r k2}
//            and stores the r-th result into CTA r's shared memory; after a
//            cluster barrier every CTA runs the inverse M-point FFT over k2
//            (giving its rows y = r + kCR m) and the inverse x FFT with the
//            output epilogue (plain store, dot product or the fused
//            Steihaug-CG update of the x-inverse pass).
//
// Sec. 2.1 / Eq. (5): the same G : zeta = F^-1 Ghat F as the five-pass
// product; the z pass with the projection in between is unchanged.  Tile
// bodies, the FFT engine and the spectrum layout are those of hv_tiles.cuh.
// The tangent is applied per component: sigma_c = (1 - D) (2 mu eps_c +
// lambda tr(eps) [c < 3]), so the clusters of the three normal components
// also read eps_0..2 (L2 hits: the six clusters of a plane are consecutive
// in the launch).
#include "hv_cluster.cuh"
#include "hv_tiles.cuh"

namespace rve {

constexpr int kCR = 4;  // CTAs per cluster (portable size)

// ----------------------------------------------------- cluster primitives
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster arrives (release) and waits
// (acquire): shared-memory writes before it are visible cluster-wide after
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cl_map(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 cl_ld(unsigned a) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ void cl_st(unsigned a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y));
}

// packed line pairs per x batch: a divisor of M/2 within the block budget
template <int N> constexpr int cl_nlb_from(int d) {
  return (d <= 1) ? 1 : ((((N / kCR) / 2) % d == 0 && d <= kFBudget / N) ? d : cl_nlb_from<N>(d - 1));
}
template <int N> constexpr int cl_nlb() { return cl_nlb_from<N>((N / kCR) / 2); }
template <int N> constexpr size_t cl_smem() {
  return (size_t)(N / kCR) * (N / 2 + 1) * sizeof(float2) + (size_t)N * (cl_nlb<N>() + 1) * sizeof(float2);
}

// ------------------------------------------------------------- forward
// MODE 0: plain; 1: secant tangent, with the block's share of
// in : (tangent : in) in partials[blockIdx.x] when partials is set.
template <int N, int MODE>
__global__ void __cluster_dims__(kCR, 1, 1) __launch_bounds__(kFT, 2)
    kc_xyfwd(const float* __restrict__ in, const uint8_t* __restrict__ phase, const float* __restrict__ dmg,
             const MatTable<float> mt, float2* __restrict__ spec, const int nz, const long long nvox,
             const float2* __restrict__ twn, const float2* __restrict__ twm, double* __restrict__ partials) {
  constexpr int M = N / kCR, NXH = N / 2 + 1, LY = NXH;
  constexpr int NLB = cl_nlb<N>(), BR = 2 * NLB, NBT = M / BR;
  constexpr int NLW = NLB + 1;  // odd line stride of the x batch: consecutive x on distinct banks
  constexpr int K2 = M / kCR;  // frequencies k2 finished by each CTA
  static_assert(M % BR == 0 && M % kCR == 0, "cluster split");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* yb = reinterpret_cast<float2*>(smem_raw);  // element m of column kx at m * LY + kx
  float2* wb = yb + M * LY;                          // x batch: element x of line p at x * NLW + p
  __shared__ double red[32];
  const int r = (int)cl_rank();
  const int cid = blockIdx.x / kCR, c = cid % 6, z = cid / 6;
  const long long pvox = (long long)z * N * N;
  float acc = 0.f;
  for (int bt = 0; bt < NBT; ++bt) {
    if (bt > 0) __syncthreads();  // the previous batch's separation has read wb
    // rows i of the batch: y = r + kCR (bt BR + i); consecutive threads take
    // consecutive x
    constexpr int ITEMS = BR * N, STEPS = (ITEMS + kFT - 1) / kFT, BATCH = STEPS < 4 ? STEPS : 4;
    for (int s0 = 0; s0 < STEPS; s0 += BATCH) {
      float v[BATCH];
#pragma unroll
      for (int b = 0; b < BATCH; ++b) {
        const int idx = threadIdx.x + (s0 + b) * kFT;
        const bool ok = s0 + b < STEPS && idx < ITEMS;
        const int i = idx / N, x = idx - (idx / N) * N;
        const long long vox = pvox + (long long)(r + kCR * (bt * BR + i)) * N + x;
        float e = ok ? __ldg(in + c * nvox + vox) : 0.f;
        if (MODE == 1 && ok) {
          const float keep = 1.f - __ldg(dmg + vox);
          const int ph = __ldg(phase + vox);
          float sg = 2.f * mt.mu[ph] * keep * e;
          if (c < 3) sg += mt.lam[ph] * keep * (__ldg(in + vox) + __ldg(in + nvox + vox) + __ldg(in + 2 * nvox + vox));
          acc += e * sg;
          e = sg;
        }
        v[b] = e;
      }
#pragma unroll
      for (int b = 0; b < BATCH; ++b) {
        const int idx = threadIdx.x + (s0 + b) * kFT;
        if (s0 + b < STEPS && idx < ITEMS) {
          const int i = idx / N, x = idx - (idx / N) * N;
          reinterpret_cast<float*>(&wb[x * NLW + (i >> 1)])[i & 1] = v[b];
        }
      }
    }
    __syncthreads();
    fft_ct<N, NLW, kFT, false>(wb, twn);
    // separate the two real rows of every packed line (Hermitian symmetry):
    // thread t takes bin k = t mod (N/2) of the lines t div (N/2) + j GB;
    // the Nyquist bins go to threads 0 .. NLB-1
    constexpr int KB = N / 2, GB = kFT / KB, JB = (NLB + GB - 1) / GB;
    const int g = threadIdx.x / KB, k = threadIdx.x - (threadIdx.x / KB) * KB;
    const int km = k == 0 ? 0 : N - k;
    if (g < GB) {
#pragma unroll
      for (int j = 0; j < JB; ++j) {
        const int p = g + j * GB;
        if (JB * GB == NLB || p < NLB) {
          const float2 zk = wb[k * NLW + p], zm = wb[km * NLW + p];
          const int m0 = bt * BR + 2 * p;
          yb[m0 * LY + k] = make_float2((zk.x + zm.x) * 0.5f, (zk.y - zm.y) * 0.5f);
          yb[(m0 + 1) * LY + k] = make_float2((zk.y + zm.y) * 0.5f, (zm.x - zk.x) * 0.5f);
        }
      }
    }
    if (threadIdx.x < NLB) {
      const int p = threadIdx.x;
      const float2 zn = wb[KB * NLW + p];
      const int m0 = bt * BR + 2 * p;
      yb[m0 * LY + KB] = make_float2(zn.x, 0.f);
      yb[(m0 + 1) * LY + KB] = make_float2(zn.y, 0.f);
    }
  }
  __syncthreads();
  // Y_r: M-point FFT over m of every column
  fft_ct<M, LY, kFT, false>(yb, twm);
  cl_sync();
  // X[k2 + M k1] for this CTA's k2 from the four CTAs' Y
  unsigned rb[kCR];
#pragma unroll
  for (int q = 0; q < kCR; ++q) rb[q] = cl_map(yb, q);
  float2* out = spec + ((long long)c * nz + z) * N * NXH;
  for (int it = threadIdx.x; it < K2 * NXH; it += kFT) {
    const int k2 = r * K2 + it / NXH, kx = it - (it / NXH) * NXH;
    const unsigned off = (unsigned)(k2 * LY + kx) * (unsigned)sizeof(float2);
    float2 a[kCR];
#pragma unroll
    for (int q = 0; q < kCR; ++q) a[q] = cl_ld(rb[q] + off);
#pragma unroll
    for (int q = 1; q < kCR; ++q) a[q] = cmul(a[q], __ldg(&twn[q * k2]));
    Dft<kCR, false, float2>::run(a);
#pragma unroll
    for (int k1 = 0; k1 < kCR; ++k1) out[(long long)(k2 + M * k1) * NXH + kx] = a[k1];
  }
  // no CTA leaves while the others may still read its Y
  cl_sync();
  if (MODE == 1 && partials) {
    double vv[1] = {(double)acc};
    block_sum<1>(vv, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = vv[0];
  }
}

// ------------------------------------------------------------- inverse
// Output epilogue as the x-inverse pass (xinv_rows): plain store (with the
// dot product with dotw, or with itself, in partials[blockIdx.x] when DOT),
// or (CG) z += alpha d, r += alpha Hd with r'.r', r'.r, z'.z in
// partials[3 blockIdx.x + s] while the CG runs, z += tau d on an exit.
template <int N, bool DOT, bool CG>
__global__ void __cluster_dims__(kCR, 1, 1) __launch_bounds__(kFT, 2)
    kc_yxinv(const float2* __restrict__ spec, float* __restrict__ out, const float* __restrict__ dotw,
             double* __restrict__ partials, const int nz, const long long nvox, const float2* __restrict__ twn,
             const float2* __restrict__ twm, const float scale, const bool self_dot, float* __restrict__ cz,
             float* __restrict__ cr, const float* __restrict__ cd, const int* __restrict__ cstatus,
             const double* __restrict__ calpha, const double* __restrict__ ctau) {
  constexpr int M = N / kCR, NXH = N / 2 + 1, LY = NXH;
  constexpr int NLB = cl_nlb<N>(), BR = 2 * NLB, NBT = M / BR;
  constexpr int NLW = NLB + 1;  // odd line stride of the x batch: consecutive x on distinct banks
  constexpr int K2 = M / kCR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* yb = reinterpret_cast<float2*>(smem_raw);
  float2* wb = yb + M * LY;
  __shared__ double red[3 * 32];
  const int r = (int)cl_rank();
  const int cid = blockIdx.x / kCR, c = cid % 6, z = cid / 6;
  const long long pvox = (long long)z * N * N;
  // every CTA of the cluster runs before any stores into another's memory
  cl_sync();
  unsigned rb[kCR];
#pragma unroll
  for (int q = 0; q < kCR; ++q) rb[q] = cl_map(yb, q);
  const float2* src = spec + ((long long)c * nz + z) * N * NXH;
  for (int it = threadIdx.x; it < K2 * NXH; it += kFT) {
    const int k2 = r * K2 + it / NXH, kx = it - (it / NXH) * NXH;
    float2 a[kCR];
#pragma unroll
    for (int k1 = 0; k1 < kCR; ++k1) a[k1] = src[(long long)(k2 + M * k1) * NXH + kx];
    Dft<kCR, true, float2>::run(a);
#pragma unroll
    for (int q = 1; q < kCR; ++q) a[q] = cmulc(a[q], __ldg(&twn[q * k2]));
    const unsigned off = (unsigned)(k2 * LY + kx) * (unsigned)sizeof(float2);
#pragma unroll
    for (int q = 0; q < kCR; ++q) cl_st(rb[q] + off, a[q]);
  }
  cl_sync();
  // rows y = r + kCR m: inverse M-point FFT over k2 of every column
  fft_ct<M, LY, kFT, true>(yb, twm);
  using RI = RowItems<N, BR>;
  constexpr int SB = CG ? 4 : 8;
  constexpr int NG = (RI::COUNT + SB - 1) / SB;
  constexpr int KB = N / 2, GB = kFT / KB, JB = (NLB + GB - 1) / GB;
  int status = 0;
  bool run = true, exit_tau = false;
  float al = 0.f, ta = 0.f;
  if constexpr (CG) {
    status = *cstatus;
    run = status == 0;
    exit_tau = status == 2 || status == 3;  // boundary / negative curvature
    al = (float)*calpha;
    ta = (float)*ctau;
  }
  float cs[3] = {0.f, 0.f, 0.f};
  for (int bt = 0; bt < NBT; ++bt) {
    __syncthreads();  // the y FFT / the previous batch's outputs are done with wb
    // rows m = bt BR + 2p + h packed as line p (Hermitian extension)
    const int g = threadIdx.x / KB, kk = threadIdx.x - (threadIdx.x / KB) * KB;
    if (g < GB) {
#pragma unroll
      for (int j = 0; j < JB; ++j) {
        const int p = g + j * GB;
        if (JB * GB == NLB || p < NLB) {
          const int m0 = bt * BR + 2 * p;
          float2 a = yb[m0 * LY + kk], c2 = yb[(m0 + 1) * LY + kk];
          if (kk == 0) {
            a.y = 0.f;
            c2.y = 0.f;
          }
          wb[kk * NLW + p] = make_float2(a.x - c2.y, a.y + c2.x);
          if (kk != 0) wb[(N - kk) * NLW + p] = make_float2(a.x + c2.y, c2.x - a.y);
        }
      }
    }
    if (threadIdx.x < NLB) {
      const int p = threadIdx.x, m0 = bt * BR + 2 * p;
      wb[KB * NLW + p] = make_float2(yb[m0 * LY + KB].x, yb[(m0 + 1) * LY + KB].x);  // Nyquist: real parts
    }
    __syncthreads();
    fft_ct<N, NLW, kFT, true>(wb, twn);
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
      float o[SB], w[SB], zv[SB], rv[SB], dv[SB];
      long long offv[SB];
      bool ok[SB];
#pragma unroll
      for (int b = 0; b < SB; ++b) {
        int rho, x;
        RI::at(gi * SB + b, rho, x);
        ok[b] = gi * SB + b < RI::COUNT && RI::valid(rho, x) && (!CG || run || exit_tau);
        const int y = r + kCR * (bt * BR + rho);
        offv[b] = c * nvox + pvox + (long long)y * N + x;
        o[b] = ok[b] ? reinterpret_cast<const float*>(&wb[x * NLW + (rho >> 1)])[rho & 1] * scale : 0.f;
        if constexpr (CG) {
          zv[b] = ok[b] ? cz[offv[b]] : 0.f;
          dv[b] = ok[b] ? __ldg(cd + offv[b]) : 0.f;
          rv[b] = (ok[b] && run) ? cr[offv[b]] : 0.f;
        } else {
          w[b] = (DOT && ok[b]) ? (self_dot ? o[b] : __ldg(dotw + offv[b])) : 0.f;
        }
      }
#pragma unroll
      for (int b = 0; b < SB; ++b) {
        if (!ok[b]) continue;
        if constexpr (CG) {
          if (run) {
            const float zn = zv[b] + al * dv[b], rn = rv[b] + al * o[b];
            cz[offv[b]] = zn;
            cr[offv[b]] = rn;
            cs[0] += rn * rn;
            cs[1] += rn * rv[b];
            cs[2] += zn * zn;
          } else {
            cz[offv[b]] = zv[b] + ta * dv[b];
          }
        } else {
          out[offv[b]] = o[b];
          if (DOT) cs[0] += o[b] * w[b];
        }
      }
    }
  }
  if constexpr (CG) {
    double v3[3] = {(double)cs[0], (double)cs[1], (double)cs[2]};
    block_sum<3>(v3, red);
    if (threadIdx.x == 0)
      for (int k = 0; k < 3; ++k) partials[3 * (long long)blockIdx.x + k] = v3[k];
  } else if (DOT) {
    double v1[1] = {(double)cs[0]};
    block_sum<1>(v1, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = v1[0];
  }
}

// ================================================================ host side
bool cluster_size_ok(const GridDesc& g) {
  if (g.ndim != 3 || g.nq != 1 || g.ncomp != 6 || g.nx != g.ny) return false;
  return g.nx == 64 || g.nx == 128 || g.nx == 256 || g.nx == 96 || g.nx == 192;
}

int cluster_blocks(const GridDesc& g) { return kCR * 6 * g.nz; }

// once per kernel and device (a process may run contexts on several GPUs);
// the kernel is a template argument so that every instantiation keeps its
// own flags
template <auto kernel>
static cudaError_t cl_attr(size_t smem) {
  static int done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
  return e;
}

template <int N>
static cudaError_t xyfwd_n(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                           const MatTable<float>& mt, float2* spec, const float2* twn, const float2* twm,
                           bool tangent, double* partials, cudaStream_t st) {
  constexpr size_t sm = cl_smem<N>();
  const int blocks = cluster_blocks(g);
  cudaError_t e;
  if (tangent) {
    if ((e = cl_attr<kc_xyfwd<N, 1>>(sm)) != cudaSuccess) return e;
    kc_xyfwd<N, 1><<<blocks, kFT, sm, st>>>(in, phase, dmg, mt, spec, g.nz, g.nvox, twn, twm, partials);
  } else {
    if ((e = cl_attr<kc_xyfwd<N, 0>>(sm)) != cudaSuccess) return e;
    kc_xyfwd<N, 0><<<blocks, kFT, sm, st>>>(in, phase, dmg, mt, spec, g.nz, g.nvox, twn, twm, nullptr);
  }
  return cudaGetLastError();
}

template <int N, bool DOT, bool CG>
static cudaError_t yxinv_launch(const GridDesc& g, const float2* spec, float* out, const float* dotw,
                                double* partials, const float2* twn, const float2* twm, bool self, float* z, float* r,
                                const float* d, const int* status, const double* alpha, const double* tau,
                                cudaStream_t st) {
  constexpr size_t sm = cl_smem<N>();
  cudaError_t e;
  if ((e = cl_attr<kc_yxinv<N, DOT, CG>>(sm)) != cudaSuccess) return e;
  const float scale = (float)(1.0 / (double)g.nvox);
  kc_yxinv<N, DOT, CG><<<cluster_blocks(g), kFT, sm, st>>>(spec, out, dotw, partials, g.nz, g.nvox, twn, twm, scale,
                                                           self, z, r, d, status, alpha, tau);
  return cudaGetLastError();
}

#define RVE_CL_SIZES(X) X(64) X(128) X(256) X(96) X(192)

cudaError_t cluster_xyfwd(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                          const MatTable<float>& mt, float2* spec, const float2* twn, const float2* twm, bool tangent,
                          double* partials, cudaStream_t st) {
  if (!cluster_size_ok(g) || !twm) return cudaErrorNotSupported;
#define RVE_CASE(n_) \
  if (g.nx == n_) return xyfwd_n<n_>(g, in, phase, dmg, mt, spec, twn, twm, tangent, partials, st);
  RVE_CL_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

cudaError_t cluster_yxinv(const GridDesc& g, const float2* spec, float* out, const float* dotw, double* partials,
                          const float2* twn, const float2* twm, bool dot, bool self, cudaStream_t st) {
  if (!cluster_size_ok(g) || !twm) return cudaErrorNotSupported;
#define RVE_CASE(n_)                                                                                          \
  if (g.nx == n_)                                                                                             \
    return dot ? yxinv_launch<n_, true, false>(g, spec, out, dotw, partials, twn, twm, self, nullptr, nullptr, \
                                               nullptr, nullptr, nullptr, nullptr, st)                         \
               : yxinv_launch<n_, false, false>(g, spec, out, nullptr, nullptr, twn, twm, false, nullptr,      \
                                                nullptr, nullptr, nullptr, nullptr, nullptr, st);
  RVE_CL_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

cudaError_t cluster_yxinv_cg(const GridDesc& g, const float2* spec, float* z, float* r, const float* d,
                             const int* status, const double* alpha, const double* tau, double* partials,
                             const float2* twn, const float2* twm, cudaStream_t st) {
  if (!cluster_size_ok(g) || !twm) return cudaErrorNotSupported;
#define RVE_CASE(n_)                                                                                            \
  if (g.nx == n_)                                                                                               \
    return yxinv_launch<n_, false, true>(g, spec, nullptr, nullptr, partials, twn, twm, false, z, r, d, status, \
                                         alpha, tau, st);
  RVE_CL_SIZES(RVE_CASE)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

}  // namespace rve
