// FP32 spectral passes specialised at compile time for the common axis
// lengths (powers of two from 32 to 512 and 3 * 2^k up to 384).  Same data
// layout and the same arithmetic as the generic passes in hv_passes.cu;
// only the FFT engine (fft_fast.cuh) and the staging differ: global loads
// are batched in registers before they are written to shared memory, and
// the x passes give consecutive threads consecutive x so that the
// line-interleaved shared-memory accesses stay (nearly) conflict free.
#include "fft_fast.cuh"
#include "hv_passes.cuh"
#include "hv_fast.cuh"
#include "project.cuh"

namespace rve {

constexpr int kFT = 256;       // threads of the x / y passes
constexpr int kFBudget = 4096; // complex elements per x / y block

template <int N, int NC> constexpr int xq() {
  // voxel rows per x block: NC*Q/2 lines of N, prefer an odd line count
  constexpr int nlmax = kFBudget / N;
  constexpr int q0 = (2 * nlmax) / NC;
  constexpr int q1 = (NC & 1) ? (q0 & ~1) : q0;
  constexpr int q2 = (q1 < ((NC & 1) ? 2 : 1)) ? ((NC & 1) ? 2 : 1) : q1;
  constexpr int nl = NC * q2 / 2;
  return ((nl & 1) == 0 && q2 > ((NC & 1) ? 2 : 1)) ? q2 - ((NC & 1) ? 2 : 1) : q2;
}
template <int N> constexpr int ytx() { return (kFBudget / N) < 16 ? (kFBudget / N) : 16; }
template <int N> constexpr int ztx() { return N <= 64 ? 16 : 4; }
template <int N> constexpr int zthreads() { return N >= 512 ? 512 : 256; }
template <int N> constexpr int zminblocks() { return N >= 512 ? 1 : 3; }
template <int N> constexpr int p2tx() { return (kFBudget / (3 * N)) < 16 ? (kFBudget / (3 * N)) : 16; }

// ------------------------------------------------------------ x forward
// MODE 0: plain; 1: secant tangent; 2: symmetric consistent tangent (the
// secant plus the rank-one correction of ConsTan on loading voxels).
template <int N, int NC, int MODE>
__global__ void __launch_bounds__(kFT)
    kf_xfwd(const float* __restrict__ in, const uint8_t* __restrict__ phase, const float* __restrict__ dmg,
            const MatTable<float> mt, float2* __restrict__ spec, const long long nrows, const long long nvox,
            const float2* __restrict__ tw, double* __restrict__ partials, const float* __restrict__ cdp = nullptr,
            const float* __restrict__ ca = nullptr, const float* __restrict__ cn = nullptr) {
  constexpr int Q = xq<N, NC>();
  constexpr int NL = NC * Q / 2;
  constexpr int ND = NC == 6 ? 3 : 2;
  __shared__ __align__(16) float2 buf[NL * N];
  __shared__ double red[32];
  float acc = 0.f;  // in : (tangent : in) over this thread's few voxels (MODE 1 with partials)
  const long long row0 = (long long)blockIdx.x * Q;
  // one voxel per thread per step: consecutive threads take consecutive x,
  // so the line-interleaved shared-memory writes are (nearly) conflict free
  constexpr int ITEMS = Q * N;
  constexpr int STEPS = (ITEMS + kFT - 1) / kFT;
  constexpr int BATCH = STEPS < 4 ? STEPS : 4;
  for (int s0 = 0; s0 < STEPS; s0 += BATCH) {
    float v[BATCH][NC];
#pragma unroll
    for (int b = 0; b < BATCH; ++b) {
      const int idx = threadIdx.x + (s0 + b) * kFT;
      const int q = idx / N, x = idx - (idx / N) * N;
      const long long row = row0 + q;
      const bool ok = (s0 + b < STEPS) && idx < ITEMS && row < nrows;
      const long long vox = row * N + x;
#pragma unroll
      for (int c = 0; c < NC; ++c) v[b][c] = ok ? __ldg(in + c * nvox + vox) : 0.f;
      if (MODE >= 1 && ok) {
        const float keep = 1.f - __ldg(dmg + vox);
        const int ph = __ldg(phase + vox);
        const float lam = mt.lam[ph] * keep, tmu = 2.f * mt.mu[ph] * keep;
        float tr = 0.f;
#pragma unroll
        for (int i = 0; i < ND; ++i) tr += v[b][i];
        float hdp = 0.f, nv = 0.f, av = 0.f;
        if constexpr (MODE == 2) {
          hdp = 0.5f * __ldg(cdp + vox);
          if (hdp != 0.f) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              nv += __ldg(cn + c * nvox + vox) * v[b][c];
              av += __ldg(ca + c * nvox + vox) * v[b][c];
            }
          }
        }
        float dv = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          float sg = tmu * v[b][c] + (c < ND ? lam * tr : 0.f);
          if constexpr (MODE == 2) {
            if (hdp != 0.f) sg -= hdp * (__ldg(ca + c * nvox + vox) * nv + __ldg(cn + c * nvox + vox) * av);
          }
          dv += v[b][c] * sg;
          v[b][c] = sg;
        }
        acc += dv;
      }
    }
#pragma unroll
    for (int b = 0; b < BATCH; ++b) {
      const int idx = threadIdx.x + (s0 + b) * kFT;
      if (s0 + b < STEPS && idx < ITEMS) {
        const int q = idx / N, x = idx - (idx / N) * N;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int rho = q * NC + c;
          reinterpret_cast<float*>(&buf[x * NL + (rho >> 1)])[rho & 1] = v[b][c];
        }
      }
    }
  }
  __syncthreads();
  fft_ct<N, NL, kFT, false>(buf, tw);
  constexpr int NXH = N / 2 + 1;
  for (int idx = threadIdx.x; idx < NL * NXH; idx += kFT) {
    const int p = idx / NXH, k = idx - (idx / NXH) * NXH;
    const float2 zk = buf[k * NL + p];
    const float2 zm = buf[((N - k) % N) * NL + p];
    const float2 xa = make_float2((zk.x + zm.x) * 0.5f, (zk.y - zm.y) * 0.5f);
    const float2 xb = make_float2((zk.y + zm.y) * 0.5f, (zm.x - zk.x) * 0.5f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rho = 2 * p + h;
      const int q = rho / NC, c = rho - (rho / NC) * NC;
      const long long row = row0 + q;
      if (row < nrows) spec[(c * nrows + row) * NXH + k] = h ? xb : xa;
    }
  }
  if (MODE >= 1 && partials) {
    double val[1] = {(double)acc};
    block_sum<1>(val, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = val[0];
  }
}

// ------------------------------------------------------------ x inverse
// CG: instead of storing the product Hd, apply the CG iterate / residual
// update of Algorithm 1 with it (status, alpha and tau read from the device
// scalars): running, z += alpha d and r += alpha Hd with the sums r'.r',
// r'.r and z'.z per block in partials[3 b + s]; on a boundary or
// negative-curvature exit, z += tau d.
template <int N, int NC, bool DOT, bool CG = false>
__global__ void __launch_bounds__(kFT)
    kf_xinv(const float2* __restrict__ spec, float* __restrict__ out, const float* __restrict__ dotw,
            double* __restrict__ partials, const long long nrows, const long long nvox,
            const float2* __restrict__ tw, const float scale, const bool self_dot, float* __restrict__ cz = nullptr,
            float* __restrict__ cr = nullptr, const float* __restrict__ cd = nullptr,
            const int* __restrict__ cstatus = nullptr, const double* __restrict__ calpha = nullptr,
            const double* __restrict__ ctau = nullptr) {
  constexpr int Q = xq<N, NC>();
  constexpr int NL = NC * Q / 2;
  constexpr int NXH = N / 2 + 1;
  constexpr int HALF = N / 2;
  __shared__ __align__(16) float2 buf[NL * N];
  __shared__ double red[32];
  const long long row0 = (long long)blockIdx.x * Q;
  // each half-spectrum entry kk of the two real lines packed in line p is
  // read once and fills both buf[kk] and buf[N - kk] (Hermitian symmetry)
  constexpr int LITEMS = NL * NXH;
  constexpr int LSTEPS = (LITEMS + kFT - 1) / kFT;
  constexpr int LB = LSTEPS < 4 ? LSTEPS : 4;
  for (int s0 = 0; s0 < LSTEPS; s0 += LB) {
    float2 xh[LB][2];
#pragma unroll
    for (int b = 0; b < LB; ++b) {
      const int idx = threadIdx.x + (s0 + b) * kFT;
      const int p = idx / NXH, kk = idx - (idx / NXH) * NXH;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rho = 2 * p + h;
        const int q = rho / NC, c = rho - (rho / NC) * NC;
        const long long row = row0 + q;
        xh[b][h] = (s0 + b < LSTEPS && idx < LITEMS && row < nrows) ? spec[(c * nrows + row) * NXH + kk]
                                                                   : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int b = 0; b < LB; ++b) {
      const int idx = threadIdx.x + (s0 + b) * kFT;
      if (s0 + b < LSTEPS && idx < LITEMS) {
        const int p = idx / NXH, kk = idx - (idx / NXH) * NXH;
        float2 a = xh[b][0], c2 = xh[b][1];
        if (kk == 0 || kk == HALF) {
          a.y = 0.f;
          c2.y = 0.f;
        }
        buf[kk * NL + p] = make_float2(a.x - c2.y, a.y + c2.x);
        if (kk != 0 && kk != HALF) buf[(N - kk) * NL + p] = make_float2(a.x + c2.y, c2.x - a.y);
      }
    }
  }
  __syncthreads();
  fft_ct<N, NL, kFT, true>(buf, tw);
  if constexpr (CG) {
    const int status = *cstatus;
    const bool run = status == 0, exit_tau = status == 2 || status == 3;  // running / boundary, negative curvature
    const float al = (float)*calpha, ta = (float)*ctau;
    KSum<float> cs[3];
    constexpr int SITEMS = Q * NC * N;
    constexpr int SSTEPS = (SITEMS + kFT - 1) / kFT;
    constexpr int SB = SSTEPS < 4 ? SSTEPS : 4;
    for (int s0 = 0; s0 < SSTEPS; s0 += SB) {
      float o[SB], zv[SB], rv[SB], dv[SB];
      long long off[SB];
      bool ok[SB];
#pragma unroll
      for (int b = 0; b < SB; ++b) {
        const int idx = threadIdx.x + (s0 + b) * kFT;
        const int rho = idx / N, x = idx - (idx / N) * N;
        const int q = rho / NC, c = rho - (rho / NC) * NC;
        const long long row = row0 + q;
        ok[b] = (s0 + b < SSTEPS) && idx < SITEMS && row < nrows && (run || exit_tau);
        off[b] = c * nvox + row * N + x;
        o[b] = ok[b] ? reinterpret_cast<const float*>(&buf[x * NL + (rho >> 1)])[rho & 1] * scale : 0.f;
        zv[b] = ok[b] ? cz[off[b]] : 0.f;
        dv[b] = ok[b] ? __ldg(cd + off[b]) : 0.f;
        rv[b] = (ok[b] && run) ? cr[off[b]] : 0.f;
      }
#pragma unroll
      for (int b = 0; b < SB; ++b) {
        if (!ok[b]) continue;
        if (run) {
          const float zn = zv[b] + al * dv[b], rn = rv[b] + al * o[b];
          cz[off[b]] = zn;
          cr[off[b]] = rn;
          cs[0].add(rn * rn);
          cs[1].add(rn * rv[b]);
          cs[2].add(zn * zn);
        } else {
          cz[off[b]] = zv[b] + ta * dv[b];
        }
      }
    }
    __shared__ double red3[3 * 32];
    double v3[3] = {cs[0].value(), cs[1].value(), cs[2].value()};
    block_sum<3>(v3, red3);
    if (threadIdx.x == 0)
      for (int k = 0; k < 3; ++k) partials[3 * (long long)blockIdx.x + k] = v3[k];
    return;
  }
  KSum<float> acc;
  constexpr int SITEMS = Q * NC * N;
  constexpr int SSTEPS = (SITEMS + kFT - 1) / kFT;
  constexpr int SB = SSTEPS < 8 ? SSTEPS : 8;
  for (int s0 = 0; s0 < SSTEPS; s0 += SB) {
    float o[SB], w[SB];
    long long off[SB];
    bool ok[SB];
#pragma unroll
    for (int b = 0; b < SB; ++b) {
      const int idx = threadIdx.x + (s0 + b) * kFT;
      const int rho = idx / N, x = idx - (idx / N) * N;
      const int q = rho / NC, c = rho - (rho / NC) * NC;
      const long long row = row0 + q;
      ok[b] = (s0 + b < SSTEPS) && idx < SITEMS && row < nrows;
      off[b] = c * nvox + row * N + x;
      o[b] = ok[b] ? reinterpret_cast<const float*>(&buf[x * NL + (rho >> 1)])[rho & 1] * scale : 0.f;
      w[b] = (DOT && ok[b]) ? (self_dot ? o[b] : __ldg(dotw + off[b])) : 0.f;
    }
#pragma unroll
    for (int b = 0; b < SB; ++b) {
      if (ok[b]) {
        out[off[b]] = o[b];
        if (DOT) acc.add(o[b] * w[b]);
      }
    }
  }
  if (DOT) {
    double v[1] = {acc.value()};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
  }
}

// ------------------------------------------------------------ y columns
template <int N, bool INV>
__global__ void __launch_bounds__(kFT)
    kf_ycols(float2* __restrict__ spec, const int nz, const int nxh, const float2* __restrict__ tw) {
  constexpr int TX = ytx<N>();
  __shared__ __align__(16) float2 buf[TX * N];
  const int kx0 = blockIdx.x * TX;
  const int tv = min(TX, nxh - kx0);
  const long long plane = ((long long)blockIdx.z * nz + blockIdx.y) * N;
  // the first stage reads the columns straight from global memory and the
  // last one writes them back: no staging through shared memory
  auto load = [&](int t, int y) -> float2 {
    return t < tv ? spec[(plane + y) * nxh + kx0 + t] : make_float2(0.f, 0.f);
  };
  auto store = [&](int t, int y, float2 v) {
    if (t < tv) spec[(plane + y) * nxh + kx0 + t] = v;
  };
  fft_stage0_from<N, TX, kFT, INV>(buf, load);
  fft_ct_range<N, TX, kFT, INV, 1, fft_nstages(N) - 1>(buf, tw);
  fft_stage_last_to<N, TX, kFT, INV>(buf, tw, store);
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
  const float2 ay = gay[ky], dy = gdy[ky];
  for (int pt = threadIdx.x; pt < N * TX; pt += NT) {
    const int z = pt / TX, t = pt - (pt / TX) * TX;
    const int kx = kx0 + t;
    if (t >= tv) continue;
    float2 m[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) m[c] = buf[z * NL + c * TX + t];
    const float2 ax = gax[kx], dx = gdx[kx], az = gaz[z], dz = gdz[z];
    project3<float>(m, cmul(cmul(dx, ay), az), cmul(cmul(ax, dy), az), cmul(cmul(ax, ay), dz),
                    kx == 0 && ky == 0 && z == 0, free_mask);
#pragma unroll
    for (int c = 0; c < 6; ++c) buf[z * NL + c * TX + t] = m[c];
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
template <int N>
__global__ void __launch_bounds__(kFT)
    kf_yproj2d(float2* __restrict__ spec, const int nxh, const float2* __restrict__ tw,
               const float2* __restrict__ gdx, const float2* __restrict__ gax, const float2* __restrict__ gdy,
               const float2* __restrict__ gay, const unsigned free_mask) {
  constexpr int TX = p2tx<N>();
  constexpr int NL = 3 * TX;
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
    float2 m[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) m[c] = buf[y * NL + c * TX + t];
    project2<float>(m, cmul(gdx[kx], gay[y]), cmul(gax[kx], gdy[y]), kx == 0 && y == 0, free_mask);
#pragma unroll
    for (int c = 0; c < 3; ++c) buf[y * NL + c * TX + t] = m[c];
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
    if (cons)
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
  constexpr int TX = p2tx<N>();
  const dim3 grid((g.nxh + TX - 1) / TX);
  kf_yproj2d<N><<<grid, kFT, 0, st>>>(spec, g.nxh, w.tw[1], w.gdiff[0], w.gavg[0], w.gdiff[1], w.gavg[1],
                                       w.free_mask);
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
