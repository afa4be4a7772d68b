// Tile bodies of the compile-time-specialised FP32 passes (hv_fast.cu):
// one x-forward row tile, one x-inverse row tile, one y column tile.  Sizes
// are template constants: powers of two from 32 to 512 and 3 * 2^k up to
// 384.
#pragma once

#include "fft_fast.cuh"
#include "hv_passes.cuh"

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
template <int N> constexpr int ztx() { return N <= 64 ? 16 : (N <= 256 ? 8 : 4); }
template <int N> constexpr int zthreads() { return N >= 512 || (N >= 128 && N <= 256) ? 512 : 256; }
template <int N> constexpr int zminblocks() { return N >= 512 ? 1 : (N >= 128 && N <= 256 ? 2 : 3); }
// Items (rho, x) -- real row rho of a tile of NROW rows, element x -- as
// thread threadIdx.x takes them, item i = 0 .. COUNT-1.  Where N divides the
// 256 threads (or 256 divides N) a thread keeps one x (two for N = 512) and
// steps through the rows, so that rho is a compile-time constant for
// N >= 256 and the row / component split of rho costs nothing; other N take
// consecutive elements of the flattened tile.
template <int N, int NROW> struct RowItems {
  static constexpr bool REG = (kFT % N == 0) || (N % kFT == 0);
  static constexpr int XR = N >= kFT ? 1 : kFT / N;  // rows per sweep of the block
  static constexpr int XH = N >= kFT ? N / kFT : 1;  // elements per row and thread
  static constexpr int NJ = (NROW + XR - 1) / XR;
  static constexpr int COUNT = REG ? NJ * XH : (NROW * N + kFT - 1) / kFT;
  __device__ __forceinline__ static void at(int i, int& rho, int& x) {
    if constexpr (REG) {
      const int j = i / XH, h = i - (i / XH) * XH;
      rho = (N >= kFT ? 0 : (int)threadIdx.x / N) + j * XR;
      x = (N >= kFT ? (int)threadIdx.x : (int)threadIdx.x % N) + h * kFT;
    } else {
      const int idx = threadIdx.x + i * kFT;
      rho = idx / N;
      x = idx - rho * N;
    }
  }
  __device__ __forceinline__ static bool valid(int rho, int) { return rho < NROW; }
};


// ------------------------------------------------------------ x forward
template <int N, int NC>
__device__ __forceinline__ void xfwd_fft_store(float2* buf, float2* __restrict__ spec, const long long nrows,
                                               const float2* __restrict__ tw, const long long row0,
                                               const long long row_end);

// One x-forward tile: the voxel rows [row0, row_end) (at most xq rows),
// tangent applied on load, forward FFT of the real rows packed in pairs,
// half spectrum stored.  Returns this thread's share of in : (tangent : in)
// (MODE >= 1).  `buf` holds NC * xq / 2 lines of N.  MODE 0: plain; 1:
// secant tangent; 2: symmetric consistent tangent; 3: secant tangent of
// the 2D Kuhn triangles (NC = 6 lines c * 2 + q).
template <int N, int NC, int MODE>
__device__ __forceinline__ float xfwd_rows(float2* buf, const float* __restrict__ in,
                                           const uint8_t* __restrict__ phase, const float* __restrict__ dmg,
                                           const MatTable<float>& mt, float2* __restrict__ spec,
                                           const long long nrows, const long long nvox,
                                           const float2* __restrict__ tw, const long long row0,
                                           const long long row_end, const float* __restrict__ cdp,
                                           const float* __restrict__ ca, const float* __restrict__ cn) {
  constexpr int Q = xq<N, NC>();
  constexpr int NL = NC * Q / 2;
  constexpr int ND = NC == 6 ? 3 : 2;
  float acc = 0.f;  // in : (tangent : in) over this thread's few voxels (MODE >= 1)
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
      const bool ok = (s0 + b < STEPS) && idx < ITEMS && row < row_end;
      const long long vox = row * N + x;
#pragma unroll
      for (int c = 0; c < NC; ++c) v[b][c] = ok ? __ldg(in + c * nvox + vox) : 0.f;
      if (MODE == 3 && ok) {
        // 2D Kuhn triangles: line c * 2 + q is Mandel component c of
        // triangle q, whose damage is dmg[q * nvox + vox]
        const int ph = __ldg(phase + vox);
        float dv = 0.f;
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          const float keep = 1.f - __ldg(dmg + q2 * nvox + vox);
          const float lam = mt.lam[ph] * keep, tmu = 2.f * mt.mu[ph] * keep;
          const float tr = v[b][q2] + v[b][2 + q2];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float sg = tmu * v[b][2 * c + q2] + (c < 2 ? lam * tr : 0.f);
            dv += v[b][2 * c + q2] * sg;
            v[b][2 * c + q2] = sg;
          }
        }
        acc += dv;
      }
      if ((MODE == 1 || MODE == 2) && ok) {
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
  xfwd_fft_store<N, NC>(buf, spec, nrows, tw, row0, row_end);
  return acc;
}

// The FFT and store stage of an x-forward tile whose NC * xq rows sit packed
// in pairs in `buf` (element x of line p at x * NL + p; the caller has
// synchronised): forward FFT of every line, then the two real rows of every
// line separated (Hermitian symmetry of real-input spectra) and their half
// spectra stored.  Thread t takes bin k = t mod (N/2) of the lines
// p = t div (N/2) + j (256 / (N/2)); the Nyquist bin of every line goes to
// threads 0 .. NL-1.  Row and component of the two halves follow from p
// alone, so no per-item division by the half-spectrum length.
template <int N, int NC>
__device__ __forceinline__ void xfwd_fft_store(float2* buf, float2* __restrict__ spec, const long long nrows,
                                               const float2* __restrict__ tw, const long long row0,
                                               const long long row_end) {
  constexpr int Q = xq<N, NC>();
  constexpr int NL = NC * Q / 2;
  fft_ct<N, NL, kFT, false>(buf, tw);
  constexpr int NXH = N / 2 + 1;
  constexpr int KB = N / 2, GB = kFT / KB, JB = (NL + GB - 1) / GB;
  const long long plane = nrows * NXH;
  {
    const int g = threadIdx.x / KB, k = threadIdx.x - (threadIdx.x / KB) * KB;
    const int km = k == 0 ? 0 : N - k;
    if (g < GB) {
#pragma unroll
      for (int j = 0; j < JB; ++j) {
        const int p = g + j * GB;
        if (JB * GB == NL || p < NL) {
          const float2 zk = buf[k * NL + p], zm = buf[km * NL + p];
          const float2 xa = make_float2((zk.x + zm.x) * 0.5f, (zk.y - zm.y) * 0.5f);
          const float2 xb = make_float2((zk.y + zm.y) * 0.5f, (zm.x - zk.x) * 0.5f);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int rho = 2 * p + h;
            const int q = rho / NC, c = rho - (rho / NC) * NC;
            if (row0 + q < row_end) spec[c * plane + (row0 + q) * NXH + k] = h ? xb : xa;
          }
        }
      }
    }
    if (threadIdx.x < NL) {
      const int p = threadIdx.x;
      const float2 z = buf[KB * NL + p];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rho = 2 * p + h;
        const int q = rho / NC, c = rho - (rho / NC) * NC;
        if (row0 + q < row_end) spec[c * plane + (row0 + q) * NXH + KB] = make_float2(h ? z.y : z.x, 0.f);
      }
    }
  }
}

// ------------------------------------------------------------ x inverse
// CG: instead of storing the product Hd, apply the CG iterate / residual
// update of Algorithm 1 with it (status, alpha and tau read from the device
// scalars): running, z += alpha d and r += alpha Hd with the sums r'.r',
// r'.r and z'.z per block in partials[3 b + s]; on a boundary or
// negative-curvature exit, z += tau d.
// One x-inverse tile: rows [row0, row_end); its block sums go to
// partials[pidx] (DOT) or partials[3 pidx + s] (CG).  L2LOAD: the spectrum
// was written by other blocks of the same launch, so it is read through L2
// (ld.global.cg), never from a stale L1 line.  `red` holds 3 * 32 doubles.
template <int N, int NC, bool DOT, bool CG, bool L2LOAD>
__device__ __forceinline__ void xinv_rows(float2* buf, double* red, const float2* __restrict__ spec,
                                          float* __restrict__ out, const float* __restrict__ dotw,
                                          double* __restrict__ partials, const long long nrows,
                                          const long long nvox, const float2* __restrict__ tw, const float scale,
                                          const bool self_dot, float* __restrict__ cz, float* __restrict__ cr,
                                          const float* __restrict__ cd, const int* __restrict__ cstatus,
                                          const double* __restrict__ calpha, const double* __restrict__ ctau,
                                          const long long row0, const long long row_end, const long long pidx) {
  constexpr int Q = xq<N, NC>();
  constexpr int NL = NC * Q / 2;
  constexpr int NXH = N / 2 + 1;
  // Each half-spectrum entry kk of the two real rows packed in line p is read
  // once and fills both buf[kk] and buf[N - kk] (Hermitian symmetry).
  // Thread t takes bin kk = t mod (N/2) of the lines p = t div (N/2) + j
  // (256 / (N/2)), all its loads issued before its stores; the Nyquist bin of
  // every line goes to threads 0 .. NL-1.
  constexpr int KB = N / 2, GB = kFT / KB, JB = (NL + GB - 1) / GB;
  const long long plane = nrows * NXH;
  {
    const int g = threadIdx.x / KB, kk = threadIdx.x - (threadIdx.x / KB) * KB;
    if (g < GB) {
      float2 xh[JB][2];
#pragma unroll
      for (int j = 0; j < JB; ++j) {
        const int p = g + j * GB;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rho = 2 * p + h;
          const int q = rho / NC, c = rho - (rho / NC) * NC;
          const float2* src = spec + c * plane + (row0 + q) * NXH + kk;
          xh[j][h] = ((JB * GB == NL || p < NL) && row0 + q < row_end) ? (L2LOAD ? __ldcg(src) : *src)
                                                                       : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int j = 0; j < JB; ++j) {
        const int p = g + j * GB;
        if (JB * GB == NL || p < NL) {
          float2 a = xh[j][0], c2 = xh[j][1];
          if (kk == 0) {
            a.y = 0.f;
            c2.y = 0.f;
          }
          buf[kk * NL + p] = make_float2(a.x - c2.y, a.y + c2.x);
          if (kk != 0) buf[(N - kk) * NL + p] = make_float2(a.x + c2.y, c2.x - a.y);
        }
      }
    }
    if (threadIdx.x < NL) {
      const int p = threadIdx.x;
      float2 xn[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rho = 2 * p + h;
        const int q = rho / NC, c = rho - (rho / NC) * NC;
        const float2* src = spec + c * plane + (row0 + q) * NXH + KB;
        xn[h] = row0 + q < row_end ? (L2LOAD ? __ldcg(src) : *src) : make_float2(0.f, 0.f);
      }
      buf[KB * NL + p] = make_float2(xn[0].x, xn[1].x);  // imaginary parts of the Nyquist bin dropped
    }
  }
  __syncthreads();
  fft_ct<N, NL, kFT, true>(buf, tw);
  // The Q * NC real rows of the tile leave shared memory as items (rho, x):
  // see RowItems.  A thread's partial sums are plain FP32 over its ~30 items,
  // combined in FP64 across the block and the grid.
  using RI = RowItems<N, Q * NC>;
  constexpr int SB = CG ? 4 : 8;  // items whose loads are in flight together
  constexpr int NG = (RI::COUNT + SB - 1) / SB;
  if constexpr (CG) {
    const int status = *cstatus;
    const bool run = status == 0, exit_tau = status == 2 || status == 3;  // running / boundary, negative curvature
    const float al = (float)*calpha, ta = (float)*ctau;
    float cs[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      float o[SB], zv[SB], rv[SB], dv[SB];
      long long off[SB];
      bool ok[SB];
#pragma unroll
      for (int b = 0; b < SB; ++b) {
        int rho, x;
        RI::at(g * SB + b, rho, x);
        const int q = rho / NC, c = rho - (rho / NC) * NC;
        ok[b] = g * SB + b < RI::COUNT && RI::valid(rho, x) && row0 + q < row_end && (run || exit_tau);
        off[b] = c * nvox + (row0 + q) * N + x;
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
          cs[0] += rn * rn;
          cs[1] += rn * rv[b];
          cs[2] += zn * zn;
        } else {
          cz[off[b]] = zv[b] + ta * dv[b];
        }
      }
    }
    double v3[3] = {(double)cs[0], (double)cs[1], (double)cs[2]};
    block_sum<3>(v3, red);
    if (threadIdx.x == 0)
      for (int k = 0; k < 3; ++k) partials[3 * pidx + k] = v3[k];
    return;
  }
  float acc = 0.f;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    float o[SB], w[SB];
    long long off[SB];
    bool ok[SB];
#pragma unroll
    for (int b = 0; b < SB; ++b) {
      int rho, x;
      RI::at(g * SB + b, rho, x);
      const int q = rho / NC, c = rho - (rho / NC) * NC;
      ok[b] = g * SB + b < RI::COUNT && RI::valid(rho, x) && row0 + q < row_end;
      off[b] = c * nvox + (row0 + q) * N + x;
      o[b] = ok[b] ? reinterpret_cast<const float*>(&buf[x * NL + (rho >> 1)])[rho & 1] * scale : 0.f;
      w[b] = (DOT && ok[b]) ? (self_dot ? o[b] : __ldg(dotw + off[b])) : 0.f;
    }
#pragma unroll
    for (int b = 0; b < SB; ++b) {
      if (ok[b]) {
        out[off[b]] = o[b];
        if (DOT) acc += o[b] * w[b];
      }
    }
  }
  if (DOT) {
    double v[1] = {(double)acc};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) partials[pidx] = v[0];
  }
}

// ------------------------------------------------------------ y columns
// One y tile: columns [kx0, kx0 + ytx) of the plane whose first row is
// `plane` (row index (c Nz + z) Ny), transformed in place.  L2LOAD as for
// xinv_rows.
template <int N, bool INV, bool L2LOAD>
__device__ __forceinline__ void ycols_tile(float2* buf, float2* __restrict__ spec, const long long plane,
                                           const int kx0, const int nxh, const float2* __restrict__ tw) {
  constexpr int TX = ytx<N>();
  const int tv = min(TX, nxh - kx0);
  // the first stage reads the columns straight from global memory and the
  // last one writes them back: no staging through shared memory
  auto load = [&](int t, int y) -> float2 {
    const float2* src = spec + (plane + y) * nxh + kx0 + t;
    return t < tv ? (L2LOAD ? __ldcg(src) : *src) : make_float2(0.f, 0.f);
  };
  auto store = [&](int t, int y, float2 v) {
    if (t < tv) spec[(plane + y) * nxh + kx0 + t] = v;
  };
  fft_stage0_from<N, TX, kFT, INV>(buf, load);
  fft_ct_range<N, TX, kFT, INV, 1, fft_nstages(N) - 1>(buf, tw);
  fft_stage_last_to<N, TX, kFT, INV>(buf, tw, store);
}

}  // namespace rve
