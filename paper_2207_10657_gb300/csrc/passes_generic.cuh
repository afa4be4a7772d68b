// Generic (runtime-length) spectral pass bodies and their single-grid
// kernels.  A body processes one block of one grid; the kernels call it with
// their block index, batched kernels with an index taken from a work list.
#pragma once

#include "hv_passes.cuh"
#include "project.cuh"

namespace rve {

constexpr int kXThreads = 256, kXEpt = 16;  // x passes
constexpr int kYThreads = 256, kYEpt = 16;  // y columns, 2D y+projection
constexpr int kZThreads = 512, kZEpt = 24;  // z + projection
constexpr int kSmemCap = 100 * 1024;        // dynamic shared memory cap per block
// The x and y kernels are compiled for six resident blocks per SM (at most
// 42 registers a thread): their runtime-radix stages otherwise take 200-255
// registers and leave one block (8 warps) per SM, latency-bound.  The spills
// this costs are cheaper than the idle SM (2.4x faster generic passes at
// 256^3 FP32, 1.3x in FP64 at 128^3).
constexpr int kXYMinBlocks = 6;

// ------------------------------------------------------------ x forward
// Q voxel rows per block, all ncomp components of each row.  With the
// tangent mode the damaged isotropic tangent (1-D)(lambda tr(v) 1 + 2 mu v)
// is applied on load (Eq. (13), secant reading), plus the rank-one part of
// the symmetric consistent tangent where `ct` is set.  Real rows are packed
// in pairs into one complex FFT (real + i*imag) and separated with the
// Hermitian symmetry of real-input spectra.
template <typename R, int MODE>
__device__ __forceinline__ void xfwd_body(const R* __restrict__ in, const uint8_t* __restrict__ phase,
                                          const R* __restrict__ dmg, const MatTable<R>& mt,
                                          Cx<R>* __restrict__ spec, const GridDesc& g, const int Q,
                                          const AxisPlan& px, const Cx<R>* __restrict__ tw, const int bx,
                                          const ConsTan<R> ct = ConsTan<R>{}) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int nx = g.nx, nc = g.ncomp, nd = g.ndim;
  const long long row0 = (long long)bx * Q;
  const int npair = (nc * Q) >> 1;
  for (int idx = threadIdx.x; idx < Q * nx; idx += blockDim.x) {
    const int q = idx / nx, x = idx - q * nx;
    const long long row = row0 + q;
    if (g.nq > 1) {
      // Kuhn simplices: line c * nq + p is Mandel component c of simplex p,
      // whose damage is dmg[p * nvox + vox]; the tangent acts per simplex
      const int nqp = g.nq, nm = nc / nqp;
      const long long vox = row * nx + x;
      for (int p = 0; p < nqp; ++p) {
        R m[6] = {0, 0, 0, 0, 0, 0};
        if (row < g.nrows) {
          for (int c = 0; c < nm; ++c) m[c] = in[(c * nqp + p) * g.nvox + vox];
          if (MODE == 1) {
            const int ph = phase[vox];
            const R keep = (R)1 - dmg[p * g.nvox + vox];
            const R lam = mt.lam[ph] * keep, two_mu = (R)2 * mt.mu[ph] * keep;
            R tr = 0;
            for (int i = 0; i < nd; ++i) tr += m[i];
            for (int c = 0; c < nm; ++c) m[c] = two_mu * m[c] + (c < nd ? lam * tr : (R)0);
          }
        }
        for (int c = 0; c < nm; ++c) {
          const int rho = q * nc + c * nqp + p;
          R* slot = reinterpret_cast<R*>(&buf[(rho >> 1) * nx + x]) + (rho & 1);
          *slot = m[c];
        }
      }
      continue;
    }
    R val[6] = {0, 0, 0, 0, 0, 0};
    if (row < g.nrows) {
      const long long vox = row * nx + x;
      for (int c = 0; c < nc; ++c) val[c] = in[c * g.nvox + vox];
      if (MODE == 1) {
        const int ph = phase[vox];
        const R keep = (R)1 - dmg[vox];
        const R lam = mt.lam[ph] * keep, two_mu = (R)2 * mt.mu[ph] * keep;
        R tr = 0;
        for (int i = 0; i < nd; ++i) tr += val[i];
        const R hdp = ct.dp ? (R)0.5 * ct.dp[vox] : (R)0;
        R nv = 0, av = 0;
        if (hdp != (R)0) {
          for (int c = 0; c < nc; ++c) {
            nv += ct.n[c * g.nvox + vox] * val[c];
            av += ct.a[c * g.nvox + vox] * val[c];
          }
        }
        for (int c = 0; c < nc; ++c) {
          val[c] = two_mu * val[c] + (c < nd ? lam * tr : (R)0);
          if (hdp != (R)0) val[c] -= hdp * (ct.a[c * g.nvox + vox] * nv + ct.n[c * g.nvox + vox] * av);
        }
      }
    }
    for (int c = 0; c < nc; ++c) {
      const int rho = q * nc + c;
      R* slot = reinterpret_cast<R*>(&buf[(rho >> 1) * nx + x]) + (rho & 1);
      *slot = val[c];
    }
  }
  __syncthreads();
  fft_lines<kXEpt, false, false>(buf, px, npair, LineMap{1, nx, 0, 1}, tw);
  const int nxh = g.nxh;
  for (int idx = threadIdx.x; idx < npair * nxh; idx += blockDim.x) {
    const int p = idx / nxh, k = idx - p * nxh;
    const C zk = buf[p * nx + k];
    const C zm = buf[p * nx + (k == 0 ? 0 : nx - k)];
    const C xa = C{(zk.x + zm.x) * (R)0.5, (zk.y - zm.y) * (R)0.5};
    const C xb = C{(zk.y + zm.y) * (R)0.5, (zm.x - zk.x) * (R)0.5};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rho = 2 * p + h;
      const int q = rho / nc, c = rho - q * nc;
      const long long row = row0 + q;
      if (q < Q && row < g.nrows) spec[(c * g.nrows + row) * nxh + k] = h ? xb : xa;
    }
  }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kXThreads, kXYMinBlocks)
    k_xfwd(const R* __restrict__ in, const uint8_t* __restrict__ phase, const R* __restrict__ dmg,
           const MatTable<R> mt, Cx<R>* __restrict__ spec, const GridDesc g, const int Q, const AxisPlan px,
           const Cx<R>* __restrict__ tw, const ConsTan<R> ct) {
  xfwd_body<R, MODE>(in, phase, dmg, mt, spec, g, Q, px, tw, blockIdx.x, ct);
}

// ------------------------------------------------------------ y columns
template <typename R, bool INV>
__device__ __forceinline__ void ycols_body(Cx<R>* __restrict__ spec, const GridDesc& g, const int TX,
                                           const AxisPlan& py, const Cx<R>* __restrict__ tw, const int bx,
                                           const int by, const int bz) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int ny = g.ny, nxh = g.nxh;
  const int kx0 = bx * TX;
  const int tv = min(TX, nxh - kx0);
  const long long plane = ((long long)bz * g.nz + by) * ny;
  for (int idx = threadIdx.x; idx < ny * TX; idx += blockDim.x) {
    const int y = idx / TX, t = idx - y * TX;
    buf[idx] = t < tv ? spec[(plane + y) * nxh + kx0 + t] : C{0, 0};
  }
  __syncthreads();
  fft_lines<kYEpt, INV, true>(buf, py, TX, LineMap{TX, 0, 1, TX}, tw);
  for (int idx = threadIdx.x; idx < ny * TX; idx += blockDim.x) {
    const int y = idx / TX, t = idx - y * TX;
    if (t < tv) spec[(plane + y) * nxh + kx0 + t] = buf[idx];
  }
}

template <typename R, bool INV>
__global__ void __launch_bounds__(kYThreads, kXYMinBlocks)
    k_ycols(Cx<R>* __restrict__ spec, const GridDesc g, const int TX, const AxisPlan py,
            const Cx<R>* __restrict__ tw) {
  ycols_body<R, INV>(spec, g, TX, py, tw, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ------------------------------------------------- z + projection (3D)
template <typename R>
__device__ __forceinline__ void zproj_body(Cx<R>* __restrict__ spec, const GridDesc& g, const int TX,
                                           const AxisPlan& pz, const Cx<R>* __restrict__ tw,
                                           const Cx<R>* __restrict__ gdx, const Cx<R>* __restrict__ gax,
                                           const Cx<R>* __restrict__ gdy, const Cx<R>* __restrict__ gay,
                                           const Cx<R>* __restrict__ gdz, const Cx<R>* __restrict__ gaz,
                                           const unsigned free_mask, const int bx, const int by) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int nz = g.nz, ny = g.ny, nxh = g.nxh;
  const int ncl = g.ncomp;  // lines per column: 6, or 36 for Kuhn tetrahedra
  const int kx0 = bx * TX, ky = by;
  const int tv = min(TX, nxh - kx0);
  const int plane = nz * TX;
  for (int idx = threadIdx.x; idx < ncl * plane; idx += blockDim.x) {
    const int c = idx / plane, rem = idx - c * plane;
    const int z = rem / TX, t = rem - z * TX;
    buf[idx] = t < tv ? spec[(((long long)c * nz + z) * ny + ky) * nxh + kx0 + t] : C{0, 0};
  }
  __syncthreads();
  const LineMap lm{TX, plane, 1, TX};
  fft_lines<kZEpt, false, true>(buf, pz, ncl * TX, lm, tw);
  const C ay = gay[ky], dy = gdy[ky];
  for (int pt = threadIdx.x; pt < plane; pt += blockDim.x) {
    const int z = pt / TX, t = pt - z * TX;
    const int kx = kx0 + t;
    if (t >= tv) continue;
    if (ncl == 36) {
      const C d[3] = {gdx[kx], dy, gdz[z]};
      const C e[3] = {C{(R)1 + d[0].x, d[0].y}, C{(R)1 + d[1].x, d[1].y}, C{(R)1 + d[2].x, d[2].y}};
      project_simplex3<R>(buf + pt, plane, e, d, kx == 0 && ky == 0 && z == 0, free_mask);
      continue;
    }
    C m[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) m[c] = buf[c * plane + pt];
    const C ax = gax[kx], dx = gdx[kx], az = gaz[z], dz = gdz[z];
    const C d0 = cmul(cmul(dx, ay), az);
    const C d1 = cmul(cmul(ax, dy), az);
    const C d2 = cmul(cmul(ax, ay), dz);
    project3<R>(m, d0, d1, d2, kx == 0 && ky == 0 && z == 0, free_mask);
#pragma unroll
    for (int c = 0; c < 6; ++c) buf[c * plane + pt] = m[c];
  }
  __syncthreads();
  fft_lines<kZEpt, true, true>(buf, pz, ncl * TX, lm, tw);
  for (int idx = threadIdx.x; idx < ncl * plane; idx += blockDim.x) {
    const int c = idx / plane, rem = idx - c * plane;
    const int z = rem / TX, t = rem - z * TX;
    if (t < tv) spec[(((long long)c * nz + z) * ny + ky) * nxh + kx0 + t] = buf[idx];
  }
}

template <typename R>
__global__ void __launch_bounds__(kZThreads)
    k_zproj(Cx<R>* __restrict__ spec, const GridDesc g, const int TX, const AxisPlan pz,
            const Cx<R>* __restrict__ tw, const Cx<R>* __restrict__ gdx, const Cx<R>* __restrict__ gax,
            const Cx<R>* __restrict__ gdy, const Cx<R>* __restrict__ gay, const Cx<R>* __restrict__ gdz,
            const Cx<R>* __restrict__ gaz, const unsigned free_mask) {
  zproj_body<R>(spec, g, TX, pz, tw, gdx, gax, gdy, gay, gdz, gaz, free_mask, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------- y + projection (2D)
template <typename R>
__device__ __forceinline__ void yproj2d_body(Cx<R>* __restrict__ spec, const GridDesc& g, const int TX,
                                             const AxisPlan& py, const Cx<R>* __restrict__ tw,
                                             const Cx<R>* __restrict__ gdx, const Cx<R>* __restrict__ gax,
                                             const Cx<R>* __restrict__ gdy, const Cx<R>* __restrict__ gay,
                                             const unsigned free_mask, const int bx) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int ny = g.ny, nxh = g.nxh, ncl = g.ncomp;  // lines per column: 3, or 6 for Kuhn triangles
  const int kx0 = bx * TX;
  const int tv = min(TX, nxh - kx0);
  const int plane = ny * TX;
  for (int idx = threadIdx.x; idx < ncl * plane; idx += blockDim.x) {
    const int c = idx / plane, rem = idx - c * plane;
    const int y = rem / TX, t = rem - y * TX;
    buf[idx] = t < tv ? spec[((long long)c * ny + y) * nxh + kx0 + t] : C{0, 0};
  }
  __syncthreads();
  const LineMap lm{TX, plane, 1, TX};
  fft_lines<kYEpt, false, true>(buf, py, ncl * TX, lm, tw);
  for (int pt = threadIdx.x; pt < plane; pt += blockDim.x) {
    const int y = pt / TX, t = pt - y * TX;
    const int kx = kx0 + t;
    if (t >= tv) continue;
    if (ncl == 6) {
      C m[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) m[c] = buf[c * plane + pt];
      const C dx = gdx[kx], dy = gdy[y];
      project_simplex2<R>(m, C{(R)1 + dx.x, dx.y}, dx, C{(R)1 + dy.x, dy.y}, dy, kx == 0 && y == 0, free_mask);
#pragma unroll
      for (int c = 0; c < 6; ++c) buf[c * plane + pt] = m[c];
      continue;
    }
    C m[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) m[c] = buf[c * plane + pt];
    const C d0 = cmul(gdx[kx], gay[y]);
    const C d1 = cmul(gax[kx], gdy[y]);
    project2<R>(m, d0, d1, kx == 0 && y == 0, free_mask);
#pragma unroll
    for (int c = 0; c < 3; ++c) buf[c * plane + pt] = m[c];
  }
  __syncthreads();
  fft_lines<kYEpt, true, true>(buf, py, ncl * TX, lm, tw);
  for (int idx = threadIdx.x; idx < ncl * plane; idx += blockDim.x) {
    const int c = idx / plane, rem = idx - c * plane;
    const int y = rem / TX, t = rem - y * TX;
    if (t < tv) spec[((long long)c * ny + y) * nxh + kx0 + t] = buf[idx];
  }
}

template <typename R>
__global__ void __launch_bounds__(kYThreads, kXYMinBlocks)
    k_yproj2d(Cx<R>* __restrict__ spec, const GridDesc g, const int TX, const AxisPlan py,
              const Cx<R>* __restrict__ tw, const Cx<R>* __restrict__ gdx, const Cx<R>* __restrict__ gax,
              const Cx<R>* __restrict__ gdy, const Cx<R>* __restrict__ gay, const unsigned free_mask) {
  yproj2d_body<R>(spec, g, TX, py, tw, gdx, gax, gdy, gay, free_mask, blockIdx.x);
}

// ------------------------------------------------------------ x inverse
// Pairs of half spectra are recombined as Z = Xa + i Xb over the full
// length (Hermitian extension; the imaginary parts of the k = 0 and
// Nyquist bins are dropped, as for any complex-to-real transform), one
// inverse complex FFT gives both real rows.  DOT adds sum(out * w) in FP64.
template <typename R, bool DOT>
__device__ __forceinline__ void xinv_body(const Cx<R>* __restrict__ spec, R* __restrict__ out,
                                          const R* __restrict__ dotw, double* __restrict__ partial,
                                          const GridDesc& g, const int Q, const AxisPlan& px,
                                          const Cx<R>* __restrict__ tw, const R scale, const bool self_dot,
                                          const int bx) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[32];
  const int nx = g.nx, nc = g.ncomp, nxh = g.nxh, half = nx >> 1;
  const long long row0 = (long long)bx * Q;
  const int npair = (nc * Q) >> 1;
  for (int idx = threadIdx.x; idx < npair * nx; idx += blockDim.x) {
    const int p = idx / nx, k = idx - p * nx;
    C xh[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rho = 2 * p + h;
      const int q = rho / nc, c = rho - q * nc;
      const long long row = row0 + q;
      C x = C{0, 0};
      if (q < Q && row < g.nrows) {
        const int kk = k <= half ? k : nx - k;
        x = spec[(c * g.nrows + row) * nxh + kk];
        if (kk == 0 || kk == half) x.y = 0;
        if (k > half) x.y = -x.y;
      }
      xh[h] = x;
    }
    buf[idx] = C{xh[0].x - xh[1].y, xh[0].y + xh[1].x};
  }
  __syncthreads();
  fft_lines<kXEpt, true, false>(buf, px, npair, LineMap{1, nx, 0, 1}, tw);
  KSum<R> acc;
  for (int idx = threadIdx.x; idx < 2 * npair * nx; idx += blockDim.x) {
    const int rho = idx / nx, x = idx - rho * nx;
    const int q = rho / nc, c = rho - q * nc;
    const long long row = row0 + q;
    if (q < Q && row < g.nrows) {
      const C z = buf[(rho >> 1) * nx + x];
      const R val = ((rho & 1) ? z.y : z.x) * scale;
      const long long off = c * g.nvox + row * nx + x;
      out[off] = val;
      if (DOT) acc.add(val * (self_dot ? val : dotw[off]));
    }
  }
  if (DOT) {
    double v[1] = {acc.value()};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) *partial = v[0];
  }
}

template <typename R, bool DOT>
__global__ void __launch_bounds__(kXThreads, kXYMinBlocks)
    k_xinv(const Cx<R>* __restrict__ spec, R* __restrict__ out, const R* __restrict__ dotw,
           double* __restrict__ partials, const GridDesc g, const int Q, const AxisPlan px,
           const Cx<R>* __restrict__ tw, const R scale, const bool self_dot) {
  xinv_body<R, DOT>(spec, out, dotw, DOT ? partials + blockIdx.x : nullptr, g, Q, px, tw, scale, self_dot,
                    blockIdx.x);
}

}  // namespace rve
