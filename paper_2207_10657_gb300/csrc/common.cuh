// Shared device-side definitions: complex helpers, the shared-memory
// mixed-radix Stockham FFT engine, material tables and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rve {

// ---------------------------------------------------------------- complex
template <typename R> struct CxT;
template <> struct CxT<float> { using T = float2; };
template <> struct CxT<double> { using T = double2; };
template <typename R> using Cx = typename CxT<R>::T;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return C{a.x * s, a.y * s}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}

// ------------------------------------------------------------- FFT plans
constexpr int kMaxStages = 12;
constexpr int kMaxPhases = 16;

struct AxisPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
};

// Line addressing inside a shared-memory tile: line l starts at
// (l / lpg) * gs + (l % lpg) * ls and its elements are es apart.
struct LineMap {
  int lpg, gs, ls, es;
  __device__ __forceinline__ int base(int l) const { return (l / lpg) * gs + (l % lpg) * ls; }
};

// ------------------------------------------------------ radix butterflies
// Small DFTs with the constants of the R-th roots of unity written out.
template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<2, INV, C> {
  __device__ __forceinline__ static void run(C* a) {
    C t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};

template <bool INV, typename C> struct Dft<4, INV, C> {
  __device__ __forceinline__ static void run(C* a) {
    C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    C t2 = cadd(a[1], a[3]), t3 = rot90<INV>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};

template <bool INV, typename C> struct Dft<8, INV, C> {
  __device__ __forceinline__ static void run(C* a) {
    using R = decltype(a[0].x);
    const R h = (R)0.70710678118654752440;  // sqrt(2)/2
    C e[4] = {a[0], a[2], a[4], a[6]};
    C o[4] = {a[1], a[3], a[5], a[7]};
    Dft<4, INV, C>::run(e);
    Dft<4, INV, C>::run(o);
    // twiddles w8^k, k = 0..3 (w8 = e^{-i pi/4} forward)
    C o1 = INV ? C{h * (o[1].x - o[1].y), h * (o[1].x + o[1].y)}
               : C{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};
    C o2 = rot90<INV>(o[2]);
    C o3 = INV ? C{-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y)}
               : C{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};
    a[0] = cadd(e[0], o[0]);
    a[4] = csub(e[0], o[0]);
    a[1] = cadd(e[1], o1);
    a[5] = csub(e[1], o1);
    a[2] = cadd(e[2], o2);
    a[6] = csub(e[2], o2);
    a[3] = cadd(e[3], o3);
    a[7] = csub(e[3], o3);
  }
};

template <bool INV, typename C> struct Dft<3, INV, C> {
  __device__ __forceinline__ static void run(C* a) {
    using R = decltype(a[0].x);
    const R c = (R)-0.5;
    const R s = (R)0.86602540378443864676;  // sin(2 pi / 3)
    C t = cadd(a[1], a[2]);
    C u = csub(a[1], a[2]);
    C m = C{a[0].x + c * t.x, a[0].y + c * t.y};
    C w = rot90<INV>(C{s * u.x, s * u.y});
    a[0] = cadd(a[0], t);
    a[1] = cadd(m, w);
    a[2] = csub(m, w);
  }
};

template <bool INV, typename C> struct Dft<5, INV, C> {
  __device__ __forceinline__ static void run(C* a) {
    using R = decltype(a[0].x);
    const R c1 = (R)0.30901699437494742410, s1 = (R)0.95105651629515357212;
    const R c2 = (R)-0.80901699437494742410, s2 = (R)0.58778525229247312917;
    C t1 = cadd(a[1], a[4]), u1 = csub(a[1], a[4]);
    C t2 = cadd(a[2], a[3]), u2 = csub(a[2], a[3]);
    C m1 = C{a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y};
    C m2 = C{a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y};
    C w1 = rot90<INV>(C{s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y});
    C w2 = rot90<INV>(C{s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y});
    a[0] = cadd(a[0], cadd(t1, t2));
    a[1] = cadd(m1, w1);
    a[4] = csub(m1, w1);
    a[2] = cadd(m2, w2);
    a[3] = csub(m2, w2);
  }
};

// ---------------------------------------------------- Stockham FFT engine
// One radix-R stage of the self-sorting (Stockham) FFT over `nlines`
// lines of length n held in shared memory, in place: every thread first
// loads and transforms its butterflies into registers, the block
// synchronises, then every thread stores.  Stage with current span Ns:
// butterfly j of a line reads elements j + r*n/R, multiplies by the
// twiddle w_n^{r*(j mod Ns)*n/(Ns*R)}, applies the R-point DFT and writes
// element (j/Ns)*Ns*R + (j mod Ns) + r*Ns.  `LINE_FAST` maps consecutive
// threads to consecutive lines (for tiles whose lines are interleaved in
// shared memory) instead of consecutive butterflies of one line.
template <int R, int EPT, bool INV, bool LINE_FAST, typename C>
__device__ __forceinline__ void stockham_stage(C* buf, int n, int Ns, int nlines, const LineMap lm,
                                               const C* __restrict__ tw) {
  constexpr int MAXB = (EPT + R - 1) / R;
  const int nbl = n / R;
  const int total = nlines * nbl;
  const int tstep = n / (Ns * R);
  C v[MAXB][R];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * blockDim.x;
    if (b < total) {
      int l, j;
      if (LINE_FAST) { j = b / nlines; l = b - j * nlines; }
      else { l = b / nbl; j = b - l * nbl; }
      const int k = j % Ns;
      const int base = lm.base(l);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = buf[base + (j + r * nbl) * lm.es];
        if (r > 0 && k > 0) {
          C w = __ldg(&tw[r * k * tstep]);
          x = INV ? cmulc(x, w) : cmul(x, w);
        }
        v[i][r] = x;
      }
      Dft<R, INV, C>::run(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * blockDim.x;
    if (b < total) {
      int l, j;
      if (LINE_FAST) { j = b / nlines; l = b - j * nlines; }
      else { l = b / nbl; j = b - l * nbl; }
      const int k = j % Ns;
      const int base = lm.base(l);
      const int d0 = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[base + (d0 + r * Ns) * lm.es] = v[i][r];
    }
  }
  __syncthreads();
}

// Full transform of every line (forward: sum x_j e^{-2 pi i jk/n}; inverse:
// conjugate kernel, unnormalised).  Caller synchronises before the call.
template <int EPT, bool INV, bool LINE_FAST, typename C>
__device__ void fft_lines(C* buf, const AxisPlan& p, int nlines, const LineMap lm, const C* __restrict__ tw) {
  int Ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s];
    switch (R) {
      case 8: stockham_stage<8, EPT, INV, LINE_FAST>(buf, p.n, Ns, nlines, lm, tw); break;
      case 4: stockham_stage<4, EPT, INV, LINE_FAST>(buf, p.n, Ns, nlines, lm, tw); break;
      case 2: stockham_stage<2, EPT, INV, LINE_FAST>(buf, p.n, Ns, nlines, lm, tw); break;
      case 3: stockham_stage<3, EPT, INV, LINE_FAST>(buf, p.n, Ns, nlines, lm, tw); break;
      default: stockham_stage<5, EPT, INV, LINE_FAST>(buf, p.n, Ns, nlines, lm, tw); break;
    }
    Ns *= R;
  }
}

// ------------------------------------------------------- material tables
template <typename R> struct MatTable {
  int nphase;
  R lam[kMaxPhases], mu[kMaxPhases];
  R kappa0[kMaxPhases], kappaf[kMaxPhases];
  int damaging[kMaxPhases];
};

// --------------------------------------------------------- reductions
// Neumaier-compensated FP32/FP64 per-thread sums, FP64 across threads.
template <typename R> struct KSum {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R x) {
    R t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Block-wide FP64 sum of NS values; result valid in thread 0.  `sh` must
// hold NS * 32 doubles.
template <int NS>
__device__ __forceinline__ void block_sum(double (&v)[NS], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[s * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = lane < nw ? sh[s * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[s] = x;
    }
  }
  __syncthreads();
}

// out[s] = sum_b part[b * NS + s], s < NS, summed by one block as the
// separate reduction kernel k_reduce_partials does -- thread t < 256 (every
// thread of a smaller block) adds blocks t, t + 256, ... in that order, then
// the block-wide FP64 sum -- so the results agree bit for bit.  The NS sums
// share one sweep whose loads are issued U blocks at a time: ten thousand
// partials cost a few L2 round trips rather than one per partial.  The
// partials are read through L2 (other blocks of the grid wrote them).
// Called by every thread of the block; `sh` holds NS * 32 doubles, free on
// entry; thread 0 writes out.
template <int NS>
__device__ void block_reduce_partials(const double* part, int nblocks, double* out, double* sh) {
  constexpr int U = 8;
  const int stride = blockDim.x < 256 ? (int)blockDim.x : 256;
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  if ((int)threadIdx.x < stride) {
    int b = threadIdx.x;
#pragma unroll 1
    for (; b + (U - 1) * stride < nblocks; b += U * stride) {
      double v[U][NS];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int s = 0; s < NS; ++s) v[u][s] = __ldcg(part + (long long)(b + u * stride) * NS + s);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int s = 0; s < NS; ++s) acc[s] += v[u][s];
    }
#pragma unroll 1
    for (; b < nblocks; b += stride)
#pragma unroll
      for (int s = 0; s < NS; ++s) acc[s] += __ldcg(part + (long long)b * NS + s);
  }
  block_sum<NS>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) out[s] = acc[s];
  }
}

// Called by every thread of every block once thread 0 has written the
// block's NS partial sums to part[block * NS + s].  The last block to arrive
// (thread 0 fences its partials, then one atomic on `counter`) sums them with
// block_reduce_partials, resets the counter for the next launch and returns
// true; the other blocks return false.  No block waits on another.  Meant
// for grids of a few hundred blocks: the fence holds thread 0 until its
// stores are visible, which a grid of many short-lived blocks would pay once
// per block.  `sh` holds NS * 32 doubles, free on entry.
template <int NS>
__device__ bool reduce_in_last_block(const double* part, int nblocks, double* out, unsigned* counter, double* sh) {
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(counter, 1u) == (unsigned)nblocks - 1u ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  block_reduce_partials<NS>(part, nblocks, out, sh);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

}  // namespace rve
