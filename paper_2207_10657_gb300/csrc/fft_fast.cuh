// Compile-time-specialised Stockham FFT for lines held in shared memory.
//
// All sizes are template constants so the per-stage index arithmetic
// reduces to shifts and multiplies and each stage keeps only its own radix
// in registers.  Shared-memory layout is line-interleaved: element j of
// line l lives at buf[j * NL + l], so consecutive threads work on
// consecutive lines and both the reads and the writes of a stage are
// (nearly) bank-conflict free.
#pragma once

#include "common.cuh"

namespace rve {

// Radix policy: radix 8 as far as possible, 4 (or 4x4) for the remaining
// factors of two, then 3s, then 5s.
constexpr int fft_twos(int n) { return (n % 2 == 0) ? 1 + fft_twos(n / 2) : 0; }
constexpr int fft_odd(int n) { return (n % 2 == 0) ? fft_odd(n / 2) : n; }
constexpr int fft_threes(int m) { return (m % 3 == 0) ? 1 + fft_threes(m / 3) : 0; }
constexpr int fft_fives(int m) { return (m % 5 == 0) ? 1 + fft_fives(m / 5) : 0; }
constexpr int fft_n8(int n) {
  return (fft_twos(n) % 3 == 1 && fft_twos(n) >= 4) ? fft_twos(n) / 3 - 1 : fft_twos(n) / 3;
}
constexpr int fft_n4(int n) {
  return (fft_twos(n) % 3 == 2) ? 1 : ((fft_twos(n) % 3 == 1 && fft_twos(n) >= 4) ? 2 : 0);
}
constexpr int fft_n2(int n) { return (fft_twos(n) % 3 == 1 && fft_twos(n) < 4) ? 1 : 0; }
constexpr int fft_nstages(int n) {
  return fft_n8(n) + fft_n4(n) + fft_n2(n) + fft_threes(fft_odd(n)) + fft_fives(fft_odd(n));
}
constexpr int fft_radix(int n, int s) {
  return s < fft_n8(n) ? 8
         : s < fft_n8(n) + fft_n4(n) ? 4
         : s < fft_n8(n) + fft_n4(n) + fft_n2(n) ? 2
         : s < fft_n8(n) + fft_n4(n) + fft_n2(n) + fft_threes(fft_odd(n)) ? 3
                                                                            : 5;
}
constexpr int fft_span(int n, int s) { return s == 0 ? 1 : fft_span(n, s - 1) * fft_radix(n, s - 1); }

// One stage (see stockham_stage in common.cuh for the index scheme).
template <int N, int NL, int NT, bool INV, int S, typename C>
__device__ __forceinline__ void fft_stage_ct(C* buf, const C* __restrict__ tw) {
  constexpr int R = fft_radix(N, S);
  constexpr int NS = fft_span(N, S);
  constexpr int NBL = N / R;
  constexpr int TOTAL = NL * NBL;
  constexpr int PER = (TOTAL + NT - 1) / NT;
  constexpr int TSTEP = N / (NS * R);
  C v[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = threadIdx.x + i * NT;
    if ((TOTAL % NT) == 0 || b < TOTAL) {
      const int j = b / NL, l = b - (b / NL) * NL;
      const int k = j % NS;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = buf[(j + r * NBL) * NL + l];
        if (NS > 1 && r > 0) {
          const C w = __ldg(&tw[r * k * TSTEP]);
          x = INV ? cmulc(x, w) : cmul(x, w);
        }
        v[i][r] = x;
      }
      Dft<R, INV, C>::run(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = threadIdx.x + i * NT;
    if ((TOTAL % NT) == 0 || b < TOTAL) {
      const int j = b / NL, l = b - (b / NL) * NL;
      const int k = j % NS;
      const int d0 = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(d0 + r * NS) * NL + l] = v[i][r];
    }
  }
  __syncthreads();
}

// Stages [S, SEND) in shared memory.
template <int N, int NL, int NT, bool INV, int S, int SEND, typename C>
__device__ __forceinline__ void fft_ct_range(C* buf, const C* __restrict__ tw) {
  if constexpr (S < SEND) {
    fft_stage_ct<N, NL, NT, INV, S>(buf, tw);
    fft_ct_range<N, NL, NT, INV, S + 1, SEND>(buf, tw);
  }
}

// First stage with its inputs read through load(line, element) (global
// memory) instead of from a staged copy in shared memory; its outputs go to
// `buf`.  The stage has span 1 (no twiddles).  `buf` must not be in use by
// other threads.  Ends with a barrier.
template <int N, int NL, int NT, bool INV, typename C, typename LoadF>
__device__ __forceinline__ void fft_stage0_from(C* buf, LoadF load) {
  constexpr int R = fft_radix(N, 0);
  constexpr int NBL = N / R;
  constexpr int TOTAL = NL * NBL;
  constexpr int PER = (TOTAL + NT - 1) / NT;
  C v[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = threadIdx.x + i * NT;
    if ((TOTAL % NT) == 0 || b < TOTAL) {
      const int j = b / NL, l = b - (b / NL) * NL;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = load(l, j + r * NBL);
    }
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = threadIdx.x + i * NT;
    if ((TOTAL % NT) == 0 || b < TOTAL) {
      const int j = b / NL, l = b - (b / NL) * NL;
      Dft<R, INV, C>::run(v[i]);
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(j * R + r) * NL + l] = v[i][r];
    }
  }
  __syncthreads();
}

// Last stage reading `buf` and handing its outputs to store(line, element,
// value) (global memory) instead of writing them back.  The caller has
// synchronised after the previous stage.
template <int N, int NL, int NT, bool INV, typename C, typename StoreF>
__device__ __forceinline__ void fft_stage_last_to(const C* buf, const C* __restrict__ tw, StoreF store) {
  constexpr int S = fft_nstages(N) - 1;
  constexpr int R = fft_radix(N, S);
  constexpr int NS = fft_span(N, S);
  constexpr int NBL = N / R;
  constexpr int TOTAL = NL * NBL;
  constexpr int PER = (TOTAL + NT - 1) / NT;
  constexpr int TSTEP = N / (NS * R);
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = threadIdx.x + i * NT;
    if ((TOTAL % NT) == 0 || b < TOTAL) {
      const int j = b / NL, l = b - (b / NL) * NL;
      const int k = j % NS;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = buf[(j + r * NBL) * NL + l];
        if (NS > 1 && r > 0) {
          const C w = __ldg(&tw[r * k * TSTEP]);
          x = INV ? cmulc(x, w) : cmul(x, w);
        }
        v[r] = x;
      }
      Dft<R, INV, C>::run(v);
      const int d0 = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) store(l, d0 + r * NS, v[r]);
    }
  }
}

template <int N, int NL, int NT, bool INV, int S = 0, typename C>
__device__ __forceinline__ void fft_ct(C* buf, const C* __restrict__ tw) {
  if constexpr (S < fft_nstages(N)) {
    fft_stage_ct<N, NL, NT, INV, S>(buf, tw);
    fft_ct<N, NL, NT, INV, S + 1>(buf, tw);
  }
}

}  // namespace rve
