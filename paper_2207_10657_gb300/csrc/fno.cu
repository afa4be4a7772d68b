// Spectral neural operator of the learned warm start: forward, backward and
// Adam, all on the GPU in hand-written kernels.
//
// Dense contractions run on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation): the 1x1 channel mixes, the truncated DFTs
// (written as real matrix products along one axis at a time, the complex
// (Re, Im) pair folded into the transformed axis) and the per-mode mixing.
// Activations are FP32 in memory and rounded to BF16 when staged as
// operands; the per-mode weights are stored in BF16.
//
// Network (channels last, [B][Nz][Ny][Nx][C]): h0 = X Wl + bl; for each
// layer u = K(h) + h W + b, h = GELU(u) (not after the last layer);
// Y = h Wq + bq.  K: forward DFT, keep kx in [0, m), ky, kz in [-m/2, m/2),
// map each mode's (Re, Im) channel pairs by a real 2C x 2C matrix, real
// inverse DFT of the half spectrum.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/rve.h"
#include "common.cuh"

namespace {

using rve::block_sum;

// ================================================================ GEMM
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b], op(A) M x K, op(B) K x N.
// A(m,k) = TA ? A[k*lda + m] : A[m*lda + k]; B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n].
struct GemmArgs {
  int M, N, K;
  const void* A;
  long long lda, sA;
  const void* B;
  long long ldb, sB;
  float* C;
  long long ldc, sC;
  float alpha, beta;
  int batch, ksplit, kchunk;  // ksplit > 1: K is cut in chunks whose products are added atomically into C
  int vecA, vecB;              // operand rows and batch strides are 16-byte aligned: float4 staging
};

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

template <typename T> __device__ __forceinline__ float ldf(const T* p, long long i);
template <> __device__ __forceinline__ float ldf<float>(const float* p, long long i) { return p[i]; }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename TA_T, typename TB_T, bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];  // [n][k]
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  for (int zz = blockIdx.z; zz < g.batch * g.ksplit; zz += gridDim.z) {
    const int bz = zz / g.ksplit, ks0 = zz - bz * g.ksplit;
    const TA_T* A = static_cast<const TA_T*>(g.A) + bz * g.sA;
    const TB_T* B = static_cast<const TB_T*>(g.B) + bz * g.sB;
    float* C = g.C + bz * g.sC;
    const int kbeg = ks0 * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
      // Stage the A and B tiles as BF16.  With aligned operands every
      // thread moves 4 consecutive elements of the contiguous dimension per
      // float4 load; ragged edges fall back to guarded scalar loads.
      if (g.vecA) {
        constexpr int CH = GBM * GBK / 4;
        for (int e = threadIdx.x; e < CH; e += 128) {
          float v[4];
          if (TA) {  // contiguous along m
            const int kk = e / (GBM / 4), mm = 4 * (e % (GBM / 4));
            const int gm = m0 + mm, gk = k0 + kk;
            if (gk < kend && gm + 3 < g.M) {
              const float4 q = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(A) + (long long)gk * g.lda + gm);
              v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                v[i] = (gk < kend && gm + i < g.M) ? ldf<TA_T>(A, (long long)gk * g.lda + gm + i) : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) As[mm + i][kk] = __float2bfloat16(v[i]);
          } else {  // contiguous along k
            const int mm = e / (GBK / 4), kk = 4 * (e % (GBK / 4));
            const int gm = m0 + mm, gk = k0 + kk;
            if (gm < g.M && gk + 3 < kend) {
              const float4 q = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(A) + (long long)gm * g.lda + gk);
              v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                v[i] = (gm < g.M && gk + i < kend) ? ldf<TA_T>(A, (long long)gm * g.lda + gk + i) : 0.f;
            }
            __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t*>(&lo);
            w.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(&As[mm][kk]) = w;
          }
        }
      } else {
        for (int e = threadIdx.x; e < GBM * GBK; e += 128) {
          int mm, kk;
          if (TA) { mm = e % GBM; kk = e / GBM; }  // consecutive threads: consecutive m (contiguous)
          else { kk = e % GBK; mm = e / GBK; }
          const int gm = m0 + mm, gk = k0 + kk;
          float v = 0.f;
          if (gm < g.M && gk < kend)
            v = ldf<TA_T>(A, TA ? (long long)gk * g.lda + gm : (long long)gm * g.lda + gk);
          As[mm][kk] = __float2bfloat16(v);
        }
      }
      if (g.vecB) {
        constexpr int CH = GBN * GBK / 4;
        for (int e = threadIdx.x; e < CH; e += 128) {
          float v[4];
          if (TB) {  // contiguous along k
            const int nn = e / (GBK / 4), kk = 4 * (e % (GBK / 4));
            const int gn = n0 + nn, gk = k0 + kk;
            if (gn < g.N && gk + 3 < kend) {
              const float4 q = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(B) + (long long)gn * g.ldb + gk);
              v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                v[i] = (gn < g.N && gk + i < kend) ? ldf<TB_T>(B, (long long)gn * g.ldb + gk + i) : 0.f;
            }
            __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t*>(&lo);
            w.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(&Bs[nn][kk]) = w;
          } else {  // contiguous along n
            const int kk = e / (GBN / 4), nn = 4 * (e % (GBN / 4));
            const int gn = n0 + nn, gk = k0 + kk;
            if (gk < kend && gn + 3 < g.N) {
              const float4 q = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(B) + (long long)gk * g.ldb + gn);
              v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                v[i] = (gk < kend && gn + i < g.N) ? ldf<TB_T>(B, (long long)gk * g.ldb + gn + i) : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) Bs[nn + i][kk] = __float2bfloat16(v[i]);
          }
        }
      } else {
        for (int e = threadIdx.x; e < GBN * GBK; e += 128) {
          int nn, kk;
          if (TB) { kk = e % GBK; nn = e / GBK; }
          else { nn = e % GBN; kk = e / GBN; }
          const int gn = n0 + nn, gk = k0 + kk;
          float v = 0.f;
          if (gn < g.N && gk < kend)
            v = ldf<TB_T>(B, TB ? (long long)gn * g.ldb + gk : (long long)gk * g.ldb + gn);
          Bs[nn][kk] = __float2bfloat16(v);
        }
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < GBK; ks += 16) {
        uint32_t af[2][4], bf[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int r = wm + i * 16 + gq;
          af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq]);
          af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq]);
          af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq + 8]);
          af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int cidx = wn + j * 8 + gq;
          bf[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[cidx][ks + 2 * tq]);
          bf[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[cidx][ks + 2 * tq + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = m0 + wm + i * 16 + gq + (q >= 2 ? 8 : 0);
          const int cc = n0 + wn + j * 8 + 2 * tq + (q & 1);
          if (r < g.M && cc < g.N) {
            float* p = C + (long long)r * g.ldc + cc;
            const float v = g.alpha * acc[i][j][q];
            if (g.ksplit > 1) atomicAdd(p, v);
            else *p = (g.beta == 0.f) ? v : v + g.beta * *p;
          }
        }
  }
}

// ============================================================ mode mixing
// S layout [b][s][m][c] (s = Re/Im, m = retained mode, c < C = 32), per-mode
// weights R[m][(s_o, o)][(s_i, c)] (64 x 64, BF16).  One warp per mode.
//  mode 0: out = R S        (forward)
//  mode 1: out = R^T S      (input gradient)
constexpr int kW = 32, kW2 = 64;

template <int MODE>
__global__ void __launch_bounds__(128)
    k_modemix(const __nv_bfloat16* __restrict__ R, const float* __restrict__ S, float* __restrict__ out, int nmodes,
              int batch) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nmodes) return;
  const int m = warp, gq = lane >> 2, tq = lane & 3;
  const __nv_bfloat16* Rm = R + (long long)m * kW2 * kW2;
  const long long sstride = (long long)nmodes * kW;  // between s = 0 and s = 1
  const long long bstride = 2 * sstride;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
  // B fragment: k = (s_i, c), n = batch index gq
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    uint32_t bf[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = kt * 16 + 2 * tq + 8 * h;
      const int si = k >> 5, c = k & 31;
      float v0 = 0.f, v1 = 0.f;
      if (gq < batch) {
        const float* p = S + gq * bstride + si * sstride + (long long)m * kW + c;
        v0 = p[0];
        v1 = p[1];
      }
      __nv_bfloat162 t = __floats2bfloat162_rn(v0, v1);
      bf[h] = *reinterpret_cast<uint32_t*>(&t);
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      uint32_t af[4];
      const int r = mt * 16 + gq;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rr = r + ((q & 1) ? 8 : 0);
        const int kk = kt * 16 + 2 * tq + ((q & 2) ? 8 : 0);
        __nv_bfloat162 t;
        if (MODE == 0) {
          t = *reinterpret_cast<const __nv_bfloat162*>(Rm + rr * kW2 + kk);
        } else {
          t.x = Rm[kk * kW2 + rr];
          t.y = Rm[(kk + 1) * kW2 + rr];
        }
        af[q] = *reinterpret_cast<uint32_t*>(&t);
      }
      mma_bf16(acc[mt], af, bf);
    }
  }
  // C fragment: rows (s_o, o), column = batch index 2tq + {0,1}
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = mt * 16 + gq + (q >= 2 ? 8 : 0);
      const int b = 2 * tq + (q & 1);
      if (b < batch) {
        const int so = row >> 5, o = row & 31;
        out[b * bstride + so * sstride + (long long)m * kW + o] = acc[mt][q];
      }
    }
}

// dR[m] += dOut_m (64 x B) In_m^T (B x 64); K = batch (<= 16), one warp per mode.
__global__ void __launch_bounds__(128)
    k_modemix_grad(const float* __restrict__ dOut, const float* __restrict__ In, float* __restrict__ dR, int nmodes,
                   int batch) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nmodes) return;
  const int m = warp, gq = lane >> 2, tq = lane & 3;
  const long long sstride = (long long)nmodes * kW, bstride = 2 * sstride;
  auto at = [&](const float* T, int b, int row) -> float {
    if (b >= batch) return 0.f;
    return T[b * bstride + (row >> 5) * sstride + (long long)m * kW + (row & 31)];
  };
  float* dRm = dR + (long long)m * kW2 * kW2;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    uint32_t af[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = mt * 16 + gq + ((q & 1) ? 8 : 0);
      const int k = 2 * tq + ((q & 2) ? 8 : 0);
      __nv_bfloat162 t = __floats2bfloat162_rn(at(dOut, k, row), at(dOut, k + 1, row));
      af[q] = *reinterpret_cast<uint32_t*>(&t);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t bf[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * tq + 8 * h, col = nt * 8 + gq;
        __nv_bfloat162 t = __floats2bfloat162_rn(at(In, k, col), at(In, k + 1, col));
        bf[h] = *reinterpret_cast<uint32_t*>(&t);
      }
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(acc, af, bf);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = mt * 16 + gq + (q >= 2 ? 8 : 0);
        const int col = nt * 8 + 2 * tq + (q & 1);
        dRm[row * kW2 + col] += acc[q];
      }
    }
  }
}

// ============================================================ elementwise
__device__ __forceinline__ float gelu_f(float x) {
  const float k = 0.7978845608028654f;  // sqrt(2/pi)
  return 0.5f * x * (1.f + tanhf(k * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_g(float x) {
  const float k = 0.7978845608028654f;
  const float t = tanhf(k * (x + 0.044715f * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * k * (1.f + 3.f * 0.044715f * x * x);
}

// u += bias (per channel); h = act ? gelu(u) : u
__global__ void k_bias_act(float* __restrict__ u, const float* __restrict__ bias, float* __restrict__ h, long long n,
                           int C, int act) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = u[i] + bias[i % C];
    u[i] = v;
    h[i] = act ? gelu_f(v) : v;
  }
}

__global__ void k_gelu_back(const float* __restrict__ dh, const float* __restrict__ u, float* __restrict__ du,
                            long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    du[i] = dh[i] * gelu_g(u[i]);
}

// [A][d1][d2][inner] -> [A][d2][d1][inner]
__global__ void k_swap(const float* __restrict__ in, float* __restrict__ out, long long A, int d1, int d2,
                       long long inner) {
  const long long n = A * d1 * d2 * inner;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i % inner;
    long long t = i / inner;
    const int j2 = (int)(t % d2);
    t /= d2;
    const int j1 = (int)(t % d1);
    const long long a = t / d1;
    out[((a * d2 + j2) * d1 + j1) * inner + r] = in[i];
  }
}

// MSE: loss partials and dY = 2 (Y - T) / n
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY, long long n,
                      double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = (float)(2.0 * d / (double)n);
    acc += (double)d * d;
  }
  double v[1] = {acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0] / (double)n;
}

// column sums (bias gradients): out[c] += sum_rows in[r][c]; one block per column
__global__ void k_colsum(const float* __restrict__ in, long long rows, int C, float* __restrict__ out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (long long r = threadIdx.x; r < rows; r += blockDim.x) acc += in[r * C + c];
  double v[1] = {acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) out[c] += (float)v[0];
}

// Adam on the packed parameter vector (FP32 master), BF16 refresh of the
// per-mode weights (their offsets listed in ranges).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// Features for the warm start, channels last [Nz][Ny][Nx][cin]: phase
// one-hot (2), damage (1), previous two fluctuation increments (SoA Mandel
// fields, ncomp each) times `scale`, then (if given and cin > 3 + 2 ncomp)
// the history variable kappa times `kscale`; remaining channels zero.
__global__ void k_pack(const uint8_t* __restrict__ phase, const float* __restrict__ dmg, const float* __restrict__ kap,
                       float kscale, const float* __restrict__ d1, const float* __restrict__ d2, long long nvox, int nc,
                       float scale, int cin, float* __restrict__ X) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
    float* x = X + v * cin;
    const int ph = phase[v];
    int k = 0;
    x[k++] = ph == 0 ? 1.f : 0.f;
    x[k++] = ph == 1 ? 1.f : 0.f;
    x[k++] = dmg ? dmg[v] : 0.f;
    for (int c = 0; c < nc; ++c) x[k++] = d1 ? d1[c * nvox + v] * scale : 0.f;
    for (int c = 0; c < nc; ++c) x[k++] = d2 ? d2[c * nvox + v] * scale : 0.f;
    if (k < cin) x[k++] = kap ? kap[v] * kscale : 0.f;
    for (; k < cin; ++k) x[k] = 0.f;
  }
}

// channels-last [V][cout] -> SoA [cout][V]: out = base + scale * Y (base may be NULL)
__global__ void k_unpack(const float* __restrict__ Y, const float* __restrict__ base, long long nvox, int cout,
                         float scale, float* __restrict__ out) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x)
    for (int c = 0; c < cout; ++c) out[c * nvox + v] = (base ? base[c * nvox + v] : 0.f) + Y[v * cout + c] * scale;
}

// SoA [cout][V] -> channels-last [V][cout]: T = scale * (f - base) (training targets; base may be NULL)
__global__ void k_pack_target(const float* __restrict__ f, const float* __restrict__ base, long long nvox, int cout,
                              float scale, float* __restrict__ T) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x)
    for (int c = 0; c < cout; ++c) T[v * cout + c] = (f[c * nvox + v] - (base ? base[c * nvox + v] : 0.f)) * scale;
}

// fluctuation increment: out = eps_new - eps_old - dE (uniform per component)
__global__ void k_incr(const float* __restrict__ a, const float* __restrict__ b, long long nvox, int ncomp, float d0,
                       float d1, float d2, float d3, float d4, float d5, float* __restrict__ out) {
  const float dE[6] = {d0, d1, d2, d3, d4, d5};
  const long long n = nvox * ncomp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i] - dE[i / nvox];
}

int nblk(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 16); }

}  // namespace

// ================================================================ network
struct rve_fno_ctx {
  int cin = 16, C = 32, cout = 6, L = 4, m = 16;
  cudaStream_t st = nullptr;
  long long nparam = 0;
  float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // packed master / grad / Adam moments
  __nv_bfloat16* Rbf = nullptr;                                     // per-mode weights, BF16 (all layers)
  long long offWl = 0, offbl = 0, offWq = 0, offbq = 0;
  std::vector<long long> offW, offb, offR;
  long long nR = 0;  // per layer R size
  int adam_t = 0;
  double* part = nullptr;
  float* tmpf = nullptr;
  // per-grid transform matrices (Fx, Fy, Fz, Gx, Gy, Gz)
  std::map<std::tuple<int, int, int>, std::vector<float*>> mats;
  // activations (grown on demand)
  std::vector<float*> H, U, S;  // per layer input h, pre-activation u, retained spectrum
  float *T1 = nullptr, *T2 = nullptr, *Y = nullptr, *dA = nullptr, *dB = nullptr, *dY = nullptr, *Xbuf = nullptr,
        *Tb = nullptr;
  long long cap_vox = 0;
  int cap_batch = 0;
  long long launches = 0;
  std::string err = "no error";
};

namespace {

thread_local std::string g_fno_err = "no error";

rve_status ffail(rve_fno_ctx* c, rve_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_fno_err = msg;
  return s;
}

#define FCK(call, where)                                                                              \
  do {                                                                                                \
    cudaError_t e__ = (call);                                                                         \
    if (e__ != cudaSuccess)                                                                           \
      return ffail(c, e__ == cudaErrorMemoryAllocation ? RVE_ERR_OOM : RVE_ERR_CUDA,                   \
                   std::string(where) + ": " + cudaGetErrorString(e__));                              \
  } while (0)

template <typename TA_T, typename TB_T>
cudaError_t gemm(rve_fno_ctx* c, bool ta, bool tb, int M, int N, int K, const TA_T* A, long long lda, long long sA,
                 const TB_T* B, long long ldb, long long sB, float* Cm, long long ldc, long long sC, int batch,
                 float alpha = 1.f, float beta = 0.f) {
  // long reductions with a single output tile are split along K
  // (only for a single, densely stored output with beta = 0, which is
  // zeroed first and then accumulated atomically)
  int ksplit = 1;
  const long long tiles = (long long)((M + GBM - 1) / GBM) * ((N + GBN - 1) / GBN) * batch;
  if (tiles < 152 && K > 4096 && batch == 1 && ldc == N && beta == 0.f) {
    ksplit = (int)std::min<long long>((K + 2047) / 2048, 1024);
    cudaError_t e = cudaMemsetAsync(Cm, 0, (size_t)M * N * sizeof(float), c->st);
    if (e != cudaSuccess) return e;
  }
  const int kchunk = ((K + ksplit - 1) / ksplit + GBK - 1) / GBK * GBK;
  auto al16 = [](const void* p, long long ld, long long st) {
    return ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld % 4 == 0 && st % 4 == 0) ? 1 : 0;
  };
  GemmArgs g{M, N, K, A, lda, sA, B, ldb, sB, Cm, ldc, sC, alpha, beta, batch, ksplit, kchunk,
             al16(A, lda, sA), al16(B, ldb, sB)};
  const int zdim = (int)std::min<long long>((long long)batch * ksplit, 65535);
  dim3 grid((M + GBM - 1) / GBM, (N + GBN - 1) / GBN, zdim);
  if (ta && tb) k_gemm<TA_T, TB_T, true, true><<<grid, 128, 0, c->st>>>(g);
  else if (ta) k_gemm<TA_T, TB_T, true, false><<<grid, 128, 0, c->st>>>(g);
  else if (tb) k_gemm<TA_T, TB_T, false, true><<<grid, 128, 0, c->st>>>(g);
  else k_gemm<TA_T, TB_T, false, false><<<grid, 128, 0, c->st>>>(g);
  ++c->launches;
  return cudaGetLastError();
}

cudaError_t swap_dims(rve_fno_ctx* c, const float* in, float* out, long long A, int d1, int d2, long long inner) {
  k_swap<<<nblk(A * d1 * d2 * inner), 256, 0, c->st>>>(in, out, A, d1, d2, inner);
  ++c->launches;
  return cudaGetLastError();
}

// transform matrices for grid (nx, ny, nz), m retained modes
rve_status get_mats(rve_fno_ctx* c, int nx, int ny, int nz, std::vector<float*>& out) {
  auto key = std::make_tuple(nx, ny, nz);
  auto it = c->mats.find(key);
  if (it != c->mats.end()) {
    out = it->second;
    return RVE_OK;
  }
  const int m = c->m, mh = m / 2;
  const double N = (double)nx * ny * nz;
  const double tau = 6.283185307179586476925286766559;
  // Fx [(s,kx)=2m][x]: cos, -sin
  std::vector<float> Fx(2 * m * nx), Gx((size_t)nx * 2 * m);
  for (int k = 0; k < m; ++k)
    for (int x = 0; x < nx; ++x) {
      const double th = tau * k * x / nx, cs = std::cos(th), sn = std::sin(th);
      Fx[k * nx + x] = (float)cs;
      Fx[(m + k) * nx + x] = (float)(-sn);
      const double w = (k == 0 ? 1.0 : 2.0) / N;
      Gx[(size_t)x * 2 * m + k] = (float)(w * cs);        // Re part
      Gx[(size_t)x * 2 * m + m + k] = (float)(-w * sn);   // Im part
    }
  // complex axis transforms: F (2m x 2n) rows (s_o, k), cols (s_i, j), e^{-i};
  // G (2n x 2m) rows (s_o, j), cols (s_i, k), e^{+i}
  auto cplx = [&](int n, std::vector<float>& F, std::vector<float>& G) {
    F.assign((size_t)2 * m * 2 * n, 0.f);
    G.assign((size_t)2 * n * 2 * m, 0.f);
    for (int q = 0; q < m; ++q) {
      const int k = q - mh;
      for (int j = 0; j < n; ++j) {
        const double th = tau * k * j / n, cs = std::cos(th), sn = std::sin(th);
        // forward: re_o = cs re + sn im; im_o = -sn re + cs im
        F[(size_t)q * 2 * n + j] = (float)cs;
        F[(size_t)q * 2 * n + n + j] = (float)sn;
        F[(size_t)(m + q) * 2 * n + j] = (float)(-sn);
        F[(size_t)(m + q) * 2 * n + n + j] = (float)cs;
        // inverse: re_o = cs re - sn im; im_o = sn re + cs im
        G[(size_t)j * 2 * m + q] = (float)cs;
        G[(size_t)j * 2 * m + m + q] = (float)(-sn);
        G[(size_t)(n + j) * 2 * m + q] = (float)sn;
        G[(size_t)(n + j) * 2 * m + m + q] = (float)cs;
      }
    }
  };
  std::vector<float> Fy, Gy, Fz, Gz;
  cplx(ny, Fy, Gy);
  cplx(nz, Fz, Gz);
  std::vector<std::vector<float>*> host = {&Fx, &Fy, &Fz, &Gx, &Gy, &Gz};
  std::vector<float*> dev;
  for (auto* h : host) {
    float* d = nullptr;
    FCK(cudaMalloc(&d, h->size() * sizeof(float)), "transform matrices");
    FCK(cudaMemcpy(d, h->data(), h->size() * sizeof(float), cudaMemcpyHostToDevice), "transform matrices");
    dev.push_back(d);
  }
  c->mats[key] = dev;
  out = dev;
  return RVE_OK;
}

rve_status ensure(rve_fno_ctx* c, int batch, long long nvox) {
  if (batch <= c->cap_batch && nvox <= c->cap_vox) return RVE_OK;
  const int B = std::max(batch, c->cap_batch);
  const long long V = std::max(nvox, c->cap_vox);
  for (float* q : c->H) cudaFree(q);
  for (float* q : c->U) cudaFree(q);
  for (float* q : c->S) cudaFree(q);
  float* bufs[] = {c->T1, c->T2, c->Y, c->dA, c->dB, c->dY, c->Xbuf, c->Tb};
  for (float* q : bufs)
    if (q) cudaFree(q);
  c->H.assign(c->L + 1, nullptr);
  c->U.assign(c->L, nullptr);
  c->S.assign(c->L, nullptr);
  const long long act = (long long)B * V * c->C;
  const long long spec = (long long)B * 2 * c->m * c->m * c->m * c->C;
  // the largest intermediate of a spectral stage: after the y-transform,
  // B * Nz * 2m * m * C  <=  B * V * C * 2 (m <= Ny, Nx): bound by 2 * act
  const long long tmp = std::max(2 * act, 4 * spec);
  for (int l = 0; l <= c->L; ++l) FCK(cudaMalloc(&c->H[l], act * sizeof(float)), "activations");
  for (int l = 0; l < c->L; ++l) FCK(cudaMalloc(&c->U[l], act * sizeof(float)), "activations");
  for (int l = 0; l < c->L; ++l) FCK(cudaMalloc(&c->S[l], spec * sizeof(float)), "spectra");
  FCK(cudaMalloc(&c->T1, tmp * sizeof(float)), "workspace");
  FCK(cudaMalloc(&c->T2, tmp * sizeof(float)), "workspace");
  FCK(cudaMalloc(&c->dA, act * sizeof(float)), "workspace");
  FCK(cudaMalloc(&c->dB, act * sizeof(float)), "workspace");
  FCK(cudaMalloc(&c->Y, (long long)B * V * c->cout * sizeof(float)), "output");
  FCK(cudaMalloc(&c->dY, (long long)B * V * c->cout * sizeof(float)), "output");
  FCK(cudaMalloc(&c->Xbuf, (long long)B * V * c->cin * sizeof(float)), "input");
  FCK(cudaMalloc(&c->Tb, (long long)B * V * c->cout * sizeof(float)), "targets");
  c->cap_batch = B;
  c->cap_vox = V;
  return RVE_OK;
}

// K(h) into out (overwrites), keeping the retained spectrum in Sret.
rve_status spectral(rve_fno_ctx* c, int B, int nx, int ny, int nz, const std::vector<float*>& Mx, const float* h,
                    const __nv_bfloat16* R, float* Sret, float* out) {
  const int m = c->m, C = c->C, m2 = 2 * m;
  const long long inner_y = (long long)m * C;         // kx * c
  const long long inner_z = (long long)m * m * C;     // ky * kx * c
  const int nmodes = m * m * m;
  float *T1 = c->T1, *T2 = c->T2;
  // x: T1[b,z,y][(s,kx)][c] = Fx . h[b,z,y][x][c]
  FCK(gemm(c, false, false, m2, C, nx, Mx[0], nx, 0, h, C, (long long)nx * C, T1, C, (long long)m2 * C,
           B * nz * ny),
      "dft x");
  FCK(swap_dims(c, T1, T2, (long long)B * nz, ny, 2, inner_y), "permute");  // -> [b,z][s][y][kx c]
  // y: T1[b,z][(s,ky)][kx c] = Fy . T2[b,z][(s,y)][kx c]
  FCK(gemm(c, false, false, m2, (int)inner_y, 2 * ny, Mx[1], 2 * ny, 0, T2, inner_y, 2 * ny * inner_y, T1, inner_y,
           m2 * inner_y, B * nz),
      "dft y");
  FCK(swap_dims(c, T1, T2, B, nz, 2, inner_z), "permute");  // -> [b][s][z][ky kx c]
  // z: Sret[b][(s,kz)][ky kx c] = Fz . T2[b][(s,z)][...]
  FCK(gemm(c, false, false, m2, (int)inner_z, 2 * nz, Mx[2], 2 * nz, 0, T2, inner_z, 2 * nz * inner_z, Sret, inner_z,
           m2 * inner_z, B),
      "dft z");
  // per-mode mixing: T1 = R Sret (layout [b][s][m][c])
  k_modemix<0><<<(nmodes * 32 + 127) / 128, 128, 0, c->st>>>(R, Sret, T1, nmodes, B);
  ++c->launches;
  FCK(cudaGetLastError(), "mode mix");
  // inverse z: T2[b][(s,z)][...] = Gz . T1[b][(s,kz)][...]
  FCK(gemm(c, false, false, 2 * nz, (int)inner_z, m2, Mx[5], m2, 0, T1, inner_z, m2 * inner_z, T2, inner_z,
           2 * nz * inner_z, B),
      "idft z");
  FCK(swap_dims(c, T2, T1, B, 2, nz, inner_z), "permute");  // -> [b][z][s][ky kx c]
  // inverse y: T2[b,z][(s,y)][kx c] = Gy . T1[b,z][(s,ky)][kx c]
  FCK(gemm(c, false, false, 2 * ny, (int)inner_y, m2, Mx[4], m2, 0, T1, inner_y, m2 * inner_y, T2, inner_y,
           2 * ny * inner_y, B * nz),
      "idft y");
  FCK(swap_dims(c, T2, T1, (long long)B * nz, 2, ny, inner_y), "permute");  // -> [b,z][y][s][kx c]
  // inverse x: out[b,z,y][x][c] = Gx . T1[b,z,y][(s,kx)][c]
  FCK(gemm(c, false, false, nx, C, m2, Mx[3], m2, 0, T1, C, (long long)m2 * C, out, C, (long long)nx * C,
           B * nz * ny),
      "idft x");
  return RVE_OK;
}

// adjoint of K: dh (accumulated with beta) and dR (accumulated)
rve_status spectral_adj(rve_fno_ctx* c, int B, int nx, int ny, int nz, const std::vector<float*>& Mx, const float* du,
                        const __nv_bfloat16* R, const float* Sret, float* dR, float* dh) {
  const int m = c->m, C = c->C, m2 = 2 * m;
  const long long inner_y = (long long)m * C, inner_z = (long long)m * m * C;
  const int nmodes = m * m * m;
  float *T1 = c->T1, *T2 = c->T2;
  // inverse x adjoint: T1[b,z,y][(s,kx)][c] = Gx^T . du[b,z,y][x][c]
  FCK(gemm(c, true, false, m2, C, nx, Mx[3], m2, 0, du, C, (long long)nx * C, T1, C, (long long)m2 * C, B * nz * ny),
      "idft x adj");
  FCK(swap_dims(c, T1, T2, (long long)B * nz, ny, 2, inner_y), "permute");  // [b,z][y][s] -> [b,z][s][y]
  // inverse y adjoint: T1[b,z][(s,ky)] = Gy^T . T2[b,z][(s,y)]
  FCK(gemm(c, true, false, m2, (int)inner_y, 2 * ny, Mx[4], m2, 0, T2, inner_y, 2 * ny * inner_y, T1, inner_y,
           m2 * inner_y, B * nz),
      "idft y adj");
  FCK(swap_dims(c, T1, T2, B, nz, 2, inner_z), "permute");  // [b][z][s] -> [b][s][z]
  // inverse z adjoint: T1[b][(s,kz)] = Gz^T . T2[b][(s,z)]
  FCK(gemm(c, true, false, m2, (int)inner_z, 2 * nz, Mx[5], m2, 0, T2, inner_z, 2 * nz * inner_z, T1, inner_z,
           m2 * inner_z, B),
      "idft z adj");
  // mode mixing adjoint: dR += dSm Sret^T; T2 = R^T dSm
  k_modemix_grad<<<(nmodes * 32 + 127) / 128, 128, 0, c->st>>>(T1, Sret, dR, nmodes, B);
  k_modemix<1><<<(nmodes * 32 + 127) / 128, 128, 0, c->st>>>(R, T1, T2, nmodes, B);
  c->launches += 2;
  FCK(cudaGetLastError(), "mode mix adj");
  // forward z adjoint: T1[b][(s,z)] = Fz^T . T2[b][(s,kz)]
  FCK(gemm(c, true, false, 2 * nz, (int)inner_z, m2, Mx[2], 2 * nz, 0, T2, inner_z, m2 * inner_z, T1, inner_z,
           2 * nz * inner_z, B),
      "dft z adj");
  FCK(swap_dims(c, T1, T2, B, 2, nz, inner_z), "permute");  // [b][s][z] -> [b][z][s]
  // forward y adjoint: T1[b,z][(s,y)] = Fy^T . T2[b,z][(s,ky)]
  FCK(gemm(c, true, false, 2 * ny, (int)inner_y, m2, Mx[1], 2 * ny, 0, T2, inner_y, m2 * inner_y, T1, inner_y,
           2 * ny * inner_y, B * nz),
      "dft y adj");
  FCK(swap_dims(c, T1, T2, (long long)B * nz, 2, ny, inner_y), "permute");  // [b,z][s][y] -> [b,z][y][s]
  // forward x adjoint: dh[b,z,y][x][c] += Fx^T . T2[b,z,y][(s,kx)][c]
  FCK(gemm(c, true, false, nx, C, m2, Mx[0], nx, 0, T2, C, (long long)m2 * C, dh, C, (long long)nx * C, B * nz * ny,
           1.f, 1.f),
      "dft x adj");
  return RVE_OK;
}

rve_status forward_impl(rve_fno_ctx* c, int B, const int dims[3], const float* X, float* Yout) {
  const int nx = dims[0], ny = dims[1], nz = dims[2];
  const long long V = (long long)nx * ny * nz, rows = B * V;
  if (nx < 2 * c->m || ny < c->m || nz < c->m)
    return ffail(c, RVE_ERR_ARG, "grid too small for the retained modes (need Nx >= 2 modes, Ny, Nz >= modes)");
  rve_status s = ensure(c, B, V);
  if (s != RVE_OK) return s;
  std::vector<float*> Mx;
  if ((s = get_mats(c, nx, ny, nz, Mx)) != RVE_OK) return s;
  const int C = c->C;
  // lift
  FCK(gemm(c, false, false, (int)std::min<long long>(rows, 1LL << 30), C, c->cin, X, c->cin, 0, c->p + c->offWl, C, 0,
           c->U[0], C, 0, 1),
      "lift");
  k_bias_act<<<nblk(rows * C), 256, 0, c->st>>>(c->U[0], c->p + c->offbl, c->H[0], rows * C, C, 0);
  ++c->launches;
  for (int l = 0; l < c->L; ++l) {
    const __nv_bfloat16* R = c->Rbf + (long long)l * c->nR;
    if ((s = spectral(c, B, nx, ny, nz, Mx, c->H[l], R, c->S[l], c->U[l])) != RVE_OK) return s;
    FCK(gemm(c, false, false, (int)rows, C, C, c->H[l], C, 0, c->p + c->offW[l], C, 0, c->U[l], C, 0, 1, 1.f, 1.f),
        "channel mix");
    k_bias_act<<<nblk(rows * C), 256, 0, c->st>>>(c->U[l], c->p + c->offb[l], c->H[l + 1], rows * C, C,
                                                  l < c->L - 1 ? 1 : 0);
    ++c->launches;
    FCK(cudaGetLastError(), "bias/act");
  }
  FCK(gemm(c, false, false, (int)rows, c->cout, C, c->H[c->L], C, 0, c->p + c->offWq, c->cout, 0, Yout, c->cout, 0,
           1),
      "projection");
  // bias of the projection (no activation)
  k_bias_act<<<nblk(rows * c->cout), 256, 0, c->st>>>(Yout, c->p + c->offbq, Yout, rows * c->cout, c->cout, 0);
  ++c->launches;
  return cudaGetLastError() == cudaSuccess ? RVE_OK : ffail(c, RVE_ERR_CUDA, "forward");
}

// gradient of the MSE loss w.r.t. every parameter into c->g (overwritten)
rve_status backward_impl(rve_fno_ctx* c, int B, const int dims[3], const float* X, const float* T, double* loss) {
  const int nx = dims[0], ny = dims[1], nz = dims[2];
  const long long V = (long long)nx * ny * nz, rows = B * V;
  // allocate the activations before c->Y is read as the forward's output
  rve_status s = ensure(c, B, V);
  if (s != RVE_OK) return s;
  if ((s = forward_impl(c, B, dims, X, c->Y)) != RVE_OK) return s;
  std::vector<float*> Mx;
  if ((s = get_mats(c, nx, ny, nz, Mx)) != RVE_OK) return s;
  const int C = c->C;
  FCK(cudaMemsetAsync(c->g, 0, c->nparam * sizeof(float), c->st), "memset");
  const long long ny_ = rows * c->cout;
  const int nb = 152 * 4;
  k_mse<<<nb, 256, 0, c->st>>>(c->Y, T, c->dY, ny_, c->part);
  ++c->launches;
  std::vector<double> hp(nb);
  // projection
  FCK(gemm(c, true, false, C, c->cout, (int)rows, c->H[c->L], C, 0, c->dY, c->cout, 0, c->g + c->offWq, c->cout, 0,
           1),
      "dWq");
  k_colsum<<<c->cout, 256, 0, c->st>>>(c->dY, rows, c->cout, c->g + c->offbq);
  ++c->launches;
  float* dh = c->dA;
  float* du = c->dB;
  FCK(gemm(c, false, true, (int)rows, C, c->cout, c->dY, c->cout, 0, c->p + c->offWq, c->cout, 0, dh, C, 0, 1),
      "dh");
  for (int l = c->L - 1; l >= 0; --l) {
    if (l < c->L - 1) {
      k_gelu_back<<<nblk(rows * C), 256, 0, c->st>>>(dh, c->U[l], du, rows * C);
      ++c->launches;
    } else {
      FCK(cudaMemcpyAsync(du, dh, rows * C * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
    }
    FCK(gemm(c, true, false, C, C, (int)rows, c->H[l], C, 0, du, C, 0, c->g + c->offW[l], C, 0, 1), "dW");
    k_colsum<<<C, 256, 0, c->st>>>(du, rows, C, c->g + c->offb[l]);
    ++c->launches;
    // dh_in = du W^T + K^T du
    FCK(gemm(c, false, true, (int)rows, C, C, du, C, 0, c->p + c->offW[l], C, 0, dh, C, 0, 1), "dh");
    const __nv_bfloat16* R = c->Rbf + (long long)l * c->nR;
    if ((s = spectral_adj(c, B, nx, ny, nz, Mx, du, R, c->S[l], c->g + c->offR[l], dh)) != RVE_OK) return s;
  }
  // lift: dWl = X^T dh0, dbl = colsum(dh0)
  FCK(gemm(c, true, false, c->cin, C, (int)rows, X, c->cin, 0, dh, C, 0, c->g + c->offWl, C, 0, 1), "dWl");
  k_colsum<<<C, 256, 0, c->st>>>(dh, rows, C, c->g + c->offbl);
  ++c->launches;
  FCK(cudaMemcpyAsync(hp.data(), c->part, nb * sizeof(double), cudaMemcpyDeviceToHost, c->st), "loss");
  FCK(cudaStreamSynchronize(c->st), "synchronize");
  double L = 0;
  for (double v : hp) L += v;
  if (loss) *loss = L;
  return RVE_OK;
}

void fno_free(rve_fno_ctx* c) {
  if (!c) return;
  for (auto& kv : c->mats)
    for (float* q : kv.second) cudaFree(q);
  for (float* q : c->H) cudaFree(q);
  for (float* q : c->U) cudaFree(q);
  for (float* q : c->S) cudaFree(q);
  void* bufs[] = {c->T1, c->T2, c->Y, c->dA, c->dB, c->dY, c->Xbuf, c->Tb, c->p, c->g, c->m1, c->m2, c->Rbf, c->part,
                  c->tmpf};
  for (void* q : bufs)
    if (q) cudaFree(q);
  delete c;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

rve_status rve_fno_create(int cin, int width, int cout, int layers, int modes, unsigned long long seed, void* stream,
                          rve_fno_t* out) {
  if (!out) return ffail(nullptr, RVE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (width != 32) return ffail(nullptr, RVE_ERR_ARG, "width must be 32");
  if (cin < 1 || cin > 64 || cout < 1 || cout > 64 || layers < 1 || layers > 16 || modes < 2 || modes > 32 ||
      (modes & 1))
    return ffail(nullptr, RVE_ERR_ARG, "bad network shape");
  rve_fno_ctx* c = new (std::nothrow) rve_fno_ctx();
  if (!c) return ffail(nullptr, RVE_ERR_OOM, "host allocation failed");
  c->cin = cin;
  c->C = width;
  c->cout = cout;
  c->L = layers;
  c->m = modes;
  c->st = static_cast<cudaStream_t>(stream);
  long long off = 0;
  c->offWl = off;
  off += (long long)cin * width;
  c->offbl = off;
  off += width;
  c->nR = (long long)modes * modes * modes * 4 * width * width;
  for (int l = 0; l < layers; ++l) {
    c->offW.push_back(off);
    off += (long long)width * width;
    c->offb.push_back(off);
    off += width;
    c->offR.push_back(off);
    off += c->nR;
  }
  c->offWq = off;
  off += (long long)width * cout;
  c->offbq = off;
  off += cout;
  c->nparam = off;
  // deterministic initialisation (host), same scales as the oracle's
  std::vector<float> h(off, 0.f);
  uint64_t s = seed * 0x2545F4914F6CDD1DULL + 1;
  auto gauss = [&]() {
    const double u1 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  for (long long i = 0; i < (long long)cin * width; ++i) h[c->offWl + i] = (float)(gauss() / std::sqrt((double)cin));
  for (int l = 0; l < layers; ++l) {
    for (long long i = 0; i < (long long)width * width; ++i) h[c->offW[l] + i] = (float)(gauss() / std::sqrt(32.0));
    for (long long i = 0; i < c->nR; ++i) h[c->offR[l] + i] = (float)(gauss() / (2.0 * width) * 0.1);
  }
  for (long long i = 0; i < (long long)width * cout; ++i) h[c->offWq + i] = (float)(gauss() / std::sqrt(32.0));
  if (cudaMalloc(&c->p, off * sizeof(float)) != cudaSuccess || cudaMalloc(&c->g, off * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->m1, off * sizeof(float)) != cudaSuccess || cudaMalloc(&c->m2, off * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->Rbf, (long long)layers * c->nR * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&c->part, 152 * 4 * sizeof(double)) != cudaSuccess) {
    fno_free(c);
    return ffail(nullptr, RVE_ERR_OOM, "parameter allocation failed");
  }
  rve_status st = rve_fno_set_params(c, h.data());
  if (st != RVE_OK) {
    g_fno_err = c->err;
    fno_free(c);
    return st;
  }
  *out = c;
  return RVE_OK;
}

long long rve_fno_param_count(rve_fno_t c) { return c ? c->nparam : 0; }

rve_status rve_fno_set_params(rve_fno_t c, const float* params_host) {
  if (!c || !params_host) return RVE_ERR_ARG;
  FCK(cudaMemcpyAsync(c->p, params_host, c->nparam * sizeof(float), cudaMemcpyHostToDevice, c->st), "params");
  FCK(cudaMemsetAsync(c->m1, 0, c->nparam * sizeof(float), c->st), "memset");
  FCK(cudaMemsetAsync(c->m2, 0, c->nparam * sizeof(float), c->st), "memset");
  for (int l = 0; l < c->L; ++l) {
    k_to_bf16<<<nblk(c->nR), 256, 0, c->st>>>(c->p + c->offR[l], c->Rbf + (long long)l * c->nR, c->nR);
    ++c->launches;
  }
  c->adam_t = 0;
  FCK(cudaStreamSynchronize(c->st), "synchronize");
  return RVE_OK;
}

rve_status rve_fno_get_params(rve_fno_t c, float* params_host, float* grad_host) {
  if (!c) return RVE_ERR_ARG;
  if (params_host) FCK(cudaMemcpyAsync(params_host, c->p, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, c->st), "copy");
  if (grad_host) FCK(cudaMemcpyAsync(grad_host, c->g, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, c->st), "copy");
  FCK(cudaStreamSynchronize(c->st), "synchronize");
  return RVE_OK;
}

rve_status rve_fno_forward(rve_fno_t c, int batch, const int dims[3], const float* x_dev, float* y_dev) {
  if (!c || !dims || !x_dev || !y_dev || batch < 1 || batch > 8) return c ? ffail(c, RVE_ERR_ARG, "bad arguments") : RVE_ERR_ARG;
  return forward_impl(c, batch, dims, x_dev, y_dev);
}

rve_status rve_fno_loss_grad(rve_fno_t c, int batch, const int dims[3], const float* x_dev, const float* t_dev,
                             double* loss_host) {
  if (!c || !dims || !x_dev || !t_dev || batch < 1 || batch > 8) return c ? ffail(c, RVE_ERR_ARG, "bad arguments") : RVE_ERR_ARG;
  return backward_impl(c, batch, dims, x_dev, t_dev, loss_host);
}

rve_status rve_fno_adam_step(rve_fno_t c, double lr) {
  if (!c) return RVE_ERR_ARG;
  c->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)c->adam_t), c2 = 1.f - std::pow(b2, (float)c->adam_t);
  k_adam<<<nblk(c->nparam), 256, 0, c->st>>>(c->p, c->g, c->m1, c->m2, c->nparam, (float)lr, b1, b2, 1e-8f, c1, c2);
  ++c->launches;
  for (int l = 0; l < c->L; ++l) {
    k_to_bf16<<<nblk(c->nR), 256, 0, c->st>>>(c->p + c->offR[l], c->Rbf + (long long)l * c->nR, c->nR);
    ++c->launches;
  }
  FCK(cudaGetLastError(), "adam");
  return RVE_OK;
}

rve_status rve_fno_pack_features(rve_fno_t c, const int dims[3], const uint8_t* phase_dev, const float* damage_dev,
                                 const float* kappa_dev, float kappa_scale, const float* d1_dev, const float* d2_dev,
                                 float scale, float* x_dev) {
  if (!c || !dims || !phase_dev || !x_dev) return RVE_ERR_ARG;
  if (c->cin < 15) return ffail(c, RVE_ERR_ARG, "feature packing needs cin >= 15");
  const long long V = (long long)dims[0] * dims[1] * dims[2];
  k_pack<<<nblk(V), 256, 0, c->st>>>(phase_dev, damage_dev, kappa_dev, kappa_scale, d1_dev, d2_dev, V, 6, scale,
                                     c->cin, x_dev);
  ++c->launches;
  FCK(cudaGetLastError(), "pack");
  return RVE_OK;
}

rve_status rve_fno_unpack_output(rve_fno_t c, const int dims[3], const float* y_dev, float scale, const float* base_dev,
                                 float* out_dev) {
  if (!c || !dims || !y_dev || !out_dev) return RVE_ERR_ARG;
  const long long V = (long long)dims[0] * dims[1] * dims[2];
  k_unpack<<<nblk(V), 256, 0, c->st>>>(y_dev, base_dev, V, c->cout, scale, out_dev);
  ++c->launches;
  FCK(cudaGetLastError(), "unpack");
  return RVE_OK;
}

rve_status rve_fno_pack_target(rve_fno_t c, const int dims[3], const float* field_dev, const float* base_dev, float scale,
                               float* t_dev) {
  if (!c || !dims || !field_dev || !t_dev) return RVE_ERR_ARG;
  const long long V = (long long)dims[0] * dims[1] * dims[2];
  k_pack_target<<<nblk(V), 256, 0, c->st>>>(field_dev, base_dev, V, c->cout, scale, t_dev);
  ++c->launches;
  FCK(cudaGetLastError(), "pack target");
  return RVE_OK;
}

rve_status rve_fno_increment(rve_fno_t c, const int dims[3], const float* eps_new_dev, const float* eps_old_dev,
                             const double dE_host[6], float* out_dev) {
  if (!c || !dims || !eps_new_dev || !eps_old_dev || !dE_host || !out_dev) return RVE_ERR_ARG;
  const long long V = (long long)dims[0] * dims[1] * dims[2];
  k_incr<<<nblk(V * c->cout), 256, 0, c->st>>>(eps_new_dev, eps_old_dev, V, c->cout, (float)dE_host[0],
                                                (float)dE_host[1], (float)dE_host[2], (float)dE_host[3],
                                                (float)dE_host[4], (float)dE_host[5], out_dev);
  ++c->launches;
  FCK(cudaGetLastError(), "increment");
  return RVE_OK;
}

const char* rve_fno_last_error(rve_fno_t c) { return c ? c->err.c_str() : g_fno_err.c_str(); }
long long rve_fno_launch_count(rve_fno_t c) { return c ? c->launches : 0; }
void rve_fno_destroy(rve_fno_t c) { fno_free(c); }

}  // extern "C"
