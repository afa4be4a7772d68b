// x-forward pass with its input tiles moved by the tensor-memory accelerator
// (3D FP32, NC = 6, plain or secant tangent; Nx a compiled length <= 256).
//
// A persistent CTA walks the x-row tiles of the grid.  Thread 0 issues one
// 3D bulk tensor copy of the tile's six strain components (box Nx x Q x 6)
// and, with the tangent, two 2D copies of its damage and phase rows into a
// shared-memory staging area, all completing on one mbarrier; the threads
// apply the tangent from shared memory and scatter into the packed FFT
// buffer, then the copies of the CTA's next tile are issued before the FFT
// and the half-spectrum stores of the current one, so the next tile's loads
// overlap this tile's transform.  Sec. 2.1 / Eq. (13): the same tangent and
// r2c transform as kf_xfwd (hv_fast.cu); only the data movement differs.
//
// Every wait on the mbarrier is bounded: a copy that never completes sets
// the wait-error word of the device scalars, the CTA waits (bounded) once
// more for its copies in flight and leaves; the host reports RVE_ERR_TIMEOUT.
#include <algorithm>
#include <cstdint>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "hv_tiles.cuh"
#include "hv_tma.cuh"
#include "scalar_logic.cuh"

namespace rve {
namespace {

constexpr int kTmaBlocksPerSM = 2;
constexpr long long kWaitLimit = 1LL << 20;  // try_wait rounds before giving up (well under a second)

__device__ __forceinline__ unsigned sm_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(b)), "r"(bytes) : "memory");
}
// true once phase `parity` of the barrier has completed
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sm_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(sm_addr(dst)), "l"(tm), "r"(x), "r"(y), "r"(z), "r"(sm_addr(b))
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(sm_addr(dst)), "l"(tm), "r"(x), "r"(y), "r"(sm_addr(b))
      : "memory");
}

// shared-memory layout of one CTA (byte offsets; every TMA destination on a
// 128-byte boundary)
template <int N> struct TmaLayout {
  static constexpr int Q = xq<N, 6>(), NL = 6 * Q / 2;
  static constexpr int IN = 0;                                       // [6][Q][N] floats
  static constexpr int DMG = IN + 6 * Q * N * 4;                     // [Q][N] floats
  static constexpr int PH = ((DMG + Q * N * 4) + 127) / 128 * 128;   // [Q][N] bytes
  static constexpr int BUF = ((PH + Q * N) + 127) / 128 * 128;       // [N][NL] float2
  static constexpr int BYTES = BUF + N * NL * 8;
  static constexpr unsigned TX_IN = 6u * Q * N * 4, TX_STATE = (unsigned)Q * N * 5;
};

}  // namespace

template <int N>
__device__ __noinline__ void tma_fft_store(float2* buf, float2* spec, const long long nrows, const float2* tw,
                                           const long long row0, const long long row_end) {
  xfwd_fft_store<N, 6>(buf, spec, nrows, tw, row0, row_end);
}

// MODE 0: plain (the gradient G : sigma); 1: secant tangent, with this
// CTA's share of in : (tangent : in) in partials[blockIdx.x] when set; with
// S as well, the last CTA to finish sums the shares into S->dHd and takes
// Algorithm 1's step-length decision.
template <int N, int MODE>
__global__ void __launch_bounds__(kFT, kTmaBlocksPerSM)
    kt_xfwd(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_dmg,
            const __grid_constant__ CUtensorMap tm_ph, const MatTable<float> mt, float2* __restrict__ spec,
            const long long nrows, const float2* __restrict__ tw, double* __restrict__ partials, const int ntiles,
            int* __restrict__ wait_err, DevScalars* __restrict__ S) {
  using L = TmaLayout<N>;
  constexpr int Q = L::Q, NL = L::NL;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the dynamic area is 128-byte aligned by construction of its base
  unsigned char* base = smem_raw + ((128 - (sm_addr(smem_raw) & 127)) & 127);
  float* st_in = reinterpret_cast<float*>(base + L::IN);
  float* st_d = reinterpret_cast<float*>(base + L::DMG);
  uint8_t* st_p = base + L::PH;
  float2* buf = reinterpret_cast<float2*>(base + L::BUF);
  __shared__ __align__(8) uint64_t bar;
  __shared__ double red[32];
  const unsigned tx = L::TX_IN + (MODE == 1 ? L::TX_STATE : 0u);
  auto issue = [&](int tile) {
    const int row0 = tile * Q;
    mbar_expect_tx(&bar, tx);
    tma_load_3d(st_in, &tm_in, 0, row0, 0, &bar);
    if (MODE == 1) {
      tma_load_2d(st_d, &tm_dmg, 0, row0, &bar);
      tma_load_2d(st_p, &tm_ph, 0, row0, &bar);
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x);
  double acc = 0.0;
  unsigned parity = 0;
#pragma unroll 1
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, parity ^= 1u) {
    // the tile's copies have landed (bounded wait; every thread of the CTA
    // takes the same decision)
    const bool ok = mbar_wait(&bar, parity);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(wait_err, 1);
        mbar_wait(&bar, parity);  // once more, bounded: the copies in flight target this CTA's memory
      }
      break;  // still arrives at the reduction below, so its counter stays consistent
    }
    // tangent from the staged rows, scattered into the packed FFT lines;
    // consecutive threads take consecutive x
    float tacc = 0.f;
    constexpr int ITEMS = Q * N, STEPS = (ITEMS + kFT - 1) / kFT;
#pragma unroll 1
    for (int s = 0; s < STEPS; ++s) {
      const int idx = threadIdx.x + s * kFT;
      if (idx < ITEMS) {
        const int q = idx / N, x = idx - (idx / N) * N;
        float v[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = st_in[(c * Q + q) * N + x];
        if (MODE == 1) {
          const float keep = 1.f - st_d[q * N + x];
          const int ph = st_p[q * N + x];
          const float lam = mt.lam[ph] * keep, tmu = 2.f * mt.mu[ph] * keep;
          const float tr = v[0] + v[1] + v[2];
          float dv = 0.f;
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const float sg = tmu * v[c] + (c < 3 ? lam * tr : 0.f);
            dv += v[c] * sg;
            v[c] = sg;
          }
          tacc += dv;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const int rho = q * 6 + c;
          reinterpret_cast<float*>(&buf[x * NL + (rho >> 1)])[rho & 1] = v[c];
        }
      }
    }
    acc += (double)tacc;
    __syncthreads();  // staging consumed, FFT buffer complete
    const int next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(next);
    }
    const long long row0 = (long long)tile * Q;
    const long long row_end = row0 + Q < nrows ? row0 + Q : nrows;
    // a called (not inlined) transform: inlined into the tile loop, the
    // compiler hoists its loop-invariant index arithmetic out of the loop and
    // holds it in registers across tiles
    tma_fft_store<N>(buf, spec, nrows, tw, row0, row_end);
    __syncthreads();  // the stores have read buf before the next tile's scatter
  }
  if (MODE == 1 && partials) {
    double vv[1] = {acc};
    block_sum<1>(vv, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = vv[0];
    if (S && reduce_in_last_block<1>(partials, gridDim.x, &S->dHd, &S->red_cnt[0], red) && threadIdx.x == 0)
      cg_alpha_scalars(S);
  }
}

// ================================================================ host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// tensor map over `rank` dims (x fastest) with the box `box`; false when the
// encoder refuses it
bool encode(CUtensorMap* m, CUtensorMapDataType dt, cuuint32_t rank, const void* ptr, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
  const cuuint32_t es[3] = {1, 1, 1};
  return encoder()(m, dt, rank, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N>
cudaError_t tma_xfwd_n(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                       const MatTable<float>& mt, float2* spec, const float2* tw, bool tangent, double* partials,
                       int* nblocks, cudaStream_t st, int* wait_err, DevScalars* S) {
  using L = TmaLayout<N>;
  constexpr int Q = L::Q;
  // the copies' alignment rules: 16-byte base addresses, row strides and box
  // rows in multiples of 16 bytes (N floats; N bytes of phase ids), x = 0
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  if (!al16(in) || (tangent && (!al16(dmg) || !al16(phase))) || (N % 16) != 0) return cudaErrorNotSupported;
  CUtensorMap tin, tdm, tph;
  const cuuint64_t nr = (cuuint64_t)g.nrows;
  const cuuint64_t d3[3] = {(cuuint64_t)N, nr, 6}, s3[2] = {(cuuint64_t)N * 4, nr * N * 4};
  const cuuint32_t b3[3] = {(cuuint32_t)N, (cuuint32_t)Q, 6};
  if (!encode(&tin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, in, d3, s3, b3)) return cudaErrorNotSupported;
  tdm = tph = tin;
  if (tangent) {
    const cuuint64_t d2[2] = {(cuuint64_t)N, nr}, sd[1] = {(cuuint64_t)N * 4}, sp[1] = {(cuuint64_t)N};
    const cuuint32_t b2[2] = {(cuuint32_t)N, (cuuint32_t)Q};
    if (!encode(&tdm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, dmg, d2, sd, b2)) return cudaErrorNotSupported;
    if (!encode(&tph, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, phase, d2, sp, b2)) return cudaErrorNotSupported;
  }
  const int ntiles = (int)((g.nrows + Q - 1) / Q);
  const int grid = std::min(ntiles, kTmaBlocksPerSM * sm_count());
  const size_t smem = (size_t)L::BYTES + 128;
  // once per kernel and device
  static int attr[2][64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int mi = tangent ? 1 : 0;
  if (dev < 0 || dev >= 64 || !attr[mi][dev]) {
    cudaError_t e = tangent ? cudaFuncSetAttribute(kt_xfwd<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(kt_xfwd<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[mi][dev] = 1;
  }
  if (tangent)
    kt_xfwd<N, 1><<<grid, kFT, smem, st>>>(tin, tdm, tph, mt, spec, g.nrows, tw, partials, ntiles, wait_err,
                                           partials ? S : nullptr);
  else
    kt_xfwd<N, 0><<<grid, kFT, smem, st>>>(tin, tdm, tph, mt, spec, g.nrows, tw, nullptr, ntiles, wait_err, nullptr);
  *nblocks = grid;
  return cudaGetLastError();
}

}  // namespace

cudaError_t tma_xfwd(const GridDesc& g, const float* in, const uint8_t* phase, const float* dmg,
                     const MatTable<float>& mt, float2* spec, const float2* tw, bool tangent, double* partials,
                     int* nblocks, cudaStream_t st, int* wait_err, DevScalars* S) {
  if (g.ndim != 3 || g.ncomp != 6 || g.nq != 1 || !wait_err || !encoder()) return cudaErrorNotSupported;
#define RVE_CASE(n_) \
  if (g.nx == n_) return tma_xfwd_n<n_>(g, in, phase, dmg, mt, spec, tw, tangent, partials, nblocks, st, wait_err, S);
  RVE_CASE(32) RVE_CASE(64) RVE_CASE(96) RVE_CASE(128) RVE_CASE(192) RVE_CASE(256)
#undef RVE_CASE
  return cudaErrorNotSupported;
}

}  // namespace rve
