// rve_project_noalloc: the compatibility projection (FP32) for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: loops that
// fixed their device-memory budget at initialisation (real-time or embedded
// solvers, frameworks whose caching allocator owns all device memory), and
// code that must not trigger the implicit device-wide synchronisation that
// cudaMalloc / cudaFree can cause.  This entry point needs no context and
// allocates nothing: its scratch -- the 1D twiddle and gradient tables of
// the three axes and the half spectrum -- lives in one file-scope
// __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.
#include <mutex>

#include "../../include/rve.h"
#include "hv_passes.cuh"

namespace {

using rve::GridDesc;
using rve::SpecWork;

constexpr int kMaxAxis = 1024;
constexpr size_t kTableElems = 9 * (size_t)kMaxAxis;      // tw, gdiff, gavg for 3 axes
constexpr size_t kScratchBytes = (size_t)16 << 20;        // 16 MiB
constexpr size_t kScratchElems = kScratchBytes / sizeof(float2);
constexpr size_t kMaxSpecElems = kScratchElems - kTableElems;  // 2,087,936 complex values

static __device__ __align__(256) float2 g_noalloc_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_scratch_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Twiddles e^{-2 pi i k/n} and the gradient factors e^{i th} - 1 (0 at
// k = 0) and (1 + e^{i th})/2 (0 at 2k = n) of one axis, computed on the
// device from sincospi in double and rounded once to float.
__global__ void k_axis_tables(float2* base, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    base[k] = make_float2((float)c, (float)(-s));
    base[kMaxAxis + k] = (k == 0) ? make_float2(0.f, 0.f) : make_float2((float)(c - 1.0), (float)s);
    base[2 * kMaxAxis + k] = (2 * k == n) ? make_float2(0.f, 0.f)
                                          : make_float2((float)((1.0 + c) * 0.5), (float)(s * 0.5));
  }
}

bool five_smooth_even(int n) {
  if (n < 2 || n > kMaxAxis || (n & 1)) return false;
  int m = n;
  for (int p : {2, 3, 5})
    while (m % p == 0) m /= p;
  return m == 1;
}

// Failures are reported by status code only (there is no context to hold a
// message); `why` documents each site.
rve_status fail(rve_status s, const char* why) {
  (void)why;
  return s;
}

// Device address of the scratch array on the current device (set up once
// per device; must not happen while a stream on that device is capturing).
rve_status scratch_for_current_device(float2** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return fail(RVE_ERR_CUDA, "cudaGetDevice failed");
  if (dev >= kMaxDevices) return fail(RVE_ERR_ARG, "device ordinal too large for rve_project_noalloc");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(RVE_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    g_scratch_dev[dev] = static_cast<float2*>(p);
  }
  *out = g_scratch_dev[dev];
  return RVE_OK;
}

}  // namespace

extern "C" {

rve_status rve_project_noalloc(const int dims[3], int ndim, const float* v_dev, float* out_dev,
                               const uint8_t free_mask_host[6], void* stream) {
  if (!dims || !v_dev || !out_dev) return fail(RVE_ERR_ARG, "NULL argument");
  // An error left pending by earlier, unrelated work on this thread would be
  // reported by the launch checks below as this call's own; refuse to start
  // instead, and leave that error for its owner to read.
  if (cudaPeekAtLastError() != cudaSuccess) return fail(RVE_ERR_CUDA, "an earlier CUDA error is pending");
  if (ndim != 2 && ndim != 3) return fail(RVE_ERR_ARG, "ndim must be 2 or 3");
  for (int a = 0; a < ndim; ++a)
    if (!five_smooth_even(dims[a]))
      return fail(RVE_ERR_ARG, "every dim must be even, in [2, 1024], with prime factors 2, 3, 5 only");
  GridDesc g{};
  g.ndim = ndim;
  g.nx = dims[0];
  g.ny = dims[1];
  g.nz = ndim == 3 ? dims[2] : 1;
  g.nxh = g.nx / 2 + 1;
  g.ncomp = ndim == 3 ? 6 : 3;
  g.nvox = (long long)g.nx * g.ny * g.nz;
  g.nrows = (long long)g.ny * g.nz;
  if ((size_t)g.ncomp * (size_t)g.nrows * (size_t)g.nxh > kMaxSpecElems)
    return fail(RVE_ERR_ARG,
                "grid too large for rve_project_noalloc: ncomp*Ny*Nz*(Nx/2+1) must be <= 2087936");
  float2* scratch = nullptr;
  rve_status s = scratch_for_current_device(&scratch);
  if (s != RVE_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SpecWork<float> w;
  if (rve::spectral_plan<float>(g, w) != cudaSuccess) return fail(RVE_ERR_CUDA, "kernel attribute setup failed");
  const int ns[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < g.ndim; ++a) {
    float2* base = scratch + (size_t)a * 3 * kMaxAxis;
    k_axis_tables<<<(ns[a] + 255) / 256, 256, 0, st>>>(base, ns[a]);
    w.tw[a] = base;
    w.gdiff[a] = base + kMaxAxis;
    w.gavg[a] = base + 2 * kMaxAxis;
  }
  if (cudaGetLastError() != cudaSuccess) return fail(RVE_ERR_CUDA, "table kernel launch failed");
  w.spec = scratch + kTableElems;  // fully written by the first pass before it is read
  unsigned bits = 0;
  if (free_mask_host)
    for (int c = 0; c < g.ncomp; ++c)
      if (free_mask_host[c]) bits |= 1u << c;
  w.free_mask = bits;
  rve::MatTable<float> mt{};
  cudaError_t e = rve::spectral_apply<float>(g, w, mt, v_dev, nullptr, nullptr, rve::XIn::Plain, out_dev, nullptr,
                                             nullptr, st, nullptr);
  if (e != cudaSuccess) return fail(RVE_ERR_CUDA, "projection launch failed");
  return RVE_OK;
}

}  // extern "C"
