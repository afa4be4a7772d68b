// Batched solver: many RVEs of uneven sizes (2D and 3D mixed) advanced in
// lockstep through Algorithm 2 / Algorithm 1, FP32 fields.
//
// Every step of the path (tangent + FFT passes + projection, CG updates,
// constitutive update, scalar control) is ONE persistent launch over all
// member RVEs: each pass has a work list of (RVE, block) items laid out as
// a prefix-summed range per RVE, and the CTAs of the launch pull items from
// an atomic counter (dynamic load balancing across uneven grid sizes).
// Per-RVE scalars live in a device array; kernels gate each RVE on a host
// bit mask or on its device-side CG status, so the inner CG iteration is a
// fixed launch sequence that is captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rve.h"
#include "consistent.cuh"
#include "passes_generic.cuh"
#include "scalar_logic.cuh"
#include "solver_kernels.cuh"

namespace {

using namespace rve;
using R = float;
using C = float2;

constexpr int kMaxBatch = 256;
constexpr long long kVecChunk = 16384;  // field elements per vector item (multiple of 4)
constexpr long long kVoxChunk = 4096;   // voxels per constitutive item (multiple of 4)

enum BPass : int { BP_X = 0, BP_Y = 1, BP_Z = 2, BP_2D = 3, BP_VEC = 4, BP_VOX = 5, BP_N = 6 };

struct BDesc {
  GridDesc g;
  AxisPlan px, py, pz;
  const C* tw[3];
  const C* gd[3];
  const C* ga[3];
  C* spec;
  int qx, ty, tz;
  unsigned free_mask;
  long long foff;  // first field element of this RVE in the batched vectors
  long long voff;  // first voxel of this RVE in the batched scalar fields
};

// Which RVEs a launch works on.
enum GateMode : int { G_BITS = 0, G_RUN = 1, G_RESTART = 2, G_UPDATE = 3 };
struct Gate {
  int mode;
  unsigned bits[kMaxBatch / 32];
};

__device__ __forceinline__ bool gate_ok(const Gate& gt, const DevScalars* S, int i) {
  switch (gt.mode) {
    case G_BITS: return (gt.bits[i >> 5] >> (i & 31)) & 1u;
    case G_RUN: return S[i].status == CG_RUN;
    case G_RESTART: return S[i].status == CG_RUN && S[i].restart != 0;
    default: return S[i].status == CG_RUN || S[i].pad0 != 0;  // update: running, or an exit to apply
  }
}

// Work lists over the ACTIVE members only, rebuilt on the device by
// kb_compact before every gated operation (so a launch enumerates the items
// of the members that take part, however many members are idle).
struct WLists {
  int count;                          // active members
  int total[BP_N];                    // active items per pass
  int idx[kMaxBatch];                 // member id of the k-th active member
  int start[BP_N][kMaxBatch + 1];     // item prefix over active members
};

// Pull the next item of pass `pass`; false when exhausted.  Uniform across
// the block.  *v is the item's index (also its partial-sum slot).
__device__ __forceinline__ bool fetch(const WLists* __restrict__ wl, int pass, int* counter, int* s_item, int* v,
                                      int* member, int* local) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
  __syncthreads();
  const int it = *s_item;
  if (it >= wl->total[pass]) return false;
  const int* st = wl->start[pass];
  int lo = 0, hi = wl->count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (st[mid] <= it) lo = mid;
    else hi = mid - 1;
  }
  *v = it;
  *member = wl->idx[lo];
  *local = it - st[lo];
  return true;
}

// One block: the members passing the gate, in order, and their item
// prefixes for every pass (nb: BP_N x n block counts).
__global__ void kb_compact(WLists* wl, const int* __restrict__ nb, int n, Gate gt, const DevScalars* S) {
  __shared__ int flag[kMaxBatch];
  for (int i = threadIdx.x; i < n; i += blockDim.x) flag[i] = gate_ok(gt, S, i) ? 1 : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < n; ++i)
      if (flag[i]) wl->idx[k++] = i;
    wl->count = k;
    for (int p = 0; p < BP_N; ++p) {
      int sum = 0;
      for (int q = 0; q < k; ++q) {
        wl->start[p][q] = sum;
        sum += nb[p * n + wl->idx[q]];
      }
      wl->start[p][k] = sum;
      wl->total[p] = sum;
    }
  }
}

// ------------------------------------------------------ spectral passes
// XMODE: 0 plain x-forward, 1 tangent x-forward.  YINV: y direction.
// DOT for the x-inverse: 0 none, 1 with dotw, 2 self.
// cdp, ca, cn (batched like the state, may be NULL): the rank-one part of
// the symmetric consistent tangent (ConsTan), applied with XMODE 1.
template <int XMODE>
__global__ void __launch_bounds__(kXThreads, kXYMinBlocks)
    kb_xfwd(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter,
            const DevScalars* __restrict__ S, const MatTable<R> mt, const R* __restrict__ in,
            const uint8_t* __restrict__ phase, const R* __restrict__ dmg, const R* __restrict__ cdp,
            const R* __restrict__ ca, const R* __restrict__ cn) {
  __shared__ int s_item;
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_X, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    const ConsTan<R> ct{cdp ? cdp + d.voff : nullptr, ca ? ca + d.foff : nullptr, cn ? cn + d.foff : nullptr};
    xfwd_body<R, XMODE>(in + d.foff, phase + d.voff, dmg + d.voff, mt, d.spec, d.g, d.qx, d.px, d.tw[0],
                        lb, ct);
  }
}

template <bool YINV>
__global__ void __launch_bounds__(kYThreads, kXYMinBlocks)
    kb_ycols(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter) {
  __shared__ int s_item;
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_Y, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    const int b = lb;
    const int nbx = (d.g.nxh + d.ty - 1) / d.ty;
    const int bx = b % nbx, rest = b / nbx;
    ycols_body<R, YINV>(d.spec, d.g, d.ty, d.py, d.tw[1], bx, rest % d.g.nz, rest / d.g.nz);
  }
}

__global__ void __launch_bounds__(kZThreads)
    kb_zproj(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter) {
  __shared__ int s_item;
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_Z, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    const int b = lb;
    const int nbx = (d.g.nxh + d.tz - 1) / d.tz;
    zproj_body<R>(d.spec, d.g, d.tz, d.pz, d.tw[2], d.gd[0], d.ga[0], d.gd[1], d.ga[1], d.gd[2], d.ga[2],
                  d.free_mask, b % nbx, b / nbx);
  }
}

__global__ void __launch_bounds__(kYThreads, kXYMinBlocks)
    kb_yproj2d(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter) {
  __shared__ int s_item;
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_2D, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    yproj2d_body<R>(d.spec, d.g, d.tz, d.py, d.tw[1], d.gd[0], d.ga[0], d.gd[1], d.ga[1], d.free_mask,
                    lb);
  }
}

template <int DOT>
__global__ void __launch_bounds__(kXThreads, kXYMinBlocks)
    kb_xinv(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter,
            const DevScalars* __restrict__ S, R* __restrict__ out, const R* __restrict__ dotw,
            double* __restrict__ partials) {
  __shared__ int s_item;
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_X, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    const R scale = (R)(1.0 / (double)d.g.nvox);
    xinv_body<R, DOT != 0>(d.spec, out + d.foff, DOT == 1 ? dotw + d.foff : nullptr,
                           DOT ? partials + v : nullptr, d.g, d.qx, d.px, d.tw[0], scale, DOT == 2, lb);
  }
}

// Sum per-item partials over each gated RVE's item range into a DevScalars
// field group (ns consecutive doubles at byte offset `off`).
__global__ void kb_seg_reduce(const double* __restrict__ part, const WLists* __restrict__ wl, int pass, int ns,
                              DevScalars* S, int off) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  if (k >= wl->count) return;
  const int i = wl->idx[k];
  const int s0 = wl->start[pass][k], s1 = wl->start[pass][k + 1];
  double* dst = reinterpret_cast<double*>(reinterpret_cast<char*>(&S[i]) + off);
  for (int s = 0; s < ns; ++s) {
    double acc = 0.0;
    for (int b = s0 + threadIdx.x; b < s1; b += blockDim.x) acc += part[(long long)b * ns + s];
    double v[1] = {acc};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) dst[s] = v[0];
    __syncthreads();
  }
}

// ------------------------------------------------------ vector kernels
enum VecOp : int { V_INIT = 0, V_UPDATE = 1, V_RESTART = 2, V_DUPDATE = 3, V_AXPY = 4, V_COPY = 5, V_ADDE = 6 };

template <int OP, int NS>
__global__ void __launch_bounds__(256)
    kb_vec(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter,
           DevScalars* __restrict__ S, R* __restrict__ a, R* __restrict__ b, R* __restrict__ c,
           const R* __restrict__ x, const R* __restrict__ y, const double* __restrict__ dE6,
           double* __restrict__ part) {
  __shared__ int s_item;
  __shared__ double red[NS > 0 ? NS * 32 : 32];
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_VEC, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    const long long nf = (long long)d.g.ncomp * d.g.nvox;
    const long long e0 = (long long)(lb) * kVecChunk;
    const long long e1 = min(nf, e0 + kVecChunk);
    KSum<R> acc[NS > 0 ? NS : 1];
    const DevScalars& s = S[i];
    const R alpha = (R)s.alpha, beta = (R)s.beta, tau = (R)s.tau;
    const bool exiting = (OP == V_UPDATE) && s.status != CG_RUN;
    for (long long e = e0 + 4 * threadIdx.x; e < e1; e += 4 * blockDim.x) {
      const long long o = d.foff + e;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long k = o + q;
        if (OP == V_INIT) {  // a=z, b=r, c=d, x=g
          const R gi = x[k];
          a[k] = 0;
          b[k] = gi;
          c[k] = -gi;
          acc[0].add(gi * gi);
        } else if (OP == V_UPDATE) {  // a=z, b=r, x=d, y=Hd
          if (exiting) {
            a[k] += tau * x[k];
          } else {
            const R zz = a[k] + alpha * x[k];
            const R ro = b[k];
            const R rn = ro + alpha * y[k];
            a[k] = zz;
            b[k] = rn;
            acc[0].add(rn * rn);
            acc[1].add(rn * ro);
            acc[2].add(zz * zz);
          }
        } else if (OP == V_RESTART) {  // b=r, x=Hz, y=g
          const R ri = x[k] + y[k];
          b[k] = ri;
          acc[0].add(ri * ri);
        } else if (OP == V_DUPDATE) {  // x=z, b=r(read), c=d
          const R rv = b[k];
          const R dv = -rv + beta * c[k];
          c[k] = dv;
          acc[0].add(dv * dv);
          acc[1].add(x[k] * dv);
          acc[2].add(rv * dv);
        } else if (OP == V_AXPY) {  // a += x
          a[k] += x[k];
        } else if (OP == V_COPY) {  // a = x
          a[k] = x[k];
        } else {  // V_ADDE: a += dE[comp]
          const int comp = (int)((e + q) / d.g.nvox);
          a[k] += (R)dE6[6 * i + comp];
        }
      }
    }
    if constexpr (NS > 0) {
      double vv[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) vv[q] = acc[q].value();
      block_sum<NS>(vv, red);
      if (threadIdx.x == 0)
        for (int q = 0; q < NS; ++q) part[(long long)v * NS + q] = vv[q];
    }
  }
}

// scalar-field copy (damage, kappa) over voxel items: a = x
__global__ void __launch_bounds__(256)
    kb_scopy(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter, R* __restrict__ a,
             const R* __restrict__ x) {
  __shared__ int s_item;
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_VOX, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    const long long v0 = (long long)(lb) * kVoxChunk;
    const long long v1 = min(d.g.nvox, v0 + kVoxChunk);
    for (long long k = v0 + threadIdx.x; k < v1; k += blockDim.x) a[d.voff + k] = x[d.voff + k];
  }
}

// Constitutive trial evaluation over voxel items (same arithmetic as the
// single-grid kernel); 6 sums per item.  MEANS instead sums sigma and eps
// per component (12 sums).
template <bool MEANS>
__global__ void __launch_bounds__(256)
    kb_trial(const BDesc* __restrict__ D, const WLists* __restrict__ wl, int* counter, const MatTable<R> mt,
             const uint8_t* __restrict__ phase,
             const R* __restrict__ eps, const R* __restrict__ p, const R* __restrict__ khist,
             const R* __restrict__ sig0, const R* __restrict__ D0, R* __restrict__ sig_t, R* __restrict__ D_t,
             R* __restrict__ kap_t, double* __restrict__ part, const R* __restrict__ cdp = nullptr,
             const R* __restrict__ ca = nullptr, const R* __restrict__ cn = nullptr) {
  __shared__ int s_item;
  constexpr int NS = MEANS ? 12 : 6;
  __shared__ double red[NS * 32];
  for (;;) {
    int v, i, lb;
    if (!fetch(wl, BP_VOX, counter, &s_item, &v, &i, &lb)) break;
    const BDesc& d = D[i];
    const int nc = d.g.ncomp, nd = d.g.ndim;
    const long long nv = d.g.nvox;
    const long long v0 = (long long)(lb) * kVoxChunk;
    const long long v1 = min(nv, v0 + kVoxChunk);
    KSum<R> acc[NS];
    for (long long k = v0 + threadIdx.x; k < v1; k += blockDim.x) {
      const long long fo = d.foff + k;
      if constexpr (MEANS) {
        for (int c = 0; c < nc; ++c) {
          acc[c].add(sig0[fo + c * nv]);
          acc[6 + c].add(eps[fo + c * nv]);
        }
      } else {
      R e[6], pv[6];
      for (int c = 0; c < nc; ++c) {
        pv[c] = p ? p[fo + c * nv] : (R)0;
        e[c] = eps[fo + c * nv] + pv[c];
      }
      const int ph = phase[d.voff + k];
      const R lam = mt.lam[ph], mu = mt.mu[ph];
      R Dv = 0, kap = 0;
      if (mt.damaging[ph]) {
        const R kt = kappa_tension<R>(e, nd);
        const R khk = khist[d.voff + k];
        const R kk = kt > khk ? kt : khk;  // keeps a NaN history (fmax would drop it)
        kap = kk;
        Dv = damage_of<R>(kk, mt.kappa0[ph], mt.kappaf[ph]);
      }
      const R keep = (R)1 - Dv;
      R tr = 0, trp = 0;
      for (int q = 0; q < nd; ++q) {
        tr += e[q];
        trp += pv[q];
      }
      const R keep0 = D0 ? (R)1 - D0[d.voff + k] : (R)1;
      // p:B0:p of the model with the Hessian of the state: the secant, plus
      // the consistent tangent's rank-one part where cdp is set
      const R hdp = (cdp && p) ? (R)0.5 * cdp[d.voff + k] : (R)0;
      R np_ = 0, ap_ = 0;
      if (hdp != (R)0) {
        for (int c = 0; c < nc; ++c) {
          np_ += cn[fo + c * nv] * pv[c];
          ap_ += ca[fo + c * nv] * pv[c];
        }
      }
      for (int c = 0; c < nc; ++c) {
        const R sv = keep * ((R)2 * mu * e[c] + (c < nd ? lam * tr : (R)0));
        sig_t[fo + c * nv] = sv;
        R bp = keep0 * ((R)2 * mu * pv[c] + (c < nd ? lam * trp : (R)0));
        if (hdp != (R)0) bp -= hdp * (ca[fo + c * nv] * np_ + cn[fo + c * nv] * ap_);
        if (sig0) acc[0].add(sig0[fo + c * nv] * pv[c]);
        acc[1].add(sv * pv[c]);
        acc[2].add(pv[c] * bp);
        acc[3].add(sv * sv);
        acc[4].add(pv[c] * pv[c]);
        acc[5].add(e[c] * e[c]);
      }
      D_t[d.voff + k] = Dv;
      kap_t[d.voff + k] = kap;
      }
    }
    double vv[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) vv[q] = acc[q].value();
    block_sum<NS>(vv, red);
    if (threadIdx.x == 0)
      for (int q = 0; q < NS; ++q) part[(long long)v * NS + q] = vv[q];
  }
}

// ------------------------------------------------------ scalar kernels
enum ScOp : int { S_PARAMS = 0, S_INIT = 1, S_ALPHA = 2, S_BETA = 3, S_RESTART = 4, S_DECIDE = 5, S_PARK = 6,
                  S_RADIUS = 7, S_ENERGY = 8 };

__global__ void kb_scalar(int op, int n, Gate gt, DevScalars* S, double eta_cg, double thr, int max_cg,
                          double eta_up, const double* __restrict__ R0, const double* __restrict__ Rmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  DevScalars* s = &S[i];
  if (op == S_PARK) {  // RVEs outside the gate leave the CG loop idle
    if (!gate_ok(gt, S, i)) {
      s->status = CG_ZERO;
      s->restart = 0;
      s->pad0 = 0;
    }
    return;
  }
  if (!gate_ok(gt, S, i)) return;
  switch (op) {
    case S_RADIUS:
      s->R = R0[i];
      s->Rmax = Rmax[i];
      break;
    case S_PARAMS:
      s->tol = eta_cg * sqrt(s->gg);
      s->thr = thr;
      s->max_cg = max_cg;
      s->eta_up = eta_up;
      s->pad0 = 0;
      break;
    case S_INIT: cg_init_scalars(s); break;
    case S_ALPHA: {
      const int before = s->status;
      cg_alpha_scalars(s);
      if (before == CG_RUN && (s->status == CG_BOUNDARY || s->status == CG_NEGCURV)) s->pad0 = 1;
      break;
    }
    case S_BETA:
      cg_beta_scalars(s);
      s->pad0 = 0;
      break;
    case S_RESTART: cg_restart_scalars(s); break;
    case S_DECIDE: tr_decide_scalars(s); break;
    default:  // S_ENERGY
      break;
  }
}

bool five_smooth_even(int n) {
  if (n < 2 || n > 1024 || (n & 1)) return false;
  int m = n;
  for (int p : {2, 3, 5})
    while (m % p == 0) m /= p;
  return m == 1;
}

}  // namespace

// ================================================================ context
struct rve_batch_ctx {
  int n = 0;
  cudaStream_t st = nullptr;
  rve_solver_opts opts{};
  MatTable<R> mt{};
  std::vector<GridDesc> g;
  std::vector<SpecWork<R>> sw;
  std::vector<BDesc> desc;
  BDesc* dD = nullptr;
  int* dnb = nullptr;      // BP_N x n block counts (device)
  WLists* wl = nullptr;    // compacted work lists (device)
  std::vector<int> hstart[BP_N];
  int total[BP_N] = {};
  size_t smem[BP_N] = {};
  int* counters = nullptr;  // one slot per launch in a sequence (reset by memset)
  int ncounters = 64;
  int cslot = 0;
  long long nfield = 0, nvox = 0;
  R *eps = nullptr, *sig = nullptr, *sig_t = nullptr, *gv = nullptr, *z = nullptr, *r = nullptr, *d = nullptr,
    *Hd = nullptr, *tmp = nullptr;
  R *D = nullptr, *D_t = nullptr, *kap = nullptr, *kap_t = nullptr, *khist = nullptr;
  // symmetric consistent tangent (opts.hessian = 1): D'(kappa) per voxel, C:eps
  // and eps^(t)/kappa per field element, refreshed for every accepted state
  R *cdp = nullptr, *ca = nullptr, *cn = nullptr;
  uint8_t* phase = nullptr;
  DevScalars* S = nullptr;
  DevScalars* Sh = nullptr;
  double* part = nullptr;
  double* dE = nullptr;    // n x 6 device
  double* hbuf = nullptr;  // pinned staging: n x 6 dE, n R0, n Rmax
  double* dR = nullptr;    // n R0 + n Rmax device
  std::vector<char> radius_set;
  bool any3d = false, any2d = false;
  cudaGraphExec_t g_iter = nullptr, g_dir = nullptr;
  cudaStream_t cap = nullptr;  // private stream the graphs are captured on (launched on st)
  int part_items = 0;           // capacity of `part` in work items (12 doubles each)
  int sched[4] = {1, 1, 1, 0};  // schedule: x / y / z tile divisors, reversed radix order
  long long launches = 0, hv = 0;
  std::string err = "no error";
};

namespace {

thread_local std::string g_batch_create_error = "no error";

rve_status bfail(rve_batch_ctx* c, rve_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_batch_create_error = msg;
  return s;
}

#define BCK(call, where)                                                                              \
  do {                                                                                                \
    cudaError_t e__ = (call);                                                                         \
    if (e__ != cudaSuccess)                                                                           \
      return bfail(c, e__ == cudaErrorMemoryAllocation ? RVE_ERR_OOM : RVE_ERR_CUDA,                   \
                   std::string(where) + ": " + cudaGetErrorString(e__));                              \
  } while (0)

Gate gate_bits(const std::vector<char>& m) {
  Gate g{};
  g.mode = G_BITS;
  for (size_t i = 0; i < m.size(); ++i)
    if (m[i]) g.bits[i >> 5] |= 1u << (i & 31);
  return g;
}
Gate gate_mode(int mode) {
  Gate g{};
  g.mode = mode;
  return g;
}

int grid_for(int total, int per_sm) { return std::max(1, std::min(total, 152 * per_sm)); }

// counter slot for the next work-list launch; the caller resets slots with
// reset_counters() at the start of every launch sequence
int* next_counter(rve_batch_ctx* c) { return c->counters + (c->cslot++ % c->ncounters); }
cudaError_t reset_counters(rve_batch_ctx* c) {
  c->cslot = 0;
  return cudaMemsetAsync(c->counters, 0, c->ncounters * sizeof(int), c->st);
}

cudaError_t compact(rve_batch_ctx* c, Gate gt) {
  kb_compact<<<1, 256, 0, c->st>>>(c->wl, c->dnb, c->n, gt, c->S);
  ++c->launches;
  return cudaGetLastError();
}

// per-member sums over the items of the last compacted work list
cudaError_t seg_reduce(rve_batch_ctx* c, int pass, int ns, size_t off) {
  kb_seg_reduce<<<c->n, 256, 0, c->st>>>(c->part, c->wl, pass, ns, c->S, (int)off);
  ++c->launches;
  return cudaGetLastError();
}

// Hessian-vector product (tangent) or projection (plain) of every gated RVE:
// out = G : (B : in) or G : in; with dot, sum(out * dotw) (or |out|^2 when
// dotw == out) into DevScalars at byte offset dot_off.
cudaError_t batch_apply(rve_batch_ctx* c, const R* in, R* out, bool tangent, const R* dotw, size_t dot_off, Gate gt) {
  cudaError_t e;
  if ((e = compact(c, gt)) != cudaSuccess) return e;
  {
    const int tot = c->total[BP_X];
    // hessian = 1: every tangent product carries the consistent tangent's
    // rank-one part of the current state (refreshed whenever eps or the
    // history change), also inside the captured CG graphs
    const bool cons = c->cdp != nullptr;
    if (tangent)
      kb_xfwd<1><<<grid_for(tot, kXYMinBlocks), kXThreads, c->smem[BP_X], c->st>>>(
          c->dD, c->wl, next_counter(c), c->S, c->mt, in, c->phase, c->D, cons ? c->cdp : nullptr,
          cons ? c->ca : nullptr, cons ? c->cn : nullptr);
    else
      kb_xfwd<0><<<grid_for(tot, kXYMinBlocks), kXThreads, c->smem[BP_X], c->st>>>(
          c->dD, c->wl, next_counter(c), c->S, c->mt, in, c->phase, c->D, nullptr, nullptr, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c->any3d) {
    kb_ycols<false><<<grid_for(c->total[BP_Y], kXYMinBlocks), kYThreads, c->smem[BP_Y], c->st>>>(
        c->dD, c->wl, next_counter(c));
    kb_zproj<<<grid_for(c->total[BP_Z], 2), kZThreads, c->smem[BP_Z], c->st>>>(c->dD, c->wl, next_counter(c));
    kb_ycols<true><<<grid_for(c->total[BP_Y], kXYMinBlocks), kYThreads, c->smem[BP_Y], c->st>>>(
        c->dD, c->wl, next_counter(c));
    c->launches += 3;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c->any2d) {
    kb_yproj2d<<<grid_for(c->total[BP_2D], kXYMinBlocks), kYThreads, c->smem[BP_2D], c->st>>>(
        c->dD, c->wl, next_counter(c));
    ++c->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int tot = c->total[BP_X];
  if (!dotw) {
    kb_xinv<0><<<grid_for(tot, kXYMinBlocks), kXThreads, c->smem[BP_X], c->st>>>(c->dD, c->wl,
                                                                      next_counter(c), c->S, out, nullptr,
                                                                      nullptr);
  } else if (dotw == out) {
    kb_xinv<2><<<grid_for(tot, kXYMinBlocks), kXThreads, c->smem[BP_X], c->st>>>(c->dD, c->wl,
                                                                      next_counter(c), c->S, out, nullptr,
                                                                      c->part);
  } else {
    kb_xinv<1><<<grid_for(tot, kXYMinBlocks), kXThreads, c->smem[BP_X], c->st>>>(c->dD, c->wl,
                                                                      next_counter(c), c->S, out, dotw,
                                                                      c->part);
  }
  c->launches += 2;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (dotw) return seg_reduce(c, BP_X, 1, dot_off);
  return cudaSuccess;
}

template <int OP, int NS>
cudaError_t vec(rve_batch_ctx* c, Gate gt, R* a, R* b, R* cc, const R* x, const R* y, size_t sum_off) {
  cudaError_t e = compact(c, gt);
  if (e != cudaSuccess) return e;
  const int tot = c->total[BP_VEC];
  kb_vec<OP, NS><<<grid_for(tot, 8), 256, 0, c->st>>>(c->dD, c->wl, next_counter(c), c->S, a, b, cc, x, y, c->dE,
                                                       c->part);
  ++c->launches;
  e = cudaGetLastError();
  if (e != cudaSuccess || NS == 0) return e;
  return seg_reduce(c, BP_VEC, NS, sum_off);
}

cudaError_t scopy(rve_batch_ctx* c, Gate gt, R* a, const R* x) {
  cudaError_t e = compact(c, gt);
  if (e != cudaSuccess) return e;
  const int tot = c->total[BP_VOX];
  kb_scopy<<<grid_for(tot, 8), 256, 0, c->st>>>(c->dD, c->wl, next_counter(c), a, x);
  ++c->launches;
  return cudaGetLastError();
}

cudaError_t trial(rve_batch_ctx* c, Gate gt, const R* p, bool with_state) {
  cudaError_t e0 = compact(c, gt);
  if (e0 != cudaSuccess) return e0;
  const int tot = c->total[BP_VOX];
  kb_trial<false><<<grid_for(tot, 8), 256, 0, c->st>>>(c->dD, c->wl, next_counter(c), c->mt, c->phase, c->eps, p,
                                                       c->khist,
                                                       with_state ? c->sig : nullptr, with_state ? c->D : nullptr,
                                                       with_state ? c->sig_t : c->sig, with_state ? c->D_t : c->D,
                                                       with_state ? c->kap_t : c->kap, c->part,
                                                       with_state ? c->cdp : nullptr, c->ca, c->cn);
  ++c->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return seg_reduce(c, BP_VOX, 6, offsetof(DevScalars, sp));
}

cudaError_t scalar(rve_batch_ctx* c, int op, Gate gt) {
  kb_scalar<<<(c->n + 127) / 128, 128, 0, c->st>>>(op, c->n, gt, c->S, c->opts.eta_cg, c->opts.restart_thr,
                                                   c->opts.max_cg, c->opts.eta_up, c->dR, c->dR + c->n);
  ++c->launches;
  return cudaGetLastError();
}

rve_status read_all(rve_batch_ctx* c) {
  BCK(cudaMemcpyAsync(c->Sh, c->S, c->n * sizeof(DevScalars), cudaMemcpyDeviceToHost, c->st), "read scalars");
  BCK(cudaStreamSynchronize(c->st), "synchronize");
  return RVE_OK;
}

// The inner CG iteration (Hv of d, alpha, z/r update, beta) and the
// direction update, as fixed launch sequences gated on device-side status.
cudaError_t issue_iter(rve_batch_ctx* c) {
  cudaError_t e;
  if ((e = reset_counters(c)) != cudaSuccess) return e;
  const Gate run = gate_mode(G_RUN);
  if ((e = batch_apply(c, c->d, c->Hd, true, c->d, offsetof(DevScalars, dHd), run)) != cudaSuccess) return e;
  if ((e = scalar(c, S_ALPHA, run)) != cudaSuccess) return e;
  const Gate upd = gate_mode(G_UPDATE);
  if ((e = vec<V_UPDATE, 3>(c, upd, c->z, c->r, nullptr, c->d, c->Hd, offsetof(DevScalars, rr_new))) != cudaSuccess)
    return e;
  return scalar(c, S_BETA, upd);
}
cudaError_t issue_dir(rve_batch_ctx* c) {
  cudaError_t e;
  if ((e = reset_counters(c)) != cudaSuccess) return e;
  return vec<V_DUPDATE, 3>(c, gate_mode(G_RUN), nullptr, c->r, c->d, c->z, nullptr, offsetof(DevScalars, dd));
}

rve_status build_graph(rve_batch_ctx* c, cudaGraphExec_t* out, cudaError_t (*issue)(rve_batch_ctx*)) {
  // capture on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graph is launched on the caller's
  if (!c->cap) BCK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "capture stream");
  cudaGraph_t graph = nullptr;
  cudaStream_t user = c->st;
  BCK(cudaStreamSynchronize(user), "synchronize");
  c->st = c->cap;
  cudaError_t e0 = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
  if (e0 != cudaSuccess) {
    c->st = user;
    return bfail(c, RVE_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e0));
  }
  cudaError_t e = issue(c);
  cudaError_t e2 = cudaStreamEndCapture(c->st, &graph);
  c->st = user;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(c, RVE_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  }
  BCK(e2, "end capture");
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  BCK(e, "graph instantiate");
  return RVE_OK;
}

rve_status run_graph(rve_batch_ctx* c, cudaGraphExec_t* g, cudaError_t (*issue)(rve_batch_ctx*)) {
  if (!*g) {
    rve_status s = build_graph(c, g, issue);
    if (s != RVE_OK) return s;
  }
  BCK(cudaGraphLaunch(*g, c->st), "graph launch");
  ++c->launches;
  return RVE_OK;
}

// Steihaug CG on every RVE in `mask` (Algorithm 1), in lockstep.
rve_status batch_cg(rve_batch_ctx* c, const std::vector<char>& mask, rve_step_report* reps) {
  const Gate gm = gate_bits(mask);
  BCK(reset_counters(c), "memset");
  BCK(scalar(c, S_PARAMS, gm), "cg params");
  BCK((vec<V_INIT, 1>(c, gm, c->z, c->r, c->d, c->gv, nullptr, offsetof(DevScalars, rr))), "cg init");
  BCK(scalar(c, S_INIT, gm), "cg init scalars");
  BCK(scalar(c, S_PARK, gm), "park");
  rve_status s = read_all(c);
  if (s != RVE_OK) return s;
  auto any_run = [&]() {
    for (int i = 0; i < c->n; ++i)
      if (c->Sh[i].status == CG_RUN) return true;
    return false;
  };
  while (any_run()) {
    for (int i = 0; i < c->n; ++i)
      if (c->Sh[i].status == CG_RUN) {
        ++c->hv;
        ++reps[i].hv_products;
      }
    if ((s = run_graph(c, &c->g_iter, issue_iter)) != RVE_OK) return s;
    if ((s = read_all(c)) != RVE_OK) return s;
    bool any_restart = false;
    for (int i = 0; i < c->n; ++i)
      if (c->Sh[i].status == CG_RUN && c->Sh[i].restart) {
        any_restart = true;
        ++c->hv;
        ++reps[i].hv_products;
      }
    if (any_restart) {
      const Gate rg = gate_mode(G_RESTART);
      BCK(reset_counters(c), "memset");
      BCK(batch_apply(c, c->z, c->tmp, true, nullptr, 0, rg), "restart hessp");
      BCK((vec<V_RESTART, 1>(c, rg, nullptr, c->r, nullptr, c->tmp, c->gv, offsetof(DevScalars, rr_new))),
          "restart");
      BCK(scalar(c, S_RESTART, rg), "restart scalars");
    }
    if (any_run())
      if ((s = run_graph(c, &c->g_dir, issue_dir)) != RVE_OK) return s;
  }
  for (int i = 0; i < c->n; ++i)
    if (mask[i]) {
      reps[i].cg_iters += c->Sh[i].iters;
      reps[i].restarts += c->Sh[i].restarts;
      if (c->Sh[i].status == CG_NONFINITE) return bfail(c, RVE_ERR_NONFINITE, "non-finite value in CG");
    }
  return RVE_OK;
}

// The consistent tangent's per-voxel data for the current state (eps,
// khist) of every member: one preparation launch per member (outside the
// captured CG iteration; once per accepted Newton state).
rve_status batch_refresh_hessian(rve_batch_ctx* c) {
  if (!c->cdp) return RVE_OK;
  const EigTable<R> none{};
  for (int i = 0; i < c->n; ++i) {
    const BDesc& d = c->desc[i];
    BCK(cons_prep<R>(c->g[i], c->mt, none, c->phase + d.voff, c->eps + d.foff, c->khist + d.voff, c->cdp + d.voff,
                     c->ca + d.foff, c->cn + d.foff, c->st, &c->launches),
        "consistent tangent");
  }
  return RVE_OK;
}

rve_status batch_solve(rve_batch_ctx* c, const double* dE, rve_step_report* reps) {
  const int n = c->n;
  std::vector<char> all(n, 1);
  const Gate ga = gate_bits(all);
  rve_status s0 = RVE_OK;
  // radius defaults per RVE (first load step)
  bool upload_r = false;
  for (int i = 0; i < n; ++i) {
    std::memset(&reps[i], 0, sizeof(rve_step_report));
    if (!c->radius_set[i]) {
      double n2 = 0;
      for (int q = 0; q < c->g[i].ncomp; ++q) n2 += dE[6 * i + q] * dE[6 * i + q];
      const double def = 10.0 * std::sqrt((double)c->g[i].nvox) * std::sqrt(n2);
      double R0 = c->opts.R0 > 0 ? c->opts.R0 : def;
      double Rm = c->opts.Rmax > 0 ? c->opts.Rmax : std::max(R0, def);
      if (!(R0 > 0)) R0 = Rm = 1.0;
      c->hbuf[6 * n + i] = R0;
      c->hbuf[7 * n + i] = Rm;
      c->radius_set[i] = 1;
      upload_r = true;
    } else {
      c->hbuf[6 * n + i] = -1.0;
    }
  }
  std::memcpy(c->hbuf, dE, 6 * n * sizeof(double));
  BCK(cudaMemcpyAsync(c->dE, c->hbuf, 6 * n * sizeof(double), cudaMemcpyHostToDevice, c->st), "dE upload");
  if (upload_r) {
    BCK(cudaMemcpyAsync(c->dR, c->hbuf + 6 * n, 2 * n * sizeof(double), cudaMemcpyHostToDevice, c->st), "R upload");
    std::vector<char> fresh(n, 0);
    for (int i = 0; i < n; ++i) fresh[i] = c->hbuf[6 * n + i] > 0;
    BCK(scalar(c, S_RADIUS, gate_bits(fresh)), "radius");
  }
  BCK(reset_counters(c), "memset");
  BCK((vec<V_ADDE, 0>(c, ga, c->eps, nullptr, nullptr, nullptr, nullptr, 0)), "load increment");
  BCK(trial(c, ga, nullptr, false), "stress");
  if ((s0 = batch_refresh_hessian(c)) != RVE_OK) return s0;
  BCK(batch_apply(c, c->sig, c->gv, false, c->gv, offsetof(DevScalars, gg), ga), "gradient");
  rve_status s = read_all(c);
  if (s != RVE_OK) return s;
  std::vector<char> conv(n, 0), active(n, 0);
  std::vector<double> rel(n, 0.0);
  for (int i = 0; i < n; ++i) {
    rel[i] = c->Sh[i].sts > 0 ? std::sqrt(c->Sh[i].gg / c->Sh[i].sts) : 0.0;
    conv[i] = rel[i] <= c->opts.eta_eq;
  }
  for (;;) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      active[i] = !conv[i] && reps[i].nr_iters < c->opts.max_nr;
      any = any || active[i];
    }
    if (!any) break;
    for (int i = 0; i < n; ++i)
      if (active[i]) reps[i].nr_iters++;
    if ((s = batch_cg(c, active, reps)) != RVE_OK) return s;
    const Gate gm = gate_bits(active);
    BCK(reset_counters(c), "memset");
    BCK(trial(c, gm, c->z, true), "trial stress");
    BCK(scalar(c, S_DECIDE, gm), "ratio test");
    if ((s = read_all(c)) != RVE_OK) return s;
    std::vector<char> acc(n, 0);
    bool any_acc = false;
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      if (c->Sh[i].nonfinite) return bfail(c, RVE_ERR_NONFINITE, "non-finite trial state");
      if (c->Sh[i].on_boundary) reps[i].boundary_hits++;
      if (c->Sh[i].accept) {
        acc[i] = 1;
        any_acc = true;
      } else {
        reps[i].rejected++;
      }
    }
    if (!any_acc) continue;
    std::vector<double> pp(n), ee(n), sts(n);
    std::vector<char> onb(n);
    for (int i = 0; i < n; ++i) {
      pp[i] = c->Sh[i].pp;
      ee[i] = c->Sh[i].ee;
      sts[i] = c->Sh[i].sts;
      onb[i] = c->Sh[i].on_boundary;
    }
    const Gate gacc = gate_bits(acc);
    BCK(reset_counters(c), "memset");
    BCK((vec<V_AXPY, 0>(c, gacc, c->eps, nullptr, nullptr, c->z, nullptr, 0)), "accept step");
    BCK((vec<V_COPY, 0>(c, gacc, c->sig, nullptr, nullptr, c->sig_t, nullptr, 0)), "accept stress");
    BCK(scopy(c, gacc, c->D, c->D_t), "accept damage");
    BCK(scopy(c, gacc, c->kap, c->kap_t), "accept kappa");
    if ((s = batch_refresh_hessian(c)) != RVE_OK) return s;
    BCK(batch_apply(c, c->sig, c->gv, false, c->gv, offsetof(DevScalars, gg), gacc), "gradient");
    if ((s = read_all(c)) != RVE_OK) return s;
    for (int i = 0; i < n; ++i) {
      if (!acc[i]) continue;
      rel[i] = sts[i] > 0 ? std::sqrt(c->Sh[i].gg / sts[i]) : 0.0;
      const double rnr = ee[i] > 0 ? std::sqrt(pp[i] / ee[i]) : 0.0;
      if (!onb[i] && (rel[i] <= c->opts.eta_eq || (c->opts.eta_nr > 0 && rnr <= c->opts.eta_nr))) conv[i] = 1;
    }
  }
  // homogenised stress / strain, history commit for converged RVEs
  BCK(reset_counters(c), "memset");
  {
    const int tot = c->total[BP_VOX];
    BCK(compact(c, ga), "means");
    kb_trial<true><<<grid_for(tot, 8), 256, 0, c->st>>>(c->dD, c->wl, next_counter(c), c->mt, c->phase, c->eps,
                                                        nullptr, c->khist, c->sig, nullptr, nullptr, nullptr,
                                                        nullptr, c->part);
    ++c->launches;
    BCK(cudaGetLastError(), "means");
    BCK(seg_reduce(c, BP_VOX, 12, offsetof(DevScalars, msig)), "means");
  }
  BCK(scopy(c, gate_bits(conv), c->khist, c->kap), "commit");
  if ((s = batch_refresh_hessian(c)) != RVE_OK) return s;
  if ((s = read_all(c)) != RVE_OK) return s;
  bool all_conv = true;
  for (int i = 0; i < n; ++i) {
    for (int q = 0; q < 6; ++q) {
      reps[i].mean_stress[q] = c->Sh[i].msig[q] / (double)c->g[i].nvox;
      reps[i].mean_strain[q] = c->Sh[i].meps[q] / (double)c->g[i].nvox;
    }
    reps[i].rel_residual = rel[i];
    reps[i].R = c->Sh[i].R;
    reps[i].converged = conv[i];
    all_conv = all_conv && conv[i];
  }
  if (!all_conv) return bfail(c, RVE_ERR_NOT_CONVERGED, "a member load step did not converge within max_nr");
  return RVE_OK;
}

void batch_free(rve_batch_ctx* c) {
  if (!c) return;
  for (auto& w : c->sw) spectral_free(w);
  void* ptrs[] = {c->dD, c->counters, c->eps, c->sig, c->sig_t, c->gv, c->z, c->r, c->d, c->Hd, c->tmp,
                  c->D, c->D_t, c->kap, c->kap_t, c->khist, c->phase, c->S, c->part, c->dE, c->dR,
                  c->cdp, c->ca, c->cn};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->dnb) cudaFree(c->dnb);
  if (c->wl) cudaFree(c->wl);
  if (c->Sh) cudaFreeHost(c->Sh);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  if (c->g_iter) cudaGraphExecDestroy(c->g_iter);
  if (c->g_dir) cudaGraphExecDestroy(c->g_dir);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

rve_status batch_init(rve_batch_ctx* c, const int* dims, const int* ndims, const uint8_t* const* ids,
                      const rve_phase* phases, int nphase) {
  const int n = c->n;
  c->mt.nphase = nphase;
  for (int i = 0; i < nphase; ++i) {
    const double E = phases[i].E, nu = phases[i].nu;
    c->mt.lam[i] = (R)(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
    c->mt.mu[i] = (R)(E / (2.0 * (1.0 + nu)));
    c->mt.damaging[i] = phases[i].damaging ? 1 : 0;
    c->mt.kappa0[i] = (R)phases[i].kappa0;
    c->mt.kappaf[i] = (R)phases[i].kappaf;
  }
  c->g.resize(n);
  c->sw.resize(n);
  c->desc.resize(n);
  c->radius_set.assign(n, 0);
  for (int p = 0; p < BP_N; ++p) c->hstart[p].assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    GridDesc& g = c->g[i];
    g.ndim = ndims[i];
    g.nx = dims[3 * i];
    g.ny = dims[3 * i + 1];
    g.nz = g.ndim == 3 ? dims[3 * i + 2] : 1;
    g.nxh = g.nx / 2 + 1;
    g.ncomp = g.ndim == 3 ? 6 : 3;
    g.nvox = (long long)g.nx * g.ny * g.nz;
    g.nrows = (long long)g.ny * g.nz;
    if (g.ndim == 3) c->any3d = true;
    else c->any2d = true;
    BCK(spectral_setup<R>(g, c->sw[i]), "spectral setup");
    const SpecWork<R>& w = c->sw[i];
    BDesc& d = c->desc[i];
    d.g = g;
    d.px = w.px;
    d.py = w.py;
    d.pz = w.pz;
    for (int a = 0; a < 3; ++a) {
      d.tw[a] = w.tw[a];
      d.gd[a] = w.gdiff[a];
      d.ga[a] = w.gavg[a];
    }
    d.spec = w.spec;
    d.qx = w.qx;
    d.ty = w.ty;
    d.tz = w.tz;
    d.free_mask = 0;
    d.foff = c->nfield;
    d.voff = c->nvox;
    c->nfield += (long long)g.ncomp * g.nvox;
    c->nvox += g.nvox;
    const int nb[BP_N] = {
        (int)((g.nrows + w.qx - 1) / w.qx),
        g.ndim == 3 ? ((g.nxh + w.ty - 1) / w.ty) * g.nz * g.ncomp : 0,
        g.ndim == 3 ? ((g.nxh + w.tz - 1) / w.tz) * g.ny : 0,
        g.ndim == 2 ? (g.nxh + w.tz - 1) / w.tz : 0,
        (int)(((long long)g.ncomp * g.nvox + kVecChunk - 1) / kVecChunk),
        (int)((g.nvox + kVoxChunk - 1) / kVoxChunk),
    };
    for (int p = 0; p < BP_N; ++p) c->hstart[p][i + 1] = c->hstart[p][i] + nb[p];
    const size_t xs = (size_t)((g.ncomp * w.qx) / 2) * g.nx * sizeof(C);
    c->smem[BP_X] = std::max(c->smem[BP_X], xs);
    if (g.ndim == 3) {
      c->smem[BP_Y] = std::max(c->smem[BP_Y], (size_t)w.ty * g.ny * sizeof(C));
      c->smem[BP_Z] = std::max(c->smem[BP_Z], (size_t)6 * w.tz * g.nz * sizeof(C));
    } else {
      c->smem[BP_2D] = std::max(c->smem[BP_2D], (size_t)3 * w.tz * g.ny * sizeof(C));
    }
  }
  std::vector<int> nbh((size_t)BP_N * n);
  for (int p = 0; p < BP_N; ++p) {
    c->total[p] = c->hstart[p][n];
    for (int i = 0; i < n; ++i) nbh[(size_t)p * n + i] = c->hstart[p][i + 1] - c->hstart[p][i];
  }
  BCK(cudaMalloc(&c->dnb, nbh.size() * sizeof(int)), "schedule");
  BCK(cudaMemcpy(c->dnb, nbh.data(), nbh.size() * sizeof(int), cudaMemcpyHostToDevice), "schedule");
  BCK(cudaMalloc(&c->wl, sizeof(WLists)), "work lists");
  BCK(cudaMalloc(&c->dD, n * sizeof(BDesc)), "descriptors");
  BCK(cudaMemcpy(c->dD, c->desc.data(), n * sizeof(BDesc), cudaMemcpyHostToDevice), "descriptors");
  BCK(cudaMalloc(&c->counters, c->ncounters * sizeof(int)), "counters");
  const size_t fb = (size_t)c->nfield * sizeof(R), vb = (size_t)c->nvox * sizeof(R);
  R** fields[] = {&c->eps, &c->sig, &c->sig_t, &c->gv, &c->z, &c->r, &c->d, &c->Hd, &c->tmp};
  for (R** f : fields) BCK(cudaMalloc(f, fb), "field allocation");
  R** sfields[] = {&c->D, &c->D_t, &c->kap, &c->kap_t, &c->khist};
  for (R** f : sfields) BCK(cudaMalloc(f, vb), "scalar-field allocation");
  if (c->opts.hessian == 1) {
    BCK(cudaMalloc(&c->cdp, vb), "consistent-tangent allocation");
    BCK(cudaMalloc(&c->ca, fb), "consistent-tangent allocation");
    BCK(cudaMalloc(&c->cn, fb), "consistent-tangent allocation");
    BCK(cudaMemsetAsync(c->cdp, 0, vb, c->st), "memset");
  }
  BCK(cudaMalloc(&c->phase, c->nvox), "phase allocation");
  for (int i = 0; i < n; ++i)
    BCK(cudaMemcpyAsync(c->phase + c->desc[i].voff, ids[i], c->g[i].nvox, cudaMemcpyDeviceToDevice, c->st),
        "phase copy");
  std::vector<uint8_t> hid(c->nvox);
  BCK(cudaMemcpyAsync(hid.data(), c->phase, c->nvox, cudaMemcpyDeviceToHost, c->st), "phase check");
  BCK(cudaStreamSynchronize(c->st), "synchronize");
  for (long long k = 0; k < c->nvox; ++k)
    if (hid[k] >= nphase) return bfail(c, RVE_ERR_ARG, "phase id out of range");
  BCK(cudaMalloc(&c->S, n * sizeof(DevScalars)), "scalars");
  BCK(cudaMemsetAsync(c->S, 0, n * sizeof(DevScalars), c->st), "memset");
  BCK(cudaMallocHost(&c->Sh, n * sizeof(DevScalars)), "pinned scalars");
  BCK(cudaMallocHost(&c->hbuf, 8 * n * sizeof(double)), "pinned staging");
  BCK(cudaMalloc(&c->dE, 6 * n * sizeof(double)), "increments");
  BCK(cudaMalloc(&c->dR, 2 * n * sizeof(double)), "radii");
  const int maxitems = std::max({c->total[BP_X], c->total[BP_VEC], c->total[BP_VOX]});
  BCK(cudaMalloc(&c->part, (size_t)maxitems * 12 * sizeof(double)), "partials");
  c->part_items = maxitems;
  BCK(cudaMemsetAsync(c->eps, 0, fb, c->st), "memset");
  BCK(cudaMemsetAsync(c->khist, 0, vb, c->st), "memset");
  BCK(cudaMemsetAsync(c->kap, 0, vb, c->st), "memset");
  // kernel attributes for the largest dynamic shared memory
  BCK((cudaFuncSetAttribute(kb_xfwd<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_xfwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_xinv<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_xinv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_xinv<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_ycols<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_ycols<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_zproj, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  BCK((cudaFuncSetAttribute(kb_yproj2d, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap)), "attr");
  // state eps = 0: sigma = 0, D = 0
  std::vector<char> all(n, 1);
  BCK(reset_counters(c), "memset");
  BCK(trial(c, gate_bits(all), nullptr, false), "initial state");
  BCK(cudaStreamSynchronize(c->st), "synchronize");
  return RVE_OK;
}

// ---------------------------------------------------------------- autotune
// A schedule of the batched spectral passes: every member's x / y / z tile
// (rows per x item, kx columns per y item and per z item) divided by
// sx / sy / sz (the tiles of spectral_setup are the largest the per-thread
// element budgets allow, so only smaller ones are candidates), and the
// radix order of every axis plan natural or reversed (any order is a valid
// Stockham factorisation).  Work-item counts, dynamic shared memory, the
// partial-sum buffer and the device descriptors follow; captured graphs are
// dropped so that they are recaptured with the new schedule.
void reverse_plan(AxisPlan& p) {
  for (int a = 0, b = p.nstages - 1; a < b; ++a, --b) std::swap(p.radix[a], p.radix[b]);
}

rve_status apply_schedule(rve_batch_ctx* c, const int sched[4]) {
  const int n = c->n;
  const int passes[4] = {BP_X, BP_Y, BP_Z, BP_2D};
  for (int p : passes) c->smem[p] = 0;
  for (int i = 0; i < n; ++i) {
    const GridDesc& g = c->g[i];
    const SpecWork<R>& w = c->sw[i];
    BDesc& d = c->desc[i];
    int qx = std::max(1, w.qx / sched[0]);
    if (g.ncomp & 1) qx = std::max(2, qx & ~1);
    d.qx = qx;
    d.ty = std::max(1, w.ty / sched[1]);
    d.tz = std::max(1, w.tz / sched[2]);
    d.px = w.px;
    d.py = w.py;
    d.pz = w.pz;
    if (sched[3]) {
      reverse_plan(d.px);
      reverse_plan(d.py);
      reverse_plan(d.pz);
    }
    const int nb[4] = {
        (int)((g.nrows + d.qx - 1) / d.qx),
        g.ndim == 3 ? ((g.nxh + d.ty - 1) / d.ty) * g.nz * g.ncomp : 0,
        g.ndim == 3 ? ((g.nxh + d.tz - 1) / d.tz) * g.ny : 0,
        g.ndim == 2 ? (g.nxh + d.tz - 1) / d.tz : 0,
    };
    for (int k = 0; k < 4; ++k) c->hstart[passes[k]][i + 1] = c->hstart[passes[k]][i] + nb[k];
    c->smem[BP_X] = std::max(c->smem[BP_X], (size_t)((g.ncomp * d.qx) / 2) * g.nx * sizeof(C));
    if (g.ndim == 3) {
      c->smem[BP_Y] = std::max(c->smem[BP_Y], (size_t)d.ty * g.ny * sizeof(C));
      c->smem[BP_Z] = std::max(c->smem[BP_Z], (size_t)6 * d.tz * g.nz * sizeof(C));
    } else {
      c->smem[BP_2D] = std::max(c->smem[BP_2D], (size_t)3 * d.tz * g.ny * sizeof(C));
    }
  }
  std::vector<int> nbh((size_t)BP_N * n);
  for (int p = 0; p < BP_N; ++p) {
    c->total[p] = c->hstart[p][n];
    for (int i = 0; i < n; ++i) nbh[(size_t)p * n + i] = c->hstart[p][i + 1] - c->hstart[p][i];
  }
  BCK(cudaStreamSynchronize(c->st), "synchronize");
  BCK(cudaMemcpy(c->dnb, nbh.data(), nbh.size() * sizeof(int), cudaMemcpyHostToDevice), "schedule");
  BCK(cudaMemcpy(c->dD, c->desc.data(), n * sizeof(BDesc), cudaMemcpyHostToDevice), "descriptors");
  const int maxitems = std::max({c->total[BP_X], c->total[BP_VEC], c->total[BP_VOX]});
  if (maxitems > c->part_items) {
    BCK(cudaFree(c->part), "partials");
    c->part = nullptr;
    BCK(cudaMalloc(&c->part, (size_t)maxitems * 12 * sizeof(double)), "partials");
    c->part_items = maxitems;
  }
  if (c->g_iter) cudaGraphExecDestroy(c->g_iter);
  if (c->g_dir) cudaGraphExecDestroy(c->g_dir);
  c->g_iter = c->g_dir = nullptr;
  for (int k = 0; k < 4; ++k) c->sched[k] = sched[k];
  return RVE_OK;
}

// mean time of one batched Hessian-vector product of every member (ms)
rve_status time_products(rve_batch_ctx* c, int reps, double* ms) {
  std::vector<char> all(c->n, 1);
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "event");
  BCK(cudaEventCreate(&e1), "event");
  cudaError_t e = cudaSuccess;
  // one untimed product (first use of the schedule), then `reps` timed
  for (int k = 0; k <= reps && e == cudaSuccess; ++k) {
    if (k == 1) e = cudaEventRecord(e0, c->st);
    if (e == cudaSuccess) e = reset_counters(c);
    if (e == cudaSuccess) e = batch_apply(c, c->d, c->Hd, true, nullptr, 0, gate_bits(all));
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BCK(e, "timed products");
  *ms = (double)t / reps;
  return RVE_OK;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

rve_status rve_batch_create(int n, const int* dims, const int* ndims, const uint8_t* const* phase_ids_dev,
                            const rve_phase* phases, int nphase, const rve_solver_opts* opts, void* stream,
                            rve_batch_t* out) {
  if (!out) return bfail(nullptr, RVE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > kMaxBatch) return bfail(nullptr, RVE_ERR_ARG, "batch size must be in [1, 256]");
  if (!dims || !ndims || !phase_ids_dev || !phases) return bfail(nullptr, RVE_ERR_ARG, "NULL argument");
  if (nphase < 1 || nphase > kMaxPhases) return bfail(nullptr, RVE_ERR_ARG, "nphase must be in [1, 16]");
  for (int i = 0; i < nphase; ++i) {
    const rve_phase& p = phases[i];
    if (!(p.E > 0) || !(p.nu > -1.0 && p.nu < 0.5)) return bfail(nullptr, RVE_ERR_ARG, "invalid elastic constants");
    if (p.damaging && !(p.kappa0 > 0 && p.kappaf > p.kappa0))
      return bfail(nullptr, RVE_ERR_ARG, "damaging phase needs 0 < kappa0 < kappaf");
  }
  for (int i = 0; i < n; ++i) {
    if (ndims[i] != 2 && ndims[i] != 3) return bfail(nullptr, RVE_ERR_ARG, "ndim must be 2 or 3");
    if (!phase_ids_dev[i]) return bfail(nullptr, RVE_ERR_ARG, "NULL phase ids");
    for (int a = 0; a < ndims[i]; ++a)
      if (!five_smooth_even(dims[3 * i + a]))
        return bfail(nullptr, RVE_ERR_ARG, "every dim must be even, in [2, 1024], with prime factors 2, 3, 5 only");
  }
  rve_batch_ctx* c = new (std::nothrow) rve_batch_ctx();
  if (!c) return bfail(nullptr, RVE_ERR_OOM, "host allocation failed");
  c->n = n;
  c->st = static_cast<cudaStream_t>(stream);
  if (opts) c->opts = *opts;
  else rve_default_opts(&c->opts);
  if (c->opts.precision != 32) {
    delete c;
    return bfail(nullptr, RVE_ERR_ARG, "batched solver supports precision 32 only");
  }
  if (c->opts.hessian != 0 && c->opts.hessian != 1) {
    delete c;
    return bfail(nullptr, RVE_ERR_ARG, "hessian must be 0 (secant) or 1 (symmetric consistent)");
  }
  if (c->opts.element != 0) {
    delete c;
    return bfail(nullptr, RVE_ERR_ARG, "batched solver supports element 0 only");
  }
  rve_status s = batch_init(c, dims, ndims, phase_ids_dev, phases, nphase);
  if (s != RVE_OK) {
    g_batch_create_error = c->err;
    batch_free(c);
    return s;
  }
  *out = c;
  return RVE_OK;
}

rve_status rve_batch_solve_step(rve_batch_t c, const double* dE, const uint8_t* free_mask, rve_step_report* reps) {
  if (!c) return RVE_ERR_ARG;
  if (!dE || !reps) return bfail(c, RVE_ERR_ARG, "NULL argument");
  if (free_mask) {
    for (int i = 0; i < c->n; ++i) {
      unsigned bits = 0;
      for (int q = 0; q < c->g[i].ncomp; ++q)
        if (free_mask[6 * i + q]) bits |= 1u << q;
      c->desc[i].free_mask = bits;
    }
    BCK(cudaMemcpyAsync(c->dD, c->desc.data(), c->n * sizeof(BDesc), cudaMemcpyHostToDevice, c->st), "masks");
    BCK(cudaStreamSynchronize(c->st), "synchronize");
  }
  return batch_solve(c, dE, reps);
}

rve_status rve_batch_hessp(rve_batch_t c, const float* const* v_dev, float* const* out_dev) {
  if (!c) return RVE_ERR_ARG;
  if (!v_dev || !out_dev) return bfail(c, RVE_ERR_ARG, "NULL argument");
  for (int i = 0; i < c->n; ++i) {
    const size_t b = (size_t)c->g[i].ncomp * c->g[i].nvox * sizeof(R);
    BCK(cudaMemcpyAsync(c->d + c->desc[i].foff, v_dev[i], b, cudaMemcpyDeviceToDevice, c->st), "input copy");
  }
  std::vector<char> all(c->n, 1);
  BCK(reset_counters(c), "memset");
  BCK(batch_apply(c, c->d, c->Hd, true, nullptr, 0, gate_bits(all)), "hessp");
  c->hv += c->n;
  for (int i = 0; i < c->n; ++i) {
    const size_t b = (size_t)c->g[i].ncomp * c->g[i].nvox * sizeof(R);
    BCK(cudaMemcpyAsync(out_dev[i], c->Hd + c->desc[i].foff, b, cudaMemcpyDeviceToDevice, c->st), "output copy");
  }
  return RVE_OK;
}

rve_status rve_batch_set_schedule(rve_batch_t c, const int* schedule_host) {
  if (!c) return RVE_ERR_ARG;
  if (!schedule_host) return bfail(c, RVE_ERR_ARG, "NULL schedule");
  for (int k = 0; k < 3; ++k)
    if (schedule_host[k] != 1 && schedule_host[k] != 2 && schedule_host[k] != 4)
      return bfail(c, RVE_ERR_ARG, "tile divisors must be 1, 2 or 4");
  if (schedule_host[3] != 0 && schedule_host[3] != 1) return bfail(c, RVE_ERR_ARG, "radix order flag must be 0 or 1");
  return apply_schedule(c, schedule_host);
}

rve_status rve_batch_autotune(rve_batch_t c, int reps, double* base_ms_host, double* best_ms_host,
                              int* schedule_host) {
  if (!c) return RVE_ERR_ARG;
  if (reps < 1 || reps > 1000) return bfail(c, RVE_ERR_ARG, "reps must be in [1, 1000]");
  // the CG scratch vectors d (zeroed) and Hd carry the timed products
  BCK(cudaMemsetAsync(c->d, 0, (size_t)c->nfield * sizeof(R), c->st), "memset");
  int best[4] = {1, 1, 1, 0};
  rve_status s = apply_schedule(c, best);
  if (s != RVE_OK) return s;
  double tbest = 0;
  if ((s = time_products(c, reps, &tbest)) != RVE_OK) return s;
  if (base_ms_host) *base_ms_host = tbest;
  // coordinate search: tile divisors 2 and 4 per pass, then the radix order;
  // a candidate must beat the incumbent by 2 % to replace it
  for (int axis = 0; axis < 4; ++axis) {
    const int cands[2] = {axis < 3 ? 2 : 1, axis < 3 ? 4 : 0};
    for (int v : cands) {
      if (axis == 3 && v == 0) continue;
      int cand[4] = {best[0], best[1], best[2], best[3]};
      cand[axis] = v;
      if ((s = apply_schedule(c, cand)) != RVE_OK) return s;
      double t = 0;
      if ((s = time_products(c, reps, &t)) != RVE_OK) return s;
      if (t < 0.98 * tbest) {
        tbest = t;
        for (int k = 0; k < 4; ++k) best[k] = cand[k];
      }
    }
  }
  if ((s = apply_schedule(c, best)) != RVE_OK) return s;
  if (best_ms_host) *best_ms_host = tbest;
  if (schedule_host)
    for (int k = 0; k < 4; ++k) schedule_host[k] = best[k];
  return RVE_OK;
}

rve_status rve_batch_set_damage(rve_batch_t c, int i, const float* damage_dev) {
  if (!c) return RVE_ERR_ARG;
  if (i < 0 || i >= c->n || !damage_dev) return bfail(c, RVE_ERR_ARG, "bad member or NULL");
  BCK(cudaMemcpyAsync(c->D + c->desc[i].voff, damage_dev, c->g[i].nvox * sizeof(R), cudaMemcpyDeviceToDevice,
                      c->st),
      "damage copy");
  return RVE_OK;
}

rve_status rve_batch_get_state(rve_batch_t c, int i, float* strain_dev, float* kappa_dev, float* stress_dev,
                               float* damage_dev) {
  if (!c) return RVE_ERR_ARG;
  if (i < 0 || i >= c->n) return bfail(c, RVE_ERR_ARG, "bad member");
  const size_t fb = (size_t)c->g[i].ncomp * c->g[i].nvox * sizeof(R), vb = c->g[i].nvox * sizeof(R);
  if (strain_dev)
    BCK(cudaMemcpyAsync(strain_dev, c->eps + c->desc[i].foff, fb, cudaMemcpyDeviceToDevice, c->st), "copy");
  if (stress_dev)
    BCK(cudaMemcpyAsync(stress_dev, c->sig + c->desc[i].foff, fb, cudaMemcpyDeviceToDevice, c->st), "copy");
  if (kappa_dev)
    BCK(cudaMemcpyAsync(kappa_dev, c->khist + c->desc[i].voff, vb, cudaMemcpyDeviceToDevice, c->st), "copy");
  if (damage_dev)
    BCK(cudaMemcpyAsync(damage_dev, c->D + c->desc[i].voff, vb, cudaMemcpyDeviceToDevice, c->st), "copy");
  return RVE_OK;
}

rve_status rve_batch_reset(rve_batch_t c) {
  if (!c) return RVE_ERR_ARG;
  BCK(cudaMemsetAsync(c->eps, 0, (size_t)c->nfield * sizeof(R), c->st), "memset");
  BCK(cudaMemsetAsync(c->khist, 0, (size_t)c->nvox * sizeof(R), c->st), "memset");
  std::vector<char> all(c->n, 1);
  BCK(reset_counters(c), "memset");
  BCK(trial(c, gate_bits(all), nullptr, false), "state stress");
  return batch_refresh_hessian(c);
}

const char* rve_batch_last_error(rve_batch_t c) { return c ? c->err.c_str() : g_batch_create_error.c_str(); }
long long rve_batch_hv_count(rve_batch_t c) { return c ? c->hv : 0; }
long long rve_batch_launch_count(rve_batch_t c) { return c ? c->launches : 0; }
void rve_batch_destroy(rve_batch_t c) { batch_free(c); }

}  // extern "C"
