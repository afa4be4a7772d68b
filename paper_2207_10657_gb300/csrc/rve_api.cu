// C ABI: context management, the Hessian-vector product entry points and
// the trust-region Newton / Steihaug-CG load step (Algorithms 1 and 2).
// The control loop runs on the host; every arithmetic step (fields and
// FP64 scalars) runs in the kernels of hv_passes.cu and solver_kernels.cu,
// and the host only reads back the small scalar block to branch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rve.h"
#include "consistent.cuh"
#include "homogenize.cuh"
#include "hv_passes.cuh"
#include "lbfgs.cuh"
#include "solver_kernels.cuh"

using namespace rve;

namespace {

thread_local std::string g_create_error = "no error";

__global__ void k_set_cg_params(DevScalars* S, double R, double eta_cg, double thr, int max_cg, double eta_up,
                                double Rmax) {
  S->R = R;
  S->tol = eta_cg * sqrt(S->gg);
  S->thr = thr;
  S->max_cg = max_cg;
  S->eta_up = eta_up;
  S->Rmax = Rmax;
}

__global__ void k_energy_s(DevScalars* S) {
  S->dm = S->sp + 0.5 * S->pBp;
  S->dW = 0.5 * (S->sp + S->stp);
}

template <typename R>
struct Impl {
  SpecWork<R> sw;
  MatTable<R> mt;
  EigTable<R> eg{};
  uint8_t* phase = nullptr;
  R *eps = nullptr, *sig = nullptr, *sig_t = nullptr, *g = nullptr, *z = nullptr, *r = nullptr, *d = nullptr,
    *Hd = nullptr, *tmp = nullptr;
  R *D = nullptr, *D_t = nullptr, *kap = nullptr, *kap_t = nullptr, *khist = nullptr;
  // symmetric consistent tangent of the state (opts.hessian = 1 only)
  R *cdp = nullptr, *ca = nullptr, *cn = nullptr;
  DevScalars* S = nullptr;
  // L-BFGS pairs (allocated at the first L-BFGS step; lb_mem of each)
  int lb_mem = 0;
  R* lbS[kLbMaxMemory] = {};
  R* lbY[kLbMaxMemory] = {};
  LbScalars* L = nullptr;
  LbScalars* Lh = nullptr;  // pinned host mirror
};

bool five_smooth_even(int n) {
  if (n < 2 || n > 1024 || (n & 1)) return false;
  int m = n;
  for (int p : {2, 3, 5})
    while (m % p == 0) m /= p;
  return m == 1;
}

}  // namespace

// One instantiated graph of the device-side Steihaug loop (see
// steihaug_graph) and what it was captured with.
struct CgGraph {
  cudaGraphExec_t exec = nullptr;
  const void* D = nullptr;    // damage field of the products
  const void* cdp = nullptr;  // consistent-tangent data (NULL: secant)
  unsigned free_mask = 0;
  long long per_iter = 0;     // kernel launches per iteration
  long long used = 0;         // last use, for replacement
};
constexpr int kCgGraphs = 4;

struct rve_ctx {
  int precision = 32;
  GridDesc g{};   // strain points (voxels, or the triangles of every pixel): the pointwise kernels
  GridDesc gs{};  // the spectral passes (voxels, with nq lines per Mandel component)
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;  // private stream the Steihaug graphs are captured on
  CgGraph cg_graph[kCgGraphs];
  long long cg_graph_clock = 0;
  bool cg_graph_ok = true;     // false after a graph could not be built: host-driven loop
  bool device_loop = true;     // rve_set_device_loop
  long long host_syncs = 0;    // stream synchronisations that read device scalars
  std::string err = "no error";
  long long hv = 0, launches = 0;
  rve_solver_opts opts{};
  bool radius_set = false;
  double R = 0.0, Rmax = 0.0;
  unsigned free_mask = 0;
  DevScalars* Sh = nullptr;  // pinned host mirror
  PassTimer timer;
  void* impl = nullptr;
};

namespace {

rve_status fail(rve_ctx* c, rve_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

rve_status cuda_fail(rve_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? RVE_ERR_OOM : RVE_ERR_CUDA, m);
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return cuda_fail(c, e__, where); \
  } while (0)

template <typename R>
Impl<R>* impl_of(rve_ctx* c) {
  return static_cast<Impl<R>*>(c->impl);
}

template <typename R>
void impl_free(Impl<R>* m) {
  if (!m) return;
  spectral_free(m->sw);
  void* ptrs[] = {m->phase, m->eps, m->sig, m->sig_t, m->g, m->z, m->r, m->d, m->Hd, m->tmp,
                  m->D, m->D_t, m->kap, m->kap_t, m->khist, m->cdp, m->ca, m->cn, m->S};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < kLbMaxMemory; ++i) {
    if (m->lbS[i]) cudaFree(m->lbS[i]);
    if (m->lbY[i]) cudaFree(m->lbY[i]);
  }
  if (m->L) cudaFree(m->L);
  if (m->Lh) cudaFreeHost(m->Lh);
  delete m;
}

template <typename R>
rve_status read_scalars(rve_ctx* c) {
  Impl<R>* m = impl_of<R>(c);
  CK(cudaMemcpyAsync(c->Sh, m->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->st), "read scalars");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  ++c->host_syncs;
  if (c->Sh->wait_err) return fail(c, RVE_ERR_TIMEOUT, "a pass's bulk copies did not arrive within the wait limit");
  return RVE_OK;
}

// With the consistent Hessian, refresh its per-voxel data from the state
// (strain eps, committed history); a no-op with the secant.
template <typename R>
cudaError_t refresh_hessian(rve_ctx* c) {
  Impl<R>* m = impl_of<R>(c);
  if (!m->cdp) return cudaSuccess;
  return cons_prep<R>(c->g, m->mt, m->eg, m->phase, m->eps, m->khist, m->cdp, m->ca, m->cn, c->st, &c->launches);
}

template <typename R>
rve_status create_impl(rve_ctx* c, const uint8_t* phase_ids, const rve_phase* phases, int nphase) {
  Impl<R>* m = new (std::nothrow) Impl<R>();
  if (!m) return fail(c, RVE_ERR_OOM, "host allocation failed");
  c->impl = m;
  const GridDesc& g = c->g;
  m->mt.nphase = nphase;
  for (int i = 0; i < kMaxPhases; ++i) {
    m->mt.lam[i] = m->mt.mu[i] = 0;
    m->mt.kappa0[i] = m->mt.kappaf[i] = 0;
    m->mt.damaging[i] = 0;
  }
  for (int i = 0; i < nphase; ++i) {
    const double E = phases[i].E, nu = phases[i].nu;
    m->mt.lam[i] = (R)(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
    m->mt.mu[i] = (R)(E / (2.0 * (1.0 + nu)));
    m->mt.damaging[i] = phases[i].damaging ? 1 : 0;
    m->mt.kappa0[i] = (R)phases[i].kappa0;
    m->mt.kappaf[i] = (R)phases[i].kappaf;
  }
  CK(spectral_setup<R>(c->gs, m->sw), "spectral setup");
  m->sw.timer = &c->timer;
  // the compiled passes carry up to six lines per voxel: the 36 of the
  // Kuhn tetrahedra run on the generic passes
  m->sw.generic = c->opts.passes == 1 || c->gs.ncomp > 6;
  m->sw.unfused = c->opts.passes == 2;
  m->sw.cluster = c->opts.passes == 3;
  const size_t nf = (size_t)g.ncomp * g.nvox * sizeof(R);
  const size_t ns = (size_t)g.nvox * sizeof(R);
  R** fields[] = {&m->eps, &m->sig, &m->sig_t, &m->g, &m->z, &m->r, &m->d, &m->Hd, &m->tmp};
  for (R** f : fields) CK(cudaMalloc(f, nf), "field allocation");
  R** sf[] = {&m->D, &m->D_t, &m->kap, &m->kap_t, &m->khist};
  for (R** f : sf) CK(cudaMalloc(f, ns), "scalar-field allocation");
  if (c->opts.hessian == 1) {
    CK(cudaMalloc(&m->cdp, ns), "consistent-tangent allocation");
    CK(cudaMalloc(&m->ca, nf), "consistent-tangent allocation");
    CK(cudaMalloc(&m->cn, nf), "consistent-tangent allocation");
    m->sw.cons = ConsTan<R>{m->cdp, m->ca, m->cn};
  }
  // one phase id per strain point: the voxel's id, repeated for each of its
  // triangles (point q * Nvox + v)
  const long long nv = c->gs.nvox;
  CK(cudaMalloc(&m->phase, g.nvox), "phase allocation");
  CK(cudaMalloc(&m->S, sizeof(DevScalars)), "scalar allocation");
  m->sw.wait_err = &m->S->wait_err;
  CK(cudaMemsetAsync(m->S, 0, sizeof(DevScalars), c->st), "memset");
  for (int q = 0; q < c->gs.nq; ++q)
    CK(cudaMemcpyAsync(m->phase + q * nv, phase_ids, nv, cudaMemcpyDeviceToDevice, c->st), "phase copy");
  // validate ids once
  std::vector<uint8_t> ids(nv);
  CK(cudaMemcpyAsync(ids.data(), m->phase, nv, cudaMemcpyDeviceToHost, c->st), "phase check copy");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  for (long long i = 0; i < nv; ++i)
    if (ids[i] >= nphase) return fail(c, RVE_ERR_ARG, "phase id out of range at voxel " + std::to_string(i));
  CK(cudaMemsetAsync(m->eps, 0, nf, c->st), "memset");
  CK(cudaMemsetAsync(m->khist, 0, ns, c->st), "memset");
  CK(cudaMemsetAsync(m->kap, 0, ns, c->st), "memset");
  // state eps = 0: sigma = 0, D = 0
  CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, nullptr, m->khist, nullptr, nullptr, m->sig, m->D, m->kap, m->S,
                   m->sw.partials, c->st, &c->launches),
     "initial state");
  CK(refresh_hessian<R>(c), "consistent tangent");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  return RVE_OK;
}

// One iteration of Algorithm 1 after the direction d is known: the product
// H d with the step length and the iterate / residual update (fused into
// the compiled FP32 passes, else the generic product, step length and
// update kernels), the residual scalars and the next direction.
template <typename R>
cudaError_t issue_cg_iteration(rve_ctx* c, cudaStream_t st, long long* nl) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  cudaError_t e = cudaErrorNotSupported;
  if constexpr (std::is_same<R, float>::value) {
    e = spectral_hv_cg(c->gs, m->sw, m->mt, m->d, m->phase, m->D, m->z, m->r, m->S, st, nl);
  }
  if (e == cudaErrorNotSupported) {
    e = spectral_apply<R>(c->gs, m->sw, m->mt, m->d, m->phase, m->D, XIn::Tangent, m->Hd, m->d, &m->S->dHd, st, nl);
    if (e == cudaSuccess) e = cg_alpha(m->S, st, nl);
    if (e == cudaSuccess) {
      PassScope ps(&c->timer, st, PASS_CGVEC);
      e = cg_update<R>(g, m->z, m->r, m->d, m->Hd, m->S, m->sw.partials, st, nl);
    }
    if (e == cudaSuccess) e = cg_beta(m->S, st, nl);
  }
  if (e == cudaSuccess) {
    PassScope ps(&c->timer, st, PASS_CGVEC);
    e = cg_dupdate<R>(g, m->z, m->r, m->d, m->S, m->sw.partials, st, nl);
  }
  return e;
}

// The loop condition of the device-side Steihaug loop: continue while the
// iteration runs and no restart (Eq. (20)) is pending.
__global__ void k_cg_cond(cudaGraphConditionalHandle h, const DevScalars* S) {
  cudaGraphSetConditional(h, (S->status == CG_RUN && !S->restart) ? 1u : 0u);
}

// Capture Algorithm 1's iteration as the body of a graph WHILE node.
template <typename R>
cudaError_t build_cg_graph(rve_ctx* c, CgGraph* out) {
  Impl<R>* m = impl_of<R>(c);
  cudaError_t e;
  if (!c->cap && (e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
  long long nl = 0;
  if (e == cudaSuccess) {
    cudaGraph_t body = p.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      e = issue_cg_iteration<R>(c, c->cap, &nl);
      if (e == cudaSuccess) {
        k_cg_cond<<<1, 1, 0, c->cap>>>(h, m->S);
        e = cudaGetLastError();
        ++nl;
      }
      cudaGraph_t got = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(c->cap, &got);
      if (e == cudaSuccess) e = e2;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&out->exec, g, 0);
  cudaGraphDestroy(g);
  out->per_iter = nl;
  return e;
}

// The graph for the current product operands (damage field, consistent
// tangent, mixed-control mask), built on first use and kept.
template <typename R>
CgGraph* cg_graph_for(rve_ctx* c) {
  Impl<R>* m = impl_of<R>(c);
  ++c->cg_graph_clock;
  CgGraph* victim = &c->cg_graph[0];
  for (CgGraph& gr : c->cg_graph) {
    if (gr.exec && gr.D == m->D && gr.cdp == m->sw.cons.dp && gr.free_mask == m->sw.free_mask) {
      gr.used = c->cg_graph_clock;
      return &gr;
    }
    if (!gr.exec || gr.used < victim->used) victim = &gr;
  }
  if (victim->exec) cudaGraphExecDestroy(victim->exec);
  *victim = CgGraph{};
  if (build_cg_graph<R>(c, victim) != cudaSuccess) {
    if (victim->exec) cudaGraphExecDestroy(victim->exec);
    *victim = CgGraph{};
    cudaGetLastError();  // the failed build leaves no pending error behind
    c->cg_graph_ok = false;
    return nullptr;
  }
  victim->D = m->D;
  victim->cdp = m->sw.cons.dp;
  victim->free_mask = m->sw.free_mask;
  victim->used = c->cg_graph_clock;
  return victim;
}

// Steihaug CG on H p = -g inside radius S.R (Algorithm 1).  Result in z,
// exit status in S.status.  The iterations run on the device, as a graph
// whose WHILE node repeats the iteration until an exit of Algorithm 1 or a
// restart: the host synchronises once per restart and once at the end
// instead of once per iteration.  With per-pass timing on (events cannot be
// recorded inside a conditional body), or if the graph cannot be built,
// the host drives the same iteration one launch sequence at a time.
template <typename R>
rve_status steihaug(rve_ctx* c, rve_step_report* rep) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  long long* nl = &c->launches;
  k_set_cg_params<<<1, 1, 0, c->st>>>(m->S, c->R, c->opts.eta_cg, c->opts.restart_thr, c->opts.max_cg,
                                      c->opts.eta_up, c->Rmax);
  ++*nl;
  CK(cg_init<R>(g, m->g, m->z, m->r, m->d, m->S, m->sw.partials, c->st, nl), "cg init");
  rve_status s = read_scalars<R>(c);
  if (s != RVE_OK) return s;
  if (c->Sh->status == CG_NONFINITE) return fail(c, RVE_ERR_NONFINITE, "non-finite gradient in CG");
  if (c->Sh->status != CG_RUN) return RVE_OK;
  CgGraph* gr = (c->device_loop && c->cg_graph_ok && !c->timer.on) ? cg_graph_for<R>(c) : nullptr;
  for (;;) {
    const int it0 = c->Sh->iters;
    if (gr) {
      CK(cudaGraphLaunch(gr->exec, c->st), "graph launch");
    } else {
      CK(issue_cg_iteration<R>(c, c->st, nl), "cg iteration");
    }
    if ((s = read_scalars<R>(c)) != RVE_OK) return s;
    const int done = c->Sh->iters - it0;
    c->hv += done;
    if (gr) c->launches += 1 + done * gr->per_iter;
    if (rep) rep->hv_products += done;
    if (c->Sh->status != CG_RUN) break;
    if (c->Sh->restart) {
      // Eq. (20): r = H z + g, beta = 0, then the direction
      CK(spectral_apply<R>(c->gs, m->sw, m->mt, m->z, m->phase, m->D, XIn::Tangent, m->tmp, nullptr, nullptr, c->st,
                           nl),
         "hessp (restart)");
      ++c->hv;
      if (rep) ++rep->hv_products;
      CK(cg_restart<R>(g, m->r, m->tmp, m->g, m->S, m->sw.partials, c->st, nl), "cg restart");
      PassScope ps(&c->timer, c->st, PASS_CGVEC);
      CK(cg_dupdate<R>(g, m->z, m->r, m->d, m->S, m->sw.partials, c->st, nl), "cg direction");
    }
  }
  if (rep) {
    rep->cg_iters += c->Sh->iters;
    rep->restarts += c->Sh->restarts;
  }
  if (c->Sh->status == CG_NONFINITE) return fail(c, RVE_ERR_NONFINITE, "non-finite value in CG");
  return RVE_OK;
}

// gradient g = G : sigma with |g|^2 into S.gg
template <typename R>
rve_status gradient(rve_ctx* c) {
  Impl<R>* m = impl_of<R>(c);
  CK(spectral_apply<R>(c->gs, m->sw, m->mt, m->sig, m->phase, m->D, XIn::Plain, m->g, m->g, &m->S->gg, c->st,
                       &c->launches),
     "gradient");
  return RVE_OK;
}

template <typename R>
rve_status solve_step_impl(rve_ctx* c, const double dE[6], const void* init, rve_step_report* rep) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  long long* nl = &c->launches;
  rve_step_report local{};
  rve_step_report* rp = rep ? rep : &local;
  std::memset(rp, 0, sizeof(*rp));
  if (!c->radius_set) {
    double n2 = 0;
    for (int i = 0; i < g.ncomp; ++i) n2 += dE[i] * dE[i];
    const double def = 10.0 * std::sqrt((double)g.nvox) * std::sqrt(n2);
    c->R = c->opts.R0 > 0 ? c->opts.R0 : def;
    c->Rmax = c->opts.Rmax > 0 ? c->opts.Rmax : std::max(c->R, def);
    if (!(c->R > 0)) c->R = c->Rmax = 1.0;
    c->radius_set = true;
  }
  CK(add_uniform<R>(g, m->eps, dE, c->st, nl), "load increment");
  if (init) {
    CK(spectral_apply<R>(c->gs, m->sw, m->mt, (const R*)init, m->phase, m->D, XIn::Plain, m->tmp, nullptr, nullptr,
                         c->st, nl),
       "warm start projection");
    CK(axpy<R>((long long)g.ncomp * g.nvox, (R)1, m->tmp, m->eps, c->st, nl), "warm start add");
  }
  CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, nullptr, m->khist, nullptr, nullptr, m->sig, m->D, m->kap, m->S,
                   m->sw.partials, c->st, nl),
     "stress");
  CK(refresh_hessian<R>(c), "consistent tangent");
  rve_status s = gradient<R>(c);
  if (s != RVE_OK) return s;
  if ((s = read_scalars<R>(c)) != RVE_OK) return s;
  if (!std::isfinite(c->Sh->gg) || !std::isfinite(c->Sh->sts))
    return fail(c, RVE_ERR_NONFINITE, "non-finite stress or gradient at the start of the load step");
  double rel = c->Sh->sts > 0 ? std::sqrt(c->Sh->gg / c->Sh->sts) : 0.0;
  bool converged = rel <= c->opts.eta_eq;
  while (!converged && rp->nr_iters < c->opts.max_nr) {
    rp->nr_iters++;
    if ((s = steihaug<R>(c, rp)) != RVE_OK) return s;
    {
      PassScope ps(&c->timer, c->st, PASS_TRIAL);
      CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, m->z, m->khist, m->sig, m->D, m->sig_t, m->D_t, m->kap_t,
                       m->S, m->sw.partials, c->st, nl, m->sw.cons),
         "trial stress");
    }
    CK(tr_decide(m->S, c->st, nl), "ratio test");
    if ((s = read_scalars<R>(c)) != RVE_OK) return s;
    if (c->Sh->nonfinite) return fail(c, RVE_ERR_NONFINITE, "non-finite trial state");
    c->R = c->Sh->R;
    if (c->Sh->on_boundary) rp->boundary_hits++;
    if (!c->Sh->accept) {
      rp->rejected++;
      continue;
    }
    const bool on_b = c->Sh->on_boundary;
    const double pp = c->Sh->pp, ee = c->Sh->ee, sts = c->Sh->sts;
    CK(axpy<R>((long long)g.ncomp * g.nvox, (R)1, m->z, m->eps, c->st, nl), "accept step");
    std::swap(m->sig, m->sig_t);
    std::swap(m->D, m->D_t);
    std::swap(m->kap, m->kap_t);
    CK(refresh_hessian<R>(c), "consistent tangent");
    if ((s = gradient<R>(c)) != RVE_OK) return s;
    if ((s = read_scalars<R>(c)) != RVE_OK) return s;
    rel = sts > 0 ? std::sqrt(c->Sh->gg / sts) : 0.0;
    const double rnr = ee > 0 ? std::sqrt(pp / ee) : 0.0;
    if (!on_b && (rel <= c->opts.eta_eq || (c->opts.eta_nr > 0 && rnr <= c->opts.eta_nr))) converged = true;
  }
  CK(field_means<R>(g, m->sig, m->eps, m->S, m->sw.partials, c->st, nl), "means");
  if ((s = read_scalars<R>(c)) != RVE_OK) return s;
  for (int i = 0; i < 6; ++i) {
    rp->mean_stress[i] = c->Sh->msig[i] / (double)g.nvox;
    rp->mean_strain[i] = c->Sh->meps[i] / (double)g.nvox;
  }
  rp->rel_residual = rel;
  rp->R = c->R;
  rp->converged = converged ? 1 : 0;
  if (!converged) return fail(c, RVE_ERR_NOT_CONVERGED, "load step did not converge within max_nr");
  // commit history: kappa_n <- max(kappa_n, kappa(eps)) (kap already holds the max)
  CK(cudaMemcpyAsync(m->khist, m->kap, (size_t)g.nvox * sizeof(R), cudaMemcpyDeviceToDevice, c->st), "commit");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  return RVE_OK;
}

// ------------------------------------------------------------ L-BFGS
// One load step by L-BFGS with the first-order incremental energy (Eq. (18))
// in a backtracking Armijo line search (Nocedal & Wright Alg. 7.5, the
// direction from the compact representation of the inverse Hessian, equal to
// the two-loop recursion of Alg. 7.4; the paper's remark after Eq. (20)):
// p = -H g; halve the step s = alpha p until
// 1/2 (sigma + sigma(eps + s)) : s <= c1 sigma : s; eps += s; the pair
// (s, y = g_new - g) is kept when s.y > 1e-12 |s| |y|, H0 = gamma I with
// gamma = s.y / y.y of the newest pair (before any pair 1 / max(3 lam + 2 mu)).
// Pairs are kept by pointer swaps: the accepted step (in d) and y (in r)
// become the pair's fields and the evicted ones take over d and r.
constexpr double kLbC1 = 1e-4;
constexpr int kLbMaxBacktrack = 40;

template <typename R>
rve_status lbfgs_alloc(rve_ctx* c, int mem) {
  Impl<R>* m = impl_of<R>(c);
  if (m->lb_mem == mem) return RVE_OK;
  for (int i = 0; i < kLbMaxMemory; ++i) {
    if (m->lbS[i]) cudaFree(m->lbS[i]);
    if (m->lbY[i]) cudaFree(m->lbY[i]);
    m->lbS[i] = m->lbY[i] = nullptr;
  }
  m->lb_mem = 0;
  const size_t nf = (size_t)c->g.ncomp * c->g.nvox * sizeof(R);
  for (int i = 0; i < mem; ++i) {
    CK(cudaMalloc(&m->lbS[i], nf), "L-BFGS pair allocation");
    CK(cudaMalloc(&m->lbY[i], nf), "L-BFGS pair allocation");
  }
  if (!m->L) CK(cudaMalloc(&m->L, sizeof(LbScalars)), "L-BFGS scalar allocation");
  if (!m->Lh) CK(cudaMallocHost(&m->Lh, sizeof(LbScalars)), "L-BFGS pinned allocation");
  m->lb_mem = mem;
  return RVE_OK;
}

template <typename R>
rve_status lbfgs_step_impl(rve_ctx* c, const double dE[6], int mem, int max_iter, rve_step_report* rp) {
  rve_status s = lbfgs_alloc<R>(c, mem);
  if (s != RVE_OK) return s;
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  long long* nl = &c->launches;
  const long long n = (long long)g.ncomp * g.nvox;
  double* part = m->sw.partials;
  std::memset(rp, 0, sizeof(*rp));
  double cmax = 0.0;
  for (int i = 0; i < m->mt.nphase; ++i)
    cmax = std::max(cmax, 3.0 * (double)m->mt.lam[i] + 2.0 * (double)m->mt.mu[i]);
  const double gamma0 = 1.0 / cmax;
  CK(add_uniform<R>(g, m->eps, dE, c->st, nl), "load increment");
  CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, nullptr, m->khist, nullptr, nullptr, m->sig, m->D, m->kap,
                   m->S, part, c->st, nl),
     "stress");
  if ((s = gradient<R>(c)) != RVE_OK) return s;
  if ((s = read_scalars<R>(c)) != RVE_OK) return s;
  if (!std::isfinite(c->Sh->gg) || !std::isfinite(c->Sh->sts))
    return fail(c, RVE_ERR_NONFINITE, "non-finite stress or gradient at the start of the load step");
  double rel = c->Sh->sts > 0 ? std::sqrt(c->Sh->gg / c->Sh->sts) : 0.0;
  std::vector<int> ord;  // pair slots, oldest first
  bool new_pair = false;  // a pair entered since the last direction
  double gamma = gamma0;
  double alpha = 0.0;
  // d = -H g (compact representation of the L-BFGS inverse Hessian)
  auto direction = [&]() -> cudaError_t {
    PassScope ps(&c->timer, c->st, PASS_CGVEC);
    const int k = (int)ord.size();
    if (k == 0) return lb_scale<R>(n, m->g, m->d, -gamma0, c->st, nl);
    LbRing<R> ring{};
    ring.k = k;
    for (int j = 0; j < k; ++j) {
      ring.slot[j] = ord[j];
      ring.s[j] = m->lbS[ord[j]];
      ring.y[j] = m->lbY[ord[j]];
    }
    const cudaError_t e = lb_direction<R>(n, m->g, ring, new_pair, gamma, m->d, m->L, part, c->st, nl);
    new_pair = false;
    return e;
  };
  auto trial = [&]() -> rve_status {
    ++rp->cg_iters;
    {
      PassScope ps(&c->timer, c->st, PASS_TRIAL);
      CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, m->d, m->khist, m->sig, m->D, m->sig_t, m->D_t,
                       m->kap_t, m->S, part, c->st, nl),
         "trial stress");
    }
    rve_status t = read_scalars<R>(c);
    if (t != RVE_OK) return t;
    const DevScalars& h = *c->Sh;
    if (!std::isfinite(h.sp) || !std::isfinite(h.stp) || !std::isfinite(h.sts))
      return fail(c, RVE_ERR_NONFINITE, "non-finite trial state");
    return RVE_OK;
  };
  bool failed = false;
  while (rel > c->opts.eta_eq && rp->nr_iters < max_iter) {
    rp->nr_iters++;
    CK(direction(), "L-BFGS direction");
    alpha = 1.0;
    if ((s = trial()) != RVE_OK) return s;
    if (!(c->Sh->sp < 0.0)) {
      // not a descent direction (rounding at the floor): drop the pairs and
      // take the scaled gradient step
      ord.clear();
      new_pair = false;
      gamma = gamma0;
      rp->boundary_hits++;
      CK(direction(), "L-BFGS direction");
      if ((s = trial()) != RVE_OK) return s;
    }
    bool ok = false;
    for (int b = 0; b <= kLbMaxBacktrack; ++b) {
      const double sp = c->Sh->sp, dW = 0.5 * (sp + c->Sh->stp);
      if (dW <= kLbC1 * sp) {
        ok = true;
        break;
      }
      if (b == kLbMaxBacktrack) break;
      alpha *= 0.5;
      rp->rejected++;
      CK(lb_scale<R>(n, m->d, m->d, 0.5, c->st, nl), "step halving");
      if ((s = trial()) != RVE_OK) return s;
    }
    if (!ok) {
      failed = true;
      break;
    }
    const double pp = c->Sh->pp, sts = c->Sh->sts;
    CK(axpy<R>(n, (R)1, m->d, m->eps, c->st, nl), "accept step");
    std::swap(m->sig, m->sig_t);
    std::swap(m->D, m->D_t);
    std::swap(m->kap, m->kap_t);
    CK(spectral_apply<R>(c->gs, m->sw, m->mt, m->sig, m->phase, m->D, XIn::Plain, m->r, m->r, &m->S->gg, c->st, nl),
       "gradient");
    CK(lb_pair<R>(n, m->d, m->g, m->r, m->L, part, c->st, nl), "pair update");
    CK(cudaMemcpyAsync(m->Lh, m->L, sizeof(LbScalars), cudaMemcpyDeviceToHost, c->st), "read L-BFGS scalars");
    if ((s = read_scalars<R>(c)) != RVE_OK) return s;
    const double sy = m->Lh->sy, yy = m->Lh->yy;
    if (!std::isfinite(sy) || !std::isfinite(yy) || !std::isfinite(c->Sh->gg))
      return fail(c, RVE_ERR_NONFINITE, "non-finite gradient");
    if (sy > 1e-12 * std::sqrt(pp) * std::sqrt(yy)) {
      int slot;
      if ((int)ord.size() < mem) {
        slot = 0;
        while (std::find(ord.begin(), ord.end(), slot) != ord.end()) ++slot;
      } else {
        slot = ord.front();
        ord.erase(ord.begin());
      }
      std::swap(m->lbS[slot], m->d);
      std::swap(m->lbY[slot], m->r);
      gamma = sy / yy;
      ord.push_back(slot);
      new_pair = true;
    } else {
      rp->restarts++;
    }
    rel = sts > 0 ? std::sqrt(c->Sh->gg / sts) : 0.0;
  }
  CK(refresh_hessian<R>(c), "consistent tangent");
  CK(field_means<R>(g, m->sig, m->eps, m->S, part, c->st, nl), "means");
  if ((s = read_scalars<R>(c)) != RVE_OK) return s;
  for (int i = 0; i < 6; ++i) {
    rp->mean_stress[i] = c->Sh->msig[i] / (double)g.nvox;
    rp->mean_strain[i] = c->Sh->meps[i] / (double)g.nvox;
  }
  rp->rel_residual = rel;
  rp->R = alpha;
  const bool converged = !failed && rel <= c->opts.eta_eq;
  rp->converged = converged ? 1 : 0;
  if (!converged)
    return fail(c, RVE_ERR_NOT_CONVERGED,
                failed ? "L-BFGS line search failed" : "L-BFGS load step did not converge within max_iter");
  CK(cudaMemcpyAsync(m->khist, m->kap, (size_t)g.nvox * sizeof(R), cudaMemcpyDeviceToDevice, c->st), "commit");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  return RVE_OK;
}

// ------------------------------------------------------ homogenisation
// Effective secant stiffness at the frozen damage field: for every Mandel
// unit mean strain e_j (all mean components strain-controlled), the
// fluctuation x_j solving G:B:(e_j + x_j) = 0 by Steihaug CG without a
// radius (Algorithm 1 on the Hessian-vector product of Eq. (8)); column j
// is <(1 - D) C : (e_j + x_j)>.
template <typename R>
rve_status stiffness_impl(rve_ctx* c, double tol, int max_cg, double* Cbar, int* cg_total) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  long long* nl = &c->launches;
  // the CG runs under the load-step machinery with its radius, tolerance and
  // mask replaced; everything is put back before returning
  const double R0 = c->R, Rm = c->Rmax;
  const rve_solver_opts opts0 = c->opts;
  const unsigned fm0 = m->sw.free_mask;
  const ConsTan<R> ct0 = m->sw.cons;
  m->sw.cons = ConsTan<R>{};  // the effective stiffness is the secant one
  c->R = c->Rmax = 1e300;
  c->opts.eta_cg = tol;
  c->opts.max_cg = max_cg;
  m->sw.free_mask = 0;
  auto restore = [&]() {
    c->R = R0;
    c->Rmax = Rm;
    c->opts = opts0;
    m->sw.free_mask = fm0;
    m->sw.cons = ct0;
  };
  rve_status s = RVE_OK;
  rve_step_report rep{};
  for (int j = 0; j < g.ncomp && s == RVE_OK; ++j) {
    double e[6] = {0, 0, 0, 0, 0, 0};
    e[j] = 1.0;
    cudaError_t ce = cudaMemsetAsync(m->tmp, 0, (size_t)g.ncomp * g.nvox * sizeof(R), c->st);
    if (ce == cudaSuccess) ce = add_uniform<R>(g, m->tmp, e, c->st, nl);
    if (ce == cudaSuccess)
      ce = spectral_apply<R>(c->gs, m->sw, m->mt, m->tmp, m->phase, m->D, XIn::Tangent, m->g, m->g, &m->S->gg, c->st,
                             nl);
    if (ce != cudaSuccess) {
      s = cuda_fail(c, ce, "stiffness right-hand side");
      break;
    }
    if ((s = steihaug<R>(c, &rep)) != RVE_OK) break;
    const int st = c->Sh->status;
    if (st != CG_CONVERGED && st != CG_ZERO) {
      s = fail(c, RVE_ERR_NOT_CONVERGED, "effective stiffness: CG did not reach the tolerance within max_cg");
      break;
    }
    // z = x_j (zero when the right-hand side vanishes: cg_init clears it)
    ce = add_uniform<R>(g, m->z, e, c->st, nl);
    if (ce == cudaSuccess)
      ce = tangent_sum<R>(g, m->mt, m->phase, m->D, m->z, &m->S->msig[0], m->sw.partials, c->st, nl);
    if (ce != cudaSuccess) {
      s = cuda_fail(c, ce, "stiffness column");
      break;
    }
    if ((s = read_scalars<R>(c)) != RVE_OK) break;
    for (int i = 0; i < g.ncomp; ++i) Cbar[i * g.ncomp + j] = c->Sh->msig[i] / (double)g.nvox;
  }
  if (cg_total) *cg_total = rep.cg_iters;
  restore();
  return s;
}

template <typename R>
rve_status set_state_impl(rve_ctx* c, const void* strain, const void* khist) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  CK(cudaMemcpyAsync(m->eps, strain, (size_t)g.ncomp * g.nvox * sizeof(R), cudaMemcpyDeviceToDevice, c->st),
     "state copy");
  if (khist)
    CK(cudaMemcpyAsync(m->khist, khist, (size_t)g.nvox * sizeof(R), cudaMemcpyDeviceToDevice, c->st),
       "history copy");
  else
    CK(cudaMemsetAsync(m->khist, 0, (size_t)g.nvox * sizeof(R), c->st), "history reset");
  CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, nullptr, m->khist, nullptr, nullptr, m->sig, m->D, m->kap, m->S,
                   m->sw.partials, c->st, &c->launches),
     "state stress");
  CK(refresh_hessian<R>(c), "consistent tangent");
  return RVE_OK;
}

template <typename R>
rve_status set_eig_impl(rve_ctx* c, const double* eig) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  EigTable<R> eg{};
  if (eig)
    for (int i = 0; i < m->mt.nphase; ++i)
      for (int k = 0; k < g.ncomp; ++k) {
        eg.e[i][k] = (R)eig[i * g.ncomp + k];
        if (eig[i * g.ncomp + k] != 0.0) eg.on = 1;
      }
  m->eg = eg;
  CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, nullptr, m->khist, nullptr, nullptr, m->sig, m->D, m->kap,
                   m->S, m->sw.partials, c->st, &c->launches),
     "state stress");
  CK(refresh_hessian<R>(c), "consistent tangent");
  return RVE_OK;
}

template <typename R>
rve_status get_state_impl(rve_ctx* c, void* strain, void* kappa, void* stress, void* damage) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  const size_t nf = (size_t)g.ncomp * g.nvox * sizeof(R), ns = (size_t)g.nvox * sizeof(R);
  if (strain) CK(cudaMemcpyAsync(strain, m->eps, nf, cudaMemcpyDeviceToDevice, c->st), "copy");
  if (stress) CK(cudaMemcpyAsync(stress, m->sig, nf, cudaMemcpyDeviceToDevice, c->st), "copy");
  if (kappa) CK(cudaMemcpyAsync(kappa, m->khist, ns, cudaMemcpyDeviceToDevice, c->st), "copy");
  if (damage) CK(cudaMemcpyAsync(damage, m->D, ns, cudaMemcpyDeviceToDevice, c->st), "copy");
  return RVE_OK;
}

template <typename R>
rve_status energy_grad_impl(rve_ctx* c, const void* p, double* dW, double* dm, void* grad) {
  Impl<R>* m = impl_of<R>(c);
  const GridDesc& g = c->g;
  CK(trial_eval<R>(g, m->mt, m->eg, m->phase, m->eps, (const R*)p, m->khist, m->sig, m->D, m->sig_t, m->D_t, m->kap_t,
                   m->S, m->sw.partials, c->st, &c->launches, m->sw.cons),
     "trial stress");
  k_energy_s<<<1, 1, 0, c->st>>>(m->S);
  ++c->launches;
  if (grad)
    CK(spectral_apply<R>(c->gs, m->sw, m->mt, m->sig_t, m->phase, m->D, XIn::Plain, (R*)grad, nullptr, nullptr, c->st,
                         &c->launches),
       "gradient");
  rve_status s = read_scalars<R>(c);
  if (s != RVE_OK) return s;
  if (dW) *dW = c->Sh->dW;
  if (dm) *dm = c->Sh->dm;
  return RVE_OK;
}

// Algorithm 1 alone at the state: g = G : sigma(state), then Steihaug CG
// with radius Rad and relative tolerance eta_cg; the load-step radius and
// the options are restored afterwards.
template <typename R>
rve_status steihaug_once_impl(rve_ctx* c, double Rad, double eta_cg, void* zout, rve_cg_report* rep) {
  Impl<R>* m = impl_of<R>(c);
  const double R0 = c->R, eta0 = c->opts.eta_cg;
  c->R = Rad;
  c->opts.eta_cg = eta_cg;
  rve_step_report sr{};
  rve_status s = gradient<R>(c);
  if (s == RVE_OK) s = steihaug<R>(c, &sr);
  c->R = R0;
  c->opts.eta_cg = eta0;
  if (s != RVE_OK) return s;
  CK(cudaMemcpyAsync(zout, m->z, (size_t)c->g.ncomp * c->g.nvox * sizeof(R), cudaMemcpyDeviceToDevice, c->st),
     "copy z");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  if (rep) {
    rep->status = c->Sh->status;
    rep->iters = sr.cg_iters;
    rep->hv_products = sr.hv_products;
    rep->restarts = sr.restarts;
  }
  return RVE_OK;
}

template <typename R>
rve_status apply_impl(rve_ctx* c, const void* v, void* out, bool tangent) {
  Impl<R>* m = impl_of<R>(c);
  CK(spectral_apply<R>(c->gs, m->sw, m->mt, (const R*)v, m->phase, m->D, tangent ? XIn::Tangent : XIn::Plain,
                       (R*)out, nullptr, nullptr, c->st, &c->launches),
     tangent ? "hessp" : "project");
  if (tangent) ++c->hv;
  return RVE_OK;
}

}  // namespace

// ============================================================ C ABI
extern "C" {

void rve_default_opts(rve_solver_opts* o) {
  if (!o) return;
  o->eta_eq = 1e-6;
  o->eta_nr = 0.0;
  o->eta_cg = 1e-2;
  o->eta_up = 0.1;
  o->R0 = 0.0;
  o->Rmax = 0.0;
  o->max_nr = 50;
  o->max_cg = 1000;
  o->restart_thr = 0.2;
  o->precision = 32;
  o->hessian = 0;
  o->passes = 0;
  o->element = 0;
}

rve_status rve_create(const int dims[3], int ndim, const uint8_t* phase_ids_dev, const rve_phase* phases, int nphase,
                      const rve_solver_opts* opts, void* stream, rve_t* out) {
  if (!out) return fail(nullptr, RVE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!dims || !phase_ids_dev || !phases) return fail(nullptr, RVE_ERR_ARG, "NULL argument");
  if (ndim != 2 && ndim != 3) return fail(nullptr, RVE_ERR_ARG, "ndim must be 2 or 3");
  for (int a = 0; a < ndim; ++a)
    if (!five_smooth_even(dims[a]))
      return fail(nullptr, RVE_ERR_ARG, "every dim must be even, in [2, 1024], with prime factors 2, 3, 5 only");
  if (nphase < 1 || nphase > kMaxPhases) return fail(nullptr, RVE_ERR_ARG, "nphase must be in [1, 16]");
  for (int i = 0; i < nphase; ++i) {
    const rve_phase& p = phases[i];
    if (!(p.E > 0) || !(p.nu > -1.0 && p.nu < 0.5)) return fail(nullptr, RVE_ERR_ARG, "invalid elastic constants");
    if (p.damaging && !(p.kappa0 > 0 && p.kappaf > p.kappa0))
      return fail(nullptr, RVE_ERR_ARG, "damaging phase needs 0 < kappa0 < kappaf");
  }
  rve_ctx* c = new (std::nothrow) rve_ctx();
  if (!c) return fail(nullptr, RVE_ERR_OOM, "host allocation failed");
  if (opts) c->opts = *opts;
  else rve_default_opts(&c->opts);
  if (c->opts.precision != 32 && c->opts.precision != 64) {
    delete c;
    return fail(nullptr, RVE_ERR_ARG, "precision must be 32 or 64");
  }
  if (c->opts.max_nr < 1 || c->opts.max_cg < 1) {
    delete c;
    return fail(nullptr, RVE_ERR_ARG, "max_nr and max_cg must be >= 1");
  }
  if (c->opts.hessian != 0 && c->opts.hessian != 1) {
    delete c;
    return fail(nullptr, RVE_ERR_ARG, "hessian must be 0 (secant) or 1 (symmetric consistent)");
  }
  if (c->opts.element != 0 && c->opts.element != 1) {
    delete c;
    return fail(nullptr, RVE_ERR_ARG, "element must be 0 (one element per voxel) or 1 (Kuhn simplices)");
  }
  if (c->opts.element == 1 && c->opts.hessian != 0) {
    delete c;
    return fail(nullptr, RVE_ERR_ARG, "element 1 (Kuhn simplices) takes the secant Hessian only");
  }
  if (c->opts.passes < 0 || c->opts.passes > 3) {
    delete c;
    return fail(nullptr, RVE_ERR_ARG,
                "passes must be 0 (compiled, fused CG), 1 (generic), 2 (compiled, unfused CG) or 3 (compiled, "
                "fused CG, cluster x+y passes)");
  }
  c->precision = c->opts.precision;
  c->st = static_cast<cudaStream_t>(stream);
  GridDesc& g = c->g;
  g.ndim = ndim;
  g.nx = dims[0];
  g.ny = dims[1];
  g.nz = ndim == 3 ? dims[2] : 1;
  g.nxh = g.nx / 2 + 1;
  g.ncomp = ndim == 3 ? 6 : 3;
  g.nvox = (long long)g.nx * g.ny * g.nz;
  g.nrows = (long long)g.ny * g.nz;
  c->gs = g;
  if (c->opts.element == 1) {
    // Kuhn simplices: 2 triangles per pixel / 6 tetrahedra per voxel, one
    // strain point each; the spectral passes transform the lines c * nq + q
    // of every voxel (6 in 2D, 36 in 3D)
    const int nq = ndim == 3 ? 6 : 2;
    c->gs.nq = nq;
    c->gs.ncomp = g.ncomp * nq;
    g.nq = nq;
    g.nvox = nq * c->gs.nvox;
    if (ndim == 3) {
      // the generic passes hold a tile of 36 lines: the x passes one row
      // (18 packed line pairs of nx points within 16 per thread), the z
      // pass one column (36 lines of nz points within 24 per thread and the
      // shared-memory cap)
      const size_t csz = (c->opts.precision == 32 ? 8 : 16);
      if (18LL * g.nx > 256LL * 16 || 36LL * g.nz > 512LL * 24 || 36LL * g.nz * csz > 100 * 1024) {
        delete c;
        return fail(nullptr, RVE_ERR_ARG,
                    "element 1 in 3D takes nx <= 227 and nz <= 341 (FP32) / 177 (FP64): the 36 lines of a row or "
                    "a column must fit one block");
      }
    }
  }
  cudaError_t e = cudaMallocHost(&c->Sh, sizeof(DevScalars));
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, RVE_ERR_OOM, "pinned allocation failed");
  }
  rve_status s = c->precision == 32 ? create_impl<float>(c, phase_ids_dev, phases, nphase)
                                    : create_impl<double>(c, phase_ids_dev, phases, nphase);
  if (s != RVE_OK) {
    g_create_error = c->err;
    rve_destroy(c);
    return s;
  }
  *out = c;
  return RVE_OK;
}

#define DISPATCH(c, fn, ...) ((c)->precision == 32 ? fn<float>(c, __VA_ARGS__) : fn<double>(c, __VA_ARGS__))

rve_status rve_set_state(rve_t c, const void* strain, const void* khist) {
  if (!c) return RVE_ERR_ARG;
  if (!strain) return fail(c, RVE_ERR_ARG, "strain is NULL");
  return DISPATCH(c, set_state_impl, strain, khist);
}

rve_status rve_get_state(rve_t c, void* strain, void* kappa, void* stress, void* damage) {
  if (!c) return RVE_ERR_ARG;
  return DISPATCH(c, get_state_impl, strain, kappa, stress, damage);
}

rve_status rve_set_damage(rve_t c, const void* damage) {
  if (!c) return RVE_ERR_ARG;
  if (!damage) return fail(c, RVE_ERR_ARG, "damage is NULL");
  void* D = c->precision == 32 ? (void*)impl_of<float>(c)->D : (void*)impl_of<double>(c)->D;
  const size_t es = c->precision == 32 ? sizeof(float) : sizeof(double);
  CK(cudaMemcpyAsync(D, damage, (size_t)c->g.nvox * es, cudaMemcpyDeviceToDevice, c->st), "damage copy");
  return RVE_OK;
}

rve_status rve_set_eigenstrain(rve_t c, const double* eig, int nphase) {
  if (!c) return RVE_ERR_ARG;
  const int np = c->precision == 32 ? impl_of<float>(c)->mt.nphase : impl_of<double>(c)->mt.nphase;
  if (eig) {
    if (nphase != np) return fail(c, RVE_ERR_ARG, "nphase differs from the context's phase count");
    for (int i = 0; i < nphase * c->g.ncomp; ++i)
      if (!std::isfinite(eig[i])) return fail(c, RVE_ERR_ARG, "non-finite eigenstrain entry");
  }
  return DISPATCH(c, set_eig_impl, eig);
}

rve_status rve_set_free_mask(rve_t c, const uint8_t fm[6]) {
  if (!c) return RVE_ERR_ARG;
  if (!fm) return fail(c, RVE_ERR_ARG, "free_mask is NULL");
  unsigned bits = 0;
  for (int i = 0; i < c->g.ncomp; ++i)
    if (fm[i]) bits |= 1u << i;
  c->free_mask = bits;
  if (c->precision == 32) impl_of<float>(c)->sw.free_mask = bits;
  else impl_of<double>(c)->sw.free_mask = bits;
  return RVE_OK;
}

rve_status rve_hessp(rve_t c, const void* v, void* out) {
  if (!c) return RVE_ERR_ARG;
  if (!v || !out) return fail(c, RVE_ERR_ARG, "NULL field");
  return DISPATCH(c, apply_impl, v, out, true);
}

rve_status rve_project(rve_t c, const void* v, void* out) {
  if (!c) return RVE_ERR_ARG;
  if (!v || !out) return fail(c, RVE_ERR_ARG, "NULL field");
  return DISPATCH(c, apply_impl, v, out, false);
}

rve_status rve_energy_grad(rve_t c, const void* p, double* dW, double* dm, void* grad) {
  if (!c) return RVE_ERR_ARG;
  return DISPATCH(c, energy_grad_impl, p, dW, dm, grad);
}

rve_status rve_solve_step(rve_t c, const double dE[6], const uint8_t fm[6], const void* init, rve_step_report* rep) {
  if (!c) return RVE_ERR_ARG;
  if (!dE) return fail(c, RVE_ERR_ARG, "dE is NULL");
  if (fm) {
    rve_status s = rve_set_free_mask(c, fm);
    if (s != RVE_OK) return s;
  }
  return DISPATCH(c, solve_step_impl, dE, init, rep);
}

rve_status rve_steihaug(rve_t c, double R, double eta_cg, void* z, rve_cg_report* rep) {
  if (!c) return RVE_ERR_ARG;
  if (!z) return fail(c, RVE_ERR_ARG, "z is NULL");
  if (!(R > 0.0) || !std::isfinite(R)) return fail(c, RVE_ERR_ARG, "R must be positive and finite");
  if (!(eta_cg > 0.0 && eta_cg < 1.0)) return fail(c, RVE_ERR_ARG, "eta_cg must be in (0, 1)");
  return DISPATCH(c, steihaug_once_impl, R, eta_cg, z, rep);
}

rve_status rve_solve_step_lbfgs(rve_t c, const double dE[6], const uint8_t fm[6], int memory, int max_iter,
                                rve_step_report* rep) {
  if (!c) return RVE_ERR_ARG;
  if (!dE) return fail(c, RVE_ERR_ARG, "dE is NULL");
  if (memory < 1 || memory > kLbMaxMemory) return fail(c, RVE_ERR_ARG, "memory must be in [1, 16]");
  if (max_iter < 1) return fail(c, RVE_ERR_ARG, "max_iter must be >= 1");
  if (fm) {
    rve_status s = rve_set_free_mask(c, fm);
    if (s != RVE_OK) return s;
  }
  rve_step_report local{};
  return DISPATCH(c, lbfgs_step_impl, dE, memory, max_iter, rep ? rep : &local);
}

rve_status rve_effective_stiffness(rve_t c, double tol, int max_cg, double* Cbar, int* cg_iters) {
  if (!c) return RVE_ERR_ARG;
  if (!Cbar) return fail(c, RVE_ERR_ARG, "Cbar is NULL");
  if (!(tol > 0.0 && tol < 1.0)) return fail(c, RVE_ERR_ARG, "tol must be in (0, 1)");
  if (max_cg < 1) return fail(c, RVE_ERR_ARG, "max_cg must be >= 1");
  return DISPATCH(c, stiffness_impl, tol, max_cg, Cbar, cg_iters);
}

rve_status rve_pass_timing(rve_t c, int enable) {
  if (!c) return RVE_ERR_ARG;
  if (!enable) {
    c->timer.on = false;
    return RVE_OK;
  }
  CK(c->timer.enable(16384), "timer events");
  return RVE_OK;
}

rve_status rve_pass_stats(rve_t c, long long* counts, double* ms, int n) {
  if (!c) return RVE_ERR_ARG;
  if (!counts || !ms || n < 0) return fail(c, RVE_ERR_ARG, "NULL output");
  CK(c->timer.flush(), "timer flush");
  for (int i = 0; i < n; ++i) {
    counts[i] = i < PASS_COUNT ? c->timer.counts[i] : 0;
    ms[i] = i < PASS_COUNT ? c->timer.ms[i] : 0.0;
  }
  return RVE_OK;
}

const char* rve_last_error(rve_t c) { return c ? c->err.c_str() : g_create_error.c_str(); }

long long rve_hv_count(rve_t c) { return c ? c->hv : 0; }
long long rve_launch_count(rve_t c) { return c ? c->launches : 0; }
long long rve_sync_count(rve_t c) { return c ? c->host_syncs : 0; }

rve_status rve_set_device_loop(rve_t c, int enable) {
  if (!c) return RVE_ERR_ARG;
  if (enable != 0 && enable != 1) return fail(c, RVE_ERR_ARG, "enable must be 0 or 1");
  c->device_loop = enable == 1;
  return RVE_OK;
}

void rve_destroy(rve_t c) {
  if (!c) return;
  if (c->impl) {
    if (c->precision == 32) impl_free(impl_of<float>(c));
    else impl_free(impl_of<double>(c));
  }
  if (c->Sh) cudaFreeHost(c->Sh);
  for (CgGraph& gr : c->cg_graph)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  if (c->cap) cudaStreamDestroy(c->cap);
  c->timer.destroy();
  delete c;
}

}  // extern "C"
