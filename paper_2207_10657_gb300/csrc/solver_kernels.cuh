// Pointwise constitutive update, CG vector updates and the device-side
// scalar controller of Steihaug CG / the trust region.
#pragma once

#include "common.cuh"
#include "hv_passes.cuh"

namespace rve {

// Steihaug CG status codes (Algorithm 1 exits).
enum CgStatus : int {
  CG_RUN = 0,
  CG_CONVERGED = 1,
  CG_BOUNDARY = 2,
  CG_NEGCURV = 3,
  CG_MAXITER = 4,
  CG_ZERO = 5,
  CG_NONFINITE = 6,
};

// Device-resident FP64 scalars.  Groups written by one reduction are
// contiguous (reduce_partials writes ns consecutive doubles).
struct DevScalars {
  // parameters
  double R, tol, thr, eta_up, Rmax;
  int max_cg, pad0;
  // CG reductions
  double rr;                    // r.r
  double dHd;                   // d.Hd (fused into the x-inverse pass)
  double dd, zd, rd;            // group D: after the direction update
  double rr_new, rnr, zz_new;   // group U: after the iterate/residual update
  double zz;
  double alpha, beta, tau;
  int status, restart, iters, restarts;
  // trust region (Algorithm 2)
  double sp, stp, pBp, sts, pp, ee;  // group T: trial-state sums
  double gg;                         // |G sigma|^2
  double rho, dm, dW;
  int accept, on_boundary, nonfinite;
  int wait_err;  // set by a kernel whose bounded wait on its copies ran out
  // arrival counters of the reductions done by a launch's last block (d:H:d
  // in the x-forward pass, group D in the direction update)
  unsigned red_cnt[2];
  // homogenised fields (group M: ncomp sums of sigma then ncomp of eps)
  double msig[6], meps[6];
};

// Per-phase eigenstrain (Algorithm 2: the constitutive law is evaluated at
// eps + eps_eig; Sec. 3.3 imposes it on the ASR product sites).  Passed by
// value to the constitutive kernel; `on` is 0 when every entry is zero.
template <typename R>
struct EigTable {
  int on;
  R e[kMaxPhases][6];
};

template <typename R>
struct FieldPtrs {
  GridDesc g;
  const uint8_t* phase;
  MatTable<R> mt;
};

// z = 0, r = g, d = -g; S.rr <- g.g and CG scalars initialised.
template <typename R>
cudaError_t cg_init(const GridDesc& g, const R* gvec, R* z, R* r, R* d, DevScalars* S, double* part,
                    cudaStream_t st, long long* nl);
// alpha / boundary / negative-curvature decision (1 thread).
cudaError_t cg_alpha(DevScalars* S, cudaStream_t st, long long* nl);
// z += alpha d, r += alpha Hd (or z += tau d on an exit); sums group U.
template <typename R>
cudaError_t cg_update(const GridDesc& g, R* z, R* r, const R* d, const R* Hd, DevScalars* S, double* part,
                      cudaStream_t st, long long* nl);
// convergence / restart test and beta (1 thread).
cudaError_t cg_beta(DevScalars* S, cudaStream_t st, long long* nl);
// restart: r = Hz + g, rr recomputed, beta = 0.
template <typename R>
cudaError_t cg_restart(const GridDesc& g, R* r, const R* Hz, const R* gvec, DevScalars* S, double* part,
                       cudaStream_t st, long long* nl);
// d = -r + beta d; sums group D (reduced inside the same launch).
template <typename R>
cudaError_t cg_dupdate(const GridDesc& g, const R* z, const R* r, R* d, DevScalars* S, double* part,
                       cudaStream_t st, long long* nl);

// Trial constitutive evaluation at eps + p (p may be NULL), the material seeing
// eps + p + eps_eig(phase): sigma_t, D_t, kappa_t, and group T sums against the
// stored state (sig0, D0, may be NULL); the strain norm (eps+p):(eps+p) of the
// group excludes the eigenstrain.  p:B0:p uses the state's Hessian: the secant,
// or the symmetric consistent tangent when ct is set.
template <typename R>
cudaError_t trial_eval(const GridDesc& g, const MatTable<R>& mt, const EigTable<R>& eg, const uint8_t* phase,
                       const R* eps, const R* p,
                       const R* khist, const R* sig0, const R* D0, R* sig_t, R* D_t, R* kap_t,
                       DevScalars* S, double* part, cudaStream_t st, long long* nl,
                       const ConsTan<R>& ct = ConsTan<R>{});
// rho_bar, radius update and acceptance (1 thread).
cudaError_t tr_decide(DevScalars* S, cudaStream_t st, long long* nl);
// y += a * x over ncomp * nvox entries (a from the host).
template <typename R>
cudaError_t axpy(long long n, R a, const R* x, R* y, cudaStream_t st, long long* nl);
// eps += dE[c] on component c (uniform increment).
template <typename R>
cudaError_t add_uniform(const GridDesc& g, R* eps, const double dE[6], cudaStream_t st, long long* nl);
// component means of sigma and eps into S.msig / S.meps.
template <typename R>
cudaError_t field_means(const GridDesc& g, const R* sig, const R* eps, DevScalars* S, double* part,
                        cudaStream_t st, long long* nl);
// Mandel <-> precision conversion helpers are not needed: fields are R.

}  // namespace rve
