// Vector kernels of the L-BFGS load step (quasi-Newton alternative to the
// trust-region Newton-CG solver, with the first-order incremental energy of
// Eq. (18) in its line search).  The direction d = -H g uses the compact
// representation of the L-BFGS inverse Hessian (Byrd, Nocedal & Schnabel
// 1994, Thm. 2.2; Nocedal & Wright Sec. 7.2), which gives the same H as the
// two-loop recursion of N&W Alg. 7.4 but needs two streams over the pair
// fields instead of 2k + 1:
//   pass A  a = S^T g, c = Y^T g (and, after a new pair n, S^T y_n, Y^T y_n)
//   one thread  u = R^-1 a,  p = R^-T ((D + gamma Y^T Y) u - gamma c)
//   pass C  d = -gamma g - S p + gamma Y u
// with R the upper triangle of S^T Y and D its diagonal (pairs oldest
// first).  Every pass streams fields of ncomp * Nvox reals (a multiple of 4)
// and leaves per-block FP64 partial sums for reduce_partials.
#pragma once

#include "common.cuh"

namespace rve {

constexpr int kLbMaxMemory = 16;
constexpr int kLbGroup = 8;  // pairs per stream of passes A and C

// Device scalars of one L-BFGS context.
struct LbScalars {
  double gsum[2][4 * kLbGroup];                 // pass A sums per group: a, c, e, f
  double SY[kLbMaxMemory][kLbMaxMemory];        // s_i . y_j, by slot
  double YY[kLbMaxMemory][kLbMaxMemory];        // y_i . y_j, by slot
  double cS[kLbMaxMemory], cY[kLbMaxMemory];    // coefficients of pass C, by ring position
  double sy, yy;                                // newest pair (pair kernel)
};

// Ring of stored pairs, oldest first, as seen by one launch.
template <typename R>
struct LbRing {
  int k;                       // pairs stored
  int slot[kLbMaxMemory];      // slot of ring position j
  const R* s[kLbMaxMemory];    // fields by ring position
  const R* y[kLbMaxMemory];
};

// d = -H g (compact representation): passes A, the coefficient thread and
// pass C.  new_pair: a pair entered the ring (at position k-1) since the
// last call, so its dot products with the ring are formed in pass A.
template <typename R>
cudaError_t lb_direction(long long n, const R* g, const LbRing<R>& ring, bool new_pair, double gamma, R* d,
                         LbScalars* L, double* part, cudaStream_t st, long long* nl);

// dst = c * src.
template <typename R>
cudaError_t lb_scale(long long n, const R* src, R* dst, double c, cudaStream_t st, long long* nl);

// Pair update after an accepted step s: gnew holds G:sigma at the new state;
// y = gnew - g, g = gnew, gnew <- y; L->sy = s . y, L->yy = y . y.
template <typename R>
cudaError_t lb_pair(long long n, const R* s, R* g, R* gnew, LbScalars* L, double* part, cudaStream_t st,
                    long long* nl);

}  // namespace rve
