// Vector kernels of the L-BFGS load step (quasi-Newton alternative to the
// trust-region Newton-CG solver, with the first-order incremental energy of
// Eq. (18) in its line search): the two-loop recursion of Nocedal & Wright
// Alg. 7.4 as fused "update + next dot" passes, step scaling and the pair
// update.  Every pass streams fields of ncomp * Nvox reals (a multiple of 4)
// and leaves per-block FP64 partial sums for reduce_partials.
#pragma once

#include "common.cuh"

namespace rve {

constexpr int kLbMaxMemory = 16;

// Device scalars of one L-BFGS context: a[i] of the first loop, the running
// dot product, s.y and y.y of the newest pair.
struct LbScalars {
  double a[kLbMaxMemory];
  double sum;
  double sy, yy;
};

// sum <- x . y (reduced into L->sum).
template <typename R>
cudaError_t lb_dot(long long n, const R* x, const R* y, LbScalars* L, double* part, cudaStream_t st,
                   long long* nl);

// First loop, pair i: a_i = rho_i * L->sum (stored in L->a[i]);
// q = src - a_i y; L->sum <- w . q (w may be NULL).
template <typename R>
cudaError_t lb_loop1(long long n, const R* src, R* q, const R* y, const R* w, double rho, int i, LbScalars* L,
                     double* part, cudaStream_t st, long long* nl);

// Second loop, pair i: with v = f * src, b = rho_i * f * L->sum (L->sum =
// y_i . src), out = sgn * (v + (a_i - b) s); L->sum <- w . (v + (a_i - b) s)
// (w may be NULL).  f = gamma on the first pair of the loop, 1 after;
// sgn = -1 on the last pair (out is then the search direction).
template <typename R>
cudaError_t lb_loop2(long long n, const R* src, R* out, const R* s, const R* w, double rho, double f, double sgn,
                     int i, LbScalars* L, double* part, cudaStream_t st, long long* nl);

// dst = c * src.
template <typename R>
cudaError_t lb_scale(long long n, const R* src, R* dst, double c, cudaStream_t st, long long* nl);

// Pair update after an accepted step s: gnew holds G:sigma at the new state;
// y = gnew - g, g = gnew, gnew <- y; L->sy = s . y, L->yy = y . y.
template <typename R>
cudaError_t lb_pair(long long n, const R* s, R* g, R* gnew, LbScalars* L, double* part, cudaStream_t st,
                    long long* nl);

}  // namespace rve
