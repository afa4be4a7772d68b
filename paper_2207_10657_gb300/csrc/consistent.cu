// Symmetric consistent damage tangent: per-voxel preparation (positive part
// of the strain by cyclic Jacobi rotations, D'(kappa), C : eps).
#include <cmath>

#include "consistent.cuh"

namespace rve {

namespace {

constexpr int kCThreads = 256;
constexpr int kCBlocks = 152 * 4;

// Eigen-decomposition of a symmetric d x d matrix (d = 2 or 3) by cyclic
// Jacobi rotations: on return the diagonal of A holds the eigenvalues and
// the columns of V the eigenvectors.  Each rotation in the (p, q) plane
// zeroes A[p][q]; a few sweeps reach rounding level for d <= 3.
template <typename R, int d>
__device__ void jacobi_eig(R (&A)[3][3], R (&V)[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? (R)1 : (R)0;
  for (int sweep = 0; sweep < 8; ++sweep) {
    R off = 0, diag = 0;
    for (int p = 0; p < d; ++p) {
      diag += A[p][p] * A[p][p];
      for (int q = p + 1; q < d; ++q) off += A[p][q] * A[p][q];
    }
    if (off == (R)0 || off <= (R)1e-36 * diag) break;
    for (int p = 0; p < d - 1; ++p)
      for (int q = p + 1; q < d; ++q) {
        const R apq = A[p][q];
        if (apq == (R)0) continue;
        const R theta = (A[q][q] - A[p][p]) / ((R)2 * apq);
        const R t = (theta >= (R)0 ? (R)1 : (R)-1) / (fabs(theta) + sqrt(theta * theta + (R)1));
        const R c = (R)1 / sqrt(t * t + (R)1), s = t * c;
        for (int k = 0; k < d; ++k) {  // A <- A J
          const R akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < d; ++k) {  // A <- J^T A
          const R apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < d; ++k) {  // V <- V J
          const R vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// eps^(t) = sum_i max(eps_i, 0) q_i (x) q_i in Mandel form (plane strain:
// the in-plane 2 x 2 block; its zero out-of-plane eigenvalue adds nothing).
template <typename R, int NC>
__device__ void positive_part(const R (&e)[6], R (&ep)[6]) {
  constexpr int d = NC == 6 ? 3 : 2;
  const R is2 = (R)0.70710678118654752440, s2 = (R)1.41421356237309504880;
  R A[3][3] = {}, V[3][3];
  A[0][0] = e[0];
  A[1][1] = e[1];
  if constexpr (NC == 6) {
    A[2][2] = e[2];
    A[1][2] = A[2][1] = e[3] * is2;
    A[0][2] = A[2][0] = e[4] * is2;
    A[0][1] = A[1][0] = e[5] * is2;
  } else {
    A[0][1] = A[1][0] = e[2] * is2;
  }
  jacobi_eig<R, d>(A, V);
  R T[3][3] = {};
  for (int k = 0; k < d; ++k) {
    const R l = fmax(A[k][k], (R)0);
    if (l == (R)0) continue;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) T[i][j] += l * V[i][k] * V[j][k];
  }
  ep[0] = T[0][0];
  ep[1] = T[1][1];
  if constexpr (NC == 6) {
    ep[2] = T[2][2];
    ep[3] = s2 * T[1][2];
    ep[4] = s2 * T[0][2];
    ep[5] = s2 * T[0][1];
  } else {
    ep[2] = s2 * T[0][1];
  }
}

template <typename R, int NC>
__global__ void __launch_bounds__(kCThreads)
    k_cons_prep(const GridDesc g, const MatTable<R> mt, const EigTable<R> eg, const uint8_t* __restrict__ phase,
                const R* __restrict__ eps, const R* __restrict__ khist, R* __restrict__ dp, R* __restrict__ a,
                R* __restrict__ n) {
  constexpr int nd = NC == 6 ? 3 : 2;
  const long long nv = g.nvox;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    const int ph = phase[v];
    R dpv = 0;
    if (mt.damaging[ph]) {
      R e[6] = {0, 0, 0, 0, 0, 0}, ep[6] = {0, 0, 0, 0, 0, 0};
      for (int c = 0; c < NC; ++c) e[c] = eps[c * nv + v] + (eg.on ? eg.e[ph][c] : (R)0);
      positive_part<R, NC>(e, ep);
      R kt2 = 0;
      for (int c = 0; c < NC; ++c) kt2 += ep[c] * ep[c];
      const R kt = sqrt(kt2), kh = khist[v];
      const R k = kt > kh ? kt : kh, k0 = mt.kappa0[ph], kf = mt.kappaf[ph];
      if (kt > kh && k > k0 && k < kf) {
        dpv = kf * k0 / (k * k * (kf - k0));
        const R lam = mt.lam[ph], mu = mt.mu[ph];
        R tr = 0;
        for (int i = 0; i < nd; ++i) tr += e[i];
        for (int c = 0; c < NC; ++c) {
          a[c * nv + v] = (R)2 * mu * e[c] + (c < nd ? lam * tr : (R)0);
          n[c * nv + v] = ep[c] / kt;
        }
      }
    }
    dp[v] = dpv;
  }
}

}  // namespace

template <typename R>
cudaError_t cons_prep(const GridDesc& g, const MatTable<R>& mt, const EigTable<R>& eg, const uint8_t* phase,
                      const R* eps, const R* khist, R* dp, R* a, R* n, cudaStream_t st, long long* nl) {
  if (g.ncomp == 6) k_cons_prep<R, 6><<<kCBlocks, kCThreads, 0, st>>>(g, mt, eg, phase, eps, khist, dp, a, n);
  else k_cons_prep<R, 3><<<kCBlocks, kCThreads, 0, st>>>(g, mt, eg, phase, eps, khist, dp, a, n);
  ++*nl;
  return cudaGetLastError();
}

template cudaError_t cons_prep<float>(const GridDesc&, const MatTable<float>&, const EigTable<float>&,
                                      const uint8_t*, const float*, const float*, float*, float*, float*,
                                      cudaStream_t, long long*);
template cudaError_t cons_prep<double>(const GridDesc&, const MatTable<double>&, const EigTable<double>&,
                                       const uint8_t*, const double*, const double*, double*, double*, double*,
                                       cudaStream_t, long long*);

}  // namespace rve
