// Per-frequency compatibility projection Ghat(k) (Sec. 2.1, Eq. (9)) for
// small strain, in Mandel components.
#pragma once

#include "common.cuh"

namespace rve {

// ------------------------------------------------------------ projection
// Ghat(k) : zeta for one frequency, Mandel components m (complex).
// n = Dhat/|Dhat|, v = zeta n*, s = n*^T zeta n*,
// Ghat:zeta = n (x) v + v (x) n - s n (x) n.  Ghat = 0 where Dhat = 0
// (k != 0); Ghat(0) keeps the stress-controlled (free) components.
template <typename R>
__device__ __forceinline__ void project3(Cx<R> (&m)[6], Cx<R> d0, Cx<R> d1, Cx<R> d2, bool k0,
                                         unsigned free_mask) {
  using C = Cx<R>;
  if (k0) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (!((free_mask >> c) & 1u)) m[c] = C{0, 0};
    return;
  }
  const R n2 = d0.x * d0.x + d0.y * d0.y + d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y;
  if (n2 == (R)0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) m[c] = C{0, 0};
    return;
  }
  const R inv = (R)1 / sqrt(n2);
  const C n[3] = {cscale(d0, inv), cscale(d1, inv), cscale(d2, inv)};
  const R is2 = (R)0.70710678118654752440, s2 = (R)1.41421356237309504880;
  const C t00 = m[0], t11 = m[1], t22 = m[2];
  const C t12 = cscale(m[3], is2), t02 = cscale(m[4], is2), t01 = cscale(m[5], is2);
  // v_i = sum_j T_ij conj(n_j)
  const C v0 = cadd(cadd(cmulc(t00, n[0]), cmulc(t01, n[1])), cmulc(t02, n[2]));
  const C v1 = cadd(cadd(cmulc(t01, n[0]), cmulc(t11, n[1])), cmulc(t12, n[2]));
  const C v2 = cadd(cadd(cmulc(t02, n[0]), cmulc(t12, n[1])), cmulc(t22, n[2]));
  // s = sum_i conj(n_i) v_i
  const C s = cadd(cadd(cmulc(v0, n[0]), cmulc(v1, n[1])), cmulc(v2, n[2]));
  auto o = [&](C ni, C nj, C vi, C vj) { return csub(cadd(cmul(ni, vj), cmul(vi, nj)), cmul(s, cmul(ni, nj))); };
  m[0] = o(n[0], n[0], v0, v0);
  m[1] = o(n[1], n[1], v1, v1);
  m[2] = o(n[2], n[2], v2, v2);
  m[3] = cscale(o(n[1], n[2], v1, v2), s2);
  m[4] = cscale(o(n[0], n[2], v0, v2), s2);
  m[5] = cscale(o(n[0], n[1], v0, v1), s2);
}

template <typename R>
__device__ __forceinline__ void project2(Cx<R> (&m)[3], Cx<R> d0, Cx<R> d1, bool k0, unsigned free_mask) {
  using C = Cx<R>;
  if (k0) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (!((free_mask >> c) & 1u)) m[c] = C{0, 0};
    return;
  }
  const R n2 = d0.x * d0.x + d0.y * d0.y + d1.x * d1.x + d1.y * d1.y;
  if (n2 == (R)0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) m[c] = C{0, 0};
    return;
  }
  const R inv = (R)1 / sqrt(n2);
  const C n0 = cscale(d0, inv), n1 = cscale(d1, inv);
  const R is2 = (R)0.70710678118654752440, s2 = (R)1.41421356237309504880;
  const C t00 = m[0], t11 = m[1], t01 = cscale(m[2], is2);
  const C v0 = cadd(cmulc(t00, n0), cmulc(t01, n1));
  const C v1 = cadd(cmulc(t01, n0), cmulc(t11, n1));
  const C s = cadd(cmulc(v0, n0), cmulc(v1, n1));
  auto o = [&](C ni, C nj, C vi, C vj) { return csub(cadd(cmul(ni, vj), cmul(vi, nj)), cmul(s, cmul(ni, nj))); };
  m[0] = o(n0, n0, v0, v0);
  m[1] = o(n1, n1, v1, v1);
  m[2] = cscale(o(n0, n1, v0, v1), s2);
}

}  // namespace rve
