// Per-frequency compatibility projection Ghat(k) (Sec. 2.1, Eq. (9)) for
// small strain, in Mandel components.
#pragma once

#include "common.cuh"

namespace rve {

// ------------------------------------------------------------ projection
// Ghat(k) : zeta for one frequency, Mandel components m (complex), from the
// unnormalised symbol D = Dhat(k).  With n = D/|D|, v = zeta n* and
// s = n*^T zeta n*, Ghat:zeta = n (x) v + v (x) n - s n (x) n.  Written with
// D itself: v' = zeta D*, s' = D*^T v', w = v' - (s' / (2 |D|^2)) D, and
// Ghat:zeta = (D (x) w + w (x) D) / |D|^2 -- the same operator, one
// reciprocal instead of a normalisation, and two products per output entry
// instead of four.  Ghat = 0 where D = 0 (k != 0); Ghat(0) keeps the
// stress-controlled (free) components.
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
  const R inv = (R)1 / n2;
  const R is2 = (R)0.70710678118654752440, s2 = (R)1.41421356237309504880;
  const C t00 = m[0], t11 = m[1], t22 = m[2];
  const C t12 = cscale(m[3], is2), t02 = cscale(m[4], is2), t01 = cscale(m[5], is2);
  // v_i = sum_j T_ij conj(D_j)
  const C v0 = cadd(cadd(cmulc(t00, d0), cmulc(t01, d1)), cmulc(t02, d2));
  const C v1 = cadd(cadd(cmulc(t01, d0), cmulc(t11, d1)), cmulc(t12, d2));
  const C v2 = cadd(cadd(cmulc(t02, d0), cmulc(t12, d1)), cmulc(t22, d2));
  // s = sum_i conj(D_i) v_i, scaled by -1 / (2 |D|^2)
  const C sh = cscale(cadd(cadd(cmulc(v0, d0), cmulc(v1, d1)), cmulc(v2, d2)), (R)-0.5 * inv);
  const C w0 = cadd(v0, cmul(sh, d0)), w1 = cadd(v1, cmul(sh, d1)), w2 = cadd(v2, cmul(sh, d2));
  const R i2 = (R)2 * inv, is = s2 * inv;
  m[0] = cscale(cmul(d0, w0), i2);
  m[1] = cscale(cmul(d1, w1), i2);
  m[2] = cscale(cmul(d2, w2), i2);
  m[3] = cscale(cadd(cmul(d1, w2), cmul(w1, d2)), is);
  m[4] = cscale(cadd(cmul(d0, w2), cmul(w0, d2)), is);
  m[5] = cscale(cadd(cmul(d0, w1), cmul(w0, d1)), is);
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

// Ghat(k) for the 2D Kuhn-triangle discretisation (every pixel split along
// its main diagonal into two linear triangles, one strain each; Sec. 2.1
// builds the projection from any FE gradient).  m holds the six lines
// c * 2 + q: Mandel component c (11, 22, sqrt2*12) of triangle q.  The
// triangle of axis order (x, y) has derivative symbols Dx0 = e^{i thx} - 1,
// Dy0 = e^{i thx} (e^{i thy} - 1); the one of order (y, x) has
// Dy1 = e^{i thy} - 1, Dx1 = e^{i thy} (e^{i thx} - 1).  The compatible
// strains are B a (a in C^2, B stacking sym(Dq (x) a) over q) and the
// orthogonal projector is B (B^H B)^-1 B^H: b = B^H m, a = M^-1 b with the
// 2 x 2 Hermitian M = B^H B (non-singular for k != 0: linear triangles have
// no zero-energy modes), m = B a.  At k = 0 a compatible field has the same
// mean strain on both triangles: the free components keep the triangle
// average, the strain-controlled ones vanish.  ex, ey: e^{i th}; dx, dy:
// e^{i th} - 1 (exact zero at k = 0).
template <typename R>
__device__ __forceinline__ void project_simplex2(Cx<R> (&m)[6], Cx<R> ex, Cx<R> dx, Cx<R> ey, Cx<R> dy, bool k0,
                                                 unsigned free_mask) {
  using C = Cx<R>;
  if (k0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C avg = ((free_mask >> c) & 1u) ? cscale(cadd(m[2 * c], m[2 * c + 1]), (R)0.5) : C{0, 0};
      m[2 * c] = avg;
      m[2 * c + 1] = avg;
    }
    return;
  }
  const R is2 = (R)0.70710678118654752440;
  const C Dx[2] = {dx, cmul(ey, dx)}, Dy[2] = {cmul(ex, dy), dy};
  C bx{0, 0}, by{0, 0}, mxy{0, 0};
  R mxx = 0, myy = 0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const R ax = Dx[q].x * Dx[q].x + Dx[q].y * Dx[q].y, ay = Dy[q].x * Dy[q].x + Dy[q].y * Dy[q].y;
    mxx += ax + (R)0.5 * ay;
    myy += ay + (R)0.5 * ax;
    mxy = cadd(mxy, cscale(cmulc(Dx[q], Dy[q]), (R)0.5));  // conj(Dy) Dx / 2
    const C s12 = cscale(m[4 + q], is2);
    bx = cadd(bx, cadd(cmulc(m[q], Dx[q]), cmulc(s12, Dy[q])));
    by = cadd(by, cadd(cmulc(m[2 + q], Dy[q]), cmulc(s12, Dx[q])));
  }
  const R det = mxx * myy - (mxy.x * mxy.x + mxy.y * mxy.y);
  const R inv = (R)1 / det;
  // a = M^-1 b with M = [[mxx, mxy], [conj(mxy), myy]]
  const C ax = cscale(csub(cscale(bx, myy), cmul(mxy, by)), inv);
  const C ay = cscale(csub(cscale(by, mxx), cmulc(bx, mxy)), inv);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    m[q] = cmul(Dx[q], ax);
    m[2 + q] = cmul(Dy[q], ay);
    m[4 + q] = cscale(cadd(cmul(Dy[q], ax), cmul(Dx[q], ay)), is2);
  }
}

}  // namespace rve
