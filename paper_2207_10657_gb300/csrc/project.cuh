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

// Ghat(k) for the 3D Kuhn tetrahedra (every voxel split along its main
// diagonal into the six tetrahedra of the axis permutations pi, in
// lexicographic order of pi; Sec. 2.1 builds the projection from any FE
// gradient).  The 36 lines c * 6 + q -- Mandel component c (11, 22, 33,
// sqrt2*23, sqrt2*13, sqrt2*12) of tetrahedron q -- sit at p[(c * 6 + q) *
// stride].  Tetrahedron pi has vertices v0 = 0, v_j = v_{j-1} + e_{pi_j};
// its derivative symbol along pi_j is e^{i (th_{pi_1} + ... + th_{pi_{j-1}})}
// (e^{i th_{pi_j}} - 1).  As for the triangles: b = B^H m, a = M^-1 b with
// the 3 x 3 Hermitian M = B^H B (non-singular for k != 0), m = B a; at
// k = 0 the free components keep their tetrahedron average and the
// strain-controlled ones vanish.  e[a]: e^{i th_a}; d[a]: e^{i th_a} - 1
// (exact zero at k = 0).
template <typename R>
__device__ __forceinline__ void project_simplex3(Cx<R>* p, const int stride, const Cx<R> (&e)[3],
                                                 const Cx<R> (&d)[3], bool k0, unsigned free_mask) {
  using C = Cx<R>;
  constexpr int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  if (k0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      C avg{0, 0};
      if ((free_mask >> c) & 1u) {
#pragma unroll
        for (int q = 0; q < 6; ++q) avg = cadd(avg, p[(c * 6 + q) * stride]);
        avg = cscale(avg, (R)1 / (R)6);
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) p[(c * 6 + q) * stride] = avg;
    }
    return;
  }
  auto symbol = [&](int q, C (&D)[3]) {
    C pre{1, 0};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int a = kPerm[q][s];
      D[a] = cmul(pre, d[a]);
      pre = cmul(pre, e[a]);
    }
  };
  const R is2 = (R)0.70710678118654752440;
  R m00 = 0, m11 = 0, m22 = 0;
  C m01{0, 0}, m02{0, 0}, m12{0, 0}, b0{0, 0}, b1{0, 0}, b2{0, 0};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    C D[3];
    symbol(q, D);
    const R a0 = D[0].x * D[0].x + D[0].y * D[0].y, a1 = D[1].x * D[1].x + D[1].y * D[1].y,
            a2 = D[2].x * D[2].x + D[2].y * D[2].y;
    m00 += a0 + (R)0.5 * (a1 + a2);
    m11 += a1 + (R)0.5 * (a0 + a2);
    m22 += a2 + (R)0.5 * (a0 + a1);
    m01 = cadd(m01, cscale(cmulc(D[0], D[1]), (R)0.5));  // D0 conj(D1) / 2
    m02 = cadd(m02, cscale(cmulc(D[0], D[2]), (R)0.5));
    m12 = cadd(m12, cscale(cmulc(D[1], D[2]), (R)0.5));
    const C v0 = p[(0 * 6 + q) * stride], v1 = p[(1 * 6 + q) * stride], v2 = p[(2 * 6 + q) * stride];
    const C s3 = cscale(p[(3 * 6 + q) * stride], is2), s4 = cscale(p[(4 * 6 + q) * stride], is2),
            s5 = cscale(p[(5 * 6 + q) * stride], is2);
    b0 = cadd(b0, cadd(cmulc(v0, D[0]), cadd(cmulc(s4, D[2]), cmulc(s5, D[1]))));
    b1 = cadd(b1, cadd(cmulc(v1, D[1]), cadd(cmulc(s3, D[2]), cmulc(s5, D[0]))));
    b2 = cadd(b2, cadd(cmulc(v2, D[2]), cadd(cmulc(s3, D[1]), cmulc(s4, D[0]))));
  }
  // a = M^-1 b through the adjugate (M Hermitian: i10 = conj(i01), ...)
  const R i00 = m11 * m22 - (m12.x * m12.x + m12.y * m12.y);
  const R i11 = m00 * m22 - (m02.x * m02.x + m02.y * m02.y);
  const R i22 = m00 * m11 - (m01.x * m01.x + m01.y * m01.y);
  const C i01 = csub(cmulc(m02, m12), cscale(m01, m22));  // m02 conj(m12) - m01 m22
  const C i02 = csub(cmul(m01, m12), cscale(m02, m11));   // m01 m12 - m02 m11
  const C i12 = csub(cmulc(m02, m01), cscale(m12, m00));  // m02 conj(m01) - m00 m12
  const R det = m00 * i00 + (m01.x * i01.x + m01.y * i01.y) + (m02.x * i02.x + m02.y * i02.y);
  const R inv = (R)1 / det;
  C a[3];
  a[0] = cscale(cadd(cscale(b0, i00), cadd(cmul(i01, b1), cmul(i02, b2))), inv);
  a[1] = cscale(cadd(cmulc(b0, i01), cadd(cscale(b1, i11), cmul(i12, b2))), inv);
  a[2] = cscale(cadd(cmulc(b0, i02), cadd(cmulc(b1, i12), cscale(b2, i22))), inv);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    C D[3];
    symbol(q, D);
    p[(0 * 6 + q) * stride] = cmul(D[0], a[0]);
    p[(1 * 6 + q) * stride] = cmul(D[1], a[1]);
    p[(2 * 6 + q) * stride] = cmul(D[2], a[2]);
    p[(3 * 6 + q) * stride] = cscale(cadd(cmul(D[1], a[2]), cmul(D[2], a[1])), is2);
    p[(4 * 6 + q) * stride] = cscale(cadd(cmul(D[0], a[2]), cmul(D[2], a[0])), is2);
    p[(5 * 6 + q) * stride] = cscale(cadd(cmul(D[0], a[1]), cmul(D[1], a[0])), is2);
  }
}

}  // namespace rve
