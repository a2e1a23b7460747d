// FP64 recomputation and exact intersection of face pairs (the rare stage).
//
// - tri_dist2_f64: squared distance between two closed faces in double, in a
//   frame at the first vertex of face A, as the minimum over the 6
//   vertex-face and 9 edge-edge feature pairs (Sec. 3.2.2, Eq. 3).
// - tri_isect_exact: whether two closed faces share a point, decided exactly
//   (Sec. 3.2.3, Eq. 4 without the division): each edge of one face against
//   the other face by orientation signs; a segment lying in the face plane is
//   decided in 2D on a coordinate projection that is injective on the plane;
//   a degenerate face is the union of its edges.  Each sign is first taken in
//   double with a forward error bound; when that cannot certify it, the
//   determinant is evaluated exactly with floating-point expansions
//   (two-sum / two-product, grow- and scale-expansion with zero elimination,
//   after Shewchuk 1997, "Adaptive Precision Floating-Point Arithmetic and
//   Fast Robust Geometric Predicates").
// Valid for coordinates 0 or 2^-200 <= |x| <= 2^200 (no underflow/overflow
// of any product).
#pragma once
#include "closest.cuh"
#include "internal.cuh"

namespace g3d {

// ---------------------------------------------------------------------------
// FP64 distance
// ---------------------------------------------------------------------------
__device__ __forceinline__ double d2of64(double3 P, double3 Q) {
  double3 d = P - Q;
  return dot(d, d);
}

__device__ inline double tri_dist2_f64(const double* A, const double* B) {
  double3 a0 = make_double3(0.0, 0.0, 0.0);
  double3 a1 = make_double3(A[3] - A[0], A[4] - A[1], A[5] - A[2]);
  double3 a2 = make_double3(A[6] - A[0], A[7] - A[1], A[8] - A[2]);
  double3 b0 = make_double3(B[0] - A[0], B[1] - A[1], B[2] - A[2]);
  double3 b1 = make_double3(B[3] - A[0], B[4] - A[1], B[5] - A[2]);
  double3 b2 = make_double3(B[6] - A[0], B[7] - A[1], B[8] - A[2]);
  double best = d2of64(a0, closest_on_tri(a0, b0, b1, b2));
  best = fmin(best, d2of64(a1, closest_on_tri(a1, b0, b1, b2)));
  best = fmin(best, d2of64(a2, closest_on_tri(a2, b0, b1, b2)));
  best = fmin(best, d2of64(b0, closest_on_tri(b0, a0, a1, a2)));
  best = fmin(best, d2of64(b1, closest_on_tri(b1, a0, a1, a2)));
  best = fmin(best, d2of64(b2, closest_on_tri(b2, a0, a1, a2)));
  const double3 ea[3][2] = {{a0, a1}, {a1, a2}, {a2, a0}};
  const double3 eb[3][2] = {{b0, b1}, {b1, b2}, {b2, b0}};
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double3 p, q;
      closest_seg_seg(ea[i][0], ea[i][1], eb[j][0], eb[j][1], p, q);
      best = fmin(best, d2of64(p, q));
    }
  return best;
}

// ---------------------------------------------------------------------------
// floating-point expansions (components in increasing magnitude, no zeros)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  double bv = __dsub_rn(x, a);
  double av = __dsub_rn(x, bv);
  double br = __dsub_rn(b, bv);
  double ar = __dsub_rn(a, av);
  y = __dadd_rn(ar, br);
}

__device__ __forceinline__ void two_diff(double a, double b, double& x, double& y) {
  x = __dsub_rn(a, b);
  double bv = __dsub_rn(a, x);
  double av = __dadd_rn(x, bv);
  double br = __dsub_rn(bv, b);
  double ar = __dsub_rn(a, av);
  y = __dadd_rn(ar, br);
}

__device__ __forceinline__ void two_prod(double a, double b, double& x, double& y) {
  x = __dmul_rn(a, b);
  y = __fma_rn(a, b, -x);
}

// h = e + b, in place allowed (h == e); returns the new length (<= n + 1)
__device__ inline int grow_exp(int n, double* e, double b) {
  double Q = b, hh;
  int k = 0;
  for (int i = 0; i < n; i++) {
    double Qn;
    two_sum(Q, e[i], Qn, hh);
    Q = Qn;
    if (hh != 0.0) e[k++] = hh;
  }
  if (Q != 0.0 || k == 0) e[k++] = Q;
  return k;
}

// e += f (e must have room for n + m components); returns the new length
__device__ inline int add_exp(int n, double* e, int m, const double* f) {
  for (int j = 0; j < m; j++) n = grow_exp(n, e, f[j]);
  return n;
}

// h = e * b (h has room for 2 n); returns the length
__device__ inline int scale_exp(int n, const double* e, double b, double* h) {
  int k = 0;
  double Q, hh, p1, p0, s;
  two_prod(e[0], b, Q, hh);
  if (hh != 0.0) h[k++] = hh;
  for (int i = 1; i < n; i++) {
    two_prod(e[i], b, p1, p0);
    two_sum(Q, p0, s, hh);
    if (hh != 0.0) h[k++] = hh;
    two_sum(p1, s, Q, hh);
    if (hh != 0.0) h[k++] = hh;
  }
  if (Q != 0.0 || k == 0) h[k++] = Q;
  return k;
}

// h = e * f (h has room for 2 n m); tmp has room for 2 n
__device__ inline int mul_exp(int n, const double* e, int m, const double* f, double* h, double* tmp) {
  int k = scale_exp(n, e, f[0], h);
  for (int j = 1; j < m; j++) {
    int t = scale_exp(n, e, f[j], tmp);
    k = add_exp(k, h, t, tmp);
  }
  return k;
}

__device__ __forceinline__ int exp_sign(int n, const double* e) {
  double top = e[n - 1];
  return (top > 0.0) - (top < 0.0);
}

__device__ __forceinline__ int diff_exp(double a, double b, double* h) {
  double x, y;
  two_diff(a, b, x, y);
  int k = 0;
  if (y != 0.0) h[k++] = y;
  h[k++] = x;  // x == 0 only when y == 0; keeps a single zero component
  return k;
}

__device__ __forceinline__ void negate_exp(int n, double* e) {
  for (int i = 0; i < n; i++) e[i] = -e[i];
}

// exact sign of det[a-d; b-d; c-d]
__device__ inline int orient3d_exact(const double* a, const double* b, const double* c,
                                     const double* d) {
  double ad[3][2], bd[3][2], cd[3][2];
  int nad[3], nbd[3], ncd[3];
  for (int k = 0; k < 3; k++) {
    nad[k] = diff_exp(a[k], d[k], ad[k]);
    nbd[k] = diff_exp(b[k], d[k], bd[k]);
    ncd[k] = diff_exp(c[k], d[k], cd[k]);
  }
  double det[200], m[16], p[8], tmp[8], t[64], tmp2[32];
  int ndet = 0;
  // det = adz (bdx cdy - bdy cdx) + bdz (cdx ady - cdy adx) + cdz (adx bdy - ady bdx)
  const double* X[3][4] = {{bd[0], cd[1], bd[1], cd[0]}, {cd[0], ad[1], cd[1], ad[0]}, {ad[0], bd[1], ad[1], bd[0]}};
  const int NX[3][4] = {{nbd[0], ncd[1], nbd[1], ncd[0]}, {ncd[0], nad[1], ncd[1], nad[0]}, {nad[0], nbd[1], nad[1], nbd[0]}};
  const double* Z[3] = {ad[2], bd[2], cd[2]};
  const int NZ[3] = {nad[2], nbd[2], ncd[2]};
  for (int r = 0; r < 3; r++) {
    int nm = mul_exp(NX[r][0], X[r][0], NX[r][1], X[r][1], m, tmp);
    int np = mul_exp(NX[r][2], X[r][2], NX[r][3], X[r][3], p, tmp);
    negate_exp(np, p);
    nm = add_exp(nm, m, np, p);
    int nt = mul_exp(nm, m, NZ[r], Z[r], t, tmp2);
    if (r == 0) {
      for (int i = 0; i < nt; i++) det[i] = t[i];
      ndet = nt;
    } else {
      ndet = add_exp(ndet, det, nt, t);
    }
  }
  return exp_sign(ndet, det);
}

// exact sign of det[a-c; b-c] (2D)
__device__ inline int orient2d_exact(const double* a, const double* b, const double* c) {
  double ac[2][2], bc[2][2], m[16], p[8], tmp[8];
  int nac[2], nbc[2];
  for (int k = 0; k < 2; k++) {
    nac[k] = diff_exp(a[k], c[k], ac[k]);
    nbc[k] = diff_exp(b[k], c[k], bc[k]);
  }
  int nm = mul_exp(nac[0], ac[0], nbc[1], bc[1], m, tmp);
  int np = mul_exp(nac[1], ac[1], nbc[0], bc[0], p, tmp);
  negate_exp(np, p);
  nm = add_exp(nm, m, np, p);
  return exp_sign(nm, m);
}

// ---------------------------------------------------------------------------
// filtered predicates: double evaluation with a forward error bound first
// ---------------------------------------------------------------------------
constexpr double kU64 = 1.1102230246251565e-16;  // 2^-53

struct ExactCounter {
  unsigned int orients = 0;
};

__device__ inline int orient3d_f64(const double* a, const double* b, const double* c,
                                   const double* d, ExactCounter& ctr) {
  double adx = a[0] - d[0], ady = a[1] - d[1], adz = a[2] - d[2];
  double bdx = b[0] - d[0], bdy = b[1] - d[1], bdz = b[2] - d[2];
  double cdx = c[0] - d[0], cdy = c[1] - d[1], cdz = c[2] - d[2];
  double bc1 = bdx * cdy, bc2 = bdy * cdx;
  double ca1 = cdx * ady, ca2 = cdy * adx;
  double ab1 = adx * bdy, ab2 = ady * bdx;
  double det = adz * (bc1 - bc2) + bdz * (ca1 - ca2) + cdz * (ab1 - ab2);
  double perm = __fma_ru(__dadd_ru(fabs(bc1), fabs(bc2)), fabs(adz),
                         __fma_ru(__dadd_ru(fabs(ca1), fabs(ca2)), fabs(bdz),
                                  __dmul_ru(__dadd_ru(fabs(ab1), fabs(ab2)), fabs(cdz))));
  double eb = __dmul_ru(8.0 * kU64, perm);
  if (det > eb) return 1;
  if (-det > eb) return -1;
  ctr.orients++;
  return orient3d_exact(a, b, c, d);
}

__device__ inline int orient2d_f64(const double* a, const double* b, const double* c,
                                   ExactCounter& ctr) {
  double acx = a[0] - c[0], acy = a[1] - c[1], bcx = b[0] - c[0], bcy = b[1] - c[1];
  double l = acx * bcy, r = acy * bcx;
  double det = l - r;
  double eb = __dmul_ru(4.0 * kU64, __dadd_ru(fabs(l), fabs(r)));
  if (det > eb) return 1;
  if (-det > eb) return -1;
  ctr.orients++;
  return orient2d_exact(a, b, c);
}

// ---------------------------------------------------------------------------
// exact closed-face intersection
// ---------------------------------------------------------------------------
__device__ __forceinline__ void drop_axis(const double* p, int ax, double* q) {
  q[0] = p[ax == 0 ? 1 : 0];
  q[1] = p[ax == 2 ? 1 : 2];
}

__device__ __forceinline__ bool in_range(double a, double b, double x) {
  return fmin(a, b) <= x && x <= fmax(a, b);
}

// closed 2D segments pq, rs meet (either may be a point)
__device__ inline bool segs_meet_2d(const double* p, const double* q, const double* r,
                                    const double* s, ExactCounter& ctr) {
  int o1 = orient2d_f64(p, q, r, ctr), o2 = orient2d_f64(p, q, s, ctr);
  int o3 = orient2d_f64(r, s, p, ctr), o4 = orient2d_f64(r, s, q, ctr);
  if (o1 * o2 < 0 && o3 * o4 < 0) return true;
  if (o1 == 0 && in_range(p[0], q[0], r[0]) && in_range(p[1], q[1], r[1])) return true;
  if (o2 == 0 && in_range(p[0], q[0], s[0]) && in_range(p[1], q[1], s[1])) return true;
  if (o3 == 0 && in_range(r[0], s[0], p[0]) && in_range(r[1], s[1], p[1])) return true;
  if (o4 == 0 && in_range(r[0], s[0], q[0]) && in_range(r[1], s[1], q[1])) return true;
  return false;
}

__device__ inline bool point_in_face_2d(const double* p, const double* a, const double* b,
                                        const double* c, ExactCounter& ctr) {
  int s0 = orient2d_f64(a, b, p, ctr), s1 = orient2d_f64(b, c, p, ctr), s2 = orient2d_f64(c, a, p, ctr);
  return (s0 >= 0 && s1 >= 0 && s2 >= 0) || (s0 <= 0 && s1 <= 0 && s2 <= 0);
}

// closed 3D segments meet: coplanar, and their projections meet on all three
// coordinate planes (one of which is injective on their common plane / line)
__device__ inline bool segs_meet_3d(const double* p0, const double* p1, const double* q0,
                                    const double* q1, ExactCounter& ctr) {
  if (orient3d_f64(p0, p1, q0, q1, ctr) != 0) return false;
  for (int ax = 0; ax < 3; ax++) {
    double a[2], b[2], c[2], d[2];
    drop_axis(p0, ax, a); drop_axis(p1, ax, b); drop_axis(q0, ax, c); drop_axis(q1, ax, d);
    if (!segs_meet_2d(a, b, c, d, ctr)) return false;
  }
  return true;
}

// closed segment P0P1 meets closed face V0V1V2
__device__ inline bool seg_meets_face(const double* P0, const double* P1, const double* V0,
                                      const double* V1, const double* V2, ExactCounter& ctr) {
  int ax = -1;
  for (int k = 2; k >= 0; k--) {
    double a[2], b[2], c[2];
    drop_axis(V0, k, a); drop_axis(V1, k, b); drop_axis(V2, k, c);
    if (orient2d_f64(a, b, c, ctr) != 0) { ax = k; break; }
  }
  if (ax < 0)  // degenerate face: union of its edges
    return segs_meet_3d(P0, P1, V0, V1, ctr) || segs_meet_3d(P0, P1, V1, V2, ctr) ||
           segs_meet_3d(P0, P1, V2, V0, ctr);
  int s0 = orient3d_f64(V0, V1, V2, P0, ctr), s1 = orient3d_f64(V0, V1, V2, P1, ctr);
  if (s0 * s1 > 0) return false;
  if (s0 != 0 || s1 != 0) {
    int a = orient3d_f64(P0, P1, V0, V1, ctr);
    int b = orient3d_f64(P0, P1, V1, V2, ctr);
    int c = orient3d_f64(P0, P1, V2, V0, ctr);
    return (a >= 0 && b >= 0 && c >= 0) || (a <= 0 && b <= 0 && c <= 0);
  }
  double p[2], q[2], a[2], b[2], c[2];
  drop_axis(P0, ax, p); drop_axis(P1, ax, q);
  drop_axis(V0, ax, a); drop_axis(V1, ax, b); drop_axis(V2, ax, c);
  if (point_in_face_2d(p, a, b, c, ctr) || point_in_face_2d(q, a, b, c, ctr)) return true;
  return segs_meet_2d(p, q, a, b, ctr) || segs_meet_2d(p, q, b, c, ctr) ||
         segs_meet_2d(p, q, c, a, ctr);
}

__device__ inline bool tri_isect_exact(const double* A, const double* B, ExactCounter& ctr) {
  for (int i = 0; i < 3; i++) {
    int j = (i + 1) % 3;
    if (seg_meets_face(A + 3 * i, A + 3 * j, B, B + 3, B + 6, ctr)) return true;
    if (seg_meets_face(B + 3 * i, B + 3 * j, A, A + 3, A + 6, ctr)) return true;
  }
  return false;
}

}  // namespace g3d
