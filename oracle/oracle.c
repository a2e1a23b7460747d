/*
 * CPU oracle for 3D distance and 3D intersection between triangle meshes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product path never
 * does.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes (arxiv 1808.09571):
 *  - A geometry is a polyhedral surface / TIN: the union of its closed
 *    triangles A_i (Sec. 3.2.1, the face set A_i, i = 0..N-1; supported
 *    geometry types in Sec. 2.2).
 *  - 3D distance (Sec. 3.2.2): the minimum over face pairs of the distance
 *    between faces, each face-face distance being the minimum of the squared
 *    distance Q of Eq. 3 extended to two parametric triangles.  It is
 *    evaluated as the minimum over the 6 vertex-face and 9 edge-edge feature
 *    pairs, which contains the minimiser whenever the faces are disjoint; if
 *    the faces intersect, the distance is exactly 0.
 *  - 3D intersection (Sec. 3.2.3): the segment-triangle test of Eq. 4 ("cut
 *    the face plane, then check the barycentric constraints") applied to the
 *    6 edges of the two faces, taken in exact arithmetic and without the
 *    division: the segment meets the plane when the two orientation signs of
 *    its end points are not equal and strict, and the meeting point lies in
 *    the closed face when the three edge orientations agree.  A segment that
 *    lies in the plane is decided in 2D.  All constraints are inclusive
 *    (0 <= u, v, u + v <= 1, 0 <= t <= 1), so touching counts.
 *  - Readings where the paper is silent: d = P1 - P0 (so t in [0,1] spans the
 *    segment), the P of Eq. 4 is P0, degenerate faces are their closed point
 *    or segment sets.
 *
 * Arithmetic: distances in IEEE double, translated to a frame at the first
 * vertex of the first face before any other operation, squared distance kept
 * through the minimum and one sqrt at the end.  Orientation signs are exact:
 * every double is an integer times a power of two, so the coordinates of a
 * predicate are scaled to integers and the determinant is evaluated in a
 * signed big-integer type written here.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -shared -fPIC oracle.c -lpthread
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* signed big integers (sign-magnitude, 32-bit limbs, little endian)          */
/* ------------------------------------------------------------------------- */

#define BI_LIMBS 80 /* 2560 bits: orient3d of doubles in [2^-200, 2^200] */

typedef struct {
  int sign; /* -1, 0, +1 */
  int n;    /* used limbs */
  uint32_t d[BI_LIMBS];
} bigint;

static volatile int g_bi_overflow = 0;

static void bi_trim(bigint *a) {
  while (a->n > 0 && a->d[a->n - 1] == 0) a->n--;
  if (a->n == 0) a->sign = 0;
}

/* a = m * 2^shift, m a signed 64-bit integer with |m| < 2^62 */
static void bi_from_shifted(bigint *a, int64_t m, int shift) {
  memset(a, 0, sizeof(*a));
  if (m == 0) return;
  a->sign = m < 0 ? -1 : 1;
  uint64_t u = m < 0 ? (uint64_t)(-m) : (uint64_t)m;
  int limb = shift / 32, bit = shift % 32;
  if (limb + 3 > BI_LIMBS) { g_bi_overflow = 1; a->sign = 0; return; }
  unsigned __int128 v = (unsigned __int128)u << bit;
  a->d[limb] = (uint32_t)v;
  a->d[limb + 1] = (uint32_t)(v >> 32);
  a->d[limb + 2] = (uint32_t)(v >> 64);
  a->n = limb + 3;
  bi_trim(a);
}

static int bi_cmp_mag(const bigint *a, const bigint *b) {
  if (a->n != b->n) return a->n < b->n ? -1 : 1;
  for (int i = a->n - 1; i >= 0; i--)
    if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
  return 0;
}

/* |r| = |a| + |b| */
static void bi_add_mag(bigint *r, const bigint *a, const bigint *b) {
  int n = a->n > b->n ? a->n : b->n;
  uint64_t carry = 0;
  bigint t;
  memset(&t, 0, sizeof(t));
  for (int i = 0; i < n; i++) {
    uint64_t s = carry;
    if (i < a->n) s += a->d[i];
    if (i < b->n) s += b->d[i];
    t.d[i] = (uint32_t)s;
    carry = s >> 32;
  }
  if (carry) {
    if (n >= BI_LIMBS) { g_bi_overflow = 1; n = BI_LIMBS - 1; }
    t.d[n++] = (uint32_t)carry;
  }
  t.n = n;
  t.sign = 1;
  *r = t;
  bi_trim(r);
}

/* |r| = |a| - |b|, requires |a| >= |b| */
static void bi_sub_mag(bigint *r, const bigint *a, const bigint *b) {
  int64_t borrow = 0;
  bigint t;
  memset(&t, 0, sizeof(t));
  for (int i = 0; i < a->n; i++) {
    int64_t s = (int64_t)a->d[i] - borrow - (i < b->n ? (int64_t)b->d[i] : 0);
    borrow = s < 0;
    if (s < 0) s += ((int64_t)1 << 32);
    t.d[i] = (uint32_t)s;
  }
  t.n = a->n;
  t.sign = 1;
  *r = t;
  bi_trim(r);
}

static void bi_add(bigint *r, const bigint *a, const bigint *b) {
  if (a->sign == 0) { *r = *b; return; }
  if (b->sign == 0) { *r = *a; return; }
  if (a->sign == b->sign) {
    int s = a->sign;
    bi_add_mag(r, a, b);
    if (r->sign) r->sign = s;
    return;
  }
  int c = bi_cmp_mag(a, b);
  if (c == 0) { memset(r, 0, sizeof(*r)); return; }
  if (c > 0) { int s = a->sign; bi_sub_mag(r, a, b); if (r->sign) r->sign = s; }
  else       { int s = b->sign; bi_sub_mag(r, b, a); if (r->sign) r->sign = s; }
}

static void bi_neg(bigint *a) { a->sign = -a->sign; }

static void bi_sub(bigint *r, const bigint *a, const bigint *b) {
  bigint nb = *b;
  bi_neg(&nb);
  bi_add(r, a, &nb);
}

static void bi_mul(bigint *r, const bigint *a, const bigint *b) {
  bigint t;
  memset(&t, 0, sizeof(t));
  if (a->sign == 0 || b->sign == 0) { *r = t; return; }
  if (a->n + b->n > BI_LIMBS) { g_bi_overflow = 1; *r = t; return; }
  for (int i = 0; i < a->n; i++) {
    uint64_t carry = 0;
    for (int j = 0; j < b->n; j++) {
      uint64_t cur = (uint64_t)a->d[i] * b->d[j] + t.d[i + j] + carry;
      t.d[i + j] = (uint32_t)cur;
      carry = cur >> 32;
    }
    int k = i + b->n;
    while (carry) {
      uint64_t cur = (uint64_t)t.d[k] + carry;
      t.d[k] = (uint32_t)cur;
      carry = cur >> 32;
      k++;
    }
  }
  t.n = a->n + b->n;
  t.sign = a->sign * b->sign;
  *r = t;
  bi_trim(r);
}

/* Decompose a finite double into m * 2^e with m a 53-bit signed integer. */
static void dbl_split(double x, int64_t *m, int *e) {
  if (x == 0.0) { *m = 0; *e = 0; return; }
  int k;
  double f = frexp(x, &k);            /* x = f * 2^k, 0.5 <= |f| < 1 */
  *m = (int64_t)ldexp(f, 53);         /* exact */
  *e = k - 53;
}

/* Load n doubles as big integers sharing the smallest exponent. */
static void bi_load(const double *x, int n, bigint *out) {
  int64_t m[12];
  int e[12], emin = 1 << 30;
  for (int i = 0; i < n; i++) {
    dbl_split(x[i], &m[i], &e[i]);
    if (m[i] != 0 && e[i] < emin) emin = e[i];
  }
  for (int i = 0; i < n; i++) bi_from_shifted(&out[i], m[i], m[i] ? e[i] - emin : 0);
}

/* sign of det [a-d; b-d; c-d], exact */
int orc_orient3d(const double *a, const double *b, const double *c, const double *d) {
  double x[12] = {a[0], a[1], a[2], b[0], b[1], b[2], c[0], c[1], c[2], d[0], d[1], d[2]};
  bigint v[12], r[9], t1, t2, m, acc, tmp;
  bi_load(x, 12, v);
  for (int i = 0; i < 3; i++)
    for (int k = 0; k < 3; k++) bi_sub(&r[3 * i + k], &v[3 * i + k], &v[9 + k]);
  /* cofactor expansion along the first row */
  memset(&acc, 0, sizeof(acc));
  /* r0 * (r4 r8 - r5 r7) */
  bi_mul(&t1, &r[4], &r[8]); bi_mul(&t2, &r[5], &r[7]); bi_sub(&m, &t1, &t2);
  bi_mul(&tmp, &r[0], &m); bi_add(&acc, &acc, &tmp);
  /* - r1 * (r3 r8 - r5 r6) */
  bi_mul(&t1, &r[3], &r[8]); bi_mul(&t2, &r[5], &r[6]); bi_sub(&m, &t1, &t2);
  bi_mul(&tmp, &r[1], &m); bi_sub(&acc, &acc, &tmp);
  /* + r2 * (r3 r7 - r4 r6) */
  bi_mul(&t1, &r[3], &r[7]); bi_mul(&t2, &r[4], &r[6]); bi_sub(&m, &t1, &t2);
  bi_mul(&tmp, &r[2], &m); bi_add(&acc, &acc, &tmp);
  return acc.sign;
}

/* sign of det [a-c; b-c] in 2D, exact */
int orc_orient2d(const double *a, const double *b, const double *c) {
  double x[6] = {a[0], a[1], b[0], b[1], c[0], c[1]};
  bigint v[6], r[4], t1, t2, acc;
  bi_load(x, 6, v);
  bi_sub(&r[0], &v[0], &v[4]); bi_sub(&r[1], &v[1], &v[5]);
  bi_sub(&r[2], &v[2], &v[4]); bi_sub(&r[3], &v[3], &v[5]);
  bi_mul(&t1, &r[0], &r[3]); bi_mul(&t2, &r[1], &r[2]);
  bi_sub(&acc, &t1, &t2);
  return acc.sign;
}

int orc_bigint_overflowed(void) { return g_bi_overflow; }

/* ------------------------------------------------------------------------- */
/* exact closed segment / triangle tests                                      */
/* ------------------------------------------------------------------------- */

/* drop axis `ax` of a 3D point */
static void proj(const double *p, int ax, double *q) {
  int k = 0;
  for (int i = 0; i < 3; i++) if (i != ax) q[k++] = p[i];
}

static int within(double a, double b, double x) {
  double lo = a < b ? a : b, hi = a < b ? b : a;
  return lo <= x && x <= hi;
}

/* r on closed 2D segment pq, given that p, q, r are collinear */
static int on_seg2(const double *p, const double *q, const double *r) {
  return within(p[0], q[0], r[0]) && within(p[1], q[1], r[1]);
}

/* closed 2D segments pq and rs share a point (either may be degenerate) */
static int seg_seg_2d(const double *p, const double *q, const double *r, const double *s) {
  int o1 = orc_orient2d(p, q, r), o2 = orc_orient2d(p, q, s);
  int o3 = orc_orient2d(r, s, p), o4 = orc_orient2d(r, s, q);
  if (o1 * o2 < 0 && o3 * o4 < 0) return 1;
  if (o1 == 0 && on_seg2(p, q, r)) return 1;
  if (o2 == 0 && on_seg2(p, q, s)) return 1;
  if (o3 == 0 && on_seg2(r, s, p)) return 1;
  if (o4 == 0 && on_seg2(r, s, q)) return 1;
  return 0;
}

/* 2D point in closed triangle (triangle non-degenerate) */
static int pt_in_tri_2d(const double *p, const double *a, const double *b, const double *c) {
  int s0 = orc_orient2d(a, b, p), s1 = orc_orient2d(b, c, p), s2 = orc_orient2d(c, a, p);
  return (s0 >= 0 && s1 >= 0 && s2 >= 0) || (s0 <= 0 && s1 <= 0 && s2 <= 0);
}

/* closed 3D segments share a point.  Both lie in some common plane iff the
 * orientation of the four end points is zero; then they meet iff their
 * projections meet on all three coordinate planes (one of them is injective
 * on the common plane or line). */
static int seg_seg_3d(const double *p0, const double *p1, const double *q0, const double *q1) {
  if (orc_orient3d(p0, p1, q0, q1) != 0) return 0;
  for (int ax = 0; ax < 3; ax++) {
    double a[2], b[2], c[2], d[2];
    proj(p0, ax, a); proj(p1, ax, b); proj(q0, ax, c); proj(q1, ax, d);
    if (!seg_seg_2d(a, b, c, d)) return 0;
  }
  return 1;
}

/* closed segment P0P1 meets closed triangle V0V1V2 */
static int seg_tri(const double *P0, const double *P1,
                   const double *V0, const double *V1, const double *V2) {
  /* degenerate triangle: it is the union of its three edges */
  int ax = -1;
  for (int k = 2; k >= 0 && ax < 0; k--) {
    double a[2], b[2], c[2];
    proj(V0, k, a); proj(V1, k, b); proj(V2, k, c);
    if (orc_orient2d(a, b, c) != 0) ax = k;
  }
  if (ax < 0) {
    return seg_seg_3d(P0, P1, V0, V1) || seg_seg_3d(P0, P1, V1, V2) ||
           seg_seg_3d(P0, P1, V2, V0);
  }
  int s0 = orc_orient3d(V0, V1, V2, P0), s1 = orc_orient3d(V0, V1, V2, P1);
  if ((s0 > 0 && s1 > 0) || (s0 < 0 && s1 < 0)) return 0;
  if (s0 != 0 || s1 != 0) {
    /* the segment crosses or touches the plane at one point: the line
     * through it meets the closed triangle iff the three edge orientations
     * do not disagree in strict sign */
    int a = orc_orient3d(P0, P1, V0, V1);
    int b = orc_orient3d(P0, P1, V1, V2);
    int c = orc_orient3d(P0, P1, V2, V0);
    return (a >= 0 && b >= 0 && c >= 0) || (a <= 0 && b <= 0 && c <= 0);
  }
  /* segment in the triangle's plane: decide on the injective projection */
  double p[2], q[2], a[2], b[2], c[2];
  proj(P0, ax, p); proj(P1, ax, q); proj(V0, ax, a); proj(V1, ax, b); proj(V2, ax, c);
  if (pt_in_tri_2d(p, a, b, c) || pt_in_tri_2d(q, a, b, c)) return 1;
  return seg_seg_2d(p, q, a, b) || seg_seg_2d(p, q, b, c) || seg_seg_2d(p, q, c, a);
}

/* Closed triangles T1, T2 (9 doubles each) share a point, exactly. */
int orc_tri_intersects(const double *T1, const double *T2) {
  const double *a[3] = {T1, T1 + 3, T1 + 6}, *b[3] = {T2, T2 + 3, T2 + 6};
  for (int i = 0; i < 3; i++) {
    int j = (i + 1) % 3;
    if (seg_tri(a[i], a[j], b[0], b[1], b[2])) return 1;
    if (seg_tri(b[i], b[j], a[0], a[1], a[2])) return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* FP64 distances (Eq. 3 minimised over the feature pairs)                    */
/* ------------------------------------------------------------------------- */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double *a, const double *b, double *r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static void cross3(const double *a, const double *b, double *r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

/* squared distance from p to the closed segment ab */
double orc_pt_seg_d2(const double *p, const double *a, const double *b) {
  double ab[3], ap[3], r[3];
  sub3(b, a, ab); sub3(p, a, ap);
  double L = dot3(ab, ab);
  double t = 0.0;
  if (L > 0.0) {
    t = dot3(ap, ab) / L;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
  }
  for (int k = 0; k < 3; k++) r[k] = ap[k] - t * ab[k];
  return dot3(r, r);
}

/* squared distance from p to the closed triangle abc */
double orc_pt_tri_d2(const double *p, const double *a, const double *b, const double *c) {
  double e0[3], e1[3], n[3];
  sub3(b, a, e0); sub3(c, a, e1); cross3(e0, e1, n);
  double nn = dot3(n, n);
  double best = orc_pt_seg_d2(p, a, b);
  double t = orc_pt_seg_d2(p, b, c); if (t < best) best = t;
  t = orc_pt_seg_d2(p, c, a); if (t < best) best = t;
  if (nn > 0.0) {
    /* projection inside the triangle: the three sub-triangle normals agree with n */
    double x[3], y[3], w[3], ap[3], bp[3], cp[3], bc[3], ca[3];
    sub3(p, a, ap); sub3(p, b, bp); sub3(p, c, cp);
    sub3(c, b, bc); sub3(a, c, ca);
    cross3(e0, ap, x); cross3(bc, bp, y); cross3(ca, cp, w);
    if (dot3(x, n) >= 0.0 && dot3(y, n) >= 0.0 && dot3(w, n) >= 0.0) {
      double h = dot3(ap, n);
      double d2 = h * h / nn;
      if (d2 < best) best = d2;
    }
  }
  return best;
}

/* squared distance between closed segments p0p1 and q0q1 */
double orc_seg_seg_d2(const double *p0, const double *p1, const double *q0, const double *q1) {
  double best = orc_pt_seg_d2(p0, q0, q1);
  double t = orc_pt_seg_d2(p1, q0, q1); if (t < best) best = t;
  t = orc_pt_seg_d2(q0, p0, p1); if (t < best) best = t;
  t = orc_pt_seg_d2(q1, p0, p1); if (t < best) best = t;
  double d1[3], d2[3], r[3];
  sub3(p1, p0, d1); sub3(q1, q0, d2); sub3(p0, q0, r);
  double a = dot3(d1, d1), e = dot3(d2, d2), b = dot3(d1, d2);
  double c = dot3(d1, r), f = dot3(d2, r);
  double det = a * e - b * b;
  if (det > 0.0) {
    /* stationary point of |r + s d1 - t d2|^2 */
    double s = (b * f - c * e) / det;
    double u = (a * f - b * c) / det;
    if (s > 0.0 && s < 1.0 && u > 0.0 && u < 1.0) {
      double w[3];
      for (int k = 0; k < 3; k++) w[k] = r[k] + s * d1[k] - u * d2[k];
      double dd = dot3(w, w);
      if (dd < best) best = dd;
    }
  }
  return best;
}

/* Squared distance between closed triangles, ignoring intersection (the
 * minimum over the 15 feature pairs), in a frame at T1's first vertex. */
double orc_tri_feature_d2(const double *T1, const double *T2) {
  double a[3][3], b[3][3];
  for (int i = 0; i < 3; i++)
    for (int k = 0; k < 3; k++) {
      a[i][k] = T1[3 * i + k] - T1[k];
      b[i][k] = T2[3 * i + k] - T1[k];
    }
  double best = INFINITY, t;
  for (int i = 0; i < 3; i++) {
    t = orc_pt_tri_d2(a[i], b[0], b[1], b[2]); if (t < best) best = t;
    t = orc_pt_tri_d2(b[i], a[0], a[1], a[2]); if (t < best) best = t;
  }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      t = orc_seg_seg_d2(a[i], a[(i + 1) % 3], b[j], b[(j + 1) % 3]);
      if (t < best) best = t;
    }
  return best;
}

/* exact closed-box overlap of two triangles (no arithmetic) */
static int tri_boxes_overlap(const double *T1, const double *T2) {
  for (int k = 0; k < 3; k++) {
    double lo1 = fmin(fmin(T1[k], T1[3 + k]), T1[6 + k]);
    double hi1 = fmax(fmax(T1[k], T1[3 + k]), T1[6 + k]);
    double lo2 = fmin(fmin(T2[k], T2[3 + k]), T2[6 + k]);
    double hi2 = fmax(fmax(T2[k], T2[3 + k]), T2[6 + k]);
    if (hi1 < lo2 || hi2 < lo1) return 0;
  }
  return 1;
}

/* Distance between closed triangles: 0 if they intersect. */
double orc_tri_distance(const double *T1, const double *T2) {
  if (tri_boxes_overlap(T1, T2) && orc_tri_intersects(T1, T2)) return 0.0;
  return sqrt(orc_tri_feature_d2(T1, T2));
}

/* ------------------------------------------------------------------------- */
/* mesh level: brute force                                                    */
/* ------------------------------------------------------------------------- */

static void gather(const double *V, const uint32_t *I, int64_t t, double *T) {
  for (int i = 0; i < 3; i++)
    for (int k = 0; k < 3; k++) T[3 * i + k] = V[3 * (int64_t)I[3 * t + i] + k];
}

/* min over all face pairs; writes the lowest (i, j) attaining it */
double orc_mesh_distance_brute(const double *VA, const uint32_t *IA, int64_t ntA,
                               const double *VB, const uint32_t *IB, int64_t ntB,
                               int64_t *arg_i, int64_t *arg_j) {
  double best2 = INFINITY;
  int64_t bi = -1, bj = -1;
  double T1[9], T2[9];
  /* any intersecting pair makes the distance 0 (lowest pair reported) */
  for (int64_t i = 0; i < ntA; i++) {
    gather(VA, IA, i, T1);
    for (int64_t j = 0; j < ntB; j++) {
      gather(VB, IB, j, T2);
      if (tri_boxes_overlap(T1, T2) && orc_tri_intersects(T1, T2)) {
        if (arg_i) *arg_i = i;
        if (arg_j) *arg_j = j;
        return 0.0;
      }
    }
  }
  for (int64_t i = 0; i < ntA; i++) {
    gather(VA, IA, i, T1);
    for (int64_t j = 0; j < ntB; j++) {
      gather(VB, IB, j, T2);
      double d2 = orc_tri_feature_d2(T1, T2);
      if (d2 < best2) { best2 = d2; bi = i; bj = j; }
    }
  }
  if (arg_i) *arg_i = bi;
  if (arg_j) *arg_j = bj;
  return sqrt(best2);
}

int orc_mesh_intersects_brute(const double *VA, const uint32_t *IA, int64_t ntA,
                              const double *VB, const uint32_t *IB, int64_t ntB) {
  double T1[9], T2[9];
  for (int64_t i = 0; i < ntA; i++) {
    gather(VA, IA, i, T1);
    for (int64_t j = 0; j < ntB; j++) {
      gather(VB, IB, j, T2);
      if (tri_boxes_overlap(T1, T2) && orc_tri_intersects(T1, T2)) return 1;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* mesh level: pruned by a CPU bounding-box tree                              */
/*                                                                            */
/* Same definitions; node pairs are skipped only when no face pair inside can */
/* reach the running minimum: the box gap is a lower bound of every face      */
/* distance below it, and a node pair is dropped only when that bound exceeds */
/* the best value so far by a margin far above double rounding (1e-9 relative */
/* plus 1e-12 absolute), so the minimising pair is never dropped and the      */
/* result equals the brute-force one.  Intersection search skips node pairs   */
/* whose closed boxes are disjoint (exact comparisons).                       */
/* ------------------------------------------------------------------------- */

typedef struct {
  double lo[3], hi[3];
  int64_t left, right; /* children, or -1 */
  int64_t first, count; /* face range in perm[] for leaves */
} onode;

typedef struct {
  const double *V;
  const uint32_t *I;
  int64_t nt;
  int64_t *perm;
  double *cen;
  onode *nodes;
  int64_t nn;
} otree;

/* order faces by centroid coordinate `axis`, ties by face id */
static int cen_less(const double *cen, int axis, int64_t a, int64_t b) {
  double ca = cen[3 * a + axis], cb = cen[3 * b + axis];
  if (ca != cb) return ca < cb;
  return a < b;
}

/* rearrange perm[lo, hi) so that position k holds the k-th face in that
 * order, smaller ones before it and larger ones after (Hoare selection) */
static void select_kth(int64_t *perm, int64_t lo, int64_t hi, int64_t k,
                       const double *cen, int axis) {
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    int64_t pv = perm[mid];
    int64_t i = lo, j = hi - 1;
    while (i <= j) {
      while (cen_less(cen, axis, perm[i], pv)) i++;
      while (cen_less(cen, axis, pv, perm[j])) j--;
      if (i <= j) { int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t; i++; j--; }
    }
    if (k <= j) hi = j + 1;
    else if (k >= i) lo = i;
    else return;
  }
}

static int64_t otree_build_rec(otree *t, int64_t first, int64_t count) {
  int64_t id = t->nn++;
  onode *n = &t->nodes[id];
  for (int k = 0; k < 3; k++) { n->lo[k] = INFINITY; n->hi[k] = -INFINITY; }
  for (int64_t q = first; q < first + count; q++) {
    int64_t f = t->perm[q];
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) {
        double x = t->V[3 * (int64_t)t->I[3 * f + i] + k];
        if (x < n->lo[k]) n->lo[k] = x;
        if (x > n->hi[k]) n->hi[k] = x;
      }
  }
  n->first = first;
  n->count = count;
  n->left = n->right = -1;
  if (count <= 4) return id;
  int axis = 0;
  double ext = -1;
  for (int k = 0; k < 3; k++)
    if (n->hi[k] - n->lo[k] > ext) { ext = n->hi[k] - n->lo[k]; axis = k; }
  int64_t h = count / 2;
  select_kth(t->perm, first, first + count, first + h, t->cen, axis);
  int64_t l = otree_build_rec(t, first, h);
  int64_t r = otree_build_rec(t, first + h, count - h);
  t->nodes[id].left = l;
  t->nodes[id].right = r;
  return id;
}

static void otree_build(otree *t, const double *V, const uint32_t *I, int64_t nt) {
  t->V = V; t->I = I; t->nt = nt;
  t->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt);
  t->cen = (double *)malloc(sizeof(double) * 3 * (size_t)nt);
  t->nodes = (onode *)malloc(sizeof(onode) * (size_t)(2 * nt + 1));
  t->nn = 0;
  for (int64_t f = 0; f < nt; f++) {
    t->perm[f] = f;
    for (int k = 0; k < 3; k++)
      t->cen[3 * f + k] = (V[3 * (int64_t)I[3 * f] + k] + V[3 * (int64_t)I[3 * f + 1] + k] +
                           V[3 * (int64_t)I[3 * f + 2] + k]) / 3.0;
  }
  otree_build_rec(t, 0, nt);
}

static void otree_free(otree *t) { free(t->perm); free(t->cen); free(t->nodes); }

static double box_gap2(const onode *a, const onode *b) {
  double s = 0;
  for (int k = 0; k < 3; k++) {
    double g = 0;
    if (b->lo[k] > a->hi[k]) g = b->lo[k] - a->hi[k];
    else if (a->lo[k] > b->hi[k]) g = a->lo[k] - b->hi[k];
    s += g * g;
  }
  return s;
}

static int box_overlap(const onode *a, const onode *b) {
  for (int k = 0; k < 3; k++)
    if (a->hi[k] < b->lo[k] || b->hi[k] < a->lo[k]) return 0;
  return 1;
}

typedef struct {
  const otree *A, *B;
  double best; /* distance */
  int hit;
  int64_t tests;
} qstate;

static int prunable(double gap2, double best) {
  if (!(best < INFINITY)) return 0;
  double lb = sqrt(gap2);
  return lb > best * (1.0 + 1e-9) + 1e-12;
}

static void dist_rec(qstate *s, int64_t na, int64_t nb) {
  if (s->hit) return;
  const onode *a = &s->A->nodes[na], *b = &s->B->nodes[nb];
  if (prunable(box_gap2(a, b), s->best)) return;
  int la = a->left < 0, lb = b->left < 0;
  if (la && lb) {
    double T1[9], T2[9];
    for (int64_t p = a->first; p < a->first + a->count; p++) {
      gather(s->A->V, s->A->I, s->A->perm[p], T1);
      for (int64_t q = b->first; q < b->first + b->count; q++) {
        gather(s->B->V, s->B->I, s->B->perm[q], T2);
        s->tests++;
        if (tri_boxes_overlap(T1, T2) && orc_tri_intersects(T1, T2)) { s->hit = 1; s->best = 0.0; return; }
        double d = sqrt(orc_tri_feature_d2(T1, T2));
        if (d < s->best) s->best = d;
      }
    }
    return;
  }
  /* descend the larger box first; visit the nearer child pair first */
  int split_a = lb || (!la && a->count >= b->count);
  if (split_a) {
    const onode *c0 = &s->A->nodes[a->left], *c1 = &s->A->nodes[a->right];
    if (box_gap2(c0, b) <= box_gap2(c1, b)) { dist_rec(s, a->left, nb); dist_rec(s, a->right, nb); }
    else { dist_rec(s, a->right, nb); dist_rec(s, a->left, nb); }
  } else {
    const onode *c0 = &s->B->nodes[b->left], *c1 = &s->B->nodes[b->right];
    if (box_gap2(a, c0) <= box_gap2(a, c1)) { dist_rec(s, na, b->left); dist_rec(s, na, b->right); }
    else { dist_rec(s, na, b->right); dist_rec(s, na, b->left); }
  }
}

static void isect_rec(qstate *s, int64_t na, int64_t nb) {
  if (s->hit) return;
  const onode *a = &s->A->nodes[na], *b = &s->B->nodes[nb];
  if (!box_overlap(a, b)) return;
  int la = a->left < 0, lb = b->left < 0;
  if (la && lb) {
    double T1[9], T2[9];
    for (int64_t p = a->first; p < a->first + a->count; p++) {
      gather(s->A->V, s->A->I, s->A->perm[p], T1);
      for (int64_t q = b->first; q < b->first + b->count; q++) {
        gather(s->B->V, s->B->I, s->B->perm[q], T2);
        s->tests++;
        if (tri_boxes_overlap(T1, T2) && orc_tri_intersects(T1, T2)) { s->hit = 1; return; }
      }
    }
    return;
  }
  int split_a = lb || (!la && a->count >= b->count);
  if (split_a) { isect_rec(s, a->left, nb); isect_rec(s, a->right, nb); }
  else { isect_rec(s, na, b->left); isect_rec(s, na, b->right); }
}

typedef struct {
  const double *VA, *VB;
  const uint32_t *IA, *IB;
  int64_t ntA, ntB;
  int op; /* 0 distance, 1 intersects */
  double result;
  int64_t tests;
} ojob;

static void run_job(ojob *j) {
  otree A, B;
  otree_build(&A, j->VA, j->IA, j->ntA);
  otree_build(&B, j->VB, j->IB, j->ntB);
  qstate s = {&A, &B, INFINITY, 0, 0};
  if (j->op == 0) {
    dist_rec(&s, 0, 0);
    j->result = s.hit ? 0.0 : s.best;
  } else {
    isect_rec(&s, 0, 0);
    j->result = s.hit ? 1.0 : 0.0;
  }
  j->tests = s.tests;
  otree_free(&A);
  otree_free(&B);
}

double orc_mesh_distance_pruned(const double *VA, const uint32_t *IA, int64_t ntA,
                                const double *VB, const uint32_t *IB, int64_t ntB,
                                int64_t *tests) {
  ojob j = {VA, VB, IA, IB, ntA, ntB, 0, 0, 0};
  run_job(&j);
  if (tests) *tests = j.tests;
  return j.result;
}

int orc_mesh_intersects_pruned(const double *VA, const uint32_t *IA, int64_t ntA,
                               const double *VB, const uint32_t *IB, int64_t ntB,
                               int64_t *tests) {
  ojob j = {VA, VB, IA, IB, ntA, ntB, 1, 0, 0};
  run_job(&j);
  if (tests) *tests = j.tests;
  return j.result != 0.0;
}

/* Many independent queries on `nthreads` POSIX threads (timing mode).
 * Query q uses meshes (a[q], b[q]) from the mesh table and operation op[q]. */
typedef struct {
  ojob *jobs;
  int64_t n;
  int64_t next;
  pthread_mutex_t mu;
} opool;

static void *pool_worker(void *arg) {
  opool *p = (opool *)arg;
  for (;;) {
    pthread_mutex_lock(&p->mu);
    int64_t i = p->next++;
    pthread_mutex_unlock(&p->mu);
    if (i >= p->n) break;
    run_job(&p->jobs[i]);
  }
  return NULL;
}

int orc_batch_pruned(int64_t n, const double *const *V, const uint32_t *const *I,
                     const int64_t *nt, const int64_t *qa, const int64_t *qb,
                     const int32_t *op, double *out, int64_t *tests, int nthreads) {
  ojob *jobs = (ojob *)calloc((size_t)n, sizeof(ojob));
  if (!jobs) return -1;
  for (int64_t q = 0; q < n; q++) {
    jobs[q].VA = V[qa[q]]; jobs[q].IA = I[qa[q]]; jobs[q].ntA = nt[qa[q]];
    jobs[q].VB = V[qb[q]]; jobs[q].IB = I[qb[q]]; jobs[q].ntB = nt[qb[q]];
    jobs[q].op = op[q];
  }
  opool p;
  p.jobs = jobs; p.n = n; p.next = 0;
  pthread_mutex_init(&p.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  pthread_t th[256];
  if (nthreads > 256) nthreads = 256;
  for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, pool_worker, &p);
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  for (int64_t q = 0; q < n; q++) {
    out[q] = jobs[q].result;
    if (tests) tests[q] = jobs[q].tests;
  }
  pthread_mutex_destroy(&p.mu);
  free(jobs);
  return 0;
}
