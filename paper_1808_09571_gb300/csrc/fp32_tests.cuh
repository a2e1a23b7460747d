// Certified FP32 face-pair tests (the leaf work of the traversal).
//
// Distance (Sec. 3.2.2, Eq. 3): the minimum of the squared distance between
// two closed faces is reached on one of 6 vertex-face or 9 edge-edge feature
// pairs when the faces are disjoint.  The test evaluates those 15 terms in
// float32 in a frame at the first vertex of face A and keeps the closest
// point pair (P on A, Q on B).  It returns two certified bounds on the exact
// distance of the stored faces, independent of whether the float32 search
// picked the right feature (it only has to produce points ON the faces):
//   ub = |P - Q| + 64 u M           (u = 2^-24, M = largest |coordinate| in the frame)
//   lb = gap(n) / |n| (1 - 8u) - 16 u M,  n = Q - P,
// where gap(n) is the separation of the two faces' vertex projections on n:
// any axis separating the faces bounds their distance from below, and Q - P
// is the optimal axis when P, Q are the closest points.  The constants cover
// the rounding of the frame translation, of constructing P and Q, of the
// norm and of the projections (derivation in the design notes); all bound
// arithmetic is done with directed rounding.
//
// Intersection (Sec. 3.2.3, Eq. 4 without the division): each of the 6 edges
// is tested against the other face with orientation signs.  An orientation
// is certified when |det| exceeds 8u times its permanent (a forward error
// bound for this evaluation order, as in Shewchuk's adaptive predicates);
// otherwise the face pair is UNCERTAIN and goes to the FP64 / exact stage.
#pragma once
#include "internal.cuh"
#include "closest.cuh"

namespace g3d {

constexpr float kU = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of float32
constexpr float kAbsSlop = 1e-20f;            // covers float32 underflow

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }

__device__ __forceinline__ float d2of(float3 P, float3 Q) {
  float3 d = P - Q;
  return dot(d, d);
}

struct PairBounds {
  float lb;  // certified lower bound of the distance (rounded down)
  float ub;  // certified upper bound (rounded up)
};

// Certified bounds of the distance between faces A = (A0,A1,A2) and
// B = (B0,B1,B2) (stored float32 coordinates).
__device__ __forceinline__ PairBounds tri_pair_bounds(float3 A0, float3 A1, float3 A2,
                                                      float3 B0, float3 B1, float3 B2) {
  // frame at A0
  float3 a0 = make_float3(0.f, 0.f, 0.f), a1 = A1 - A0, a2 = A2 - A0;
  float3 b0 = B0 - A0, b1 = B1 - A0, b2 = B2 - A0;
  float M = fmaxf(fmaxf(amax3(a1), amax3(a2)), fmaxf(amax3(b0), fmaxf(amax3(b1), amax3(b2))));

  float best;
  float3 P = a0, Q = closest_on_tri(a0, b0, b1, b2);
  best = d2of(P, Q);
#define G3D_TRY(PP, QQ)                                     \
  {                                                         \
    float3 _p = (PP), _q = (QQ);                            \
    float _d = d2of(_p, _q);                                \
    if (_d < best) { best = _d; P = _p; Q = _q; }           \
  }
  G3D_TRY(a1, closest_on_tri(a1, b0, b1, b2));
  G3D_TRY(a2, closest_on_tri(a2, b0, b1, b2));
  G3D_TRY(closest_on_tri(b0, a0, a1, a2), b0);
  G3D_TRY(closest_on_tri(b1, a0, a1, a2), b1);
  G3D_TRY(closest_on_tri(b2, a0, a1, a2), b2);
  const float3 ea[3][2] = {{a0, a1}, {a1, a2}, {a2, a0}};
  const float3 eb[3][2] = {{b0, b1}, {b1, b2}, {b2, b0}};
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      float3 p, q;
      closest_seg_seg(ea[i][0], ea[i][1], eb[j][0], eb[j][1], p, q);
      G3D_TRY(p, q);
    }
#undef G3D_TRY

  float uM = __fmul_ru(kU, __fmul_ru(M, 1.0000005f));
  PairBounds r;
  float3 n = Q - P;
  float nn = dot(n, n);
  float dist = sqrtf(nn);
  r.ub = __fadd_ru(__fadd_ru(dist, __fmul_ru(64.f, uM)), kAbsSlop);
  r.lb = 0.f;
  if (nn > 0.f) {
    float pa = fmaxf(fmaxf(dot(n, a0), dot(n, a1)), dot(n, a2));
    float pb = fminf(fminf(dot(n, b0), dot(n, b1)), dot(n, b2));
    float gap = pb - pa;
    if (gap > 0.f) {
      float q = __fdiv_rd(gap, dist);
      float lb = __fsub_rd(__fsub_rd(__fmul_rd(q, 1.f - 8.f * kU), __fmul_ru(16.f, uM)), kAbsSlop);
      r.lb = fmaxf(lb, 0.f);
    }
  }
  return r;
}

// Same bounds, with the 15 feature terms evaluated in a rolled loop over two
// faces stored as 9 consecutive floats each (shared memory): far fewer live
// registers than the unrolled form, identical arithmetic per term (every
// local-frame coordinate is recomputed as the same single rounding).
// Vertex k of a face whose vertices are S floats apart (S = 3: 9 consecutive
// floats; S = 64: the planes of a staged leaf, 16 float4 apart), in the
// frame at vertex 0 of the face at O (same stride).
template <int S>
__device__ __forceinline__ float3 lvert_s(const float* F, const float* O, int k) {
  return make_float3(F[S * k] - O[0], F[S * k + 1] - O[1], F[S * k + 2] - O[2]);
}

template <int S>
static __device__ __noinline__ PairBounds tri_pair_bounds_rolled_s(const float* A, const float* B) {
#define lvert lvert_s<S>
  float M = 0.f;
#pragma unroll 1
  for (int k = 0; k < 3; k++) M = fmaxf(M, fmaxf(amax3(lvert(A, A, k)), amax3(lvert(B, A, k))));
  float best = INFINITY;
  float3 P = make_float3(0.f, 0.f, 0.f), Q = P;
#pragma unroll 1
  for (int t = 0; t < 15; t++) {
    float3 p, q;
    if (t < 3) {
      p = lvert(A, A, t);
      q = closest_on_tri(p, lvert(B, A, 0), lvert(B, A, 1), lvert(B, A, 2));
    } else if (t < 6) {
      q = lvert(B, A, t - 3);
      p = closest_on_tri(q, lvert(A, A, 0), lvert(A, A, 1), lvert(A, A, 2));
    } else {
      const int i = (t - 6) / 3, j = (t - 6) - 3 * i;
      const int i1 = i == 2 ? 0 : i + 1, j1 = j == 2 ? 0 : j + 1;
      closest_seg_seg(lvert(A, A, i), lvert(A, A, i1), lvert(B, A, j), lvert(B, A, j1), p, q);
    }
    const float d = d2of(p, q);
    if (d < best) { best = d; P = p; Q = q; }
  }
  const float uM = __fmul_ru(kU, __fmul_ru(M, 1.0000005f));
  PairBounds r;
  const float3 n = Q - P;
  const float nn = dot(n, n);
  const float dist = sqrtf(nn);
  r.ub = __fadd_ru(__fadd_ru(dist, __fmul_ru(64.f, uM)), kAbsSlop);
  r.lb = 0.f;
  if (nn > 0.f) {
    float pa = -INFINITY, pb = INFINITY;
#pragma unroll 1
    for (int k = 0; k < 3; k++) {
      pa = fmaxf(pa, dot(n, lvert(A, A, k)));
      pb = fminf(pb, dot(n, lvert(B, A, k)));
    }
    const float gap = pb - pa;
    if (gap > 0.f) {
      const float q = __fdiv_rd(gap, dist);
      const float lb = __fsub_rd(__fsub_rd(__fmul_rd(q, 1.f - 8.f * kU), __fmul_ru(16.f, uM)), kAbsSlop);
      r.lb = fmaxf(lb, 0.f);
    }
  }
  return r;
#undef lvert
}

__device__ __forceinline__ PairBounds tri_pair_bounds_rolled(const float* A, const float* B) {
  return tri_pair_bounds_rolled_s<3>(A, B);
}

// The same certified bounds with the 15 feature terms spread over the 16
// lanes of a half-warp: lane f of the half evaluates term f (lane 15 none),
// a 4-step shuffle reduction picks the closest pair (smallest squared
// distance, ties to the lowest term, as the sequential loop does), and every
// lane of the half then derives the bounds from it.  One face pair per half:
// the 16-fold shorter dependency chain is what matters when few face pairs
// are in flight.  Both halves of the warp must call it together.
__device__ __forceinline__ PairBounds tri_pair_bounds_hw(float3 A0, float3 A1, float3 A2, float3 B0, float3 B1,
                                                         float3 B2) {
  const unsigned int FULLM = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int f = lane & 15;
  const float3 a0 = make_float3(0.f, 0.f, 0.f), a1 = A1 - A0, a2 = A2 - A0;
  const float3 b0 = B0 - A0, b1 = B1 - A0, b2 = B2 - A0;
  const float M = fmaxf(fmaxf(amax3(a1), amax3(a2)), fmaxf(amax3(b0), fmaxf(amax3(b1), amax3(b2))));
  float3 p = a0, q = a0;
  float d = INFINITY;
  if (f < 3) {
    p = f == 0 ? a0 : (f == 1 ? a1 : a2);
    q = closest_on_tri(p, b0, b1, b2);
    d = d2of(p, q);
  } else if (f < 6) {
    q = f == 3 ? b0 : (f == 4 ? b1 : b2);
    p = closest_on_tri(q, a0, a1, a2);
    d = d2of(p, q);
  } else if (f < 15) {
    const int i = (f - 6) / 3, j = (f - 6) - 3 * ((f - 6) / 3);
    const float3 ai = i == 0 ? a0 : (i == 1 ? a1 : a2), ai1 = i == 0 ? a1 : (i == 1 ? a2 : a0);
    const float3 bj = j == 0 ? b0 : (j == 1 ? b1 : b2), bj1 = j == 0 ? b1 : (j == 1 ? b2 : b0);
    closest_seg_seg(ai, ai1, bj, bj1, p, q);
    d = d2of(p, q);
  }
  int best = f;
  float bd = d;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const float od = __shfl_xor_sync(FULLM, bd, o, 16);
    const int of = __shfl_xor_sync(FULLM, best, o, 16);
    if (od < bd || (od == bd && of < best)) { bd = od; best = of; }
  }
  const int src = (lane & 16) | best;
  const float3 P = make_float3(__shfl_sync(FULLM, p.x, src), __shfl_sync(FULLM, p.y, src), __shfl_sync(FULLM, p.z, src));
  const float3 Q = make_float3(__shfl_sync(FULLM, q.x, src), __shfl_sync(FULLM, q.y, src), __shfl_sync(FULLM, q.z, src));
  const float uM = __fmul_ru(kU, __fmul_ru(M, 1.0000005f));
  PairBounds r;
  const float3 n = Q - P;
  const float nn = dot(n, n);
  const float dist = sqrtf(nn);
  r.ub = __fadd_ru(__fadd_ru(dist, __fmul_ru(64.f, uM)), kAbsSlop);
  r.lb = 0.f;
  if (nn > 0.f) {
    const float pa = fmaxf(fmaxf(dot(n, a0), dot(n, a1)), dot(n, a2));
    const float pb = fminf(fminf(dot(n, b0), dot(n, b1)), dot(n, b2));
    const float gap = pb - pa;
    if (gap > 0.f) {
      const float qq = __fdiv_rd(gap, dist);
      const float lb = __fsub_rd(__fsub_rd(__fmul_rd(qq, 1.f - 8.f * kU), __fmul_ru(16.f, uM)), kAbsSlop);
      r.lb = fmaxf(lb, 0.f);
    }
  }
  return r;
}

// Orientation sign of d with respect to the plane abc: sign of
// det[a-d; b-d; c-d] when certified, else 0 (uncertain).
__device__ __forceinline__ int orient3d_f32(float3 a, float3 b, float3 c, float3 d) {
  float adx = a.x - d.x, ady = a.y - d.y, adz = a.z - d.z;
  float bdx = b.x - d.x, bdy = b.y - d.y, bdz = b.z - d.z;
  float cdx = c.x - d.x, cdy = c.y - d.y, cdz = c.z - d.z;
  float bc1 = bdx * cdy, bc2 = bdy * cdx;
  float ca1 = cdx * ady, ca2 = cdy * adx;
  float ab1 = adx * bdy, ab2 = ady * bdx;
  float det = adz * (bc1 - bc2) + bdz * (ca1 - ca2) + cdz * (ab1 - ab2);
  float perm = __fmaf_ru(__fadd_ru(fabsf(bc1), fabsf(bc2)), fabsf(adz),
                         __fmaf_ru(__fadd_ru(fabsf(ca1), fabsf(ca2)), fabsf(bdz),
                                   __fmul_ru(__fadd_ru(fabsf(ab1), fabsf(ab2)), fabsf(cdz))));
  float eb = __fadd_ru(__fmul_ru(8.f * kU, perm), 1e-36f);
  if (det > eb) return 1;
  if (-det > eb) return -1;
  return 0;
}

enum { ISECT_NO = 0, ISECT_YES = 1, ISECT_UNSURE = 2 };

// Edge P0P1 against closed face V0V1V2; s0, s1 are the certified signs of
// P0, P1 against the face plane (0 = uncertain).  Returns ISECT_*.
__device__ __forceinline__ int edge_vs_face(float3 P0, float3 P1, int s0, int s1,
                                            float3 V0, float3 V1, float3 V2) {
  if (s0 != 0 && s0 == s1) return ISECT_NO;
  int a = orient3d_f32(P0, P1, V0, V1);
  int b = orient3d_f32(P0, P1, V1, V2);
  int c = orient3d_f32(P0, P1, V2, V0);
  // two strictly opposite edge signs: the line misses the closed face
  if (a * b < 0 || b * c < 0 || a * c < 0) return ISECT_NO;
  if (s0 * s1 < 0 && a != 0 && a == b && b == c) return ISECT_YES;
  return ISECT_UNSURE;
}

__device__ __forceinline__ bool same_point(float3 p, float3 q) { return p.x == q.x && p.y == q.y && p.z == q.z; }

// Filtered closed-face intersection test.  Faces with a vertex in common
// (adjacent faces of touching meshes, shared by construction or by data)
// meet there: decided by exact comparisons before any orientation.
__device__ __forceinline__ int tri_isect_filter(float3 A0, float3 A1, float3 A2,
                                                float3 B0, float3 B1, float3 B2) {
  if (same_point(A0, B0) || same_point(A0, B1) || same_point(A0, B2) || same_point(A1, B0) ||
      same_point(A1, B1) || same_point(A1, B2) || same_point(A2, B0) || same_point(A2, B1) ||
      same_point(A2, B2))
    return ISECT_YES;
  int sb0 = orient3d_f32(A0, A1, A2, B0), sb1 = orient3d_f32(A0, A1, A2, B1),
      sb2 = orient3d_f32(A0, A1, A2, B2);
  if (sb0 != 0 && sb0 == sb1 && sb1 == sb2) return ISECT_NO;
  int sa0 = orient3d_f32(B0, B1, B2, A0), sa1 = orient3d_f32(B0, B1, B2, A1),
      sa2 = orient3d_f32(B0, B1, B2, A2);
  if (sa0 != 0 && sa0 == sa1 && sa1 == sa2) return ISECT_NO;
  bool unsure = false;
  int r;
  r = edge_vs_face(A0, A1, sa0, sa1, B0, B1, B2); if (r == ISECT_YES) return r; unsure |= r == ISECT_UNSURE;
  r = edge_vs_face(A1, A2, sa1, sa2, B0, B1, B2); if (r == ISECT_YES) return r; unsure |= r == ISECT_UNSURE;
  r = edge_vs_face(A2, A0, sa2, sa0, B0, B1, B2); if (r == ISECT_YES) return r; unsure |= r == ISECT_UNSURE;
  r = edge_vs_face(B0, B1, sb0, sb1, A0, A1, A2); if (r == ISECT_YES) return r; unsure |= r == ISECT_UNSURE;
  r = edge_vs_face(B1, B2, sb1, sb2, A0, A1, A2); if (r == ISECT_YES) return r; unsure |= r == ISECT_UNSURE;
  r = edge_vs_face(B2, B0, sb2, sb0, A0, A1, A2); if (r == ISECT_YES) return r; unsure |= r == ISECT_UNSURE;
  return unsure ? ISECT_UNSURE : ISECT_NO;
}

// The filtered test on faces stored as 9 floats (not inlined: keeps the
// traversal's register budget small).
// The filtered intersection test with its orientations spread over a
// half-warp: lanes 0-2 of the half take B's vertices against A's plane,
// lanes 3-5 A's against B's, then lanes 0-5 the six edge-against-face tests;
// the answer (YES if the faces share a vertex -- lanes 6-14 compare one
// vertex pair each -- or any edge test says so, else UNSURE if any is
// uncertain, else NO; NO at once when either face lies strictly on one side
// of the other's plane) is the sequential test's.  Both halves of the warp must call
// it together; every lane of the half returns the answer.
__device__ __forceinline__ int tri_isect_filter_hw(float3 A0, float3 A1, float3 A2, float3 B0, float3 B1, float3 B2) {
  const unsigned int FULLM = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int f = lane & 15, base = lane & 16;
  int sg = 0;
  bool shared = false;  // lanes 6-14: vertex i of A equals vertex j of B
  if (f < 3) sg = orient3d_f32(A0, A1, A2, f == 0 ? B0 : (f == 1 ? B1 : B2));
  else if (f < 6) sg = orient3d_f32(B0, B1, B2, f == 3 ? A0 : (f == 4 ? A1 : A2));
  else if (f < 15) {
    const int i = (f - 6) / 3, j = (f - 6) - 3 * ((f - 6) / 3);
    shared = same_point(i == 0 ? A0 : (i == 1 ? A1 : A2), j == 0 ? B0 : (j == 1 ? B1 : B2));
  }
  const unsigned int shm = __ballot_sync(FULLM, shared);
  const int sb0 = __shfl_sync(FULLM, sg, base + 0), sb1 = __shfl_sync(FULLM, sg, base + 1),
            sb2 = __shfl_sync(FULLM, sg, base + 2);
  const int sa0 = __shfl_sync(FULLM, sg, base + 3), sa1 = __shfl_sync(FULLM, sg, base + 4),
            sa2 = __shfl_sync(FULLM, sg, base + 5);
  const bool sep = (sb0 != 0 && sb0 == sb1 && sb1 == sb2) || (sa0 != 0 && sa0 == sa1 && sa1 == sa2);
  int r = ISECT_NO;
  if (!sep && f < 6) {
    if (f == 0) r = edge_vs_face(A0, A1, sa0, sa1, B0, B1, B2);
    else if (f == 1) r = edge_vs_face(A1, A2, sa1, sa2, B0, B1, B2);
    else if (f == 2) r = edge_vs_face(A2, A0, sa2, sa0, B0, B1, B2);
    else if (f == 3) r = edge_vs_face(B0, B1, sb0, sb1, A0, A1, A2);
    else if (f == 4) r = edge_vs_face(B1, B2, sb1, sb2, A0, A1, A2);
    else r = edge_vs_face(B2, B0, sb2, sb0, A0, A1, A2);
  }
  const unsigned int yes = __ballot_sync(FULLM, r == ISECT_YES), uns = __ballot_sync(FULLM, r == ISECT_UNSURE);
  const unsigned int half = 0xffffu << base;
  if ((yes | shm) & half) return ISECT_YES;
  return (uns & half) ? ISECT_UNSURE : ISECT_NO;
}

template <int S>
static __device__ __noinline__ int tri_isect_filter_ss(const float* A, const float* B) {
  return tri_isect_filter(make_float3(A[0], A[1], A[2]), make_float3(A[S], A[S + 1], A[S + 2]),
                          make_float3(A[2 * S], A[2 * S + 1], A[2 * S + 2]), make_float3(B[0], B[1], B[2]),
                          make_float3(B[S], B[S + 1], B[S + 2]), make_float3(B[2 * S], B[2 * S + 1], B[2 * S + 2]));
}

__device__ __forceinline__ int tri_isect_filter_s(const float* A, const float* B) {
  return tri_isect_filter_ss<3>(A, B);
}

// Closed boxes of two faces overlap (exact comparisons).
__device__ __forceinline__ bool tri_boxes_overlap(float3 A0, float3 A1, float3 A2,
                                                  float3 B0, float3 B1, float3 B2, float slack) {
  float4 alo = make_float4(fminf(A0.x, fminf(A1.x, A2.x)), fminf(A0.y, fminf(A1.y, A2.y)),
                           fminf(A0.z, fminf(A1.z, A2.z)), 0.f);
  float4 ahi = make_float4(fmaxf(A0.x, fmaxf(A1.x, A2.x)), fmaxf(A0.y, fmaxf(A1.y, A2.y)),
                           fmaxf(A0.z, fmaxf(A1.z, A2.z)), 0.f);
  float4 blo = make_float4(fminf(B0.x, fminf(B1.x, B2.x)), fminf(B0.y, fminf(B1.y, B2.y)),
                           fminf(B0.z, fminf(B1.z, B2.z)), 0.f);
  float4 bhi = make_float4(fmaxf(B0.x, fmaxf(B1.x, B2.x)), fmaxf(B0.y, fmaxf(B1.y, B2.y)),
                           fmaxf(B0.z, fmaxf(B1.z, B2.z)), 0.f);
  return box_overlap(alo, ahi, blo, bhi, slack);
}

// Lower bound of the face distance from the faces' boxes (rounded down).
__device__ __forceinline__ float tri_boxes_lb(float3 A0, float3 A1, float3 A2,
                                              float3 B0, float3 B1, float3 B2) {
  float4 alo = make_float4(fminf(A0.x, fminf(A1.x, A2.x)), fminf(A0.y, fminf(A1.y, A2.y)),
                           fminf(A0.z, fminf(A1.z, A2.z)), 0.f);
  float4 ahi = make_float4(fmaxf(A0.x, fmaxf(A1.x, A2.x)), fmaxf(A0.y, fmaxf(A1.y, A2.y)),
                           fmaxf(A0.z, fmaxf(A1.z, A2.z)), 0.f);
  float4 blo = make_float4(fminf(B0.x, fminf(B1.x, B2.x)), fminf(B0.y, fminf(B1.y, B2.y)),
                           fminf(B0.z, fminf(B1.z, B2.z)), 0.f);
  float4 bhi = make_float4(fmaxf(B0.x, fmaxf(B1.x, B2.x)), fmaxf(B0.y, fmaxf(B1.y, B2.y)),
                           fmaxf(B0.z, fmaxf(B1.z, B2.z)), 0.f);
  return box_lb(alo, ahi, blo, bhi);
}

}  // namespace g3d
