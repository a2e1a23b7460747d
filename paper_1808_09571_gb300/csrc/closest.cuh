// Closest-point primitives of the face-pair distance, for float3 and double3.
// Every returned point is a convex combination of the feature's vertices with
// coefficients in [0, 1] (clamped), so it lies on the closed feature up to
// the rounding of its construction.
#pragma once
#include <cuda_runtime.h>

namespace g3d {

__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double3 operator-(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ double dot(double3 a, double3 b) { return fma(a.x, b.x, fma(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 axpy(float t, float3 d, float3 p) {  // p + t d
  return make_float3(fmaf(t, d.x, p.x), fmaf(t, d.y, p.y), fmaf(t, d.z, p.z));
}
__device__ __forceinline__ double3 axpy(double t, double3 d, double3 p) {
  return make_double3(fma(t, d.x, p.x), fma(t, d.y, p.y), fma(t, d.z, p.z));
}
__device__ __forceinline__ float clamp01(float t) { return fminf(fmaxf(t, 0.f), 1.f); }
__device__ __forceinline__ double clamp01(double t) { return fmin(fmax(t, 0.0), 1.0); }
__device__ __forceinline__ float amax3(float3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }

// Closest point of the closed triangle abc to p (Voronoi-region walk of
// Ericson, "Real-Time Collision Detection", Sec. 5.1.5).
template <class V, class S>
__device__ __forceinline__ V closest_on_tri_t(V p, V a, V b, V c) {
  const S zero = S(0);
  V ab = b - a, ac = c - a, ap = p - a;
  S d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= zero && d2 <= zero) return a;
  V bp = p - b;
  S d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= zero && d4 <= d3) return b;
  S vc = d1 * d4 - d3 * d2;
  if (vc <= zero && d1 >= zero && d3 <= zero) {
    S den = d1 - d3;
    return axpy(den > zero ? clamp01(d1 / den) : zero, ab, a);
  }
  V cp = p - c;
  S d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= zero && d5 <= d6) return c;
  S vb = d5 * d2 - d1 * d6;
  if (vb <= zero && d2 >= zero && d6 <= zero) {
    S den = d2 - d6;
    return axpy(den > zero ? clamp01(d2 / den) : zero, ac, a);
  }
  S va = d3 * d6 - d5 * d4;
  S e43 = d4 - d3, e56 = d5 - d6;
  if (va <= zero && e43 >= zero && e56 >= zero) {
    S den = e43 + e56;
    return axpy(den > zero ? clamp01(e43 / den) : zero, c - b, b);
  }
  S s = va + vb + vc;
  if (!(s > zero)) return a;
  S v = clamp01(vb / s), w = clamp01(vc / s);
  S vw = v + w;
  if (vw > S(1)) { v = v / vw; w = w / vw; }
  return axpy(w, ac, axpy(v, ab, a));
}

// Closest points of the closed segments p0p1 and q0q1 (clamped parametric
// minimisation, Ericson Sec. 5.1.9).
template <class V, class S>
__device__ __forceinline__ void closest_seg_seg_t(V p0, V p1, V q0, V q1, V& P, V& Q) {
  const S zero = S(0);
  V d1 = p1 - p0, d2 = q1 - q0, r = p0 - q0;
  S a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  S s = zero, t = zero;
  if (a > zero || e > zero) {
    if (!(a > zero)) {
      t = clamp01(f / e);
    } else {
      S c = dot(d1, r);
      if (!(e > zero)) {
        s = clamp01(-c / a);
      } else {
        S b = dot(d1, d2);
        S den = a * e - b * b;
        s = den > zero ? clamp01((b * f - c * e) / den) : zero;
        t = (b * s + f) / e;
        if (t < zero) { t = zero; s = clamp01(-c / a); }
        else if (t > S(1)) { t = S(1); s = clamp01((b - c) / a); }
        else if (!(t >= zero)) { t = zero; s = zero; }  // NaN guard
      }
    }
  }
  P = axpy(s, d1, p0);
  Q = axpy(t, d2, q0);
}

__device__ __forceinline__ float3 closest_on_tri(float3 p, float3 a, float3 b, float3 c) {
  return closest_on_tri_t<float3, float>(p, a, b, c);
}
__device__ __forceinline__ double3 closest_on_tri(double3 p, double3 a, double3 b, double3 c) {
  return closest_on_tri_t<double3, double>(p, a, b, c);
}
__device__ __forceinline__ void closest_seg_seg(float3 p0, float3 p1, float3 q0, float3 q1, float3& P, float3& Q) {
  closest_seg_seg_t<float3, float>(p0, p1, q0, q1, P, Q);
}
__device__ __forceinline__ void closest_seg_seg(double3 p0, double3 p1, double3 q0, double3 q1, double3& P, double3& Q) {
  closest_seg_seg_t<double3, double>(p0, p1, q0, q1, P, Q);
}

}  // namespace g3d
