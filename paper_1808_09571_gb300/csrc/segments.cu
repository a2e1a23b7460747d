// Line segments and points against one polyhedral surface.
//
// The paper's operators are defined for line segment / polyhedral surface
// and point / polyhedral surface (Sec. 3.2.2): the distance is the minimum
// over the surface's faces of the segment-face distance (the squared
// distance Q(u, v, t) of Eq. 3 minimised over the closed face and the
// closed segment), and the segment intersects the surface when it meets a
// closed face (Sec. 3.2.3, Eq. 4: the segment crosses the face plane inside
// the face).  A point is a segment with P0 == P1.
//
// The paper evaluates each face in its own thread; here each segment is a
// thread that walks the mesh's BVH (single-tree branch and bound) nearest
// child first, with certified FP32 tests built like the mesh-mesh path's
// (over the segment's 5 feature pairs; the exact predicates see the
// segment as the degenerate face P0 P1 P1, i.e. its closed point set):
//   - distance: a subtree is skipped when the box lower bound exceeds the
//     certified upper bound UB; face pairs whose certified lower bound does
//     not exceed UB are kept in a small per-thread list and recomputed in
//     FP64 at the end (or when the list is full), intersecting candidates
//     decided exactly;
//   - intersects: boxes must overlap; the filtered orientation test decides
//     most faces, the rest are decided exactly.
#include <cuda_runtime.h>

#include "fp32_tests.cuh"
#include "fp64_exact.cuh"
#include "segments.cuh"

namespace g3d {

constexpr int kSegStack = 96;  // deeper than any radix tree over 30-bit keys + index bits
constexpr int kSegCand = 8;    // candidates kept per thread before an early FP64 flush

__device__ __forceinline__ void seg_face64(const MeshDev& M, int f, double* out) {
  if (M.m64) {
    for (int k = 0; k < 9; k++) out[k] = M.m64[9ll * f + k];
  } else {
    const float4 a = __ldg(&M.v0[f]), b = __ldg(&M.v1[f]), c = __ldg(&M.v2[f]);
    out[0] = a.x; out[1] = a.y; out[2] = a.z;
    out[3] = b.x; out[4] = b.y; out[5] = b.z;
    out[6] = c.x; out[7] = c.y; out[8] = c.z;
  }
}

// Filtered test of the closed segment S[0..2] S[3..5] against a closed face.
__device__ __forceinline__ int seg_isect_filter(const float* S, const float* F) {
  const float3 P0 = make_float3(S[0], S[1], S[2]), P1 = make_float3(S[3], S[4], S[5]);
  const float3 V0 = make_float3(F[0], F[1], F[2]), V1 = make_float3(F[3], F[4], F[5]),
               V2 = make_float3(F[6], F[7], F[8]);
  const int s0 = orient3d_f32(V0, V1, V2, P0), s1 = orient3d_f32(V0, V1, V2, P1);
  return edge_vs_face(P0, P1, s0, s1, V0, V1, V2);
}

// Certified bounds of the distance between the closed segment S = P0 P1
// (S[0..5]) and the closed face F (F[0..8]): the face-pair bounds of the mesh
// path (ub = |P - Q| + 64 u M, lb from the separation along Q - P) with the
// segment's own 5 feature pairs -- P0 and P1 against the face, the segment
// against the face's 3 edges -- instead of the 15 of two faces.  A face
// vertex's closest point on the segment is covered by the segment-edge
// terms of its two edges, and when a zero-area face or a zero-length segment
// makes a point-face term fall back to a vertex, the segment-edge terms
// still reach the minimum.  The error budget is the one of the face-pair
// test: the same primitives and the same frame translation, in a frame at P0.
__device__ __forceinline__ float3 sfv(const float* F, const float* O, int k) {
  return make_float3(F[3 * k] - O[0], F[3 * k + 1] - O[1], F[3 * k + 2] - O[2]);
}

static __device__ __noinline__ PairBounds seg_tri_bounds(const float* S, const float* F) {
  const float3 p0 = make_float3(0.f, 0.f, 0.f), p1 = sfv(S, S, 1);
  float M = amax3(p1);
#pragma unroll 1
  for (int k = 0; k < 3; k++) M = fmaxf(M, amax3(sfv(F, S, k)));
  float best = INFINITY;
  float3 P = p0, Q = p0;
#pragma unroll 1
  for (int t = 0; t < 5; t++) {
    float3 p, q;
    if (t < 2) {
      p = t == 0 ? p0 : p1;
      q = closest_on_tri(p, sfv(F, S, 0), sfv(F, S, 1), sfv(F, S, 2));
    } else {
      const int j = t - 2, j1 = j == 2 ? 0 : j + 1;
      closest_seg_seg(p0, p1, sfv(F, S, j), sfv(F, S, j1), p, q);
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
    const float pa = fmaxf(dot(n, p0), dot(n, p1));
    float pb = INFINITY;
#pragma unroll 1
    for (int k = 0; k < 3; k++) pb = fminf(pb, dot(n, sfv(F, S, k)));
    const float gap = pb - pa;
    if (gap > 0.f) {
      const float q = __fdiv_rd(gap, dist);
      const float lb = __fsub_rd(__fsub_rd(__fmul_rd(q, 1.f - 8.f * kU), __fmul_ru(16.f, uM)), kAbsSlop);
      r.lb = fmaxf(lb, 0.f);
    }
  }
  return r;
}

// FP64 squared distance of the closed segment S64[0..5] and the closed face
// F[0..8], over the same 5 feature pairs, in a frame at P0.
__device__ inline double seg_dist2_f64(const double* S64, const double* F) {
  const double3 p0 = make_double3(0.0, 0.0, 0.0);
  const double3 p1 = make_double3(S64[3] - S64[0], S64[4] - S64[1], S64[5] - S64[2]);
  double3 b[3];
  for (int k = 0; k < 3; k++) b[k] = make_double3(F[3 * k] - S64[0], F[3 * k + 1] - S64[1], F[3 * k + 2] - S64[2]);
  double best = d2of64(p0, closest_on_tri(p0, b[0], b[1], b[2]));
  best = fmin(best, d2of64(p1, closest_on_tri(p1, b[0], b[1], b[2])));
  for (int j = 0; j < 3; j++) {
    double3 p, q;
    closest_seg_seg(p0, p1, b[j], b[j == 2 ? 0 : j + 1], p, q);
    best = fmin(best, d2of64(p, q));
  }
  return best;
}

struct SegState {
  float ub = INFINITY;
  double best = INFINITY;  // FP64 minimum squared distance of the evaluated candidates
  bool hit = false;
  int nc = 0;
  int cf[kSegCand];
  float cl[kSegCand];
  unsigned int cx = 0;  // bit k: candidate k needs the exact intersection test
  unsigned int tests = 0, exact = 0, nodes = 0;
};

// FP64 / exact evaluation of candidate k of the list
__device__ __forceinline__ void seg_eval(const SegArgs& a, SegState& st, const double* S64, int k) {
  double F[9];
  seg_face64(a.M, st.cf[k], F);
  if ((st.cx >> k) & 1u) {
    ExactCounter ctr;
    st.exact++;
    if (seg_meets_face(S64, S64 + 3, F, F + 3, F + 6, ctr)) {
      st.hit = true;
      return;
    }
  }
  if (a.op == G3D_OP_DISTANCE) st.best = fmin(st.best, seg_dist2_f64(S64, F));
}

__device__ __forceinline__ void seg_push_cand(const SegArgs& a, SegState& st, const double* S64, int f, float lb,
                                              bool needs_exact) {
  if (st.nc == kSegCand) {  // drop what the current bound excludes, then flush the oldest
    int m = 0;
    unsigned int x = 0;
    for (int k = 0; k < kSegCand; k++) {
      if (st.cl[k] > st.ub) continue;
      st.cf[m] = st.cf[k];
      st.cl[m] = st.cl[k];
      x |= ((st.cx >> k) & 1u) << m;
      m++;
    }
    st.nc = m;
    st.cx = x;
    if (m == kSegCand) {
      seg_eval(a, st, S64, 0);
      for (int k = 1; k < kSegCand; k++) { st.cf[k - 1] = st.cf[k]; st.cl[k - 1] = st.cl[k]; }
      st.cx >>= 1;
      st.nc--;
      if (st.hit) return;
    }
  }
  st.cf[st.nc] = f;
  st.cl[st.nc] = lb;
  if (needs_exact) st.cx |= 1u << st.nc;
  st.nc++;
}

// faces of leaf `ref` (< 0) against the segment
__device__ __forceinline__ void seg_leaf(const SegArgs& a, SegState& st, const float* S, const double* S64,
                                         float4 slo, float4 shi, int ref) {
  const MeshDev& M = a.M;
  const int first = (~ref) * M.L, cnt = min(M.L, M.ntri - first);
  const float3 P0 = make_float3(S[0], S[1], S[2]), P1 = make_float3(S[3], S[4], S[5]);
  for (int t = 0; t < cnt && !st.hit; t++) {
    const int f = first + t;
    const float4 p0 = __ldg(&M.v0[f]), p1 = __ldg(&M.v1[f]), p2 = __ldg(&M.v2[f]);
    const float3 V0 = f3(p0), V1 = f3(p1), V2 = f3(p2);
    const float F[9] = {p0.x, p0.y, p0.z, p1.x, p1.y, p1.z, p2.x, p2.y, p2.z};
    if (a.op == G3D_OP_DISTANCE) {
      if (__fsub_rd(tri_boxes_lb(P0, P1, P1, V0, V1, V2), a.slack) > st.ub) continue;
      st.tests++;
      const PairBounds pb = seg_tri_bounds(S, F);
      const float plb = fmaxf(__fsub_rd(pb.lb, a.slack), 0.f);
      const float pub = __fadd_ru(pb.ub, a.slack);
      if (pub < st.ub) st.ub = pub;
      if (plb > st.ub) continue;
      bool ex = false;
      if (plb <= 0.f) {
        const int r = a.slack == 0.f ? seg_isect_filter(S, F) : ISECT_UNSURE;
        if (r == ISECT_YES) { st.hit = true; return; }
        ex = r == ISECT_UNSURE;
      }
      seg_push_cand(a, st, S64, f, plb, ex);
    } else {
      if (!tri_boxes_overlap(P0, P1, P1, V0, V1, V2, a.slack)) continue;
      st.tests++;
      const int r = a.slack == 0.f ? seg_isect_filter(S, F) : ISECT_UNSURE;
      if (r == ISECT_YES) { st.hit = true; return; }
      if (r == ISECT_UNSURE) {
        double F64[9];
        seg_face64(M, f, F64);
        ExactCounter ctr;
        st.exact++;
        if (seg_meets_face(S64, S64 + 3, F64, F64 + 3, F64 + 6, ctr)) { st.hit = true; return; }
      }
    }
  }
  (void)slo; (void)shi;
}

// every leaf below internal node r (stack overflow fallback)
__device__ __forceinline__ void seg_subtree(const SegArgs& a, SegState& st, const float* S, const double* S64,
                                            float4 slo, float4 shi, int r) {
  const int2 rg = __ldg(&a.M.nrange[r]);
  for (int k = rg.x; k <= rg.y && !st.hit; k++) seg_leaf(a, st, S, S64, slo, shi, ~k);
}

__global__ void __launch_bounds__(128) k_segments(SegArgs a) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  SegState st;
  int err = 0;
  float S[9];
  double S64[9];
  float4 slo = make_float4(0.f, 0.f, 0.f, 0.f), shi = slo;
  if (i < a.n) {
    for (int k = 0; k < 6; k++) S[k] = a.segs[6 * i + k];
    S[6] = S[3]; S[7] = S[4]; S[8] = S[5];
    for (int k = 0; k < 6; k++) {
      if (!isfinite(S[k])) err = G3D_ERR_NAN_INPUT;
      else if (fabsf(S[k]) > 1.152921504606846976e18f) err = err ? err : G3D_ERR_RANGE;  // 2^60
    }
    for (int k = 0; k < 9; k++) S64[k] = S[k];
    slo = make_float4(fminf(S[0], S[3]), fminf(S[1], S[4]), fminf(S[2], S[5]), 0.f);
    shi = make_float4(fmaxf(S[0], S[3]), fmaxf(S[1], S[4]), fmaxf(S[2], S[5]), 0.f);
  }
  const bool active = i < a.n && !err;
  const MeshDev& M = a.M;
  int stk[kSegStack];
  float slb[kSegStack];
  int sp = 0;
  if (active) {
    stk[0] = M.root;
    slb[0] = 0.f;
    sp = 1;
  }
  // Two phases per round so the lanes of a warp stay together: every lane
  // walks internal nodes until it holds a leaf (or runs out of work), then
  // the lanes holding one test its faces at the same time.
  int leaf = 0;
  bool live = active;
  while (__any_sync(0xffffffffu, live)) {
    bool have = false;
    while (live && sp > 0 && !have) {
      --sp;
      const int r = stk[sp];
      if (a.op == G3D_OP_DISTANCE && slb[sp] > st.ub) continue;
      if (r < 0) {
        leaf = r;
        have = true;
        break;
      }
      st.nodes++;
      const float4* nd = M.nodes + 4 * r;
      int ch[2];
      float lb[2];
      bool keep[2];
      for (int c = 0; c < 2; c++) {
        const float4 lo = __ldg(nd + 2 * c), hi = __ldg(nd + 2 * c + 1);
        ch[c] = __float_as_int(lo.w);
        if (a.op == G3D_OP_DISTANCE) {
          lb[c] = fmaxf(__fsub_rd(box_lb(slo, shi, lo, hi), a.slack), 0.f);
          keep[c] = lb[c] <= st.ub;
        } else {
          lb[c] = 0.f;
          keep[c] = box_overlap(slo, shi, lo, hi, a.slack);
        }
      }
      // push the farther child first so the nearer one is expanded next
      const int o = (keep[0] && keep[1] && lb[1] > lb[0]) ? 1 : 0;
      for (int j = 0; j < 2; j++) {
        const int c = j == 0 ? o : 1 - o;
        if (!keep[c]) continue;
        if (sp == kSegStack) {  // no room: the whole subtree, leaf by leaf
          if (ch[c] < 0) seg_leaf(a, st, S, S64, slo, shi, ch[c]);
          else seg_subtree(a, st, S, S64, slo, shi, ch[c]);
          continue;
        }
        stk[sp] = ch[c];
        slb[sp++] = lb[c];
      }
      if (st.hit) break;
    }
    if (have && !st.hit) seg_leaf(a, st, S, S64, slo, shi, leaf);
    live = live && !st.hit && sp > 0;
  }
  if (active) {
    // FP64 / exact stage of the kept candidates
    for (int k = 0; k < st.nc && !st.hit; k++)
      if (st.cl[k] <= st.ub) seg_eval(a, st, S64, k);
  }
  if (i < a.n) {
    double d = __longlong_as_double(0x7ff8000000000000ll);
    if (!err && a.op == G3D_OP_DISTANCE) {
      if (st.hit) d = 0.0;
      else if (isfinite(st.best)) d = sqrt(st.best);
      else err = G3D_ERR_CUDA;  // no candidate survived: internal error
    }
    if (a.dist) a.dist[i] = err ? __longlong_as_double(0x7ff8000000000000ll) : d;
    if (a.hit) a.hit[i] = err ? 0xff : (unsigned char)(st.hit ? 1 : 0);
    if (a.status) a.status[i] = err;
    if (err && !a.status && a.sticky) atomicCAS(a.sticky, 0, err);  // reported nowhere else
  }
  // counters: one atomic per warp
  unsigned int nodes = st.nodes, tests = st.tests, exact = st.exact;
  for (int o = 16; o > 0; o >>= 1) {
    nodes += __shfl_xor_sync(0xffffffffu, nodes, o);
    tests += __shfl_xor_sync(0xffffffffu, tests, o);
    exact += __shfl_xor_sync(0xffffffffu, exact, o);
  }
  if ((threadIdx.x & 31) == 0 && a.stats) {
    stat_add(a.stats, ST_NODE_PAIRS, nodes);
    stat_add(a.stats, ST_TRI_TESTS, tests);
    stat_add(a.stats, ST_EXACT_TESTS, exact);
  }
}

}  // namespace g3d
