// Internal device-side types shared by the geo3d translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/geo3d.h"

namespace g3d {

// ---------------------------------------------------------------------------
// Device layout of one mesh (HBM):
//   v0, v1, v2 : float4[nt]   faces in BVH (Morton) order, SoA; v0.w holds the
//                             original face id (int bits), v1.w / v2.w unused.
//   m64        : double[9*nt] optional FP64 master coordinates, same order.
//   nodes      : float4[4*(nleaf-1)] internal nodes of the binary radix tree,
//                each {lo0, hi0, lo1, hi1}: the boxes of its two children;
//                lo_c.w = child reference (int bits: >= 0 internal node,
//                < 0 leaf ~ref), hi_c.w = number of leaves below the child.
//   leaves     : float4[2*nleaf] {lo (w = first face), hi (w = face count)}.
// ---------------------------------------------------------------------------
struct MeshDev {
  const float4* v0;
  const float4* v1;
  const float4* v2;
  const double* m64;
  const float4* nodes;
  const float4* leaves;
  int root;   // >= 0 internal node index, < 0 leaf (~root)
  int nleaf;
  int ntri;
  float rho;  // bound on |f64 input - stored f32| over all coordinates (0 for f32)
  int L;      // faces per leaf: leaf k holds faces [k L, min(k L + L, ntri))
  int pad;
  const int2* nrange;   // [nleaf - 1] first / last leaf below each internal node
  const float* cstats;  // [64 x 16] per-cluster statistics (learned proposal)
};

struct QueryDev {
  MeshDev A, B;
  int op;       // G3D_OP_*
  float slack;  // sqrt(3) * (rho_A + rho_B), rounded up
  int link;     // distance query: index of an intersects query of the same pair, or -1
  int dlink;    // intersects query: a distance query linked to it, or -1
};

// Per-query mutable state, reset before each launch.
constexpr int kMaxProposals = 4;  // cluster pairs proposed per query (restricted dive d takes d mod n)

struct QueryState {
  unsigned int ub;          // certified upper bound of the distance (float bits)
  int done;                 // 1: an intersection was certified (result fixed)
  int ncand;                // candidate pushes for this query (may exceed pool)
  int overflow;             // a push of this query failed (pool full)
  unsigned long long best;  // FP64 minimum squared distance (double bits)
  int hit;                  // exact intersection found in finalize
  int status;               // G3D_OK or error
  int pass;                 // 1 or 2
  int phase;                // distance queries: 0 intersects, 1 distance
  int nprop;                // proposals held (0 .. kMaxProposals)
  int4 prop[kMaxProposals]; // proposal k: leaf ranges (pa0, pa1, pb0, pb1), inclusive, the restricted dives keep to
  unsigned long long witness;  // (input face id of A << 32) | input face id of B attaining the minimum
  int label;                   // cluster pair (cA * 64 + cB) of the witness, -1 if none
  unsigned int ub_seed;        // UB when the distance traversal starts (after the dives)
};

// Candidate face pair kept for the FP64 / exact stage.
// x = face of A (sorted index), y = face of B, z = lower bound (float bits),
// w = query index | flags << 24... flags live in the top bits of w.
#define CAND_NEEDS_EXACT 0x40000000
#define CAND_QMASK 0x3fffffff

// Work item: x = query, y = ref A, z = ref B, w = lower bound (float bits).

// Device counters (g3d_stats order).
enum {
  ST_NODE_PAIRS = 0, ST_LEAF_PAIRS, ST_TRI_PREFILTER, ST_TRI_TESTS, ST_CANDIDATES,
  ST_FP64_TESTS, ST_EXACT_TESTS, ST_EXACT_ORIENTS, ST_QUEUE_PUSHES, ST_SECOND_PASSES,
  ST_BUSY_NS, ST_IDLE_NS, ST_SEED_EXCESS, ST_SEED_QUERIES,
  ST_DISTINCT_NODES, ST_DISTINCT_FACES, ST_LEVELS,
  ST_COUNT = 20
};

struct Queue {
  int4* items;                    // [cap]
  int* seq;                       // [cap] slot sequence numbers
  unsigned long long* head;       // next ticket to pop
  unsigned long long* tail;       // next ticket to push
  long long* pending;             // items owned by the queue or by a working warp
  int* error;                     // sticky device error (G3D_ERR_*)
  unsigned int cap;               // power of two
};

struct CandPool {
  int4* items;
  int* count;
  int cap;
};

struct TravArgs {
  const QueryDev* q;      // [nq]
  QueryState* st;         // [nq]
  int nq;
  Queue queue;
  CandPool cand;
  unsigned long long* stats;
  unsigned long long t_limit_ns;  // wall-clock limit of every device wait
  int total_warps;
  int pass;
  int* sticky;  // first per-query error since the last g3d_sync
  int leaf_w;   // lanes per leaf-pair slot: 16 (leaves of <= 8 faces) or 32
  int* dbg;     // [8] first invalid item seen: {where, x, y, z, w}
  // optional first-visit bitmap (distinct nodes / faces counters): per
  // query, bits for mesh A's internal nodes then leaves, then mesh B's,
  // starting at bit visit_off[q]; null when not counting
  unsigned int* visit;
  const long long* visit_off;
};

// Level-synchronous traversal state.  Level k expands the node pairs of
// frontier F[k & 1] into F[(k + 1) & 1] and tests the leaf pairs of L[k & 1]
// (found while expanding level k - 1); leaf pairs found at level k go to
// L[(k + 1) & 1].  cnt holds three rotating frontier counts (index k % 3),
// three leaf counts (3 + k % 3) and three leaf work tickets (6 + k % 3); an
// item that does not fit goes to the global queue, which the persistent
// kernel drains afterwards.  The leaf tests of a level defer the face pairs
// that pass the box prefilter to FP, and all warps test them after a second
// grid barrier (a face pair that does not fit is tested where it was found).
// A distance pair goes to bucket b by its box bound against the query's bound
// when it was found (<= 1/8, 1/4, 1/2 of it, or above), and the buckets are
// tested nearest first, so the bounds the near pairs produce prune the far
// ones.
constexpr int kFPBuckets = 4;
struct FrontierArgs {
  int4* F[2];
  int4* L[2];
  int4* FP;           // face pairs the leaf tests of a level defer: {q, face of A, face of B, box bound},
                      // in kFPBuckets sublists of fpcap / kFPBuckets entries
  int fpcap;
  unsigned int* cnt;  // [28]: [16 + 2 b + (k & 1)] counts level k's deferred face pairs of bucket b
  unsigned int* bar;  // [2] grid barrier: arrivals, generation
  int fcap, lcap;
  int nblocks;
  // level trace ring: per level {ns since the launch started, level,
  // frontier node pairs, leaf pairs, ns block 0 spent expanding, ns until
  // block 0 finished its leaf tests}; trace_next counts the entries written
  unsigned long long* trace;
  unsigned int* trace_next;
  int trace_cap;  // power of 2
};

// An item's references must name nodes / leaves of its query's meshes.
__device__ __forceinline__ bool ref_ok(int r, int nleaf) {
  return r >= 0 ? r < nleaf - 1 : (~r) < nleaf;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float i2f(int x) { return __int_as_float(x); }
__device__ __forceinline__ int f2i(float x) { return __float_as_int(x); }

// order-preserving map of floats to unsigned ints (for atomic min/max)
__device__ __forceinline__ unsigned int f2ord(float f) {
  unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ void stat_add(unsigned long long* stats, int k, unsigned long long v) {
  if (stats && v) atomicAdd(&stats[k], v);
}

// Lower bound of the distance between two axis-aligned boxes, rounded down.
__device__ __forceinline__ float box_lb(float4 alo, float4 ahi, float4 blo, float4 bhi) {
  float gx = fmaxf(0.f, fmaxf(__fsub_rd(blo.x, ahi.x), __fsub_rd(alo.x, bhi.x)));
  float gy = fmaxf(0.f, fmaxf(__fsub_rd(blo.y, ahi.y), __fsub_rd(alo.y, bhi.y)));
  float gz = fmaxf(0.f, fmaxf(__fsub_rd(blo.z, ahi.z), __fsub_rd(alo.z, bhi.z)));
  float s = __fmaf_rd(gx, gx, __fmaf_rd(gy, gy, __fmul_rd(gz, gz)));
  return __fsqrt_rd(s);
}

// Closed boxes, each inflated by `slack`, overlap (exact comparisons when
// slack is 0).
__device__ __forceinline__ bool box_overlap(float4 alo, float4 ahi, float4 blo, float4 bhi,
                                            float slack) {
  if (slack == 0.f)
    return !(ahi.x < blo.x || bhi.x < alo.x || ahi.y < blo.y || bhi.y < alo.y ||
             ahi.z < blo.z || bhi.z < alo.z);
  return !(__fadd_ru(ahi.x, slack) < __fsub_rd(blo.x, slack) ||
           __fadd_ru(bhi.x, slack) < __fsub_rd(alo.x, slack) ||
           __fadd_ru(ahi.y, slack) < __fsub_rd(blo.y, slack) ||
           __fadd_ru(bhi.y, slack) < __fsub_rd(alo.y, slack) ||
           __fadd_ru(ahi.z, slack) < __fsub_rd(blo.z, slack) ||
           __fadd_ru(bhi.z, slack) < __fsub_rd(alo.z, slack));
}

}  // namespace g3d
