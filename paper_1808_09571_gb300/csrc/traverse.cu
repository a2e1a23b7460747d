// Dual-tree branch-and-bound traversal, leaf face-pair tests and the FP64 /
// exact finalisation.
//
// The paper evaluates each face of a polyhedral surface in its own GPU thread
// and reduces the per-face results with a minimum (Sec. 3.2.2, "the minimum
// distance is returned") or an any (Sec. 3.2.3).  Here the same per-face-pair
// work is pruned by the two meshes' BVHs:
//   - a work item is a pair of BVH nodes (query, refA, refB, lower bound);
//   - distance: a node pair is dropped when the box lower bound (directed
//     rounding) exceeds the query's certified upper bound UB, which every
//     warp lowers with atomicMin as leaf face pairs are tested;
//   - intersects: a node pair is dropped when the closed boxes are disjoint;
//     the first certified intersecting face pair ends the query;
//   - each warp owns a node-pair stack in shared memory and expands up to 8
//     items per step, one child pair per lane, survivors compacted with a
//     ballot; leaf pairs are tested by the whole warp;
//   - warps share work through a global ring queue (sequence-numbered slots):
//     a warp donates the bottom of its stack when the queue runs low, idle
//     warps pop from it; `pending` counts the items not yet finished and the
//     launch ends when it reaches zero.  Every wait is bounded by a
//     wall-clock limit after which the kernel records G3D_ERR_TIMEOUT.
// Face pairs whose certified lower bound does not exceed UB are kept as
// candidates; after the traversal they are recomputed in FP64, and those that
// might intersect are decided exactly (fp64_exact.cuh).
#include <cuda_runtime.h>

#include "fp32_tests.cuh"
#include "fp64_exact.cuh"
#include "traverse.cuh"

namespace g3d {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
  return *(volatile const unsigned int*)p;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}
__device__ __forceinline__ long long ld_volatile_i64(const long long* p) {
  return *(volatile const long long*)p;
}

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// record the first invalid item (never dereferenced) and flag the launch
__device__ void record_bad(const TravArgs& a, int where, int4 v) {
  if (a.dbg && atomicCAS(&a.dbg[0], 0, where) == 0) {
    a.dbg[1] = v.x; a.dbg[2] = v.y; a.dbg[3] = v.z; a.dbg[4] = v.w;
  }
  if (a.sticky) atomicCAS(a.sticky, 0, G3D_ERR_CUDA);
}

__device__ __forceinline__ bool item_ok(const TravArgs& a, int4 it) {
  if (it.x < 0 || it.x >= a.nq) return false;
  const QueryDev& Qd = a.q[it.x];
  return ref_ok(it.y, Qd.A.nleaf) && ref_ok(it.z, Qd.B.nleaf);
}

// ---------------------------------------------------------------------------
// global queue
// ---------------------------------------------------------------------------
// Push n (<= 32) items held by lanes [0, n).  Returns 1 when pushed, 0 on
// error, and -1 (nothing pushed, no error recorded) when `soft` is set and
// the queue has no room; without `soft` a full queue is an error.
__device__ int gq_push_n(const Queue& Q, int4 item, int n, unsigned long long tlim, bool soft) {
  const int lane = threadIdx.x & 31;
  unsigned long long t0 = 0;
  int ok = 1;
  if (lane == 0) {
    unsigned long long h = ld_volatile_u64(Q.head), t = ld_volatile_u64(Q.tail);
    if (t - h + (unsigned long long)n + 4096ull > Q.cap) {
      if (!soft) set_error(Q.error, G3D_ERR_CAND_OVERFLOW);
      ok = soft ? -1 : 0;
    } else {
      atomicAdd((unsigned long long*)Q.pending, (unsigned long long)n);
      __threadfence();  // pending must count the items before they can be popped
      t0 = atomicAdd(Q.tail, (unsigned long long)n);
    }
  }
  ok = __shfl_sync(FULL, ok, 0);
  if (ok != 1) return ok;
  t0 = __shfl_sync(FULL, t0, 0);
  bool good = true;
  if (lane < n) {
    unsigned long long ticket = t0 + lane;
    unsigned int slot = (unsigned int)(ticket & (Q.cap - 1));
    int want = (int)(unsigned int)ticket;
    unsigned long long start = 0;
    int spins = 0;
    while (ld_volatile_i32(&Q.seq[slot]) != want) {
      if (++spins == 64) start = globaltimer_ns();
      if (spins > 64 && globaltimer_ns() - start > tlim) { set_error(Q.error, G3D_ERR_TIMEOUT); good = false; break; }
      __nanosleep(64);
    }
    if (good) {
      Q.items[slot] = item;
      __threadfence();
      *(volatile int*)&Q.seq[slot] = want + 1;
    }
  }
  return __all_sync(FULL, good) ? 1 : 0;
}

__device__ __forceinline__ bool gq_push(const Queue& Q, int4 item, int n, unsigned long long tlim) {
  return gq_push_n(Q, item, n, tlim, false) == 1;
}

// Pop up to maxk (<= 32) items into lanes [0, got).  Returns got, or -1 on
// error.
__device__ int gq_pop(const Queue& Q, int4& item, int maxk, unsigned long long tlim) {
  const int lane = threadIdx.x & 31;
  int got = 0;
  unsigned long long t0 = 0;
  if (lane == 0) {
    for (int tries = 0; tries < 64; tries++) {
      unsigned long long h = ld_volatile_u64(Q.head), t = ld_volatile_u64(Q.tail);
      if (t <= h) break;
      unsigned long long k = t - h;
      if (k > (unsigned long long)maxk) k = maxk;
      if (atomicCAS(Q.head, h, h + k) == h) { got = (int)k; t0 = h; break; }
    }
  }
  got = __shfl_sync(FULL, got, 0);
  if (got == 0) return 0;
  t0 = __shfl_sync(FULL, t0, 0);
  bool good = true;
  if (lane < got) {
    unsigned long long ticket = t0 + lane;
    unsigned int slot = (unsigned int)(ticket & (Q.cap - 1));
    int want = (int)(unsigned int)(ticket + 1);
    unsigned long long start = 0;
    int spins = 0;
    while (ld_volatile_i32(&Q.seq[slot]) != want) {
      if (++spins == 64) start = globaltimer_ns();
      if (spins > 64 && globaltimer_ns() - start > tlim) { set_error(Q.error, G3D_ERR_TIMEOUT); good = false; break; }
      __nanosleep(32);
    }
    if (good) {
      __threadfence();
      volatile int* src = (volatile int*)&Q.items[slot];
      item = make_int4(src[0], src[1], src[2], src[3]);
      __threadfence();
      *(volatile int*)&Q.seq[slot] = (int)(unsigned int)(ticket + Q.cap);
    }
  }
  if (!__all_sync(FULL, good)) return -1;
  return got;
}

// ---------------------------------------------------------------------------
// leaf pair: all lanes test the faces of leaf la (mesh A) x leaf lb (mesh B)
// ---------------------------------------------------------------------------
struct LeafCounters {
  unsigned int pre = 0, tests = 0, cands = 0;
};

#ifndef G3D_CAND_AGG
#define G3D_CAND_AGG 1  // one atomic per group of converged lanes pushing together
#endif
__device__ __forceinline__ void push_candidate(const TravArgs& a, int q, int fa, int fb, float lb, int flags) {
#if G3D_CAND_AGG
  const unsigned int m = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(a.cand.count, __popc(m));
  base = __shfl_sync(m, base, leader);
  const int idx = base + __popc(m & ((1u << lane) - 1u));
#else
  int idx = atomicAdd(a.cand.count, 1);
#endif
  if (idx < a.cand.cap) {
    a.cand.items[idx] = make_int4(fa, fb, __float_as_int(lb), q | flags);
  } else {
    a.st[q].overflow = 1;
  }
}

__device__ __forceinline__ float3 sface(const LeafStage& S, int k, int v) {
  return make_float3(S.f[k][3 * v], S.f[k][3 * v + 1], S.f[k][3 * v + 2]);
}

// Leaf refs -> face ranges: leaf k of a mesh holds faces [k L, min(k L + L, nt)).
__device__ __forceinline__ void leaf_range(const MeshDev& M, int ref, int& first, int& count) {
  first = (~ref) * M.L;
  count = min(M.L, M.ntri - first);
}

// Test the faces of up to 32 / W leaf pairs (jobs) with the warp split into
// slots of W lanes (W = 16 when leaves hold <= 8 faces, else 32).  In a slot,
// lane k < W/2 stages face k of leaf A, lane W/2 + k face k of leaf B, and
// keeps it when its box can reach the other leaf's box (box lower bound <= UB
// for distance, closed-box overlap for intersects).  The surviving faces are
// compacted and their pairs go through the face-box prefilter and the full
// test: certified bounds (distance) or the filtered orientation test.
// The faces come through `fetch(slot, sideB, fi, M, f, p0, p1, p2)`: from
// global memory (GlobalFaces) or from a shared-memory copy staged by the bulk
// copy engine (StagedFaces).
struct GlobalFaces {
  __device__ __forceinline__ void operator()(int, bool, int, const MeshDev& M, int f, float4& p0, float4& p1,
                                             float4& p2) const {
    p0 = __ldg(&M.v0[f]);
    p1 = __ldg(&M.v1[f]);
    p2 = __ldg(&M.v2[f]);
  }
};

// faces of up to kLeafBatch leaf pairs: [job][side A / B][plane v0 / v1 / v2][face of the leaf]
#ifndef G3D_LEAF_BATCH
#define G3D_LEAF_BATCH 2  // leaf pairs a warp of the level-synchronous kernel stages per batch (2: measured fastest; a smaller staging area leaves more L1)
#endif
constexpr int kLeafBatch = G3D_LEAF_BATCH;
typedef float4 StagedLeafFaces[2][3][16];

struct StagedFaces {
  const StagedLeafFaces* jobs;  // the staged faces of the jobs passed to this call
  __device__ __forceinline__ void operator()(int slot, bool sideB, int fi, const MeshDev&, int, float4& p0,
                                             float4& p1, float4& p2) const {
    const float4* P = jobs[slot][sideB ? 1 : 0][0];
    p0 = P[fi];
    p1 = P[16 + fi];
    p2 = P[32 + fi];
  }
};

#ifndef G3D_LEAF_INLINE
#define G3D_LEAF_INLINE 1  // 0: keep the leaf tests out of line (measured slower)
#endif
template <class Fetch>
#if G3D_LEAF_INLINE
__device__ __forceinline__
#else
__device__ __noinline__
#endif
void leaf_jobs_t(const TravArgs& a, const LeafJob* jobs, int njobs, int W, LeafCounters& lc, LeafStage& S,
                 const Fetch& fetch) {
  const int lane = threadIdx.x & 31;
  const int slot = W == 32 ? 0 : lane >> 4;
  const int k = W == 32 ? lane : lane & 15;
  const int H = W >> 1;
  const bool active = slot < njobs;
  const LeafJob J = jobs[active ? slot : 0];
  const int q = J.q;
  const QueryDev& Qd = a.q[q];
  const int mode = J.mode;
  const float slack = Qd.slack;
  int fa0, na, fb0, nb;
  leaf_range(Qd.A, J.la, fa0, na);
  leaf_range(Qd.B, J.lb, fb0, nb);
  const float ub = __uint_as_float(ld_volatile_u32(&a.st[q].ub));

  const bool sideB = k >= H;
  const int fi = sideB ? k - H : k;
  const bool have = active && (sideB ? fi < nb : fi < na);
  bool keep = false;
  if (have) {
    const MeshDev& M = sideB ? Qd.B : Qd.A;
    const int f = (sideB ? fb0 : fa0) + fi;
    float4 p0, p1, p2;
    fetch(slot, sideB, fi, M, f, p0, p1, p2);
    S.f[lane][0] = p0.x; S.f[lane][1] = p0.y; S.f[lane][2] = p0.z;
    S.f[lane][3] = p1.x; S.f[lane][4] = p1.y; S.f[lane][5] = p1.z;
    S.f[lane][6] = p2.x; S.f[lane][7] = p2.y; S.f[lane][8] = p2.z;
    float4 flo = make_float4(fminf(p0.x, fminf(p1.x, p2.x)), fminf(p0.y, fminf(p1.y, p2.y)),
                             fminf(p0.z, fminf(p1.z, p2.z)), 0.f);
    float4 fhi = make_float4(fmaxf(p0.x, fmaxf(p1.x, p2.x)), fmaxf(p0.y, fmaxf(p1.y, p2.y)),
                             fmaxf(p0.z, fmaxf(p1.z, p2.z)), 0.f);
    float4 olo = sideB ? J.alo : J.blo, ohi = sideB ? J.ahi : J.bhi;
    if (mode == G3D_OP_DISTANCE) keep = __fsub_rd(box_lb(flo, fhi, olo, ohi), slack) <= ub;
    else keep = box_overlap(flo, fhi, olo, ohi, slack);
  }
  const unsigned int km = __ballot_sync(FULL, keep);
  const unsigned int segmask = W == 32 ? FULL : (0xffffu << (16 * slot));
  const unsigned int seg = (km & segmask) >> (W == 32 ? 0 : 16 * slot);
  const unsigned int hmask = (1u << H) - 1u;
  const unsigned int mA = seg & hmask, mB = (seg >> H) & hmask;
  const unsigned int below = (1u << fi) - 1u;
  const int base = slot * W;
  if (keep) S.idx[base + (sideB ? H + __popc(mB & below) : __popc(mA & below))] = (unsigned char)lane;
  __syncwarp();
  const int ka = __popc(mA), kb = __popc(mB);
  const int np = active ? ka * kb : 0;

  float my_ub = ub;
  bool hit = false;
  // rounds of W face pairs; between rounds the slot's lanes share the bound
  // they found, so later rounds skip pairs the earlier ones already beat
  const int np_max = __reduce_max_sync(FULL, (unsigned int)np);
  for (int p0 = 0; p0 < np_max; p0 += W) {
    if (p0 > 0)
      for (int o = W >> 1; o > 0; o >>= 1) my_ub = fminf(my_ub, __shfl_xor_sync(FULL, my_ub, o));
    const int p = p0 + k;
    if (p >= np) continue;
    const int i = p / kb, j = p - i * kb;
    const int sa = S.idx[base + i], sb = S.idx[base + H + j];
    const int fa = fa0 + (sa - base), fb = fb0 + (sb - base - H);
    float3 A0 = sface(S, sa, 0), A1 = sface(S, sa, 1), A2 = sface(S, sa, 2);
    float3 B0 = sface(S, sb, 0), B1 = sface(S, sb, 1), B2 = sface(S, sb, 2);
    lc.pre++;
    if (mode == G3D_OP_DISTANCE) {
      float lbt = __fsub_rd(tri_boxes_lb(A0, A1, A2, B0, B1, B2), slack);
      if (lbt > my_ub) continue;
      lc.tests++;
      PairBounds pb = tri_pair_bounds_rolled(S.f[sa], S.f[sb]);
      float plb = fmaxf(__fsub_rd(pb.lb, slack), 0.f);
      float pub = __fadd_ru(pb.ub, slack);
      if (pub < my_ub) my_ub = pub;
      if (plb <= my_ub) {
        int flags = 0;
        if (plb <= 0.f) {
          int r = slack == 0.f ? tri_isect_filter_s(S.f[sa], S.f[sb]) : ISECT_UNSURE;
          if (r == ISECT_YES) { hit = true; continue; }
          if (r == ISECT_UNSURE) flags = CAND_NEEDS_EXACT;
        }
        lc.cands++;
        push_candidate(a, q, fa, fb, plb, flags);
      }
    } else {
      if (!tri_boxes_overlap(A0, A1, A2, B0, B1, B2, slack)) continue;
      lc.tests++;
      int r = slack == 0.f ? tri_isect_filter_s(S.f[sa], S.f[sb]) : ISECT_UNSURE;
      if (r == ISECT_YES) { hit = true; continue; }
      if (r == ISECT_UNSURE) {
        lc.cands++;
        push_candidate(a, q, fa, fb, 0.f, CAND_NEEDS_EXACT);
      }
    }
  }
  __syncwarp();  // S is reused by the next call
  // reductions within each slot (xor offsets below W stay inside the slot)
  for (int o = W >> 1; o > 0; o >>= 1) my_ub = fminf(my_ub, __shfl_xor_sync(FULL, my_ub, o));
  const unsigned int hm = __ballot_sync(FULL, hit) & segmask;
  if (active && k == 0) {
    if (hm) {
      atomicExch(&a.st[q].done, 1);
      atomicMin(&a.st[q].ub, 0u);
    } else if (mode == G3D_OP_DISTANCE && my_ub < ub) {
      atomicMin(&a.st[q].ub, __float_as_uint(my_ub));
    }
  }
}

__device__ __forceinline__ void leaf_jobs(const TravArgs& a, const LeafJob* jobs, int njobs, int W, LeafCounters& lc,
                                          LeafStage& S) {
  leaf_jobs_t(a, jobs, njobs, W, lc, S, GlobalFaces{});
}

// one leaf pair with boxes taken from the leaf tables
__device__ __forceinline__ LeafJob leaf_job_from_tables(const TravArgs& a, int q, int la, int lb, int mode) {
  const QueryDev& Qd = a.q[q];
  LeafJob J;
  J.q = q; J.la = la; J.lb = lb; J.mode = mode;
  J.alo = __ldg(&Qd.A.leaves[2 * (~la)]); J.ahi = __ldg(&Qd.A.leaves[2 * (~la) + 1]);
  J.blo = __ldg(&Qd.B.leaves[2 * (~lb)]); J.bhi = __ldg(&Qd.B.leaves[2 * (~lb) + 1]);
  return J;
}

// rank of this lane's key among the lanes of `mask` (ascending, ties by
// lane); one shuffle per lane of the mask (the mask is the same in every lane)
__device__ __forceinline__ int rank_in_warp(unsigned int mask, float key) {
  const int lane = threadIdx.x & 31;
  int r = 0;
  for (unsigned int m = mask; m; m &= m - 1u) {
    const int s = __ffs(m) - 1;
    const float ks = __shfl_sync(FULL, key, s);
    r += (ks < key) || (ks == key && s < lane);
  }
  return r;
}

// Boxes of child pair c (0..3) of item (ra, rb): an internal node's child
// box comes from the node record, a leaf's box from the leaf table; with one
// side a leaf, children c and c + 2 coincide.
__device__ __forceinline__ void load_child_boxes(const QueryDev& Qd, int ra, int rb, int c, float4& alo,
                                                 float4& ahi, float4& blo, float4& bhi) {
  const bool ia = ra >= 0, ib = rb >= 0;
  if (ia && ib) {
    const float4* na = Qd.A.nodes + 4 * ra + 2 * (c >> 1);
    const float4* nb = Qd.B.nodes + 4 * rb + 2 * (c & 1);
    alo = __ldg(na); ahi = __ldg(na + 1);
    blo = __ldg(nb); bhi = __ldg(nb + 1);
  } else if (ia) {
    const float4* na = Qd.A.nodes + 4 * ra + 2 * (c & 1);
    alo = __ldg(na); ahi = __ldg(na + 1);
    blo = __ldg(&Qd.B.leaves[2 * (~rb)]); bhi = __ldg(&Qd.B.leaves[2 * (~rb) + 1]);
  } else if (ib) {
    const float4* nb = Qd.B.nodes + 4 * rb + 2 * (c & 1);
    blo = __ldg(nb); bhi = __ldg(nb + 1);
    alo = __ldg(&Qd.A.leaves[2 * (~ra)]); ahi = __ldg(&Qd.A.leaves[2 * (~ra) + 1]);
  }
}

// ---------------------------------------------------------------------------
// persistent traversal kernel
// ---------------------------------------------------------------------------
// Tuning constants (defaults chosen by measurement on GB300).
#ifndef G3D_TRAV_MINB
#define G3D_TRAV_MINB 2      // resident CTAs of 128 threads per SM the register budget targets
#endif
#ifndef G3D_POP_ITEMS
#define G3D_POP_ITEMS 16     // items a warp takes from the global queue at once
#endif
#ifndef G3D_DONATE_BELOW
#define G3D_DONATE_BELOW 256  // donate when fewer items than this wait in the queue
#endif
#ifndef G3D_DONATE_EVERY
#define G3D_DONATE_EVERY 1   // check the queue level every this many steps (power of 2)
#endif
#ifndef G3D_SPEC_LOADS
#define G3D_SPEC_LOADS 1     // 1: node boxes are loaded before the query's state is read
#endif
constexpr int kPopItems = 8;  // items expanded per step (4 lanes each)

__global__ void __launch_bounds__(128, G3D_TRAV_MINB) k_traverse(TravArgs a, int stack_cap) {
  extern __shared__ int4 smem_stack[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int4* stack = smem_stack + warp * stack_cap;
  WarpScratch& scr = ((WarpScratch*)(smem_stack + (blockDim.x >> 5) * stack_cap))[warp];
  const unsigned int smask = (unsigned int)stack_cap - 1u;
  const unsigned int lt = (1u << lane) - 1u;
  int cnt = 0;
  unsigned int bot = 0;
  long long owned = 0;
  unsigned long long idle_start = 0;
  unsigned long long busy_ns = 0, idle_ns = 0, t_mark = globaltimer_ns();
  bool working = false;  // the warp holds items (busy) since t_mark, else it waits for work
  int iter = 0;
  unsigned long long n_nodes = 0, n_leaf = 0, n_pushes = 0;
  LeafCounters lc;
  const unsigned long long t_start = globaltimer_ns();

  for (;;) {
    // the whole launch is bounded in time as well as every wait in it
    if ((iter & 255) == 255) {
      int late = 0;
      if (lane == 0) late = globaltimer_ns() - t_start > a.t_limit_ns;
      if (__shfl_sync(FULL, late, 0)) {
        if (lane == 0) set_error(a.queue.error, G3D_ERR_TIMEOUT);
        break;
      }
    }
    if (cnt == 0) {
      if (owned) {
        if (lane == 0) atomicAdd((unsigned long long*)a.queue.pending, (unsigned long long)(-owned));
        owned = 0;
      }
      if (working && lane == 0) {  // time since the last mark was spent working
        unsigned long long now = globaltimer_ns();
        busy_ns += now - t_mark;
        t_mark = now;
      }
      working = false;
      int4 it = make_int4(0, 0, 0, 0);
      int got = gq_pop(a.queue, it, G3D_POP_ITEMS, a.t_limit_ns);
      if (got < 0) break;
      if (got == 0) {
        // lane 0 decides for the warp: every lane must leave the loop together
        int stop = 0;
        if (lane == 0) {
          if (ld_volatile_i64(a.queue.pending) == 0 || ld_volatile_i32(a.queue.error) != 0) {
            stop = 1;
          } else {
            unsigned long long now = globaltimer_ns();
            if (idle_start == 0) idle_start = now;
            else if (now - idle_start > a.t_limit_ns) {
              set_error(a.queue.error, G3D_ERR_TIMEOUT);
              stop = 1;
            }
          }
        }
        if (__shfl_sync(FULL, stop, 0)) break;
        __nanosleep(200);
        continue;
      }
      idle_start = 0;
      if (lane == 0) {  // time since the last mark was spent waiting for work
        unsigned long long now = globaltimer_ns();
        idle_ns += now - t_mark;
        t_mark = now;
      }
      working = true;
      if (lane < got) stack[(bot + lane) & smask] = it;
      __syncwarp();
      cnt = got;
      owned = got;
    }

    // ---- expand up to 8 items, one child pair per lane --------------------
    const int P = min(cnt, kPopItems);
    const int k = lane >> 2, c = lane & 3;
    int4 item = make_int4(-1, 0, 0, 0);
    if (k < P) item = stack[(bot + cnt - 1 - k) & smask];
    __syncwarp();
    cnt -= P;
    if (k < P && !item_ok(a, item)) {
      if (c == 0) record_bad(a, 1, item);
      item.x = -1;
    }
    n_nodes += (k < P && c == 0);

    bool valid = false, leafpair = false, from_table = false;
    int4 child = make_int4(0, 0, 0, 0);
    int cmode = G3D_OP_INTERSECTS;
    float prio = 0.f;
    float4 alo, ahi, blo, bhi;
    if (k < P && item.x >= 0) {
      const int q = item.x;
      const QueryDev& Qd = a.q[q];
      const int ra = item.y, rb = item.z;
      const bool ia = ra >= 0, ib = rb >= 0;
#if G3D_SPEC_LOADS
      // the child boxes' loads are issued before, and overlap, the reads of
      // the query's state below (wasted for an item found dead)
      load_child_boxes(Qd, ra, rb, c, alo, ahi, blo, bhi);
#endif
      // distance queries first run an intersects phase (phase 0), then the
      // distance traversal (1)
      const int phase = a.st[q].phase;
      const int op = (Qd.op == G3D_OP_DISTANCE && phase >= 1) ? G3D_OP_DISTANCE : G3D_OP_INTERSECTS;
      bool dead = ld_volatile_i32(&a.st[q].done) != 0;
      float ub = __uint_as_float(ld_volatile_u32(&a.st[q].ub));
      if (!dead && op == G3D_OP_DISTANCE && __int_as_float(item.w) > ub) dead = true;
      if (!dead) {
        cmode = op;
        if (!ia && !ib) {
          if (c == 0) { valid = true; leafpair = true; child = item; from_table = true; }
        } else {
#if !G3D_SPEC_LOADS
          load_child_boxes(Qd, ra, rb, c, alo, ahi, blo, bhi);
#endif
          // both internal: 4 child pairs; one internal: its 2 children
          // against the other side's leaf box
          const bool act = (ia && ib) || c < 2;
          const int ca = ia ? __float_as_int(alo.w) : ra, cb = ib ? __float_as_int(blo.w) : rb;
          if (act) {
            float lbc = 0.f;
            if (op == G3D_OP_DISTANCE) {
              lbc = fmaxf(__fsub_rd(box_lb(alo, ahi, blo, bhi), Qd.slack), 0.f);
              valid = lbc <= ub;
              prio = -lbc;  // nearest pair popped first
            } else {
              valid = box_overlap(alo, ahi, blo, bhi, Qd.slack);
              prio = 0.f;  // natural order (ordering by overlap depth measured worse)
            }
            child = make_int4(q, ca, cb, __float_as_int(lbc));
            leafpair = ca < 0 && cb < 0;
          }
        }
      }
    }

    // ---- push internal survivors (compacted), donate on overflow ---------
    const unsigned int pm = __ballot_sync(FULL, valid && !leafpair);
    const int npush = __popc(pm);
    if (npush) {
      if (cnt + npush <= stack_cap) {
        // pushed in ascending priority, so the best child ends on top
        const int r = rank_in_warp(pm, prio);
        if (valid && !leafpair) stack[(bot + cnt + r) & smask] = child;
        __syncwarp();
        cnt += npush;
      } else {
        // stack full: hand the new items to the global queue
        int r = __popc(pm & lt);
        int4 mine = child;
        // gather survivors into lanes [0, npush)
        int4 g = make_int4(0, 0, 0, 0);
        for (int s = 0; s < 32; s++) {
          if (!((pm >> s) & 1u)) continue;
          int dst = __popc(pm & ((1u << s) - 1u));
          int4 v;
          v.x = __shfl_sync(FULL, mine.x, s); v.y = __shfl_sync(FULL, mine.y, s);
          v.z = __shfl_sync(FULL, mine.z, s); v.w = __shfl_sync(FULL, mine.w, s);
          if (lane == dst) g = v;
        }
        (void)r;
        if (!gq_push(a.queue, g, npush, a.t_limit_ns)) break;
        n_pushes += npush;
      }
    }

    // ---- leaf pairs: jobs staged in shared memory, W lanes each --------------
    const unsigned int lm = __ballot_sync(FULL, valid && leafpair);
    if (lm) {
      if (valid && leafpair) {
        LeafJob J;
        const bool ok = item_ok(a, child) && child.y < 0 && child.z < 0;
        if (!ok) {
          record_bad(a, 2, child);
          J.q = -1;
        } else if (from_table) {
          J = leaf_job_from_tables(a, child.x, child.y, child.z, cmode);
        } else {
          J.q = child.x; J.la = child.y; J.lb = child.z; J.mode = cmode;
          J.alo = alo; J.ahi = ahi; J.blo = blo; J.bhi = bhi;
        }
        scr.jobs[__popc(lm & lt)] = J;
      }
      __syncwarp();
      const int nj = __popc(lm);
      const int per = a.leaf_w == 32 ? 1 : 2;
      for (int j0 = 0; j0 < nj; j0 += per) {
        const int m = min(per, nj - j0);
        // drop invalid jobs (recorded above) by shrinking the call
        bool bad = false;
        for (int j = 0; j < m; j++) bad |= scr.jobs[j0 + j].q < 0;
        if (bad) continue;
        n_leaf += m;
        leaf_jobs(a, scr.jobs + j0, m, a.leaf_w, lc, scr.stage);
      }
      __syncwarp();
    }

    // ---- donate the bottom of the stack when the queue runs dry -----------
    if (((++iter) & (G3D_DONATE_EVERY - 1)) == 0 && cnt >= 2) {
      int starving = 0;
      if (lane == 0) {
        const unsigned long long h = ld_volatile_u64(a.queue.head), t = ld_volatile_u64(a.queue.tail);
        starving = (t - h) < (unsigned long long)G3D_DONATE_BELOW;
      }
      starving = __shfl_sync(FULL, starving, 0);
      if (starving) {
        int nd = min((cnt + 1) >> 1, 32);
        int4 g = make_int4(0, 0, 0, 0);
        if (lane < nd) g = stack[(bot + lane) & smask];
        __syncwarp();
        bot += nd;
        cnt -= nd;
        if (!gq_push(a.queue, g, nd, a.t_limit_ns)) break;
        n_pushes += nd;
      }
    }
  }

  // counters
  unsigned int pre = lc.pre, tests = lc.tests, cands = lc.cands;
  for (int o = 16; o > 0; o >>= 1) {
    n_nodes += __shfl_xor_sync(FULL, n_nodes, o);
    pre += __shfl_xor_sync(FULL, pre, o);
    tests += __shfl_xor_sync(FULL, tests, o);
    cands += __shfl_xor_sync(FULL, cands, o);
  }
  if (lane == 0 && a.stats) {
    stat_add(a.stats, ST_NODE_PAIRS, n_nodes);
    stat_add(a.stats, ST_LEAF_PAIRS, n_leaf);
    stat_add(a.stats, ST_TRI_PREFILTER, pre);
    stat_add(a.stats, ST_TRI_TESTS, tests);
    stat_add(a.stats, ST_CANDIDATES, cands);
    stat_add(a.stats, ST_QUEUE_PUSHES, n_pushes);
    const unsigned long long tail_ns = globaltimer_ns() - t_mark;
    stat_add(a.stats, ST_BUSY_NS, busy_ns + (working ? tail_ns : 0));
    stat_add(a.stats, ST_IDLE_NS, idle_ns + (working ? 0 : tail_ns));
  }
}

// ---------------------------------------------------------------------------
// level-synchronous traversal (one cooperative launch)
// ---------------------------------------------------------------------------
// All queries of the launch descend their dual trees together, one level of
// node pairs per step, instead of one warp following one path: each step
// every warp of the grid takes a share of the level's node pairs (4 lanes per
// pair, one child pair per lane), prunes the children against the query's
// current bound (distance) or by box overlap (intersects), and appends the
// surviving internal pairs to the next frontier and the leaf pairs to the
// next leaf list with one atomic per warp; before that, in the same step, the
// warps test the leaf pairs the previous step found (in batches dealt out by a
// ticket counter), so the bounds and finished queries they produce already
// prune this step's node pairs.  A grid barrier separates the steps.  With thousands of node
// pairs per level in flight the memory latency of a node read is paid once
// per level, not once per node pair along a warp's path.
//
// Every wait (the barrier) and the whole launch are bounded by the time
// limit: past it the launch records G3D_ERR_TIMEOUT and every block leaves.

// Bulk copies (the TMA engine's 1D form) from global into shared memory,
// completed on a per-warp mbarrier.  Sources and destinations are 16-byte
// aligned and sizes multiples of 16 (whole float4 ranges).
__device__ __forceinline__ unsigned int smem_addr(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned int bytes,
                                              unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Per-warp shared memory of the level-synchronous kernel (dynamic shared
// memory: kFrontierSmem bytes per block of 8 warps).
struct FrontierWarp {
  StagedLeafFaces faces[kLeafBatch];  // bulk-copied faces of the batch's leaf pairs
  LeafJob jobs[kLeafBatch];
  unsigned char idx[kLeafBatch][32];  // per job: surviving faces of A (0..), of B (16..)
  unsigned long long mbar;
};

// The face tests of a batch of `nb` staged leaf pairs (fw.jobs / fw.faces),
// with the surviving face pairs of all of them dealt out to the warp's lanes
// together.  Each leaf pair first culls its faces against the other leaf's
// box (H lanes per side: 16, or 8 for leaves of <= 8 faces, two leaf pairs
// per pass); the remaining face pairs, usually a handful per leaf pair, then
// go through the face-box prefilter and the full test (certified bounds for
// distance, the filtered orientation test for intersects) with one lane per
// face pair across the whole batch, instead of one leaf pair at a time.
// Append the calling lanes' face pair (q, fa, fb, box bound) to bucket b of
// the face-pair list (count[2 b], capacity cap each); false when that bucket
// is full (the caller then tests the pair itself).
__device__ __forceinline__ bool defer_face_pair(int4* fp, unsigned int* count, unsigned int cap, int b, int q, int fa,
                                                int fb, float lbt) {
  fp += (size_t)b * cap;
  count += 2 * b;
  const unsigned int m = __match_any_sync(__activemask(), b);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned int base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned int)__popc(m));
  base = __shfl_sync(m, base, leader);
  const unsigned int idx = base + (unsigned int)__popc(m & ((1u << lane) - 1u));
  if (idx >= cap) return false;
  fp[idx] = make_int4(q, fa, fb, __float_as_int(lbt));
  return true;
}

__device__ __forceinline__ void leaf_batch_packed(const TravArgs& a, FrontierWarp& fw, int nb, int H,
                                                  LeafCounters& lc, int4* fp = nullptr,
                                                  unsigned int* fp_count = nullptr, unsigned int fp_cap = 0) {
  const int lane = threadIdx.x & 31;
  const int W = 2 * H, per_pass = 32 / W;
  int ka[kLeafBatch], kb[kLeafBatch];
  float ub0[kLeafBatch], ubm[kLeafBatch], ubl[kLeafBatch];
#pragma unroll
  for (int t = 0; t < kLeafBatch; t++) { ka[t] = kb[t] = 0; ub0[t] = ubm[t] = 0.f; ubl[t] = INFINITY; }
  // ---- cull: face k of a side against the other leaf's box -----------------
#pragma unroll
  for (int t0 = 0; t0 < kLeafBatch; t0 += 1) {
    if (t0 % per_pass != 0 || t0 >= nb) continue;
    const int slot = lane / W, k = lane % W;
    const int t = t0 + slot;
    const bool sideB = k >= H;
    const int fi = sideB ? k - H : k;
    bool keep = false;
    if (t < nb) {
      const LeafJob& J = fw.jobs[t];
      const QueryDev& Qd = a.q[J.q];
      int f0, n;
      leaf_range(sideB ? Qd.B : Qd.A, sideB ? J.lb : J.la, f0, n);
      if (fi < n) {
        const float4* P = fw.faces[t][sideB ? 1 : 0][0];
        const float4 p0 = P[fi], p1 = P[16 + fi], p2 = P[32 + fi];
        const float4 flo = make_float4(fminf(p0.x, fminf(p1.x, p2.x)), fminf(p0.y, fminf(p1.y, p2.y)),
                                       fminf(p0.z, fminf(p1.z, p2.z)), 0.f);
        const float4 fhi = make_float4(fmaxf(p0.x, fmaxf(p1.x, p2.x)), fmaxf(p0.y, fmaxf(p1.y, p2.y)),
                                       fmaxf(p0.z, fmaxf(p1.z, p2.z)), 0.f);
        const float4 olo = sideB ? J.alo : J.blo, ohi = sideB ? J.ahi : J.bhi;
        const float ub = __uint_as_float(ld_volatile_u32(&a.st[J.q].ub));
        if (J.mode == G3D_OP_DISTANCE) keep = __fsub_rd(box_lb(flo, fhi, olo, ohi), Qd.slack) <= ub;
        else keep = box_overlap(flo, fhi, olo, ohi, Qd.slack);
      }
    }
    const unsigned int km = __ballot_sync(FULL, keep);
#pragma unroll
    for (int s = 0; s < 2; s++) {
      if (s >= per_pass || t0 + s >= nb) continue;
      const unsigned int seg = (km >> (W * s)) & (W == 32 ? FULL : ((1u << W) - 1u));
      const unsigned int mA = seg & ((1u << H) - 1u), mB = (seg >> H) & ((1u << H) - 1u);
      ka[t0 + s] = __popc(mA);
      kb[t0 + s] = __popc(mB);
    }
    if (keep) {
      const unsigned int seg = (km >> (W * slot)) & (W == 32 ? FULL : ((1u << W) - 1u));
      const unsigned int m = sideB ? (seg >> H) & ((1u << H) - 1u) : seg & ((1u << H) - 1u);
      fw.idx[t][(sideB ? 16 : 0) + __popc(m & ((1u << fi) - 1u))] = (unsigned char)fi;
    }
  }
  __syncwarp();
  int off[kLeafBatch + 1];
  off[0] = 0;
#pragma unroll
  for (int t = 0; t < kLeafBatch; t++) {
    off[t + 1] = off[t] + (t < nb ? ka[t] * kb[t] : 0);
    if (t < nb) {
      ub0[t] = __uint_as_float(ld_volatile_u32(&a.st[fw.jobs[t].q].ub));
      ubm[t] = ub0[t];
    }
  }
  // ---- face pairs of the whole batch, one lane each ------------------------
  // After each round of 32 face pairs the lanes share the bounds they found
  // (and read the queries' current bounds), so the later rounds of a leaf
  // pair with many candidates skip the full test of pairs the earlier ones
  // already beat.
  unsigned int hits = 0;
  const int P = off[kLeafBatch];
  for (int p0 = 0; p0 < P; p0 += 32) {
    if (p0 > 0) {
#pragma unroll
      for (int u = 0; u < kLeafBatch; u++) {
        if (u >= nb || fw.jobs[u].mode != G3D_OP_DISTANCE) continue;
        float m = fminf(ubm[u], __uint_as_float(ld_volatile_u32(&a.st[fw.jobs[u].q].ub)));
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(FULL, m, o));
        ubm[u] = m;
      }
    }
    const int p = p0 + lane;
    if (p >= P) continue;
    int t = 0;
#pragma unroll
    for (int u = 1; u < kLeafBatch; u++) t += p >= off[u];
    int r = p, nbt = 1;
#pragma unroll
    for (int u = 0; u < kLeafBatch; u++)
      if (u == t) { r = p - off[u]; nbt = kb[u]; }
    const int i = r / nbt, j = r - i * nbt;
    const LeafJob& J = fw.jobs[t];
    const QueryDev& Qd = a.q[J.q];
    const float slack = Qd.slack;
    const int sa = fw.idx[t][i], sb = fw.idx[t][16 + j];
    const float* FA = &fw.faces[t][0][0][sa].x;
    const float* FB = &fw.faces[t][1][0][sb].x;
    const float3 A0 = make_float3(FA[0], FA[1], FA[2]), A1 = make_float3(FA[64], FA[65], FA[66]),
                 A2 = make_float3(FA[128], FA[129], FA[130]);
    const float3 B0 = make_float3(FB[0], FB[1], FB[2]), B1 = make_float3(FB[64], FB[65], FB[66]),
                 B2 = make_float3(FB[128], FB[129], FB[130]);
    float my_ub = 0.f;
#pragma unroll
    for (int u = 0; u < kLeafBatch; u++)
      if (u == t) my_ub = ubm[u];
    int fa0, na, fb0, nbb;
    leaf_range(Qd.A, J.la, fa0, na);
    leaf_range(Qd.B, J.lb, fb0, nbb);
    lc.pre++;
    if (J.mode == G3D_OP_DISTANCE) {
      const float lbt = __fsub_rd(tri_boxes_lb(A0, A1, A2, B0, B1, B2), slack);
      if (lbt > my_ub) continue;
      if (fp) {
        const int bk = lbt <= 0.125f * my_ub ? 0 : (lbt <= 0.25f * my_ub ? 1 : (lbt <= 0.5f * my_ub ? 2 : 3));
        if (defer_face_pair(fp, fp_count, fp_cap, bk, J.q, fa0 + sa, fb0 + sb, lbt)) continue;
      }
      lc.tests++;
      const PairBounds pb = tri_pair_bounds_rolled_s<64>(FA, FB);
      const float plb = fmaxf(__fsub_rd(pb.lb, slack), 0.f);
      const float pub = __fadd_ru(pb.ub, slack);
      if (pub < my_ub) {
        my_ub = pub;
#pragma unroll
        for (int u = 0; u < kLeafBatch; u++)
          if (u == t) ubm[u] = pub;
      }
      if (plb <= my_ub) {
        int flags = 0;
        if (plb <= 0.f) {
          const int rr = slack == 0.f ? tri_isect_filter_ss<64>(FA, FB) : ISECT_UNSURE;
          if (rr == ISECT_YES) { hits |= 1u << t; continue; }
          if (rr == ISECT_UNSURE) flags = CAND_NEEDS_EXACT;
        }
        lc.cands++;
        push_candidate(a, J.q, fa0 + sa, fb0 + sb, plb, flags);
      }
    } else {
      if (!tri_boxes_overlap(A0, A1, A2, B0, B1, B2, slack)) continue;
      if (fp && defer_face_pair(fp, fp_count, fp_cap, 0, J.q, fa0 + sa, fb0 + sb, 0.f)) continue;
      lc.tests++;
      const int rr = slack == 0.f ? tri_isect_filter_ss<64>(FA, FB) : ISECT_UNSURE;
      if (rr == ISECT_YES) { hits |= 1u << t; continue; }
      if (rr == ISECT_UNSURE) {
        lc.cands++;
        push_candidate(a, J.q, fa0 + sa, fb0 + sb, 0.f, CAND_NEEDS_EXACT);
      }
      // a distance query of the same mesh pair runs after this intersects
      // traversal: these nearby face pairs give it a certified bound to
      // start from (it still finds and finalises its own candidates)
      if (Qd.dlink >= 0) {
        const PairBounds pb = tri_pair_bounds_rolled_s<64>(FA, FB);
        const float pub = __fadd_ru(pb.ub, slack);
#pragma unroll
        for (int u = 0; u < kLeafBatch; u++)
          if (u == t) ubl[u] = fminf(ubl[u], pub);
      }
    }
  }
  // ---- per leaf pair: certified intersection or a lower bound ---------------
#pragma unroll
  for (int t = 0; t < kLeafBatch; t++) {
    if (t >= nb) continue;
    float m = ubm[t];
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(FULL, m, o));
    const bool hit = __any_sync(FULL, (hits >> t) & 1u);
    float ml = ubl[t];
    for (int o = 16; o > 0; o >>= 1) ml = fminf(ml, __shfl_xor_sync(FULL, ml, o));
    if (lane == 0) {
      const int q = fw.jobs[t].q;
      if (hit) {
        atomicExch(&a.st[q].done, 1);
        atomicMin(&a.st[q].ub, 0u);
      } else if (fw.jobs[t].mode == G3D_OP_DISTANCE && m < ub0[t]) {
        atomicMin(&a.st[q].ub, __float_as_uint(m));
      }
      const int lq = a.q[q].dlink;
      if (fw.jobs[t].mode == G3D_OP_INTERSECTS && lq >= 0 && lq < a.nq && ml < INFINITY)
        atomicMin(&a.st[lq].ub, __float_as_uint(ml));
    }
  }
  __syncwarp();  // fw is reused by the next batch
}

// The operation an item of query q is traversed for (distance queries run
// the intersects traversal in phase 0).
__device__ __forceinline__ int item_op(const TravArgs& a, int q) {
  return (a.q[q].op == G3D_OP_DISTANCE && a.st[q].phase >= 1) ? G3D_OP_DISTANCE : G3D_OP_INTERSECTS;
}

// The deferred face pairs of a level over the whole grid, one face pair per
// half-warp: both faces loaded from global memory, then the full test
// (certified bounds, the filtered orientation test) with its terms spread
// over the 16 lanes (tri_pair_bounds_hw, tri_isect_filter_hw), against the
// query's current bound.  The work per pair is alike, so the step ends evenly
// however the pairs were spread over the leaf pairs, and each pair's chain of
// dependent operations is short.
__device__ void face_pair_stage(const TravArgs& a, const int4* __restrict__ fp, unsigned int n, long long gw,
                                long long total_w, LeafCounters& lc) {
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4, f = lane & 15;
  for (long long e0 = gw * 2; e0 < (long long)n; e0 += total_w * 2) {
    const long long e = e0 + half;
    bool active = e < (long long)n;
    int4 it = active ? fp[e] : make_int4(0, 0, 0, 0);
    int q = it.x, fa = it.y, fb = it.z;
    if (active && (q < 0 || q >= a.nq || fa < 0 || fb < 0 || fa >= a.q[q].A.ntri || fb >= a.q[q].B.ntri)) {
      if (f == 0) record_bad(a, 6, it);
      active = false;
    }
    if (active && ld_volatile_i32(&a.st[q].done)) active = false;
    int op = G3D_OP_INTERSECTS, lq = -1;
    float slack = 0.f, ub = INFINITY;
    float3 A0, A1, A2, B0, B1, B2;
    A0 = A1 = A2 = B0 = B1 = B2 = make_float3(0.f, 0.f, 0.f);
    if (active) {
      const QueryDev& Qd = a.q[q];
      op = item_op(a, q);
      slack = Qd.slack;
      lq = op == G3D_OP_INTERSECTS ? Qd.dlink : -1;
      if (lq >= a.nq) lq = -1;
      ub = __uint_as_float(ld_volatile_u32(&a.st[q].ub));
      if (op == G3D_OP_DISTANCE && __int_as_float(it.w) > ub) active = false;
      if (active) {
        A0 = f3(__ldg(&Qd.A.v0[fa])); A1 = f3(__ldg(&Qd.A.v1[fa])); A2 = f3(__ldg(&Qd.A.v2[fa]));
        B0 = f3(__ldg(&Qd.B.v0[fb])); B1 = f3(__ldg(&Qd.B.v1[fb])); B2 = f3(__ldg(&Qd.B.v2[fb]));
      }
    }
    if (active && f == 0) lc.tests++;
    // certified bounds: distance pairs, and intersects pairs that seed a
    // linked distance query
    const bool need_b = active && (op == G3D_OP_DISTANCE || lq >= 0);
    PairBounds pb;
    pb.lb = 0.f;
    pb.ub = INFINITY;
    if (__any_sync(FULL, need_b)) pb = tri_pair_bounds_hw(A0, A1, A2, B0, B1, B2);
    const float plb = fmaxf(__fsub_rd(pb.lb, slack), 0.f);
    const float pub = __fadd_ru(pb.ub, slack);
    const bool need_f = active && slack == 0.f &&
                        (op == G3D_OP_INTERSECTS || plb <= fminf(ub, pub)) && (op == G3D_OP_INTERSECTS || plb <= 0.f);
    int r = ISECT_UNSURE;
    if (__any_sync(FULL, need_f)) r = tri_isect_filter_hw(A0, A1, A2, B0, B1, B2);
    if (!need_f) r = ISECT_UNSURE;  // slack > 0: the exact stage decides
    if (!active || f != 0) continue;
    if (op == G3D_OP_DISTANCE) {
      if (pub < ub) atomicMin(&a.st[q].ub, __float_as_uint(pub));
      if (plb <= fminf(ub, pub)) {
        int flags = 0;
        if (plb <= 0.f) {
          if (r == ISECT_YES) {
            atomicExch(&a.st[q].done, 1);
            atomicMin(&a.st[q].ub, 0u);
            continue;
          }
          if (r == ISECT_UNSURE) flags = CAND_NEEDS_EXACT;
        }
        lc.cands++;
        push_candidate(a, q, fa, fb, plb, flags);
      }
    } else {
      if (r == ISECT_YES) {
        atomicExch(&a.st[q].done, 1);
        continue;
      }
      if (r == ISECT_UNSURE) {
        lc.cands++;
        push_candidate(a, q, fa, fb, 0.f, CAND_NEEDS_EXACT);
      }
      // a distance query of the same mesh pair runs after this intersects
      // traversal: the nearby face pair gives it a certified bound
      if (lq >= 0 && pub < __uint_as_float(ld_volatile_u32(&a.st[lq].ub))) atomicMin(&a.st[lq].ub, __float_as_uint(pub));
    }
  }
}

// Grid barrier over the co-resident blocks of a cooperative launch.  Returns
// false if the limit passed or an error was recorded (the caller leaves).
__device__ bool grid_sync(const FrontierArgs& f, int* err, unsigned long long tlim) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int gen, arrived;
    // the block's writes (frontier items, bounds) are released with its arrival
    __threadfence();
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(gen) : "l"(&f.bar[1]) : "memory");
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&f.bar[0]) : "memory");
    if (arrived == (unsigned int)f.nblocks - 1u) {
      f.bar[0] = 0u;
      asm volatile("red.release.gpu.add.u32 [%0], 1;" ::"l"(&f.bar[1]) : "memory");
    } else {
      const unsigned long long t0 = globaltimer_ns();
      int spins = 0;
      for (;;) {
        unsigned int g;
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(g) : "l"(&f.bar[1]) : "memory");
        if (g != gen) break;
        if (ld_volatile_i32(err) != 0) { ok = 0; break; }
        if ((++spins & 63) == 0 && globaltimer_ns() - t0 > tlim) {
          set_error(err, G3D_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (spins > 1024) __nanosleep(64);  // short waits spin without sleeping
      }
    }
    __threadfence();
    s_ok = ok && ld_volatile_i32(err) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// First visit of node / leaf `ref` of side `side` of query q: the distinct
// internal nodes and faces a query reads (algorithmic-bytes counters).
__device__ __forceinline__ void mark_visit(const TravArgs& a, int q, int side, int ref, unsigned long long& nodes,
                                           unsigned long long& faces) {
  const QueryDev& Qd = a.q[q];
  const MeshDev& M = side ? Qd.B : Qd.A;
  long long bit = a.visit_off[q] + (side ? 2ll * Qd.A.nleaf - 1 : 0);
  bit += ref >= 0 ? ref : (M.nleaf - 1) + (~ref);
  const unsigned int m = 1u << (bit & 31);
  if (atomicOr(&a.visit[bit >> 5], m) & m) return;
  if (ref >= 0) {
    nodes++;
  } else {
    const int first = (~ref) * M.L;
    faces += (unsigned long long)min(M.L, M.ntri - first);
  }
}

// Append the lanes' items flagged `mine` to buf (count at *count, capacity
// cap); items past the capacity go to the global queue instead.
__device__ bool frontier_append(const TravArgs& a, int4* buf, unsigned int* count, unsigned int cap, bool mine,
                                int4 v, unsigned long long& n_pushes) {
  const unsigned int m = __ballot_sync(FULL, mine);
  if (!m) return true;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned int base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned int)__popc(m));
  base = __shfl_sync(FULL, base, leader);
  const unsigned int idx = base + (unsigned int)__popc(m & ((1u << lane) - 1u));
  const bool fits = idx < cap;
  if (mine && fits) buf[idx] = v;
  const unsigned int om = __ballot_sync(FULL, mine && !fits);
  if (!om) return true;
  int4 g = make_int4(0, 0, 0, 0);
  for (unsigned int r = om; r; r &= r - 1u) {
    const int src = __ffs(r) - 1;
    const int dst = __popc(om & ((1u << src) - 1u));
    int4 w;
    w.x = __shfl_sync(FULL, v.x, src); w.y = __shfl_sync(FULL, v.y, src);
    w.z = __shfl_sync(FULL, v.z, src); w.w = __shfl_sync(FULL, v.w, src);
    if (lane == dst) g = w;
  }
  n_pushes += (unsigned long long)__popc(om);
  const int r = gq_push_n(a.queue, g, __popc(om), a.t_limit_ns, true);
  if (r >= 0) return r == 1;
  // neither the list nor the global queue has room: the items are dropped
  // and their queries marked, so that the second pass reruns them from
  // their roots (k_prepare_pass2)
  if (mine && !fits && v.x >= 0 && v.x < a.nq) atomicExch(&a.st[v.x].overflow, 1);
  return true;
}

// Child pair c (0..3) of node-pair item (q, refA, refB, bound), tested by
// its boxes' lower bound against the query's current bound (distance) or by
// their overlap (intersects): `valid` when it survives, `leafpair` when both
// sides are leaves.  Items of finished queries, or whose own bound exceeds
// the query's, yield nothing.
__device__ __forceinline__ void expand_child(const TravArgs& a, int4 item, int c, bool& valid, bool& leafpair,
                                             int4& child, unsigned long long& d_nodes, unsigned long long& d_faces) {
  const int q = item.x;
  const QueryDev& Qd = a.q[q];
  const int ra = item.y, rb = item.z;
  const bool ia = ra >= 0, ib = rb >= 0;
  float4 alo, ahi, blo, bhi;
  if (ia || ib) load_child_boxes(Qd, ra, rb, c, alo, ahi, blo, bhi);
  if (a.visit && c == 0) {
    if (ia) mark_visit(a, q, 0, ra, d_nodes, d_faces);
    if (ib) mark_visit(a, q, 1, rb, d_nodes, d_faces);
  }
  const int op = item_op(a, q);
  bool dead = ld_volatile_i32(&a.st[q].done) != 0;
  const float ub = __uint_as_float(ld_volatile_u32(&a.st[q].ub));
  if (!dead && op == G3D_OP_DISTANCE && __int_as_float(item.w) > ub) dead = true;
  if (!dead) {
    if (!ia && !ib) {  // a leaf-leaf root (both meshes a single leaf)
      if (c == 0) { valid = true; leafpair = true; child = item; }
    } else if ((ia && ib) || c < 2) {
      const int ca = ia ? __float_as_int(alo.w) : ra, cb = ib ? __float_as_int(blo.w) : rb;
      float lbc = 0.f;
      if (op == G3D_OP_DISTANCE) {
        lbc = fmaxf(__fsub_rd(box_lb(alo, ahi, blo, bhi), Qd.slack), 0.f);
        valid = lbc <= ub;
      } else {
        valid = box_overlap(alo, ahi, blo, bhi, Qd.slack);
      }
      child = make_int4(q, ca, cb, __float_as_int(lbc));
      leafpair = ca < 0 && cb < 0;
    }
  }
}

#ifndef G3D_FRONTIER_MINB
#define G3D_FRONTIER_MINB 2  // resident CTAs of 256 threads per SM the register budget targets
#endif

__global__ void __launch_bounds__(256, G3D_FRONTIER_MINB) k_frontier(TravArgs a, FrontierArgs f) {
  extern __shared__ __align__(16) unsigned char frontier_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  FrontierWarp& fw = ((FrontierWarp*)frontier_smem)[warp];
  if (lane == 0) {
    mbar_init(&fw.mbar, 1u);
    fence_proxy_async();
  }
  __syncwarp();
  unsigned int parity = 0;
  const long long gw = (long long)blockIdx.x * nwarps + warp;
  const long long total_w = (long long)gridDim.x * nwarps;
  unsigned long long n_nodes = 0, n_leaf = 0, n_pushes = 0, d_nodes = 0, d_faces = 0;
  LeafCounters lc;
  const unsigned long long t_start = globaltimer_ns();
  int lvl = 0;
  for (;; lvl++) {
    const int cur = lvl & 1, nxt = cur ^ 1;
    const unsigned int nF = min(ld_volatile_u32(&f.cnt[lvl % 3]), (unsigned int)f.fcap);
    const unsigned int nL = min(ld_volatile_u32(&f.cnt[3 + lvl % 3]), (unsigned int)f.lcap);
    if (nF == 0 && nL == 0) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const int z = (lvl + 2) % 3;
      f.cnt[z] = 0u;
      f.cnt[3 + z] = 0u;
      f.cnt[6 + z] = 0u;
      for (int b = 0; b < kFPBuckets; b++)  // face pairs of the next level (last read by the previous one)
        f.cnt[16 + 2 * b + ((lvl + 1) & 1)] = 0u;
    }
    unsigned long long* trace_e = nullptr;
    unsigned long long t_lvl = 0;
    if (f.trace && blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned int slot = atomicAdd(f.trace_next, 1u) & (unsigned int)(f.trace_cap - 1);
      trace_e = f.trace + 6ull * slot;
      t_lvl = globaltimer_ns();
      trace_e[0] = t_lvl - t_start;
      trace_e[1] = (unsigned long long)lvl;
      trace_e[2] = nF;
      trace_e[3] = nL;
    }
    if (lane == 0 && globaltimer_ns() - t_start > a.t_limit_ns) set_error(a.queue.error, G3D_ERR_TIMEOUT);

    // ---- leaf pairs found by the previous level ------------------------------
    // Warps take batches of up to kLeafBatch leaf pairs (fewer when the level
    // has few per warp); the batch's faces come into shared memory by bulk
    // copies, one memory round trip per batch, then its leaf pairs are tested
    // one after another from shared memory.
    const int4* Lin = f.L[cur];
    const unsigned int per_w = nL / (unsigned int)total_w;
    int JB = 1;  // the largest power of 2 up to both kLeafBatch and the leaf pairs per warp
    while (2 * JB <= kLeafBatch && (unsigned int)(2 * JB) <= per_w) JB *= 2;
    // The first batch of every warp is fixed by its index (no ticket); the
    // rest are handed out by a ticket counter past those, which no warp
    // touches when the first batches cover the level (a level of few leaf
    // pairs then costs no same-address atomics from the grid's warps).
    const unsigned long long n_static = (unsigned long long)total_w * (unsigned long long)JB;
    bool leaf_ok = true;
    for (bool first = true;; first = false) {
      unsigned long long t = 0;
      if (first) {
        t = (unsigned long long)gw * (unsigned long long)JB;
      } else {
        if (n_static >= nL) break;
        if (lane == 0) t = n_static + atomicAdd(&f.cnt[6 + lvl % 3], (unsigned int)JB);
        t = __shfl_sync(FULL, t, 0);
      }
      if (t >= nL) break;
      const int nj = min(JB, (int)(nL - t));
      LeafJob J;
      J.q = -1;
      int fa0 = 0, na = 0, fb0 = 0, nb = 0;
      const QueryDev* Qp = nullptr;
      if (lane < nj) {
        const int4 it = Lin[t + lane];
        if (!item_ok(a, it) || it.y >= 0 || it.z >= 0) {
          record_bad(a, 5, it);
        } else {
          const int q = it.x;
          const int op = item_op(a, q);
          const bool dead = ld_volatile_i32(&a.st[q].done) != 0 ||
                            (op == G3D_OP_DISTANCE &&
                             __int_as_float(it.w) > __uint_as_float(ld_volatile_u32(&a.st[q].ub)));
          if (!dead) {
            J = leaf_job_from_tables(a, q, it.y, it.z, op);
            Qp = &a.q[q];
            leaf_range(Qp->A, it.y, fa0, na);
            leaf_range(Qp->B, it.z, fb0, nb);
          }
        }
      }
      const bool live = J.q >= 0;
      const unsigned int lm = __ballot_sync(FULL, live);
      const int nlive = __popc(lm);
      if (nlive == 0) continue;
      const int slot = __popc(lm & ((1u << lane) - 1u));
      const unsigned int bytes = live ? (unsigned int)(na + nb) * 48u : 0u;
      const unsigned int total = __reduce_add_sync(FULL, bytes);
      if (live) fw.jobs[slot] = J;
      __syncwarp();
      if (lane == 0) {
        fence_proxy_async();  // earlier reads of the staging area come before the copies' writes
        mbar_arrive_expect_tx(&fw.mbar, total);
      }
      __syncwarp();
      if (live) {
        float4* dA = fw.faces[slot][0][0];
        float4* dB = fw.faces[slot][1][0];
        const unsigned int ba = (unsigned int)na * 16u, bb = (unsigned int)nb * 16u;
        bulk_copy_g2s(dA, Qp->A.v0 + fa0, ba, &fw.mbar);
        bulk_copy_g2s(dA + 16, Qp->A.v1 + fa0, ba, &fw.mbar);
        bulk_copy_g2s(dA + 32, Qp->A.v2 + fa0, ba, &fw.mbar);
        bulk_copy_g2s(dB, Qp->B.v0 + fb0, bb, &fw.mbar);
        bulk_copy_g2s(dB + 16, Qp->B.v1 + fb0, bb, &fw.mbar);
        bulk_copy_g2s(dB + 32, Qp->B.v2 + fb0, bb, &fw.mbar);
      }
      // wait for the batch's copies (bounded)
      {
        const unsigned long long t0 = globaltimer_ns();
        int spins = 0;
        bool ok = true;
        while (!mbar_try_wait(&fw.mbar, parity)) {
          if ((++spins & 63) == 0 && globaltimer_ns() - t0 > a.t_limit_ns) {
            ok = false;
            break;
          }
        }
        parity ^= 1u;
        if (!__all_sync(FULL, ok)) {
          if (lane == 0) set_error(a.queue.error, G3D_ERR_TIMEOUT);
          leaf_ok = false;
          break;
        }
      }
      if (a.visit && lane < nlive) {
        mark_visit(a, fw.jobs[lane].q, 0, fw.jobs[lane].la, d_nodes, d_faces);
        mark_visit(a, fw.jobs[lane].q, 1, fw.jobs[lane].lb, d_nodes, d_faces);
      }
      n_leaf += nlive;
      leaf_batch_packed(a, fw, nlive, a.leaf_w == 32 ? 16 : 8, lc, f.FP, &f.cnt[16 + (lvl & 1)],
                        (unsigned int)(f.fpcap / kFPBuckets));
    }
    if (!leaf_ok) break;
    // ---- the face pairs the leaf tests deferred, over the whole grid ---------
    if (!grid_sync(f, a.queue.error, a.t_limit_ns)) break;
    for (int b = 0; b < kFPBuckets; b++) {  // nearest bucket first
      const unsigned int bcap = (unsigned int)(f.fpcap / kFPBuckets);
      const unsigned int nFP = min(ld_volatile_u32(&f.cnt[16 + 2 * b + (lvl & 1)]), bcap);
      face_pair_stage(a, f.FP + (size_t)b * bcap, nFP, gw, total_w, lc);
    }
    if (trace_e) trace_e[4] = globaltimer_ns() - t_lvl;

    // ---- expand this level's node pairs: 8 per warp pass ---------------------
    const int4* Fin = f.F[cur];
    const int k = lane >> 2, c = lane & 3;
    for (long long b0 = gw * 8; b0 < (long long)nF; b0 += total_w * 8) {
      const long long ii = b0 + k;
      bool have = ii < (long long)nF;
      int4 item = have ? Fin[ii] : make_int4(-1, 0, 0, 0);
      if (have && !item_ok(a, item)) {
        if (c == 0) record_bad(a, 4, item);
        have = false;
      }
      n_nodes += (have && c == 0);
      bool valid = false, leafpair = false;
      int4 child = make_int4(0, 0, 0, 0);
      if (have) expand_child(a, item, c, valid, leafpair, child, d_nodes, d_faces);
      if (!frontier_append(a, f.F[nxt], &f.cnt[(lvl + 1) % 3], (unsigned int)f.fcap, valid && !leafpair, child,
                           n_pushes))
        break;
      if (!frontier_append(a, f.L[nxt], &f.cnt[3 + (lvl + 1) % 3], (unsigned int)f.lcap, valid && leafpair, child,
                           n_pushes))
        break;
    }
    if (trace_e) trace_e[5] = globaltimer_ns() - t_lvl;

    if (!grid_sync(f, a.queue.error, a.t_limit_ns)) break;
  }

  unsigned int pre = lc.pre, tests = lc.tests, cands = lc.cands;
  for (int o = 16; o > 0; o >>= 1) {
    n_nodes += __shfl_xor_sync(FULL, n_nodes, o);
    pre += __shfl_xor_sync(FULL, pre, o);
    tests += __shfl_xor_sync(FULL, tests, o);
    cands += __shfl_xor_sync(FULL, cands, o);
    d_nodes += __shfl_xor_sync(FULL, d_nodes, o);
    d_faces += __shfl_xor_sync(FULL, d_faces, o);
  }
  if (lane == 0 && a.stats) {
    stat_add(a.stats, ST_NODE_PAIRS, n_nodes);
    stat_add(a.stats, ST_LEAF_PAIRS, n_leaf);
    stat_add(a.stats, ST_TRI_PREFILTER, pre);
    stat_add(a.stats, ST_TRI_TESTS, tests);
    stat_add(a.stats, ST_CANDIDATES, cands);
    stat_add(a.stats, ST_QUEUE_PUSHES, n_pushes);
    stat_add(a.stats, ST_DISTINCT_NODES, d_nodes);
    stat_add(a.stats, ST_DISTINCT_FACES, d_faces);
    if (blockIdx.x == 0 && warp == 0) stat_add(a.stats, ST_LEVELS, (unsigned long long)lvl);
  }
}

size_t frontier_smem_bytes() { return 8 * sizeof(FrontierWarp); }

// The first levels of a launch, while the frontier is narrow (at most
// `max_items` node pairs), in one block of 1,024 threads: the same expansion
// as k_frontier with a block barrier between levels instead of a grid
// barrier, which costs a few microseconds per level less.  Leaf pairs it finds
// go to the first leaf list; the frontier it stops at (the first one wider
// than max_items, or empty) becomes the cooperative kernel's first level.
// Pairs that do not fit go to the global queue.
__global__ void __launch_bounds__(1024) k_frontier_top(TravArgs a, FrontierArgs f, unsigned int max_items) {
  __shared__ unsigned int s_n[2], s_l;
  __shared__ int s_err;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_n[0] = min(f.cnt[0], (unsigned int)f.fcap);
    s_n[1] = 0u;
    s_l = min(f.cnt[3], (unsigned int)f.lcap);
    s_err = 0;
  }
  __syncthreads();
  unsigned long long n_nodes = 0, n_pushes = 0, d_nodes = 0, d_faces = 0;
  int cur = 0, lvl = 0;
  for (;; lvl++) {
    const unsigned int n = s_n[cur];
    if (n == 0u || n > max_items || s_err) break;  // block-uniform
    const int nxt = cur ^ 1;
    const int k = threadIdx.x >> 2, c = threadIdx.x & 3;
    for (unsigned int b0 = 0; b0 < n; b0 += blockDim.x >> 2) {
      const unsigned int ii = b0 + (unsigned int)k;
      bool have = ii < n;
      int4 item = have ? f.F[cur][ii] : make_int4(-1, 0, 0, 0);
      if (have && !item_ok(a, item)) {
        if (c == 0) record_bad(a, 7, item);
        have = false;
      }
      n_nodes += (have && c == 0);
      bool valid = false, leafpair = false;
      int4 child = make_int4(0, 0, 0, 0);
      if (have) expand_child(a, item, c, valid, leafpair, child, d_nodes, d_faces);
      // block-shared counters: one shared atomic per warp and list
      const unsigned int lt = (1u << lane) - 1u;
      const unsigned int pm = __ballot_sync(FULL, valid && !leafpair), lm = __ballot_sync(FULL, valid && leafpair);
      unsigned int pb = 0, lb = 0;
      if (lane == 0 && pm) pb = atomicAdd(&s_n[nxt], (unsigned int)__popc(pm));
      if (lane == 0 && lm) lb = atomicAdd(&s_l, (unsigned int)__popc(lm));
      pb = __shfl_sync(FULL, pb, 0);
      lb = __shfl_sync(FULL, lb, 0);
      const unsigned int pi = pb + (unsigned int)__popc(pm & lt), li = lb + (unsigned int)__popc(lm & lt);
      const bool pfit = pi < (unsigned int)f.fcap, lfit = li < (unsigned int)f.lcap;
      if (valid && !leafpair && pfit) f.F[nxt][pi] = child;
      if (valid && leafpair && lfit) f.L[0][li] = child;
      // what does not fit goes to the global queue
      const unsigned int om = __ballot_sync(FULL, valid && ((!leafpair && !pfit) || (leafpair && !lfit)));
      if (om) {
        int4 g = make_int4(0, 0, 0, 0);
        for (unsigned int r = om; r; r &= r - 1u) {
          const int src = __ffs(r) - 1;
          const int dst = __popc(om & ((1u << src) - 1u));
          int4 w;
          w.x = __shfl_sync(FULL, child.x, src); w.y = __shfl_sync(FULL, child.y, src);
          w.z = __shfl_sync(FULL, child.z, src); w.w = __shfl_sync(FULL, child.w, src);
          if (lane == dst) g = w;
        }
        n_pushes += (unsigned long long)__popc(om);
        const int r = gq_push_n(a.queue, g, __popc(om), a.t_limit_ns, true);
        if (r == 0 && lane == 0) s_err = 1;
        if (r < 0 && valid && ((!leafpair && !pfit) || (leafpair && !lfit)) && child.x >= 0 && child.x < a.nq)
          atomicExch(&a.st[child.x].overflow, 1);  // rerun by the second pass
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_n[nxt] = min(s_n[nxt], (unsigned int)f.fcap);
      s_l = min(s_l, (unsigned int)f.lcap);
      s_n[cur] = 0u;
    }
    cur = nxt;
    __syncthreads();
  }
  // the frontier reached becomes level 0 of the cooperative kernel (F[0])
  const unsigned int n = s_n[cur];
  if (cur == 1)
    for (unsigned int i = threadIdx.x; i < n; i += blockDim.x) f.F[0][i] = f.F[1][i];
  __syncthreads();
  if (threadIdx.x == 0) {
    f.cnt[0] = n;
    f.cnt[3] = s_l;
  }
  for (int o = 16; o > 0; o >>= 1) {
    n_nodes += __shfl_xor_sync(FULL, n_nodes, o);
    d_nodes += __shfl_xor_sync(FULL, d_nodes, o);
    d_faces += __shfl_xor_sync(FULL, d_faces, o);
  }
  if (lane == 0 && a.stats) {
    stat_add(a.stats, ST_NODE_PAIRS, n_nodes);
    stat_add(a.stats, ST_QUEUE_PUSHES, n_pushes);
    stat_add(a.stats, ST_DISTINCT_NODES, d_nodes);
    stat_add(a.stats, ST_DISTINCT_FACES, d_faces);
    if (threadIdx.x == 0) stat_add(a.stats, ST_LEVELS, (unsigned long long)lvl);
  }
}

// Reset every query's state and the candidate pool (single block).
__global__ void k_reset_state(TravArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.cand.count = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.nq; q += gridDim.x * blockDim.x) {
    QueryState s;
    s.ub = __float_as_uint(INFINITY);
    s.done = 0;
    s.ncand = 0;
    s.overflow = 0;
    s.best = __double_as_longlong(INFINITY);
    s.hit = 0;
    s.status = 0;
    s.pass = 1;
    s.phase = 0;
    s.nprop = 0;
    s.witness = ~0ull;
    s.label = -1;
    s.ub_seed = __float_as_uint(INFINITY);
    a.st[q] = s;
  }
}

// Seed the frontier with one root pair per query that takes part in this
// launch (single block) and clear the level counters and the barrier.
//   which 0: intersects queries, and distance queries without a linked
//            intersects query when seed_distance is set (their intersects
//            phase);
//   which 1: the distance phase of every unfinished distance query;
//   which 2: both operators at once (intersects queries, and distance
//            queries straight in their distance phase).
// the frontier's counters and grid barrier start at zero (one block, before
// k_frontier_seed)
__global__ void k_frontier_zero(FrontierArgs f) {
  if (threadIdx.x < 28) f.cnt[threadIdx.x] = 0u;
  if (threadIdx.x < 2) f.bar[threadIdx.x] = 0u;
}

// the root pairs of the queries the phase traverses, over the grid (one
// atomic per warp; the order of the first frontier does not matter)
__global__ void k_frontier_seed(TravArgs a, FrontierArgs f, int which, int seed_distance) {
  const int lane = threadIdx.x & 31;
  const int q0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  if (q0 >= a.nq) return;  // whole warps leave together
  const int q = q0 + lane;
  bool take = false;
  int4 item = make_int4(0, 0, 0, 0);
  if (q < a.nq) {
    const QueryDev& Qd = a.q[q];
    if (which == 0) {
      take = Qd.op == G3D_OP_INTERSECTS || (seed_distance && Qd.link < 0);
    } else {
      if (Qd.op == G3D_OP_DISTANCE) {
        a.st[q].phase = 1;
        a.st[q].ub_seed = a.st[q].ub;
        const int l = Qd.link;
        if (which == 1 && l >= 0 && a.st[l].done) {  // the linked intersects query certified a hit
          a.st[q].done = 1;
          a.st[q].ub = 0u;
        }
        take = !a.st[q].done;
      } else {
        take = which == 2;
      }
    }
    item = make_int4(q, Qd.A.root, Qd.B.root, 0);
  }
  const unsigned int m = __ballot_sync(0xffffffffu, take);
  if (!m) return;
  unsigned int base = 0;
  if (lane == 0) base = atomicAdd(&f.cnt[0], (unsigned int)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  const unsigned int k = base + (unsigned int)__popc(m & ((1u << lane) - 1u));
  if (take && k < (unsigned int)f.fcap) f.F[0][k] = item;  // readers take min(count, capacity)
}

// ---------------------------------------------------------------------------
// upper-bound seeding by greedy dives
// ---------------------------------------------------------------------------
// One warp per (query of operator `op`, dive d): from the root pair,
// repeatedly take the best child pair down to a leaf pair, whose faces are
// then tested.  Distance: best = smallest box lower bound, then nearest box
// centres; the certified bounds of the leaf's face pairs lower the query's
// UB before the traversal starts.  Intersects: only child pairs whose boxes
// overlap, nearest box centres first; a certified intersection of the leaf's
// faces ends the query before the traversal.  At the first three levels
// dive d takes the ((d >> 2 l) & 3)-th best child pair instead of the best,
// so the dives of a query start in different subtrees.  Anything a dive
// finds is certified, so the result does not depend on it.  A query gets
// at most max(2, (log2 nleafA + log2 nleafB) / 2) of the `dives` dives.
// With `restricted` set, only queries holding a proposal dive, and only
// through child pairs whose leaf ranges meet the proposed clusters: with n
// proposals, dive d keeps to proposal d mod n and takes the (d / n)-th
// diversification above.  The warps cover nrows queries: rows[r] (the
// queries holding a proposal), or query r when rows is null.
__global__ void __launch_bounds__(128) k_dive(TravArgs a, int dives, int restricted, int op, const int* rows,
                                              int nrows) {
  __shared__ LeafStage stage[4];
  __shared__ LeafJob job[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (gw >= (long long)nrows * dives) return;
  const int r = (int)(gw / dives), d = (int)(gw % dives);
  const int q = rows ? rows[r] : r;  // the queries of a row list (null: rows are queries)
  if (q < 0 || q >= a.nq) return;
  const QueryDev& Qd = a.q[q];
  if (Qd.op != op || ld_volatile_i32(&a.st[q].done)) return;
  {
    const int depth = (31 - __clz(max(Qd.A.nleaf, 1))) + (31 - __clz(max(Qd.B.nleaf, 1)));
    if (d >= max(2, depth / 2)) return;
  }
  const bool isect = op == G3D_OP_INTERSECTS;
  const QueryState& S = a.st[q];
  int pa0 = 0, pa1 = -1, pb0 = 0, pb1 = -1;
  int dv = d;  // which child-pair rank the first levels take
  if (restricted) {
    const int np = min(S.nprop, kMaxProposals);
    if (np <= 0) return;  // no proposal for this query
    const int4 pr = S.prop[d % np];
    dv = d / np;  // dives of different proposals each take the best child pairs
    pa0 = pr.x; pa1 = pr.y; pb0 = pr.z; pb1 = pr.w;
    if (pa1 < pa0 || pb1 < pb0) return;
  }
  int ra = Qd.A.root, rb = Qd.B.root;
  LeafCounters lc;
  for (int level = 0; level < 200 && (ra >= 0 || rb >= 0); level++) {
    // lane c < 4 evaluates child pair c
    float lb = INFINITY;
    int ca = ra, cb = rb;
    const int c = lane;
    bool act = false;
    float4 alo, ahi, blo, bhi;
    if (ra >= 0 && rb >= 0) {
      act = c < 4;
      if (act) {
        const float4* na = Qd.A.nodes + 4 * ra + 2 * (c >> 1);
        const float4* nb = Qd.B.nodes + 4 * rb + 2 * (c & 1);
        alo = __ldg(na); ahi = __ldg(na + 1); blo = __ldg(nb); bhi = __ldg(nb + 1);
        ca = __float_as_int(alo.w); cb = __float_as_int(blo.w);
      }
    } else if (ra >= 0) {
      act = c < 2;
      if (act) {
        const float4* na = Qd.A.nodes + 4 * ra + 2 * c;
        alo = __ldg(na); ahi = __ldg(na + 1);
        blo = __ldg(&Qd.B.leaves[2 * (~rb)]); bhi = __ldg(&Qd.B.leaves[2 * (~rb) + 1]);
        ca = __float_as_int(alo.w);
      }
    } else {
      act = c < 2;
      if (act) {
        const float4* nb = Qd.B.nodes + 4 * rb + 2 * c;
        blo = __ldg(nb); bhi = __ldg(nb + 1);
        alo = __ldg(&Qd.A.leaves[2 * (~ra)]); ahi = __ldg(&Qd.A.leaves[2 * (~ra) + 1]);
        cb = __float_as_int(blo.w);
      }
    }
    if (act && restricted) {  // keep only child pairs meeting the proposed clusters
      const int2 rA = ca >= 0 ? __ldg(&Qd.A.nrange[ca]) : make_int2(~ca, ~ca);
      const int2 rB = cb >= 0 ? __ldg(&Qd.B.nrange[cb]) : make_int2(~cb, ~cb);
      act = rA.x <= pa1 && pa0 <= rA.y && rB.x <= pb1 && pb0 <= rB.y;
    }
    if (act && isect) act = box_overlap(alo, ahi, blo, bhi, Qd.slack);
    // key: the box lower bound, then (boxes that overlap all bound to 0)
    // the squared distance of the box centres
    float cd = INFINITY;
    if (act) {
      lb = isect ? 0.f : box_lb(alo, ahi, blo, bhi);
      const float dx = (alo.x + ahi.x) - (blo.x + bhi.x), dy = (alo.y + ahi.y) - (blo.y + bhi.y),
                  dz = (alo.z + ahi.z) - (blo.z + bhi.z);
      cd = dx * dx + dy * dy + dz * dz;
    }
    // rank of this lane's key among the candidates (ties by lane)
    int rank = 0;
    for (int o = 0; o < 4; o++) {
      const float lo = __shfl_sync(FULL, lb, o), co = __shfl_sync(FULL, cd, o);
      rank += (lo < lb) || (lo == lb && (co < cd || (co == cd && o < lane)));
    }
    const int want = level < 3 ? (dv >> (2 * level)) & 3 : 0;
    unsigned int pick = __ballot_sync(FULL, act && rank == want);
    if (!pick) pick = __ballot_sync(FULL, act && rank == 0);
    if (!pick) return;  // no child pair left (cannot happen when the parent met the ranges)
    const int src = __ffs(pick) - 1;
    ra = __shfl_sync(FULL, ca, src);
    rb = __shfl_sync(FULL, cb, src);
  }
  if (ra < 0 && rb < 0) {
    if (lane == 0) job[warp] = leaf_job_from_tables(a, q, ra, rb, op);
    __syncwarp();
    leaf_jobs(a, &job[warp], 1, 32, lc, stage[warp]);
  }
}

// ---------------------------------------------------------------------------
// launch set-up kernels
// ---------------------------------------------------------------------------
__global__ void k_queue_init(Queue Q) {
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q.cap; i += gridDim.x * blockDim.x)
    Q.seq[i] = (int)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *Q.head = 0;
    *Q.tail = 0;
    *Q.pending = 0;
    *Q.error = 0;
  }
}

// reset per-query state and seed one root item per query (single block);
// distance queries get an intersects phase only when seed_distance is set
__global__ void k_seed(TravArgs a, int seed_distance) {
  __shared__ unsigned long long t0;
  __shared__ int nseed;
  if (threadIdx.x == 0) {
    t0 = *a.queue.tail;
    *a.cand.count = 0;
    nseed = 0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.nq; q += blockDim.x) {
    QueryState s;
    s.ub = __float_as_uint(INFINITY);
    s.done = 0;
    s.ncand = 0;
    s.overflow = 0;
    s.best = __double_as_longlong(INFINITY);
    s.hit = 0;
    s.status = 0;
    s.pass = 1;
    s.phase = 0;
    s.nprop = 0;
    s.witness = ~0ull;
    s.label = -1;
    s.ub_seed = __float_as_uint(INFINITY);
    a.st[q] = s;
    // a distance query linked to an intersects query of the same mesh pair
    // takes its intersects phase from that query instead of repeating it
    if (a.q[q].link >= 0 || (!seed_distance && a.q[q].op == G3D_OP_DISTANCE)) continue;
    int k = atomicAdd(&nseed, 1);
    unsigned long long ticket = t0 + k;
    unsigned int slot = (unsigned int)(ticket & (a.queue.cap - 1));
    a.queue.items[slot] = make_int4(q, a.q[q].A.root, a.q[q].B.root, 0);
    __threadfence();
    a.queue.seq[slot] = (int)(unsigned int)(ticket + 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *a.queue.pending = nseed;
    __threadfence();
    *a.queue.tail = t0 + nseed;
  }
}

// record each unfinished query's proposed cluster pairs (top[r * k + j] =
// cA * 64 + cB for the query of row r, outside [0, 4096) for none;
// k <= kMaxProposals) as leaf
// ranges for the restricted dives.  Cluster c of a mesh with nt faces holds
// faces [ceil(c nt / 64), ceil((c+1) nt / 64)); the ranges keep the leaves
// covering them.
__global__ void k_set_proposal(TravArgs a, const int* __restrict__ top, int k, const int* __restrict__ rows,
                               int nrows) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int q = rows ? rows[r] : r;  // row r of top proposes for query q
  if (q < 0 || q >= a.nq) return;
  const QueryDev& Qd = a.q[q];
  QueryState& S = a.st[q];
  if (S.done) return;
  int np = 0;
  for (int j = 0; j < k && j < kMaxProposals; j++) {
    const int t = top[(long long)r * k + j];
    if (t < 0 || t >= 64 * 64) continue;  // no proposal in this slot
    const int ca = t / 64, cb = t % 64;
    const long long fa0 = ((long long)ca * Qd.A.ntri + 63) / 64, fa1 = ((long long)(ca + 1) * Qd.A.ntri + 63) / 64;
    const long long fb0 = ((long long)cb * Qd.B.ntri + 63) / 64, fb1 = ((long long)(cb + 1) * Qd.B.ntri + 63) / 64;
    if (fa1 <= fa0 || fb1 <= fb0) continue;  // empty cluster
    S.prop[np++] = make_int4((int)(fa0 / Qd.A.L), (int)((fa1 - 1) / Qd.A.L), (int)(fb0 / Qd.B.L),
                             (int)((fb1 - 1) / Qd.B.L));
  }
  S.nprop = np;
}

// after the intersects phase: seed the distance phase of every distance
// query that no certified intersection has finished (single block)
__global__ void k_seed_phase1(TravArgs a) {
  __shared__ unsigned long long t0;
  __shared__ int nseed;
  if (threadIdx.x == 0) {
    t0 = *a.queue.tail;
    nseed = 0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.nq; q += blockDim.x) {
    if (a.q[q].op != G3D_OP_DISTANCE) continue;
    a.st[q].phase = 1;
    a.st[q].ub_seed = a.st[q].ub;
    const int l = a.q[q].link;
    if (l >= 0 && a.st[l].done) {  // the linked intersects query certified a hit
      a.st[q].done = 1;
      a.st[q].ub = 0u;
    }
    if (a.st[q].done) continue;
    int k = atomicAdd(&nseed, 1);
    unsigned long long ticket = t0 + k;
    unsigned int slot = (unsigned int)(ticket & (a.queue.cap - 1));
    a.queue.items[slot] = make_int4(q, a.q[q].A.root, a.q[q].B.root, 0);
    __threadfence();
    a.queue.seq[slot] = (int)(unsigned int)(ticket + 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *a.queue.pending = nseed;
    __threadfence();
    *a.queue.tail = t0 + nseed;
  }
}

// after pass 1: if the candidate pool overflowed, or a query lost work that
// neither a frontier list nor the global queue could hold, re-seed every
// unfinished query (its UB from pass 1 is a valid certified bound) with an
// empty pool; the persistent kernel then runs them from their roots
__global__ void k_prepare_pass2(TravArgs a) {
  __shared__ unsigned long long t0;
  __shared__ int nseed;
  if (threadIdx.x == 0) {
    t0 = *a.queue.tail;
    nseed = 0;
  }
  // a query marked by a failed candidate push (pool full) or by work it could
  // not keep (frontier lists and global queue full) needs a second pass
  int mine = threadIdx.x == 0 && *a.cand.count > a.cand.cap;
  for (int q = threadIdx.x; q < a.nq && !mine; q += blockDim.x) mine = a.st[q].overflow != 0;
  if (!__syncthreads_or(mine)) return;
  if (threadIdx.x == 0) *a.cand.count = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < a.nq; q += blockDim.x) {
    a.st[q].overflow = 0;
    a.st[q].pass = 2;
    if (a.st[q].done) continue;
    int k = atomicAdd(&nseed, 1);
    unsigned long long ticket = t0 + k;
    unsigned int slot = (unsigned int)(ticket & (a.queue.cap - 1));
    a.queue.items[slot] = make_int4(q, a.q[q].A.root, a.q[q].B.root, 0);
    __threadfence();
    a.queue.seq[slot] = (int)(unsigned int)(ticket + 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (a.stats) atomicAdd(&a.stats[ST_SECOND_PASSES], (unsigned long long)nseed);
    *a.queue.pending = nseed;
    __threadfence();
    *a.queue.tail = t0 + nseed;
  }
}

// ---------------------------------------------------------------------------
// finalisation
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_face64(const MeshDev& M, int f, double* out) {
  if (M.m64) {
    for (int k = 0; k < 9; k++) out[k] = M.m64[9ll * f + k];
  } else {
    float4 a = M.v0[f], b = M.v1[f], c = M.v2[f];
    out[0] = a.x; out[1] = a.y; out[2] = a.z;
    out[3] = b.x; out[4] = b.y; out[5] = b.z;
    out[6] = c.x; out[7] = c.y; out[8] = c.z;
  }
}

__global__ void __launch_bounds__(128) k_finalize(TravArgs a) {
  int n = min(*a.cand.count, a.cand.cap);
  unsigned int n64 = 0, nex = 0, nor = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int4 c = a.cand.items[i];
    int q = c.w & CAND_QMASK;
    bool needs_exact = (c.w & CAND_NEEDS_EXACT) != 0;
    if (q >= a.nq || c.x < 0 || c.y < 0 || c.x >= a.q[q].A.ntri || c.y >= a.q[q].B.ntri) {
      record_bad(a, 3, c);
      continue;
    }
    QueryState& s = a.st[q];
    // a certified intersection (in the traversal, or an exact one found here
    // for another candidate) fixes the result: the rest need no test
    if (ld_volatile_i32(&s.done) || ld_volatile_i32(&s.hit)) continue;
    const QueryDev& Qd = a.q[q];
    if (Qd.op == G3D_OP_DISTANCE && __int_as_float(c.z) > __uint_as_float(s.ub)) continue;
    double A[9], B[9];
    load_face64(Qd.A, c.x, A);
    load_face64(Qd.B, c.y, B);
    if (needs_exact) {
      ExactCounter ctr;
      nex++;
      bool x = tri_isect_exact(A, B, ctr);
      nor += ctr.orients;
      if (x) {
        atomicExch(&s.hit, 1);
        continue;
      }
    }
    if (Qd.op == G3D_OP_DISTANCE) {
      n64++;
      double d2 = tri_dist2_f64(A, B);
      atomicMin(&s.best, (unsigned long long)__double_as_longlong(d2));
    }
  }
  if (a.stats) {
    stat_add(a.stats, ST_FP64_TESTS, n64);
    stat_add(a.stats, ST_EXACT_TESTS, nex);
    stat_add(a.stats, ST_EXACT_ORIENTS, nor);
  }
}

// input face id of a face in BVH (Morton) order: kept in v0[f].w
__device__ __forceinline__ unsigned int input_face_id(const MeshDev& M, int f) {
  return (unsigned int)__float_as_int(__ldg(&M.v0[f]).w);
}

// a candidate of an unfinished distance query attaining its FP64 minimum
__device__ __forceinline__ bool attains_min(const TravArgs& a, int4 c, int& q) {
  q = c.w & CAND_QMASK;
  if (q >= a.nq) return false;
  const QueryState& s = a.st[q];
  const QueryDev& Qd = a.q[q];
  if (Qd.op != G3D_OP_DISTANCE || s.done || s.hit) return false;
  if (__int_as_float(c.z) > __uint_as_float(s.ub)) return false;
  if (c.x < 0 || c.y < 0 || c.x >= Qd.A.ntri || c.y >= Qd.B.ntri) return false;
  double A[9], B[9];
  load_face64(Qd.A, c.x, A);
  load_face64(Qd.B, c.y, B);
  return (unsigned long long)__double_as_longlong(tri_dist2_f64(A, B)) == s.best;
}

// the face pair attaining each query's minimum, lowest (face of A, face of
// B) in input face ids among ties; run after k_finalize when a witness is
// asked for
__global__ void __launch_bounds__(128) k_witness(TravArgs a) {
  const int n = min(*a.cand.count, a.cand.cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 c = a.cand.items[i];
    int q;
    if (!attains_min(a, c, q)) continue;
    const QueryDev& Qd = a.q[q];
    atomicMin(&a.st[q].witness,
              ((unsigned long long)input_face_id(Qd.A, c.x) << 32) | input_face_id(Qd.B, c.y));
  }
}

// the cluster pair of each query's witness (clusters of 64 in BVH order:
// face f of a mesh with nt faces is in cluster floor(64 f / nt)); after k_witness
__global__ void __launch_bounds__(128) k_witness_label(TravArgs a) {
  const int n = min(*a.cand.count, a.cand.cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 c = a.cand.items[i];
    int q;
    if (!attains_min(a, c, q)) continue;
    const QueryDev& Qd = a.q[q];
    const unsigned long long w = ((unsigned long long)input_face_id(Qd.A, c.x) << 32) | input_face_id(Qd.B, c.y);
    if (w != a.st[q].witness) continue;
    const int ca = (int)(64ll * c.x / Qd.A.ntri), cb = (int)(64ll * c.y / Qd.B.ntri);
    a.st[q].label = ca * 64 + cb;  // duplicates of the pair (dive + traversal) write the same value
  }
}

__global__ void k_write_results(TravArgs a, double* dist, unsigned char* hit, int* status, long long* witness,
                                int* cluster) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nq) return;
  const QueryState& s = a.st[q];
  int qerr = *a.queue.error;
  bool x = s.done || s.hit;  // a certified intersection is final
  int st = qerr;
  if (!st && !x && s.overflow) st = G3D_ERR_CAND_OVERFLOW;
  if (a.q[q].op == G3D_OP_DISTANCE) {
    double d;
    if (st) d = __longlong_as_double(0x7ff8000000000000ll);
    else if (x) d = 0.0;
    else {
      double b = __longlong_as_double((long long)s.best);
      d = isinf(b) ? __longlong_as_double(0x7ff8000000000000ll) : sqrt(b);
      if (isinf(b)) st = G3D_ERR_CUDA;  // no candidate survived: internal error
    }
    if (dist) dist[q] = d;
    if (hit) hit[q] = st ? 0xff : (unsigned char)(x ? 1 : 0);
  } else {
    if (dist) dist[q] = __longlong_as_double(0x7ff8000000000000ll);
    if (hit) hit[q] = st ? 0xff : (unsigned char)(x ? 1 : 0);
  }
  // how far above the result the seeded bound was (proposal quality), in
  // millionths of the distance
  if (a.stats && !st && !x && a.q[q].op == G3D_OP_DISTANCE) {
    const double d = sqrt(__longlong_as_double((long long)s.best));
    const double u = (double)__uint_as_float(s.ub_seed);
    if (d > 0.0 && isfinite(u)) {
      stat_add(a.stats, ST_SEED_EXCESS, (unsigned long long)(fmax(u / d - 1.0, 0.0) * 1e6));
      stat_add(a.stats, ST_SEED_QUERIES, 1ull);
    }
  }
  if (status) status[q] = st;
  if (witness) witness[q] = (s.witness == ~0ull || x || st) ? -1ll : (long long)s.witness;
  if (cluster) cluster[q] = (s.witness == ~0ull || x || st) ? -1 : s.label;
  if (st && a.sticky) atomicCAS(a.sticky, 0, st);
}

}  // namespace g3d
