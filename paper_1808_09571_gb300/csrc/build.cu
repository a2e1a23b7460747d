// Mesh ingest and BVH construction.
//
// Ingest (Sec. 3.2.1: a mesh is its face set A_i with vertices u_i, v_i, w_i):
// validate the indexed mesh on the device, then regroup it into
// structure-of-arrays float4 faces in Morton order.
//
// BVH: 24- to 30-bit Morton codes of face centroids over the mesh's vertex
// box, LSD radix sort of (code, face id) with 8-bit digits, leaves of L consecutive faces in
// that order, a binary radix tree over the leaves (Karras 2012, "Maximizing
// parallelism in the construction of BVHs, octrees, and k-d trees"; equal
// codes are ordered by leaf index), and a bottom-up refit in which the second
// child to arrive at a node computes its box.
#include <cuda_runtime.h>
#include <stdint.h>

#include "build.cuh"

namespace g3d {

// ---------------------------------------------------------------------------
// batched ingest: one launch copies the vertex and index arrays of all meshes
// of a load call into the library's buffers and validates them on the way
// (NaN / infinite and out-of-range coordinates, out-of-range indices), also
// recording for FP64 input the largest rounding error of the float32 copy
// and, for every mesh, the box of its float32-rounded vertices (the Morton
// quantisation box of the build: every face centroid lies inside it).
// Block b works on chunk b - chunk_off[i] of item i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int item_of(const long long* __restrict__ off, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&off[mid]) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// every mesh's flags and box start empty (one thread per item)
__global__ void k_ingest_init(const IngestItem* __restrict__ items, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || items[i].kind == ING_IDX) return;
  const IngestItem it = items[i];
  it.flags[0] = 0;
  it.flags[1] = 0;
  for (int k = 0; k < 3; k++) {
    it.box[k] = f2ord(INFINITY);
    it.box[3 + k] = f2ord(-INFINITY);
  }
}

// Running checks and vertex box of one thread's elements.  The box axis of
// an element is its index mod 3; the three axes are kept in separate
// registers and updated through selects (no indexed local array).
struct IngestAcc {
  int f = 0;
  float rho = 0.f;
  float l0 = INFINITY, l1 = INFINITY, l2 = INFINITY, h0 = -INFINITY, h1 = -INFINITY, h2 = -INFINITY;
};

__device__ __forceinline__ void acc_box(IngestAcc& A, float x, int ax) {
  A.l0 = fminf(A.l0, ax == 0 ? x : INFINITY);
  A.l1 = fminf(A.l1, ax == 1 ? x : INFINITY);
  A.l2 = fminf(A.l2, ax == 2 ? x : INFINITY);
  A.h0 = fmaxf(A.h0, ax == 0 ? x : -INFINITY);
  A.h1 = fmaxf(A.h1, ax == 1 ? x : -INFINITY);
  A.h2 = fmaxf(A.h2, ax == 2 ? x : -INFINITY);
}

__device__ __forceinline__ void acc_f32(IngestAcc& A, float x, int ax) {
  if (!isfinite(x)) A.f |= VAL_NAN;
  else if (fabsf(x) > 1.152921504606846976e18f) A.f |= VAL_RANGE;  // 2^60
  acc_box(A, x, ax);
}

__device__ __forceinline__ void acc_f64(IngestAcc& A, double x, int ax) {
  if (!isfinite(x)) A.f |= VAL_NAN;
  else if (fabs(x) > 1.152921504606846976e18 || (x != 0.0 && fabs(x) < 6.223015277861142e-61))
    A.f |= VAL_RANGE;  // 2^60, 2^-200
  else {
    const float xf = __double2float_rn(x);
    A.rho = fmaxf(A.rho, __double2float_ru(fabs(x - (double)xf)));  // the difference is exact
    acc_box(A, xf, ax);
  }
}

__device__ __forceinline__ int next_axis(int ax) { return ax == 2 ? 0 : ax + 1; }

// Elements [e0, e1) of one item.  With it.vec set (source and destination on
// 16-byte boundaries; chunks start at multiples of kIngestChunk elements, so
// every chunk does too) the body moves 16 bytes per load and store, which
// keeps several times more bytes in flight per thread than 4-byte accesses;
// the remainder of the chunk, and unaligned items, go element by element.
__global__ void __launch_bounds__(256) k_ingest_many(const IngestItem* __restrict__ items,
                                                     const long long* __restrict__ chunk_off, int n) {
  __shared__ float s_box[6][8];
  __shared__ int s_f[8];
  __shared__ float s_rho[8];
  const int i = item_of(chunk_off, n, blockIdx.x);
  const IngestItem it = items[i];
  const long long c = blockIdx.x - chunk_off[i];
  const long long e0 = c * kIngestChunk, e1 = min(it.n, e0 + kIngestChunk);
  const bool copy = it.src != it.dst;
  const int tid = threadIdx.x, bd = blockDim.x;
  IngestAcc A;
  if (it.kind == ING_IDX) {
    const uint32_t* src = (const uint32_t*)it.src;
    uint32_t* dst = (uint32_t*)it.dst;
    const long long nvec = it.vec ? (e1 - e0) >> 2 : 0;
    const uint4* s4 = (const uint4*)(src + e0);
    uint4* d4 = (uint4*)(dst + e0);
    for (long long j = tid; j < nvec; j += bd) {
      const uint4 x = __ldg(&s4[j]);
      if (copy) d4[j] = x;
      if ((long long)max(max(x.x, x.y), max(x.z, x.w)) >= it.nv) A.f |= VAL_OOB;
    }
    for (long long e = e0 + 4 * nvec + tid; e < e1; e += bd) {
      const uint32_t x = __ldg(&src[e]);
      if (copy) dst[e] = x;
      if ((long long)x >= it.nv) A.f |= VAL_OOB;
    }
  } else if (it.kind == ING_F32) {
    const float* src = (const float*)it.src;
    float* dst = (float*)it.dst;
    const long long nvec = it.vec ? (e1 - e0) >> 2 : 0;
    const float4* s4 = (const float4*)(src + e0);
    float4* d4 = (float4*)(dst + e0);
    for (long long j = tid; j < nvec; j += bd) {
      const float4 x = __ldg(&s4[j]);
      if (copy) d4[j] = x;
      int ax = (int)((e0 + 4 * j) % 3);
      acc_f32(A, x.x, ax);
      ax = next_axis(ax);
      acc_f32(A, x.y, ax);
      ax = next_axis(ax);
      acc_f32(A, x.z, ax);
      ax = next_axis(ax);
      acc_f32(A, x.w, ax);
    }
    for (long long e = e0 + 4 * nvec + tid; e < e1; e += bd) {
      const float x = __ldg(&src[e]);
      if (copy) dst[e] = x;
      acc_f32(A, x, (int)(e % 3));
    }
  } else {  // FP64
    const double* src = (const double*)it.src;
    double* dst = (double*)it.dst;
    const long long nvec = it.vec ? (e1 - e0) >> 1 : 0;
    const double2* s2 = (const double2*)(src + e0);
    double2* d2 = (double2*)(dst + e0);
    for (long long j = tid; j < nvec; j += bd) {
      const double2 x = __ldg(&s2[j]);
      if (copy) d2[j] = x;
      const int ax = (int)((e0 + 2 * j) % 3);
      acc_f64(A, x.x, ax);
      acc_f64(A, x.y, next_axis(ax));
    }
    for (long long e = e0 + 2 * nvec + tid; e < e1; e += bd) {
      const double x = __ldg(&src[e]);
      if (copy) dst[e] = x;
      acc_f64(A, x, (int)(e % 3));
    }
  }
  int f = A.f;
  float rho = A.rho;
  float lo[3] = {A.l0, A.l1, A.l2}, hi[3] = {A.h0, A.h1, A.h2};
  // block reduction, then a few atomics per block on the mesh's words
  for (int o = 16; o > 0; o >>= 1) {
    f |= __shfl_xor_sync(0xffffffffu, f, o);
    rho = fmaxf(rho, __shfl_xor_sync(0xffffffffu, rho, o));
    for (int k = 0; k < 3; k++) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_f[w] = f;
    s_rho[w] = rho;
    for (int k = 0; k < 3; k++) { s_box[k][w] = lo[k]; s_box[3 + k][w] = hi[k]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
    int ff = 0;
    float rr = 0.f;
    for (int j = 0; j < nw; j++) { ff |= s_f[j]; rr = fmaxf(rr, s_rho[j]); }
    if (ff) atomicOr(it.flags, ff);
    if (rr > 0.f) atomicMax((unsigned int*)(it.flags + 1), __float_as_uint(rr));
    if (it.kind != ING_IDX) {
      for (int k = 0; k < 3; k++) {
        float l = INFINITY, h = -INFINITY;
        for (int j = 0; j < nw; j++) { l = fminf(l, s_box[k][j]); h = fmaxf(h, s_box[3 + k][j]); }
        if (l <= h) {
          atomicMin(&it.box[k], f2ord(l));
          atomicMax(&it.box[3 + k], f2ord(h));
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// batched build: every kernel runs over all faces / leaves / nodes of all the
// meshes of one build call; a flattened index is mapped to its mesh by a
// binary search over the per-mesh offsets
// ---------------------------------------------------------------------------
__device__ __forceinline__ int seg_of(const long long* __restrict__ off, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&off[mid]) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Vertex k of a mesh's raw vertex array, rounded to float32.  The two input
// types get separate code paths selected once per warp (vtx<T> below): GB300
// runs FP64 instructions, conversions included, at a small fraction of the
// FP32 rate, and a float64 path merged into the float32 one by predication
// kept the FP64 pipe of the Morton and gather kernels over 80 % busy.
//
// Three consecutive 4-byte words (a vertex, a face's indices) are read with
// one 8-byte and one 4-byte load: the pair that starts on an 8-byte boundary,
// then the remaining word.  In the gather, whose loads follow the sort
// permutation and touch a different cache line in every lane, this cuts the
// L1 wavefronts per face by a third.  The arrays start 8-byte aligned.
__device__ __forceinline__ void load3w(const unsigned int* p, unsigned int& x, unsigned int& y, unsigned int& z) {
  const bool even = ((uintptr_t)p & 7u) == 0;
  const uint2 v = *(const uint2*)(even ? p : p + 1);
  const unsigned int w = even ? p[2] : p[0];
  x = even ? v.x : w;
  y = even ? v.y : v.x;
  z = even ? w : v.y;
}

template <typename T>
__device__ __forceinline__ float3 vtx(const T* V, uint32_t k);
template <>
__device__ __forceinline__ float3 vtx<float>(const float* V, uint32_t k) {
  unsigned int x, y, z;
  load3w((const unsigned int*)(V + 3ull * k), x, y, z);
  return make_float3(__uint_as_float(x), __uint_as_float(y), __uint_as_float(z));
}
template <>
__device__ __forceinline__ float3 vtx<double>(const double* V, uint32_t k) {
  const double* p = V + 3ull * k;
  return make_float3(__double2float_rn(p[0]), __double2float_rn(p[1]), __double2float_rn(p[2]));
}

// mesh of flattened slot g; lane 0 searches and the warp shares the result
// (slot ranges are padded to multiples of 32, so a warp never straddles two
// meshes)
__device__ __forceinline__ int warp_seg_of(const long long* __restrict__ off, int n, long long g) {
  int m = 0;
  if ((threadIdx.x & 31) == 0) m = seg_of(off, n, g);
  return __shfl_sync(0xffffffffu, m, 0);
}

// Rounded operations that the compiler may not fuse into multiply-adds: the
// Morton keys follow exactly the float32 rule written here (centroid
// ((a + b) + c) * (1/3), cell trunc((centroid - lo) * cells / extent)).
__device__ __forceinline__ float3 centroid(float3 a, float3 b, float3 c) {
  const float third = 1.f / 3.f;
  return make_float3(__fmul_rn(__fadd_rn(__fadd_rn(a.x, b.x), c.x), third),
                     __fmul_rn(__fadd_rn(__fadd_rn(a.y, b.y), c.y), third),
                     __fmul_rn(__fadd_rn(__fadd_rn(a.z, b.z), c.z), third));
}

// The Morton quantisation of every mesh, from its vertex box (ingest):
// bounds[8 m + k] = lo_k and bounds[8 m + 4 + k] = cells / extent_k (0 for a
// flat axis), float bits, k = 0..2.
__global__ void k_bounds_from_ingest(BuildArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.n) return;
  const unsigned int* box = a.m[m].box;
  for (int k = 0; k < 3; k++) {
    const float lo = ord2f(box[k]);
    const float e = __fsub_rn(ord2f(box[3 + k]), lo);
    a.bounds[8 * m + k] = __float_as_uint(lo);
    a.bounds[8 * m + 4 + k] = __float_as_uint(e > 0.f ? __fdiv_rn(a.cells, e) : 0.f);
  }
}

// bits 0..9 of x moved to bits 0, 3, 6, ..., 27 (interleaving by masks in
// 32-bit arithmetic: the keys have at most 10 bits per axis)
__device__ __forceinline__ unsigned int spread10(unsigned int x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// key = Morton code of the face centroid over the mesh's vertex box (8 to 10
// bits per axis, as configured); value = face index within the mesh
// trunc(x) for 0 <= x < 2^23: x + 2^23 rounded toward zero is 2^23 + trunc(x)
// exactly (the float32 spacing there is 1), read off the mantissa bits
__device__ __forceinline__ unsigned int trunc_small(float x) {
  return __float_as_uint(__fadd_rz(x, 8388608.f)) - 0x4b000000u;
}

// key of face f of mesh M, written with its value f to flattened slot g;
// B = the mesh's quantisation (lo, scale)
template <typename T>
__device__ __forceinline__ unsigned int morton_face(const BuildMesh& M, const float* B, float cells, int f,
                                                    long long g, unsigned int* keys, unsigned int* vals) {
  const T* V = (const T*)M.V;
  unsigned int i0, i1, i2;
  load3w(M.I + 3ll * f, i0, i1, i2);
  const float3 c = centroid(vtx<T>(V, i0), vtx<T>(V, i1), vtx<T>(V, i2));
  const unsigned int qx = trunc_small(fminf(fmaxf(__fmul_rn(__fsub_rn(c.x, B[0]), B[4]), 0.f), cells));
  const unsigned int qy = trunc_small(fminf(fmaxf(__fmul_rn(__fsub_rn(c.y, B[1]), B[5]), 0.f), cells));
  const unsigned int qz = trunc_small(fminf(fmaxf(__fmul_rn(__fsub_rn(c.z, B[2]), B[6]), 0.f), cells));
  const unsigned int key = (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz);
  keys[g] = key;
  vals[g] = (unsigned int)f;
  return key;
}
// the float64 paths out of line, so that no FP64 instruction sits in the
// float32 code
__device__ __noinline__ unsigned int morton_face_f64(const BuildMesh& M, const float* B, float cells, int f,
                                                     long long g, unsigned int* keys, unsigned int* vals) {
  return morton_face<double>(M, B, cells, f, g, keys, vals);
}

// ---------------------------------------------------------------------------
// Segmented LSD radix sort of (uint32 key, uint32 value): each mesh's faces
// are sorted within their own range, 8-bit digits, stable.  A pass is
//   k_seg_hist:    one block per tile (kSortTile keys of one mesh) counts
//                  the tile's digits into the mesh's digit-major table
//                  hist[tile_off[m]*256 + digit * ntiles_m + tile];
//   k_seg_scan_rows / k_seg_scan_digits: a warp per (mesh, digit) row scans
//                  the row; a warp per mesh scans the 256 row totals, so the
//                  table becomes exclusive offsets in sorted order;
//   k_seg_scatter: one block per tile ranks its keys in shared memory and
//                  writes each digit run contiguously at its offset.
// ---------------------------------------------------------------------------
#ifndef G3D_HIST_PRIVATE
#define G3D_HIST_PRIVATE 1     // 1: per-warp counter rows (measured 35 % faster); 0: lane-group aggregation
#endif
#ifndef G3D_SCATTER_LATE_VAL
#define G3D_SCATTER_LATE_VAL 1 // 1: values read when written to shared memory (fewer registers, 5 CTAs per SM
                               // instead of 4: measured 7.5 % faster); 0: read with the keys
#endif
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = kSortTile / SORT_THREADS;
constexpr int SORT_TILE = kSortTile;

struct TileInfo {
  int m;           // mesh
  int t;           // tile within the mesh
  int ntiles;      // tiles of the mesh
  long long base;  // first face (flattened) of the tile
  int count;       // faces in the tile
  long long hbase; // start of the mesh's histogram table
};

__device__ __forceinline__ TileInfo tile_info(const BuildArgs& a, long long b) {
  TileInfo ti;
  ti.m = seg_of(a.tile_off, a.n, b);
  ti.t = (int)(b - a.tile_off[ti.m]);
  ti.ntiles = (int)(a.tile_off[ti.m + 1] - a.tile_off[ti.m]);
  ti.base = a.face_off[ti.m] + (long long)ti.t * SORT_TILE;
  ti.count = min(SORT_TILE, a.m[ti.m].nt - ti.t * SORT_TILE);
  ti.hbase = a.tile_off[ti.m] * 256;
  return ti;
}

__global__ void __launch_bounds__(SORT_THREADS) k_seg_hist(BuildArgs a, const unsigned int* __restrict__ keys,
                                                           int shift, unsigned int* __restrict__ hist) {
  const TileInfo ti = tile_info(a, blockIdx.x);
#if G3D_HIST_PRIVATE
  // one counter row per warp, plain shared-memory atomics, rows summed at the end
  __shared__ unsigned int cw[SORT_THREADS / 32][256];
#pragma unroll
  for (int w = 0; w < SORT_THREADS / 32; w++) cw[w][threadIdx.x] = 0;
  unsigned int d[SORT_ITEMS];
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++) {
    const int i = r * SORT_THREADS + threadIdx.x;
    d[r] = i < ti.count ? (keys[ti.base + i] >> shift) & 0xffu : 256u;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++)
    if (d[r] < 256u) atomicAdd(&cw[warp][d[r]], 1u);
  __syncthreads();
  unsigned int tot = 0;
#pragma unroll
  for (int w = 0; w < SORT_THREADS / 32; w++) tot += cw[w][threadIdx.x];
  hist[ti.hbase + (long long)threadIdx.x * ti.ntiles + ti.t] = tot;
#else
  __shared__ unsigned int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  // keys of a tile are mostly in Morton order, so in the high-digit passes
  // most of a warp's keys share one digit: lanes with equal digits add once
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++) {
    const int i = r * SORT_THREADS + threadIdx.x;
    const unsigned int d = i < ti.count ? (keys[ti.base + i] >> shift) & 0xffu : 256u;
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&cnt[d], (unsigned int)__popc(peers));
  }
  __syncthreads();
  hist[ti.hbase + (long long)threadIdx.x * ti.ntiles + ti.t] = cnt[threadIdx.x];
#endif
}

// Morton keys and values of one sort tile per block, and the tile's counts
// of the lowest key digit, so that the sort's first pass needs no histogram
// launch of its own (the keys are counted while still in registers).  The
// tile's keys are computed first, then counted, so that the loads of a
// thread's faces are in flight together.
#ifndef G3D_MORTON_MINB
#define G3D_MORTON_MINB 8  // resident blocks per SM the register allocation must allow (8: 32 registers, measured fastest: all warps resident hide the dependent vertex reads)
#endif
__global__ void __launch_bounds__(SORT_THREADS, G3D_MORTON_MINB) k_morton_tiles(BuildArgs a,
                                                                                unsigned int* __restrict__ hist) {
  __shared__ unsigned int cnt[256];
  const TileInfo ti = tile_info(a, blockIdx.x);
  const BuildMesh& M = a.m[ti.m];
  const float* B = (const float*)a.bounds + 8 * ti.m;
  cnt[threadIdx.x] = 0;
  const bool f32 = M.dtype == G3D_F32;
  unsigned int d[SORT_ITEMS];
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++) {
    const int i = r * SORT_THREADS + threadIdx.x;
    d[r] = 256u;
    if (i < ti.count) {
      const int f = ti.t * SORT_TILE + i;
      const long long g = ti.base + i;
      const unsigned int key = f32 ? morton_face<float>(M, B, a.cells, f, g, a.keys0, a.vals0)
                                   : morton_face_f64(M, B, a.cells, f, g, a.keys0, a.vals0);
      d[r] = key & 0xffu;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++) {
    const unsigned int peers = __match_any_sync(0xffffffffu, d[r]);
    if (d[r] < 256u && lane == __ffs(peers) - 1) atomicAdd(&cnt[d[r]], (unsigned int)__popc(peers));
  }
  __syncthreads();
  hist[ti.hbase + (long long)threadIdx.x * ti.ntiles + ti.t] = cnt[threadIdx.x];
}

// one warp per (mesh, digit) row of the digit-major table: exclusive scan of
// the row's tile counts in place, row total to totals[m * 256 + d]
__global__ void __launch_bounds__(256) k_seg_scan_rows(BuildArgs a, unsigned int* __restrict__ hist,
                                                       unsigned int* __restrict__ totals) {
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= 256ll * a.n) return;
  const int m = (int)(row >> 8), d = (int)(row & 255);
  const int ntiles = (int)(a.tile_off[m + 1] - a.tile_off[m]);
  unsigned int* r = hist + a.tile_off[m] * 256 + (long long)d * ntiles;
  unsigned int carry = 0;
  for (int base = 0; base < ntiles; base += 32) {
    const int i = base + lane;
    const unsigned int v = i < ntiles ? r[i] : 0u;
    unsigned int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (i < ntiles) r[i] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) totals[row] = carry;
}

// one warp per mesh: exclusive scan of its 256 digit totals in place
__global__ void __launch_bounds__(256) k_seg_scan_digits(BuildArgs a, unsigned int* __restrict__ totals) {
  const long long m = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (m >= a.n) return;
  unsigned int* t = totals + m * 256;
  unsigned int v[8], sum = 0;
  for (int j = 0; j < 8; j++) { v[j] = t[lane * 8 + j]; sum += v[j]; }
  unsigned int x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  unsigned int run = x - sum;
  for (int j = 0; j < 8; j++) { t[lane * 8 + j] = run; run += v[j]; }
}

__device__ __forceinline__ unsigned int block_excl_scan256(unsigned int v, unsigned int* s_warp) {
  // 256 threads; returns the exclusive prefix of v in thread order
  unsigned int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) >= o) x += y;
  }
  if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = x;
  __syncthreads();
  unsigned int add = 0;
  for (int w = 0; w < (int)(threadIdx.x >> 5); w++) add += s_warp[w];
  __syncthreads();
  return x - v + add;
}

// Ranking: warp w owns tile elements [w E, (w+1) E), E = kSortTile / 8, taken
// 32 at a time in order; within a warp, lanes with equal digits find each
// other with __match_any_sync and read / bump a warp-private digit counter, so
// the only block barriers are around the per-digit combine of the 8 warps.
// Element order in the tile is (warp, round, lane), which keeps the sort
// stable.
__global__ void __launch_bounds__(SORT_THREADS, kSortTile > 2048 ? 3 : (G3D_SCATTER_LATE_VAL ? 5 : 4)) k_seg_scatter(BuildArgs a, const unsigned int* __restrict__ kin,
                                                              const unsigned int* __restrict__ vin,
                                                              unsigned int* __restrict__ kout,
                                                              unsigned int* __restrict__ vout, int shift,
                                                              const unsigned int* __restrict__ hist,
                                                              const unsigned int* __restrict__ dbase) {
  __shared__ unsigned int s_key[SORT_TILE];
  __shared__ unsigned int s_val[SORT_TILE];
  __shared__ unsigned int s_wcnt[SORT_THREADS / 32][256];
  __shared__ unsigned int s_tstart[256];
  __shared__ unsigned int s_gbase[256];
  __shared__ unsigned int s_tmp[8];
  constexpr int E = SORT_TILE / (SORT_THREADS / 32);
  const TileInfo ti = tile_info(a, blockIdx.x);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned int lt_mask = (1u << lane) - 1u;
  s_gbase[tid] = dbase[256ll * ti.m + tid] + hist[ti.hbase + (long long)tid * ti.ntiles + ti.t];
#pragma unroll
  for (int w = 0; w < SORT_THREADS / 32; w++) s_wcnt[w][tid] = 0;
  __syncthreads();
#if G3D_SCATTER_LATE_VAL
  unsigned int key[SORT_ITEMS], dig[SORT_ITEMS], rank[SORT_ITEMS];
#else
  unsigned int key[SORT_ITEMS], val[SORT_ITEMS], dig[SORT_ITEMS], rank[SORT_ITEMS];
#endif
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++) {
    const int i = warp * E + r * 32 + lane;
    const bool ok = i < ti.count;
    key[r] = ok ? kin[ti.base + i] : 0u;
#if !G3D_SCATTER_LATE_VAL
    val[r] = ok ? vin[ti.base + i] : 0u;
#endif
    dig[r] = ok ? ((key[r] >> shift) & 0xffu) : 256u;
  }
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++) {
    const unsigned int d = dig[r];
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    const unsigned int lr = __popc(peers & lt_mask);
    const unsigned int base = d < 256 ? s_wcnt[warp][d] : 0u;
    __syncwarp();
    if (d < 256 && lr == 0) s_wcnt[warp][d] = base + __popc(peers);
    __syncwarp();
    rank[r] = base + lr;
  }
  __syncthreads();
  unsigned int run = 0;
#pragma unroll
  for (int w = 0; w < SORT_THREADS / 32; w++) {
    unsigned int c = s_wcnt[w][tid];
    s_wcnt[w][tid] = run;
    run += c;
  }
  s_tstart[tid] = block_excl_scan256(run, s_tmp);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; r++)
    if (dig[r] < 256) {
      const unsigned int p = s_tstart[dig[r]] + s_wcnt[warp][dig[r]] + rank[r];
      s_key[p] = key[r];
#if G3D_SCATTER_LATE_VAL
      s_val[p] = vin[ti.base + warp * E + r * 32 + lane];
#else
      s_val[p] = val[r];
#endif
    }
  __syncthreads();
  const long long out0 = a.face_off[ti.m];
  for (int i = tid; i < ti.count; i += SORT_THREADS) {
    unsigned int k = s_key[i];
    unsigned int d = (k >> shift) & 0xffu;
    long long dst = out0 + s_gbase[d] + (i - s_tstart[d]);
    kout[dst] = k;
    vout[dst] = s_val[i];
  }
}

// ---------------------------------------------------------------------------
// regroup faces in sorted order, leaves, radix tree, refit
// ---------------------------------------------------------------------------
// Sorted position s of mesh m's range holds its face svals[s] at local
// position p = s - face_off[m].  Mesh ranges start at multiples of 32 and L
// divides 32, so a warp covers whole leaves of one mesh: each leaf's box is
// reduced over its L lanes with xor shuffles and written by its first lane,
// together with the leaf's key for the radix tree.
struct Box3 {
  float3 lo, hi;
};

// writes face f of mesh M to sorted position p (SoA records, FP64 master
// copy); returns the face's box
template <typename T>
__device__ __forceinline__ Box3 gather_face(const BuildMesh& M, int p, int f) {
  const T* V = (const T*)M.V;
  unsigned int i0, i1, i2;
  load3w(M.I + 3ll * f, i0, i1, i2);
  const float3 A = vtx<T>(V, i0), B = vtx<T>(V, i1), C = vtx<T>(V, i2);
  M.v0[p] = make_float4(A.x, A.y, A.z, __int_as_float(f));
  M.v1[p] = make_float4(B.x, B.y, B.z, 0.f);
  M.v2[p] = make_float4(C.x, C.y, C.z, 0.f);
  if (sizeof(T) == 8 && M.m64) {
    const double* D = (const double*)M.V;
    double* o = M.m64 + 9ll * p;
    for (int k = 0; k < 3; k++) {
      o[k] = D[3ull * i0 + k];
      o[3 + k] = D[3ull * i1 + k];
      o[6 + k] = D[3ull * i2 + k];
    }
  }
  return Box3{make_float3(fminf(A.x, fminf(B.x, C.x)), fminf(A.y, fminf(B.y, C.y)), fminf(A.z, fminf(B.z, C.z))),
              make_float3(fmaxf(A.x, fmaxf(B.x, C.x)), fmaxf(A.y, fmaxf(B.y, C.y)), fmaxf(A.z, fmaxf(B.z, C.z)))};
}

__device__ __noinline__ Box3 gather_face_f64(const BuildMesh& M, int p, int f) { return gather_face<double>(M, p, f); }

__global__ void __launch_bounds__(256) k_gather_many(BuildArgs a, const unsigned int* __restrict__ skeys,
                                                     const unsigned int* __restrict__ svals) {
  const long long s0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31u);
  if (s0 >= a.total_faces) return;  // whole warps leave together
  const long long s = s0 + (threadIdx.x & 31);
  const int m = warp_seg_of(a.face_off, a.n, s0);
  const BuildMesh& M = a.m[m];
  const int p = (int)(s - a.face_off[m]);
  const bool active = p < M.nt;
  float3 lo = make_float3(INFINITY, INFINITY, INFINITY), hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
  unsigned int key = 0;
  if (active) {
    key = skeys[s];
    const int f = (int)svals[s];
    const Box3 b = M.dtype == G3D_F32 ? gather_face<float>(M, p, f) : gather_face_f64(M, p, f);
    lo = b.lo;
    hi = b.hi;
  }
  const int L = a.m[0].L;  // the same for every mesh of a build (a power of two, at most 32)
  for (int o = 1; o < L; o <<= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
    lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
    lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
  }
  if (active && (p & (L - 1)) == 0) {
    const int k = p >> (__ffs(L) - 1);
    M.leaves[2 * k] = make_float4(lo.x, lo.y, lo.z, __int_as_float(p));
    M.leaves[2 * k + 1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(min(L, M.nt - p)));
    a.lkeys[a.leaf_off[m] + k] = key;
  }
}

__device__ __forceinline__ int kdelta(const unsigned int* __restrict__ k, int m, int i, int j) {
  if (j < 0 || j >= m) return -1;
  unsigned int a = k[i], b = k[j];
  if (a == b) return 32 + __clz(i ^ j);
  return __clz(a ^ b);
}

// one thread per internal node (flattened); Karras' split search over the
// leaf keys of its mesh.  Child references are local to the mesh.
__global__ void k_radix_tree_many(BuildArgs a) {
  long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gi >= a.total_nodes) return;
  const int mi = seg_of(a.node_off, a.n, gi);
  const int i = (int)(gi - a.node_off[mi]);
  const int m = a.m[mi].nleaf;
  const unsigned int* lk = a.lkeys + a.leaf_off[mi];
  int* child = a.child + 2 * a.node_off[mi];
  int* ccount = a.ccount + 2 * a.node_off[mi];
  int* pnode = a.pnode + a.node_off[mi];
  int* pleaf = a.pleaf + a.leaf_off[mi];
  int2* nrange = a.m[mi].nrange;
  int d = (kdelta(lk, m, i, i + 1) - kdelta(lk, m, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = kdelta(lk, m, i, i - d);
  int lmax = 2;
  while (kdelta(lk, m, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (kdelta(lk, m, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = kdelta(lk, m, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (kdelta(lk, m, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int gamma = i + s * d + min(d, 0);
  int first = min(i, j), last = max(i, j);
  int left = (first == gamma) ? ~gamma : gamma;
  int right = (last == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  child[2 * i] = left;
  child[2 * i + 1] = right;
  nrange[i] = make_int2(first, last);
  ccount[2 * i] = gamma - first + 1;
  ccount[2 * i + 1] = last - gamma;
  if (left >= 0) pnode[left] = (i << 1); else pleaf[gamma] = (i << 1);
  if (right >= 0) pnode[right] = (i << 1) | 1; else pleaf[gamma + 1] = (i << 1) | 1;
}

// defensive check of the topology: every child reference in range
__global__ void k_check_tree_many(BuildArgs a, int* __restrict__ err) {
  long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gi >= a.total_nodes) return;
  const int mi = seg_of(a.node_off, a.n, gi);
  const int m = a.m[mi].nleaf;
  const int* child = a.child + 2 * gi;
  for (int c = 0; c < 2; c++) {
    int r = child[c];
    bool ok = (r > 0 && r < m - 1) || (r < 0 && ~r < m);
    if (!ok) atomicCAS(err, 0, G3D_ERR_CUDA);
  }
}

// fetch-and-add with release (the caller's earlier stores are visible to
// whoever later reads the counter with acquire) and acquire (what the earlier
// arrivers stored before their release is visible to the caller's later
// loads) semantics at GPU scope: one ordered RMW instead of a full fence on
// each side of a relaxed one
__device__ __forceinline__ int atomic_add_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(__cvta_generic_to_global(p)), "r"(v)
               : "memory");
  return old;
}

// the same at CTA scope, on a shared-memory counter
__device__ __forceinline__ int atomic_add_acq_rel_cta(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.cta.shared.add.s32 %0, [%1], %2;"
               : "=r"(old)
               : "r"((unsigned int)__cvta_generic_to_shared(p)), "r"(v)
               : "memory");
  return old;
}

// One thread per leaf; the second child to reach a node computes its box.
// A block holds kRefitBlock consecutive leaves; an internal node whose leaf
// range lies inside them has both children's climbers in the block (and is
// itself one end of its range, so it has a slot among the block's
// counters): it counts its arrivals in shared memory at CTA scope, and only
// the nodes above those go through GPU-scope atomics in global memory.
constexpr int kRefitBlock = 256;
__global__ void __launch_bounds__(kRefitBlock) k_refit_many(BuildArgs a) {
  __shared__ int sflag[kRefitBlock];
  sflag[threadIdx.x] = 0;
  __syncthreads();
  const long long g0 = (long long)blockIdx.x * kRefitBlock;  // this block's first leaf
  const long long gl = g0 + threadIdx.x;
  if (gl >= a.total_leaves) return;
  const int mi = seg_of(a.leaf_off, a.n, gl);
  const BuildMesh& M = a.m[mi];
  if (M.nleaf < 2) return;
  const int k = (int)(gl - a.leaf_off[mi]);
  const long long w0 = g0 - a.leaf_off[mi], w1 = w0 + kRefitBlock - 1;  // the block's leaves, in this mesh
  const int* child = a.child + 2 * a.node_off[mi];
  const int* ccount = a.ccount + 2 * a.node_off[mi];
  const int* pnode = a.pnode + a.node_off[mi];
  const int2* nrange = M.nrange;
  int* visit = a.visit + a.node_off[mi];
  float4* nodes = M.nodes;
  float4 lo = M.leaves[2 * k], hi = M.leaves[2 * k + 1];
  int pe = a.pleaf[a.leaf_off[mi] + k];
  for (int guard = 0; guard < 96; guard++) {
    int p = pe >> 1, c = pe & 1;
    int slot = 4 * p + 2 * c;
    // the node's parent link, loaded with the node's own tables before the
    // arrival counter (one memory round trip fewer per level of the climb)
    const int pe_up = p != 0 ? __ldg(&pnode[p]) : 0;
    const int2 rg = __ldg(&nrange[p]);
    nodes[slot] = make_float4(lo.x, lo.y, lo.z, __int_as_float(__ldg(&child[2 * p + c])));
    nodes[slot + 1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(__ldg(&ccount[2 * p + c])));
    const long long sp = (long long)p - w0;
    float4 olo, ohi;
    if (rg.x >= w0 && rg.y <= w1 && sp >= 0 && sp < kRefitBlock) {
      if (atomic_add_acq_rel_cta(&sflag[sp], 1) == 0) return;
      // the sibling's box was written by a thread of this block
      olo = nodes[4 * p + 2 * (c ^ 1)];
      ohi = nodes[4 * p + 2 * (c ^ 1) + 1];
    } else {
      if (atomic_add_acq_rel(&visit[p], 1) == 0) return;
      olo = __ldcg(&nodes[4 * p + 2 * (c ^ 1)]);
      ohi = __ldcg(&nodes[4 * p + 2 * (c ^ 1) + 1]);
    }
    lo = make_float4(fminf(lo.x, olo.x), fminf(lo.y, olo.y), fminf(lo.z, olo.z), 0.f);
    hi = make_float4(fmaxf(hi.x, ohi.x), fmaxf(hi.y, ohi.y), fmaxf(hi.z, ohi.z), 0.f);
    if (p == 0) return;
    pe = pe_up;
  }
}

}  // namespace g3d
