// Mesh volume (Sec. 3.2.1, Eq. 2): V = 1/6 sum_i u_i . ((v_i - u_i) x (w_i - u_i))
// over the faces A_i = (u_i, v_i, w_i), the divergence theorem with the field
// p / 3 on a closed, counter-clockwise mesh (signed: clockwise faces give a
// negative volume; an open mesh gets the formula's value).
//
// As in the paper each face's term is one thread's work, then a sum.  Each
// term equals the determinant det(u, v, w) = u . (v x w) (the terms in u x u
// and u . (v x u) vanish identically).
//
// Float32 meshes take an exact path: every float32 coordinate is an integer
// multiple of 2^E, E the lowest bit position over the mesh's nonzero
// coordinates, so with X = x / 2^E (at most 50 bits when the mesh's
// coordinates span at most 50 binary orders of magnitude, checked per mesh by
// a first pass) each face's determinant is an exact integer of at most 153
// bits, and the mesh's sum an exact 192-bit integer; the volume is that sum
// times 2^(3E), converted to double with one rounding, divided by 6 with a
// second.  Integer sums do not depend on their order, so the result repeats
// bit for bit.  The FP32 and integer pipes do this work (GB300's FP64 rate is
// a small fraction of its FP32 rate).
//
// Float64 meshes, and float32 meshes whose coordinates span more than 50
// orders of magnitude, take the FP64 path: each term in FP64 from the input
// coordinates, summed with compensated (two-sum) arithmetic in a fixed order
// -- per thread over a fixed stride of faces, then a fixed tree over the
// block, then the chunks of each mesh over a warp (strided, then a fixed
// butterfly) -- so the result also repeats bit for bit.  All meshes of a
// call are summed by the same three launches (a range pass over the
// vertices, one block per chunk of faces, one warp per mesh).
#include <cuda_runtime.h>

#include "volume.cuh"

namespace g3d {

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void vol_two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (s, c) += x, keeping the rounding error of every addition in c
__device__ __forceinline__ void vol_acc(double& s, double& c, double x) {
  double e;
  vol_two_sum(s, x, s, e);
  c += e;
}

__device__ __forceinline__ void vol_vertex(const VolMesh& m, unsigned int k, double* p) {
  if (m.dtype == G3D_F64) {
    const double* V = (const double*)m.V;
    p[0] = V[3ull * k]; p[1] = V[3ull * k + 1]; p[2] = V[3ull * k + 2];
  } else {
    const float* V = (const float*)m.V;
    p[0] = V[3ull * k]; p[1] = V[3ull * k + 1]; p[2] = V[3ull * k + 2];
  }
}

// ---------------------------------------------------------------------------
// exact path (float32 meshes)
// ---------------------------------------------------------------------------
constexpr int kVolMaxBits = 50;  // bits of |X| the exact path allows

// range[2 m] = smallest nonzero |x| (float bits), range[2 m + 1] = largest
// |x| (float bits) over mesh m's float32 coordinates; one block per chunk of
// kVolRangeVerts vertices.  (Bits of non-negative floats order like the
// floats.)  range starts at {0x7f800000, 0}.
__global__ void __launch_bounds__(256) k_volume_range(const VolMesh* __restrict__ meshes,
                                                      const int* __restrict__ vchunk_mesh,
                                                      const long long* __restrict__ vchunk_first,
                                                      unsigned int* __restrict__ range) {
  const int mi = vchunk_mesh[blockIdx.x];
  const VolMesh m = meshes[mi];
  if (m.dtype != G3D_F32) return;
  const float* V = (const float*)m.V;
  const long long e0 = 3 * vchunk_first[blockIdx.x];
  const long long e1 = min(e0 + 3ll * kVolRangeVerts, 3 * m.nv);
  unsigned int lo = 0x7f800000u, hi = 0u;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const unsigned int b = __float_as_uint(V[e]) & 0x7fffffffu;
    if (b != 0u) lo = min(lo, b);
    hi = max(hi, b);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&range[2 * mi], lo);
    atomicMax(&range[2 * mi + 1], hi);
  }
}

// Exponent E of the integer grid of mesh range (lo, hi) and whether the
// exact path applies (|X| < 2^kVolMaxBits).  E = lowest bit position of the
// smallest nonzero magnitude (its exponent minus 23, or -149 if subnormal).
__device__ __forceinline__ bool vol_exact_grid(unsigned int lo, unsigned int hi, int& E) {
  if (hi == 0u) {  // every coordinate is zero
    E = 0;
    return true;
  }
  if (hi >= 0x7f800000u) return false;  // not finite (cannot happen after ingest)
  const int elo = (int)(lo >> 23), ehi = (int)(hi >> 23);
  E = elo == 0 ? -149 : elo - 127 - 23;
  const int top = (ehi == 0 ? -126 : ehi - 127) + 1;  // |x| < 2^top
  return top - E <= kVolMaxBits;
}

struct I192 {
  unsigned long long w0, w1, w2;
};

__device__ __forceinline__ void add192(I192& a, unsigned long long b0, unsigned long long b1, unsigned long long b2) {
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
      : "l"(b0), "l"(b1), "l"(b2));
}

// a += x * n exactly, x < 2^50 and n < 2^102 in magnitude (two's complement)
__device__ __forceinline__ void acc_mul(I192& a, long long x, __int128 n) {
  const unsigned long long nl = (unsigned long long)n;
  const long long nh = (long long)(n >> 64);
  const __int128 p1 = (__int128)x * (__int128)nl;  // |p1| < 2^114
  const __int128 p2 = (__int128)x * (__int128)nh;  // |p2| < 2^88, weight 2^64
  const unsigned long long p1h = (unsigned long long)(p1 >> 64);
  add192(a, (unsigned long long)p1, p1h, p1 < 0 ? ~0ull : 0ull);
  add192(a, 0ull, (unsigned long long)p2, (unsigned long long)(p2 >> 64));
}

// x / 2^E as an integer, from the float's bits (integer operations only):
// |x| = m 2^(e - 150) with the 24-bit significand m (e the biased exponent,
// 1 for subnormals), and e - 150 >= E for every nonzero x of the mesh
__device__ __forceinline__ long long vol_int(float x, int E) {
  const unsigned int b = __float_as_uint(x);
  const unsigned int eb = (b >> 23) & 0xffu;
  const long long m = (long long)((b & 0x7fffffu) | (eb ? 0x800000u : 0u));
  const int sh = (eb ? (int)eb : 1) - 150 - E;  // 0 <= sh < 50 (m == 0 for a zero)
  const long long v = m == 0 ? 0ll : (m << sh);
  return (b >> 31) ? -v : v;
}

// 192-bit two's complement integer -> double, rounded to nearest
__device__ inline double i192_to_double(I192 a) {
  const bool neg = (long long)a.w2 < 0;
  if (neg) {  // magnitude
    a.w0 = ~a.w0; a.w1 = ~a.w1; a.w2 = ~a.w2;
    add192(a, 1ull, 0ull, 0ull);
  }
  int shift;
  unsigned long long top, rest;
  if (a.w2) {
    const int z = __clzll(a.w2);
    shift = 128 - z;  // value = (a >> shift) with 64 significant bits
    top = z ? (a.w2 << z) | (a.w1 >> (64 - z)) : a.w2;
    rest = (z ? (a.w1 << z) : a.w1) | a.w0;
  } else if (a.w1) {
    const int z = __clzll(a.w1);
    shift = 64 - z;
    top = z ? (a.w1 << z) | (a.w0 >> (64 - z)) : a.w1;
    rest = z ? (a.w0 << z) : a.w0;
  } else {
    shift = 0;
    top = a.w0;
    rest = 0ull;
  }
  // the discarded bits only decide ties: fold them into the lowest kept bit
  // (64 kept bits > 53 + 2, so one rounding of `top` is the correct rounding)
  if (rest) top |= 1ull;
  const double d = ldexp(__ull2double_rn(top), shift);
  return neg ? -d : d;
}

__device__ __forceinline__ void vol_vertex_i(const float* V, unsigned int k, int E, long long* p) {
  p[0] = vol_int(V[3ull * k], E);
  p[1] = vol_int(V[3ull * k + 1], E);
  p[2] = vol_int(V[3ull * k + 2], E);
}

// one block per chunk of kVolChunk faces of one mesh
__global__ void __launch_bounds__(kVolThreads) k_volume_chunks(const VolMesh* __restrict__ meshes,
                                                               const int* __restrict__ chunk_mesh,
                                                               const long long* __restrict__ chunk_first,
                                                               const unsigned int* __restrict__ range,
                                                               VolPartial* __restrict__ partial) {
  const int ch = blockIdx.x;
  const int mi = chunk_mesh[ch];
  const VolMesh m = meshes[mi];
  const long long f0 = chunk_first[ch];
  const long long f1 = min(f0 + (long long)kVolChunk, m.nt);
  int E = 0;
  if (m.dtype == G3D_F32 && vol_exact_grid(range[2 * mi], range[2 * mi + 1], E)) {
    const float* V = (const float*)m.V;
    I192 acc{0ull, 0ull, 0ull};
    for (long long f = f0 + threadIdx.x; f < f1; f += kVolThreads) {
      const unsigned int ia = m.I[3 * f], ib = m.I[3 * f + 1], ic = m.I[3 * f + 2];
      long long u[3], v[3], w[3];
      vol_vertex_i(V, ia, E, u);
      vol_vertex_i(V, ib, E, v);
      vol_vertex_i(V, ic, E, w);
      // det(u, v, w) = u . (v x w)
      const __int128 nx = (__int128)v[1] * w[2] - (__int128)v[2] * w[1];
      const __int128 ny = (__int128)v[2] * w[0] - (__int128)v[0] * w[2];
      const __int128 nz = (__int128)v[0] * w[1] - (__int128)v[1] * w[0];
      acc_mul(acc, u[0], nx);
      acc_mul(acc, u[1], ny);
      acc_mul(acc, u[2], nz);
    }
    // block sum (integer: any order gives the same bits)
    __shared__ unsigned long long sw[3][kVolThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
      I192 b{__shfl_xor_sync(0xffffffffu, acc.w0, o), __shfl_xor_sync(0xffffffffu, acc.w1, o),
             __shfl_xor_sync(0xffffffffu, acc.w2, o)};
      add192(acc, b.w0, b.w1, b.w2);
    }
    if ((threadIdx.x & 31) == 0) {
      sw[0][threadIdx.x >> 5] = acc.w0;
      sw[1][threadIdx.x >> 5] = acc.w1;
      sw[2][threadIdx.x >> 5] = acc.w2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      I192 t{0ull, 0ull, 0ull};
      for (int k = 0; k < kVolThreads / 32; k++) add192(t, sw[0][k], sw[1][k], sw[2][k]);
      VolPartial r{};
      r.w0 = t.w0; r.w1 = t.w1; r.w2 = t.w2;
      r.exact = 1;
      partial[ch] = r;
    }
    return;
  }
  double s = 0.0, c = 0.0;
  for (long long f = f0 + threadIdx.x; f < f1; f += kVolThreads) {
    const unsigned int ia = m.I[3 * f], ib = m.I[3 * f + 1], ic = m.I[3 * f + 2];
    double u[3], v[3], w[3];
    vol_vertex(m, ia, u);
    vol_vertex(m, ib, v);
    vol_vertex(m, ic, w);
    // GB300 runs FP64 at a small fraction of its FP32 rate and this loop is
    // bound by it: fused multiply-adds and one compensated addition per face
    // (22 FP64 instructions)
    const double e0x = v[0] - u[0], e0y = v[1] - u[1], e0z = v[2] - u[2];
    const double e1x = w[0] - u[0], e1y = w[1] - u[1], e1z = w[2] - u[2];
    const double nx = fma(e0y, e1z, -(e0z * e1y)), ny = fma(e0z, e1x, -(e0x * e1z)),
                 nz = fma(e0x, e1y, -(e0y * e1x));
    vol_acc(s, c, fma(u[0], nx, fma(u[1], ny, u[2] * nz)));
  }
  // fixed tree over the block: (s, c) pairs added with two-sum
  __shared__ double ss[kVolThreads], sc[kVolThreads];
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int h = kVolThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      double t, e;
      vol_two_sum(ss[threadIdx.x], ss[threadIdx.x + h], t, e);
      ss[threadIdx.x] = t;
      sc[threadIdx.x] += sc[threadIdx.x + h] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    VolPartial r{};
    r.s = ss[0];
    r.c = sc[0];
    r.exact = 0;
    partial[ch] = r;
  }
}

// per mesh the sum of its chunks, then V = sum / 6 (exact path: the integer
// sum times 2^(3E), rounded once, then divided by 6)
__global__ void k_volume_finish(int n, const long long* __restrict__ mesh_chunk0,
                                const VolPartial* __restrict__ partial, const unsigned int* __restrict__ range,
                                double* __restrict__ out) {
  // one warp per mesh: lane l takes chunks k0 + l, k0 + l + 32, ... in
  // order, then the lanes combine in a fixed butterfly (integer sums are
  // exact in any order; the compensated FP64 sums keep one fixed order, so
  // the result repeats bit for bit)
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;  // whole warps leave together
  const long long k0 = mesh_chunk0[i], k1 = mesh_chunk0[i + 1];
  if (k1 > k0 && partial[k0].exact) {
    int E = 0;
    vol_exact_grid(range[2 * i], range[2 * i + 1], E);
    I192 t{0ull, 0ull, 0ull};
    for (long long k = k0 + lane; k < k1; k += 32) add192(t, partial[k].w0, partial[k].w1, partial[k].w2);
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long b0 = __shfl_xor_sync(0xffffffffu, t.w0, o), b1 = __shfl_xor_sync(0xffffffffu, t.w1, o),
                               b2 = __shfl_xor_sync(0xffffffffu, t.w2, o);
      add192(t, b0, b1, b2);
    }
    if (lane == 0) out[i] = ldexp(i192_to_double(t), 3 * E) / 6.0;
    return;
  }
  double s = 0.0, c = 0.0;
  for (long long k = k0 + lane; k < k1; k += 32) {
    vol_acc(s, c, partial[k].s);
    c += partial[k].c;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
    // the lower lane of each pair adds the upper one's pair (a fixed order)
    double t, e;
    if ((lane & o) == 0) {
      vol_two_sum(s, os, t, e);
      s = t;
      c += oc + e;
    } else {
      vol_two_sum(os, s, t, e);
      s = t;
      c = oc + c + e;
    }
  }
  if (lane == 0) out[i] = (s + c) / 6.0;
}

}  // namespace g3d
