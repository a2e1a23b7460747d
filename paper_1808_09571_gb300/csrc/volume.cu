// Mesh volume (Sec. 3.2.1, Eq. 2): V = 1/6 sum_i u_i . ((v_i - u_i) x (w_i - u_i))
// over the faces A_i = (u_i, v_i, w_i), the divergence theorem with the field
// p / 3 on a closed, counter-clockwise mesh (signed: clockwise faces give a
// negative volume; an open mesh gets the formula's value).
//
// As in the paper each face's term is one thread's work; the terms are
// evaluated in FP64 from the mesh's input coordinates (float32 or float64,
// as loaded) and summed with compensated (two-sum) arithmetic in a fixed
// order -- per thread over a fixed stride of faces, then a fixed tree over
// the block, then the chunks of each mesh in order -- so the result does not
// depend on scheduling and repeats bit for bit.  All meshes of a call are
// summed by the same two launches (one block per chunk of faces, then one
// thread per mesh), reading each face's 3 indices and 3 vertices once.
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

// one block per chunk of kVolChunk faces of one mesh
__global__ void __launch_bounds__(kVolThreads) k_volume_chunks(const VolMesh* __restrict__ meshes,
                                                               const int* __restrict__ chunk_mesh,
                                                               const long long* __restrict__ chunk_first,
                                                               double2* __restrict__ partial) {
  const int ch = blockIdx.x;
  const VolMesh m = meshes[chunk_mesh[ch]];
  const long long f0 = chunk_first[ch];
  const long long f1 = min(f0 + (long long)kVolChunk, m.nt);
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
  if (threadIdx.x == 0) partial[ch] = make_double2(ss[0], sc[0]);
}

// one thread per mesh: its chunks in order, then V = (s + c) / 6
__global__ void k_volume_finish(int n, const long long* __restrict__ mesh_chunk0, const double2* __restrict__ partial,
                                double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0, c = 0.0;
  for (long long k = mesh_chunk0[i]; k < mesh_chunk0[i + 1]; k++) {
    vol_acc(s, c, partial[k].x);
    c += partial[k].y;
  }
  out[i] = (s + c) / 6.0;
}

}  // namespace g3d
