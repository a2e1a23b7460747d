// Declarations of the mesh-volume kernels (volume.cu).
#pragma once
#include "internal.cuh"

namespace g3d {

// One mesh as loaded: input vertices (float32 or float64) and face indices.
struct VolMesh {
  const void* V;
  const unsigned int* I;
  long long nt;
  long long nv;
  int dtype;  // G3D_F32 or G3D_F64
  int pad;
};

// Per chunk of faces: the FP64 path's compensated sum (s, c), or the exact
// path's 192-bit integer sum (w0..w2, two's complement); `exact` says which.
struct VolPartial {
  double s, c;
  unsigned long long w0, w1, w2;
  int exact;
  int pad;
};

constexpr int kVolThreads = 256;
constexpr int kVolChunk = 16 * kVolThreads;  // faces per block
constexpr int kVolRangeVerts = 8192;         // vertices per block of the range scan

__global__ void k_volume_range(const VolMesh* meshes, const int* vchunk_mesh, const long long* vchunk_first,
                               unsigned int* range);
__global__ void k_volume_chunks(const VolMesh* meshes, const int* chunk_mesh, const long long* chunk_first,
                                const unsigned int* range, VolPartial* partial);
__global__ void k_volume_finish(int n, const long long* mesh_chunk0, const VolPartial* partial,
                                const unsigned int* range, double* out);

}  // namespace g3d
