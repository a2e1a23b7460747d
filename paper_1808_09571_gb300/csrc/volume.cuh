// Declarations of the mesh-volume kernels (volume.cu).
#pragma once
#include "internal.cuh"

namespace g3d {

// One mesh as loaded: input vertices (float32 or float64) and face indices.
struct VolMesh {
  const void* V;
  const unsigned int* I;
  long long nt;
  int dtype;  // G3D_F32 or G3D_F64
  int pad;
};

constexpr int kVolThreads = 256;
constexpr int kVolChunk = 16 * kVolThreads;  // faces per block

__global__ void k_volume_chunks(const VolMesh* meshes, const int* chunk_mesh, const long long* chunk_first,
                                double2* partial);
__global__ void k_volume_finish(int n, const long long* mesh_chunk0, const double2* partial, double* out);

}  // namespace g3d
