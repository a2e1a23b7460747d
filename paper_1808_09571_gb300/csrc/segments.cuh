// Declarations of the segment / point against polyhedral surface kernel
// (segments.cu).
#pragma once
#include "internal.cuh"

namespace g3d {

struct SegArgs {
  MeshDev M;
  const float* segs;  // [n][6]: P0, P1
  long long n;
  int op;             // G3D_OP_DISTANCE or G3D_OP_INTERSECTS
  float slack;        // sqrt(3) * rho of the mesh (FP64 input), rounded up
  double* dist;       // [n] or null
  unsigned char* hit; // [n] or null
  int* status;        // [n] or null
  unsigned long long* stats;
  int* sticky;
};

__global__ void k_segments(SegArgs a);

}  // namespace g3d
