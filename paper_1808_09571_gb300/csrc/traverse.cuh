// Declarations of the traversal / finalisation kernels (traverse.cu).
#pragma once
#include "internal.cuh"

namespace g3d {

__global__ void k_traverse(TravArgs a, int stack_cap);
__global__ void k_queue_init(Queue Q);
__global__ void k_seed(TravArgs a);
__global__ void k_prepare_pass2(TravArgs a);
__global__ void k_finalize(TravArgs a);
__global__ void k_write_results(TravArgs a, double* dist, unsigned char* hit, int* status);

}  // namespace g3d
