// Declarations of the traversal / finalisation kernels (traverse.cu).
#pragma once
#include "internal.cuh"

namespace g3d {

// Per-warp shared staging of one leaf pair: 32 faces (lanes 0-15 mesh A,
// 16-31 mesh B) as 9 floats, and the compacted indices of surviving faces.
struct LeafStage {
  float f[32][9];
  unsigned char idx[32];
};

// A leaf pair waiting for its face tests, with both leaf boxes.
struct LeafJob {
  int q, la, lb, mode;
  float4 alo, ahi, blo, bhi;
};

struct WarpScratch {
  LeafStage stage;
  LeafJob jobs[32];
};

constexpr size_t kLeafStageBytes = sizeof(WarpScratch);

__global__ void k_traverse(TravArgs a, int stack_cap);
__global__ void k_frontier(TravArgs a, FrontierArgs f);
size_t frontier_smem_bytes();  // dynamic shared memory of a k_frontier block (256 threads)
__global__ void k_frontier_seed(TravArgs a, FrontierArgs f, int which, int seed_distance);
__global__ void k_frontier_zero(FrontierArgs f);
__global__ void k_frontier_top(TravArgs a, FrontierArgs f, unsigned int max_items);
__global__ void k_reset_state(TravArgs a);
__global__ void k_queue_init(Queue Q);
__global__ void k_seed(TravArgs a, int seed_distance);
__global__ void k_seed_phase1(TravArgs a);
__global__ void k_dive(TravArgs a, int dives, int restricted, int op, const int* rows, int nrows);
__global__ void k_prepare_pass2(TravArgs a);
__global__ void k_finalize(TravArgs a);
__global__ void k_write_results(TravArgs a, double* dist, unsigned char* hit, int* status, long long* witness,
                                int* cluster);
__global__ void k_witness(TravArgs a);
__global__ void k_witness_label(TravArgs a);
__global__ void k_set_proposal(TravArgs a, const int* top, int k, const int* rows, int nrows);

}  // namespace g3d
