// Declarations of the learned-proposal kernels (mlp.cu).
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace g3d {

constexpr int kClusters = 64;         // Morton-ordered face clusters per mesh
constexpr int kClusterStride = 16;    // floats of per-cluster statistics
constexpr int kFeatPerCluster = 12;   // box lo/hi (6), centroid (3), mean normal (3)
constexpr int kFeatIn = 2 * kClusters * kFeatPerCluster;  // 1536
constexpr int kHidden = 256;
constexpr int kFeatOut = kClusters * kClusters;           // 4096 cluster pairs
// flat FP32 parameter layout: W1 [1536 x 256], b1, W2 [256 x 256], b2,
// W3 [256 x 256], b3, W4 [256 x 4096], b4
constexpr long long kOffW1 = 0;
constexpr long long kOffB1 = kOffW1 + (long long)kFeatIn * kHidden;
constexpr long long kOffW2 = kOffB1 + kHidden;
constexpr long long kOffB2 = kOffW2 + (long long)kHidden * kHidden;
constexpr long long kOffW3 = kOffB2 + kHidden;
constexpr long long kOffB3 = kOffW3 + (long long)kHidden * kHidden;
constexpr long long kOffW4 = kOffB3 + kHidden;
constexpr long long kOffB4 = kOffW4 + (long long)kHidden * kFeatOut;
constexpr long long kNumParams = kOffB4 + kFeatOut;

struct GemmArgs {
  const float* A;
  long long as0, as1;  // A(i, k) = A[i * as0 + k * as1]
  const float* B;
  long long bs0, bs1;  // B(k, j) = B[k * bs0 + j * bs1]
  float* C;
  long long ldc;
  const float* bias;   // [N] or null
  int relu;
  int M, N, K;
};

struct ClusterMesh {
  const float4 *v0, *v1, *v2;
  long long nt;
  float* out;  // [64 x 16] statistics
};

struct PairFeatArgs {
  const QueryDev* q;  // queries (their meshes' cluster statistics)
  float* X;           // [rows x 1536]
  const int* rows;    // query of feature row r (null: row r is query r)
};

__global__ void k_gemm_bf16(GemmArgs g);
__global__ void k_relu_bwd(float* d, const float* post, long long n);
__global__ void k_colsum(const float* dY, int M, int N, float* db);
__global__ void k_softmax_ce(float* logits, const int* labels, int N, int B, float* loss);
__global__ void k_sample_batch(const float* X, const int* labels, long long n, unsigned long long seed, long long step,
                               float* Xb, int* Yb);
__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2);
__global__ void k_topk(const float* logits, int N, int k, int* out);
__global__ void k_cluster_stats(const ClusterMesh* ms, int n);
__global__ void k_pair_features(const PairFeatArgs a);

}  // namespace g3d
