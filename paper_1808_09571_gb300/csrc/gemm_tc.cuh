// Declarations of the tcgen05 GEMM of the proposal network (gemm_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.cuh"

namespace g3d {

// C = A B^T + bias (ReLU), A [M x K] and B [N x K] row-major BF16 in device
// memory (16-byte aligned), N a multiple of 256, K a multiple of 64; C32
// (FP32) and / or C16 (BF16) [M x N] with leading dimension ldc (either may
// be null).  err (device, may be null) receives G3D_ERR_TIMEOUT when a wait
// of the kernel exceeds limit_ns.
struct TcGemmArgs {
  int M, N, K;
  const float* bias;
  int relu;
  float* C32;
  __nv_bfloat16* C16;
  long long ldc;
  int* err;
  unsigned long long limit_ns;
};

bool tc_gemm_supported(int M, int N, int K);
int tc_gemm_setup();  // 1 when the tensor-core path is available
cudaError_t tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* Bt, TcGemmArgs g, cudaStream_t s);
cudaError_t to_bf16(const float* x, __nv_bfloat16* y, long long n, cudaStream_t s);
void transpose_bf16(const float* W, __nv_bfloat16* Wt, int K, int N, cudaStream_t s);

}  // namespace g3d
