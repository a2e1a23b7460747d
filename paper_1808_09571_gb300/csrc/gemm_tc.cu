// Forward pass of the proposal network on the 5th-generation tensor cores:
// tcgen05.mma (BF16 operands, FP32 accumulation in tensor memory), operand
// tiles brought into shared memory by TMA (cp.async.bulk.tensor with 128-byte
// swizzle), the accumulator read back with tcgen05.ld for the bias / ReLU
// epilogue.
//
// One CTA of 4 warps computes a 128 x BN tile of C = A B^T + bias, A [M x K]
// and B [N x K] both K-major BF16 (B is the layer's weight matrix transposed,
// converted once per parameter change).  BN is 64 for the 256-wide hidden
// layers (4 CTAs per 128 rows: the batches are a few hundred rows, so the
// N split is what spreads a layer over SMs) and 256 for the 4,096-wide output
// layer.  Thread 0 drives a 4-stage pipeline: it issues the MMAs of k-block
// kb (K = 16 each, 4 per 64-wide k-block) as soon as its tiles have landed,
// commits them to that stage's "free" barrier, and refills the stage of
// k-block kb - 1 (whose MMAs were issued one step earlier) with k-block
// kb + 3, so that the TMA loads of three k-blocks are in flight while the
// tensor core works.  A last commit signals the end of the accumulation; the
// 4 warps then read their 32 rows of the 128 x BN FP32 accumulator and store
// 16 bytes at a time.  Rows past M are zero (TMA fills them) and not stored.
// Every wait is bounded: past the limit the kernel records G3D_ERR_TIMEOUT,
// waits (bounded) for the loads it still has in flight, skips the epilogue
// and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "gemm_tc.cuh"

namespace g3d {

constexpr int kTcM = 128, kTcK = 64;  // CTA rows and k-block
constexpr int kTcStages = 4;
constexpr unsigned int kTcABytes = kTcM * kTcK * 2;  // 16 KB

template <int BN>
struct TcTile {
  static constexpr unsigned int kBBytes = BN * kTcK * 2;
  static constexpr unsigned int kStageBytes = kTcABytes + kBBytes;  // multiple of 1024
  static constexpr size_t kSmem = 1024 + kTcStages * kStageBytes + 256;
  // Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
  // (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits
  // 24-28.
  static constexpr unsigned int kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned int)(BN >> 3) << 17) |
                                         ((unsigned int)(kTcM >> 4) << 24);
};

__device__ __forceinline__ unsigned int tc_smem(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long tc_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool tc_try_wait(unsigned int bar, unsigned int parity) {
  unsigned int done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait on phase `parity` of mbarrier `bar`
__device__ __forceinline__ bool tc_wait(unsigned int bar, unsigned int parity, unsigned long long limit_ns) {
  const unsigned long long t0 = tc_now();
  int spins = 0;
  while (!tc_try_wait(bar, parity)) {
    if ((++spins & 255) == 0 && tc_now() - t0 > limit_ns) return false;
  }
  return true;
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// start address >> 4, leading byte offset (unused for this layout) 16 >> 4,
// stride byte offset 1024 >> 4 (8 rows of 128 bytes), descriptor version 1
// (bits 46-47), swizzle mode 2 = 128 bytes (bits 61-63).
__device__ __forceinline__ unsigned long long tc_desc(unsigned int saddr) {
  return (unsigned long long)((saddr >> 4) & 0x3fffu) | ((unsigned long long)1u << 16) |
         ((unsigned long long)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// bias + ReLU of 32 accumulator columns of one row, stored 16 bytes at a time
__device__ __forceinline__ void tc_store32(const unsigned int (&v)[32], const float* bias, int relu, float* c32,
                                           __nv_bfloat16* c16) {
  float x[32];
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 b = bias ? __ldg((const float4*)(bias + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
    x[j] = __uint_as_float(v[j]) + b.x;
    x[j + 1] = __uint_as_float(v[j + 1]) + b.y;
    x[j + 2] = __uint_as_float(v[j + 2]) + b.z;
    x[j + 3] = __uint_as_float(v[j + 3]) + b.w;
  }
  if (relu) {
#pragma unroll
    for (int j = 0; j < 32; j++) x[j] = fmaxf(x[j], 0.f);
  }
  if (c32) {
#pragma unroll
    for (int j = 0; j < 32; j += 4) *(float4*)(c32 + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
  }
  if (c16) {
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
      uint4 u;
      __nv_bfloat162 h;
      h = __floats2bfloat162_rn(x[j], x[j + 1]); u.x = *(unsigned int*)&h;
      h = __floats2bfloat162_rn(x[j + 2], x[j + 3]); u.y = *(unsigned int*)&h;
      h = __floats2bfloat162_rn(x[j + 4], x[j + 5]); u.z = *(unsigned int*)&h;
      h = __floats2bfloat162_rn(x[j + 6], x[j + 7]); u.w = *(unsigned int*)&h;
      *(uint4*)(c16 + j) = u;
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                    const __grid_constant__ CUtensorMap tb, TcGemmArgs g) {
  using T = TcTile<BN>;
  extern __shared__ unsigned char tc_raw[];
  // 1024-byte aligned staging (the 128-byte swizzle pattern repeats every 8 rows)
  const unsigned int raw = tc_smem(tc_raw);
  const unsigned int base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = tc_raw + (base - raw);
  const unsigned int bar_full = base + kTcStages * T::kStageBytes;  // [kTcStages] x 8 B
  const unsigned int bar_free = bar_full + 8 * kTcStages;           // [kTcStages] x 8 B
  const unsigned int bar_acc = bar_free + 8 * kTcStages;
  const unsigned int tmem_slot = bar_acc + 8;
  volatile unsigned int* tmem_slot_p = (volatile unsigned int*)(gbase + (tmem_slot - base));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * BN;
  const int nk = g.K / kTcK;

  if (warp == 0) {  // tensor memory: BN columns x 128 lanes of FP32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot), "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < kTcStages; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_full + 8 * s) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_free + 8 * s) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_acc) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned int tmem = *tmem_slot_p;

  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    auto load = [&](int kb, int s) {
      const unsigned int sa = base + s * T::kStageBytes, sb = sa + kTcABytes;
      const unsigned int fb = bar_full + 8 * s;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(T::kStageBytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
              "r"(sa),
          "l"((unsigned long long)&ta), "r"(kb * kTcK), "r"(m0), "r"(fb)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
              "r"(sb),
          "l"((unsigned long long)&tb), "r"(kb * kTcK), "r"(n0), "r"(fb)
          : "memory");
    };
    int issued = 0;    // k-blocks whose loads were issued (0 .. issued-1)
    int consumed = 0;  // k-blocks whose tiles have landed (waited on)
    for (; issued < kTcStages && issued < nk; issued++) load(issued, issued);
    for (int kb = 0; kb < nk; kb++) {
      const int s = kb % kTcStages;
      if (!tc_wait(bar_full + 8 * s, (unsigned int)(kb / kTcStages) & 1u, g.limit_ns)) { ok = 0; break; }
      consumed = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned int sa = base + s * T::kStageBytes, sb = sa + kTcABytes;
#pragma unroll
      for (int k = 0; k < kTcK / 16; k++) {
        const unsigned long long da = tc_desc(sa + 32 * k), db = tc_desc(sb + 32 * k);
        const unsigned int acc = (kb > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(T::kIdesc), "r"(acc)
            : "memory");
      }
      // the stage is free once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bar_free + 8 * s)
                   : "memory");
      // refill the stage of the previous k-block (its MMAs were issued a
      // step earlier, so this wait overlaps the ones just issued)
      if (kb >= 1 && issued < nk) {
        const int p = kb - 1, ps = p % kTcStages;
        if (!tc_wait(bar_free + 8 * ps, (unsigned int)(p / kTcStages) & 1u, g.limit_ns)) { ok = 0; break; }
        load(issued, ps);
        issued++;
      }
    }
    // completion of every MMA issued above
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_acc)
                 : "memory");
    // after a timeout: the loads still in flight land before the CTA ends
    for (int kb = consumed; !ok && kb < issued; kb++)
      tc_wait(bar_full + 8 * (kb % kTcStages), (unsigned int)(kb / kTcStages) & 1u, g.limit_ns);
    s_ok = ok;
  }
  __syncthreads();
  bool ok = s_ok != 0 && tc_wait(bar_acc, 0u, g.limit_ns);
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // warp w reads accumulator lanes 32 w .. 32 w + 31 = rows m0 + 32 w + lane
    const int row = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      unsigned int v[32];
      const unsigned int taddr = tmem + ((unsigned int)(32 * warp) << 16) + (unsigned int)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < g.M) {
        const size_t o = (size_t)row * g.ldc + n0 + c0;
        tc_store32(v, g.bias ? g.bias + n0 + c0 : nullptr, g.relu, g.C32 ? g.C32 + o : nullptr,
                   g.C16 ? g.C16 + o : nullptr);
      }
    }
  } else if (threadIdx.x == 0 && g.err) {
    atomicCAS(g.err, 0, G3D_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// BF16 copy of a row-major float32 matrix [R x Cc] (the activations)
__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// BF16 transpose of a row-major float32 matrix W [K x N] into Wt [N x K]
__global__ void k_transpose_bf16(const float* __restrict__ W, __nv_bfloat16* __restrict__ Wt, int K, int N) {
  __shared__ float t[32][33];
  const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, n = n0 + threadIdx.x;
    t[r][threadIdx.x] = (k < K && n < N) ? W[(size_t)k * N + n] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, k = k0 + threadIdx.x;
    if (n < N && k < K) Wt[(size_t)n * K + k] = __float2bfloat16_rn(t[threadIdx.x][r]);
  }
}

namespace {
std::mutex g_tc_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  std::lock_guard<std::mutex> lock(g_tc_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    cudaGetLastError();
  }
  return g_encode;
}

// 2D tensor map of a row-major BF16 matrix [rows x K], box 64 x box_rows,
// 128-byte swizzle, zero fill out of bounds
bool make_map(CUtensorMap* m, const void* ptr, int rows, int K, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

// N tile of a layer: 256 for wide outputs, 64 for the 256-wide hidden layers
static int tc_bn(int N) { return (N % 256 == 0 && N >= 1024) ? 256 : 64; }

bool tc_gemm_supported(int M, int N, int K) {
  return M >= 1 && N % tc_bn(N) == 0 && K % kTcK == 0 && K >= kTcK;
}

int tc_gemm_setup() {
  static int state = 0;  // 0 unknown, 1 ready, -1 unavailable
  if (state == 0) {
    state = (tensor_map_encoder() &&
             cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TcTile<64>::kSmem) == cudaSuccess &&
             cudaFuncSetAttribute(k_gemm_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TcTile<256>::kSmem) == cudaSuccess)
                ? 1
                : -1;
    cudaGetLastError();
  }
  return state;
}

cudaError_t tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* Bt, TcGemmArgs g, cudaStream_t s) {
  if (tc_gemm_setup() != 1 || !tc_gemm_supported(g.M, g.N, g.K)) return cudaErrorNotSupported;
  // 16-byte accesses: operands, outputs, bias and row pitch on 16-byte boundaries
  if (((uintptr_t)A & 15) || ((uintptr_t)Bt & 15) || ((uintptr_t)g.C32 & 15) || ((uintptr_t)g.C16 & 15) ||
      ((uintptr_t)g.bias & 15) || (g.ldc & 7) || g.ldc < g.N)
    return cudaErrorMisalignedAddress;
  const int bn = tc_bn(g.N);
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, g.M, g.K, kTcM) || !make_map(&tb, Bt, g.N, g.K, bn)) return cudaErrorInvalidValue;
  dim3 grid((g.M + kTcM - 1) / kTcM, g.N / bn);
  if (bn == 256)
    k_gemm_tc<256><<<grid, 128, TcTile<256>::kSmem, s>>>(ta, tb, g);
  else
    k_gemm_tc<64><<<grid, 128, TcTile<64>::kSmem, s>>>(ta, tb, g);
  return cudaGetLastError();
}

cudaError_t to_bf16(const float* x, __nv_bfloat16* y, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_to_bf16<<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

void transpose_bf16(const float* W, __nv_bfloat16* Wt, int K, int N, cudaStream_t s) {
  dim3 grid((N + 31) / 32, (K + 31) / 32), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, s>>>(W, Wt, K, N);
}

}  // namespace g3d
