// Distance between two triangle soups without any device allocation.
//
// Some callers cannot allocate device memory: a host application whose
// device memory is owned by its own allocator or budgeted up front (a
// database engine, a renderer or a simulation hosting this library as a
// plug-in), or a real-time pipeline that must not call cudaMalloc once it
// runs (an allocation can synchronise the device and take unbounded time).
// This entry point serves them: the caller passes the faces and the output
// in its own device memory, and the working memory (the certified upper
// bound, flags and the FP64 minimum) lives in one file-scope __device__ array
// of fixed size.  Every GPU that loads the library holds that array until the
// process exits.
//
// It is the face-pair test and finalisation of the traversal path applied to
// all face pairs (no BVH), in two passes over the same pairs so that the work
// depends only on the input:
//   1. every pair gets certified FP32 bounds; the pass lowers the shared
//      upper bound UB to the smallest certified upper bound and ends early
//      when the filtered orientation test certifies an intersection;
//   2. every pair whose certified lower bound does not exceed the final UB
//      (the only pairs that can attain the minimum) is recomputed in FP64
//      and, when it may intersect, decided exactly.
// No candidate list is kept, so nothing can overflow.
#include <cuda_runtime.h>

#include <mutex>

#include "fp32_tests.cuh"
#include "fp64_exact.cuh"
#include "internal.cuh"

namespace g3d {

constexpr long long kNoAllocMaxPairs = 1ll << 26;  // na * nb

struct NoAllocHeader {
  unsigned int ub;          // certified upper bound (float bits)
  int done;                 // an intersection was certified in pass 1
  int hit;                  // an exact intersection was found in pass 2
  int bad;                  // input flags: 1 non-finite coordinate, 2 |coordinate| > 2^60
  unsigned long long best;  // FP64 minimum squared distance (double bits)
};

constexpr size_t kNoAllocBytes = 256;

// The scratch array.  In host code this name is only a host-side stand-in:
// the device address is obtained per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void k_noalloc_reset(unsigned char* scratch) {
  NoAllocHeader* h = (NoAllocHeader*)scratch;
  h->ub = __float_as_uint(INFINITY);
  h->done = 0;
  h->hit = 0;
  h->bad = 0;
  h->best = (unsigned long long)__double_as_longlong(INFINITY);
}

// The same input rules as the mesh ingest: NaN / Inf and |x| > 2^60 (beyond
// which float32 squares and the exact predicates leave their range) are
// errors.
__global__ void k_noalloc_check(const float* __restrict__ A, long long na, const float* __restrict__ B,
                                long long nb, unsigned char* scratch) {
  NoAllocHeader* h = (NoAllocHeader*)scratch;
  const long long n = 9 * (na + nb);
  int f = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const float x = k < 9 * na ? A[k] : B[k - 9 * na];
    if (!isfinite(x)) f |= 1;
    else if (fabsf(x) > 1.152921504606846976e18f) f |= 2;
  }
  if (f) atomicOr(&h->bad, f);
}

__device__ __forceinline__ void load_pair(const float* A, const float* B, long long i, long long j, float3& A0,
                                          float3& A1, float3& A2, float3& B0, float3& B1, float3& B2) {
  const float* fa = A + 9 * i;
  const float* fb = B + 9 * j;
  A0 = make_float3(fa[0], fa[1], fa[2]); A1 = make_float3(fa[3], fa[4], fa[5]); A2 = make_float3(fa[6], fa[7], fa[8]);
  B0 = make_float3(fb[0], fb[1], fb[2]); B1 = make_float3(fb[3], fb[4], fb[5]); B2 = make_float3(fb[6], fb[7], fb[8]);
}

// pass 1: the smallest certified upper bound over all pairs, or a certified
// intersection
__global__ void __launch_bounds__(256) k_noalloc_bound(const float* __restrict__ A, long long na,
                                                       const float* __restrict__ B, long long nb,
                                                       unsigned char* scratch) {
  NoAllocHeader* h = (NoAllocHeader*)scratch;
  if (h->bad) return;
  const long long np = na * nb;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    if (*(volatile int*)&h->done) return;
    const long long i = p / nb, j = p - i * nb;
    float3 A0, A1, A2, B0, B1, B2;
    load_pair(A, B, i, j, A0, A1, A2, B0, B1, B2);
    const float ub = __uint_as_float(*(volatile unsigned int*)&h->ub);
    if (tri_boxes_lb(A0, A1, A2, B0, B1, B2) > ub) continue;
    const PairBounds pb = tri_pair_bounds_rolled(A + 9 * i, B + 9 * j);
    if (pb.ub < ub) atomicMin(&h->ub, __float_as_uint(pb.ub));
    if (pb.lb <= 0.f && tri_isect_filter_s(A + 9 * i, B + 9 * j) == ISECT_YES) {
      atomicExch(&h->done, 1);
      atomicMin(&h->ub, 0u);
      return;
    }
  }
}

// pass 2: FP64 distance (and the exact test where the faces may meet) of
// every pair whose certified lower bound does not exceed the final UB
__global__ void __launch_bounds__(128) k_noalloc_exact(const float* __restrict__ A, long long na,
                                                       const float* __restrict__ B, long long nb,
                                                       unsigned char* scratch) {
  NoAllocHeader* h = (NoAllocHeader*)scratch;
  if (h->bad || h->done) return;
  const float ub = __uint_as_float(h->ub);
  const long long np = na * nb;
  unsigned long long best = (unsigned long long)__double_as_longlong(INFINITY);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    const long long i = p / nb, j = p - i * nb;
    float3 A0, A1, A2, B0, B1, B2;
    load_pair(A, B, i, j, A0, A1, A2, B0, B1, B2);
    if (tri_boxes_lb(A0, A1, A2, B0, B1, B2) > ub) continue;
    const PairBounds pb = tri_pair_bounds_rolled(A + 9 * i, B + 9 * j);
    if (pb.lb > ub) continue;
    double fa[9], fb[9];
    for (int t = 0; t < 9; t++) {
      fa[t] = A[9 * i + t];
      fb[t] = B[9 * j + t];
    }
    if (pb.lb <= 0.f && tri_isect_filter_s(A + 9 * i, B + 9 * j) != ISECT_NO) {
      ExactCounter ctr;
      if (tri_isect_exact(fa, fb, ctr)) {
        atomicExch(&h->hit, 1);
        continue;
      }
    }
    const unsigned long long d2 = (unsigned long long)__double_as_longlong(tri_dist2_f64(fa, fb));
    if (d2 < best) best = d2;
  }
  if (best != (unsigned long long)__double_as_longlong(INFINITY)) atomicMin(&h->best, best);
}

__global__ void k_noalloc_write(const unsigned char* scratch, double* out, int* status) {
  const NoAllocHeader* h = (const NoAllocHeader*)scratch;
  int st = 0;
  double d;
  if (h->bad) {
    st = (h->bad & 1) ? G3D_ERR_NAN_INPUT : G3D_ERR_RANGE;
    d = __longlong_as_double(0x7ff8000000000000ll);
  } else if (h->done || h->hit) {
    d = 0.0;
  } else {
    d = sqrt(__longlong_as_double((long long)h->best));
  }
  *out = d;
  *status = st;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
int g_noalloc_sms[kMaxDevices] = {};

// Device address of the scratch array and the SM count of the current
// device, looked up once per device (that device must be current).
cudaError_t noalloc_setup(int* dev_out, void** ptr_out, int* sms_out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_sms[dev] = sms > 0 ? sms : 1;
    g_noalloc_ptr[dev] = p;
  }
  *dev_out = dev;
  *ptr_out = g_noalloc_ptr[dev];
  *sms_out = g_noalloc_sms[dev];
  return cudaSuccess;
}

// memory the current device `dev` can dereference: its own device memory,
// or managed memory
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

unsigned int grid_of(long long work, int block, int sms, int per_sm) {
  long long g = (work + block - 1) / block;
  const long long cap = (long long)sms * per_sm;
  if (g > cap) g = cap;
  return (unsigned int)(g > 0 ? g : 1);
}
}  // namespace

}  // namespace g3d

extern "C" int g3d_distance_soup_noalloc(const float* faces_a, int64_t na, const float* faces_b, int64_t nb,
                                         double* out, int32_t* status_out, void* stream) {
  using namespace g3d;
  if (!faces_a || !faces_b || !out || !status_out || na <= 0 || nb <= 0) return G3D_ERR_INVALID_ARG;
  if (na > kNoAllocMaxPairs / nb) return G3D_ERR_TOO_LARGE;
  int dev = -1, sms = 0;
  void* scratch = nullptr;
  if (noalloc_setup(&dev, &scratch, &sms) != cudaSuccess) return G3D_ERR_CUDA;
  if (!on_device(faces_a, dev) || !on_device(faces_b, dev) || !on_device(out, dev) || !on_device(status_out, dev))
    return G3D_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* sc = (unsigned char*)scratch;
  const long long np = (long long)na * nb;
  k_noalloc_reset<<<1, 1, 0, s>>>(sc);
  k_noalloc_check<<<grid_of(9 * (na + nb), 256, sms, 4), 256, 0, s>>>(faces_a, na, faces_b, nb, sc);
  k_noalloc_bound<<<grid_of(np, 256, sms, 8), 256, 0, s>>>(faces_a, na, faces_b, nb, sc);
  k_noalloc_exact<<<grid_of(np, 128, sms, 16), 128, 0, s>>>(faces_a, na, faces_b, nb, sc);
  k_noalloc_write<<<1, 1, 0, s>>>(sc, out, (int*)status_out);
  return cudaGetLastError() == cudaSuccess ? G3D_OK : G3D_ERR_CUDA;
}
