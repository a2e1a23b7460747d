// Distance between two triangle soups without any device allocation.
//
// Some callers cannot allocate device memory: code running while a CUDA
// graph is being captured, hosts whose memory is owned by their own
// allocator or budgeted up front, embedded or real-time pipelines that must
// not call cudaMalloc after start-up.  This entry point serves them: the
// caller passes the faces and the output in its own device memory, and the
// working memory (the certified upper bound, flags and the candidate list)
// lives in one file-scope __device__ array of fixed size.  Every GPU that
// loads the library holds that array until the process exits.
//
// It is the face-pair test and finalisation of the traversal path applied to
// all face pairs (no BVH): each pair gets certified FP32 bounds (and the
// filtered orientation test when it may intersect), pairs whose lower bound
// does not exceed the running upper bound are kept, and the kept pairs are
// recomputed in FP64 and, where needed, decided exactly.
#include <cuda_runtime.h>

#include <mutex>

#include "fp32_tests.cuh"
#include "fp64_exact.cuh"
#include "internal.cuh"

namespace g3d {

constexpr long long kNoAllocMaxPairs = 1ll << 26;  // na * nb
constexpr int kNoAllocMaxCand = 1 << 16;           // kept face pairs

struct NoAllocHeader {
  unsigned int ub;          // certified upper bound (float bits)
  int done;                 // an intersection was certified
  int ncand;                // candidate pushes (may exceed the capacity)
  int hit;                  // exact intersection found in the finalisation
  unsigned long long best;  // FP64 minimum squared distance (double bits)
};

constexpr size_t kNoAllocBytes = 256 + sizeof(int4) * (size_t)kNoAllocMaxCand;  // about 1 MiB

// The scratch array.  In host code this name is only a host-side stand-in:
// the device address is obtained per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void k_noalloc_reset(unsigned char* scratch) {
  NoAllocHeader* h = (NoAllocHeader*)scratch;
  h->ub = __float_as_uint(INFINITY);
  h->done = 0;
  h->ncand = 0;
  h->hit = 0;
  h->best = (unsigned long long)__double_as_longlong(INFINITY);
}

__global__ void __launch_bounds__(256) k_noalloc_pairs(const float* __restrict__ A, long long na,
                                                       const float* __restrict__ B, long long nb,
                                                       unsigned char* scratch) {
  NoAllocHeader* h = (NoAllocHeader*)scratch;
  int4* cand = (int4*)(scratch + 256);
  const long long np = na * nb;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    if (*(volatile int*)&h->done) return;
    const long long i = p / nb, j = p - i * nb;
    const float* fa = A + 9 * i;
    const float* fb = B + 9 * j;
    const float3 A0 = make_float3(fa[0], fa[1], fa[2]), A1 = make_float3(fa[3], fa[4], fa[5]),
                 A2 = make_float3(fa[6], fa[7], fa[8]);
    const float3 B0 = make_float3(fb[0], fb[1], fb[2]), B1 = make_float3(fb[3], fb[4], fb[5]),
                 B2 = make_float3(fb[6], fb[7], fb[8]);
    const float ub = __uint_as_float(*(volatile unsigned int*)&h->ub);
    if (tri_boxes_lb(A0, A1, A2, B0, B1, B2) > ub) continue;
    const PairBounds pb = tri_pair_bounds_rolled(fa, fb);
    if (pb.ub < ub) atomicMin(&h->ub, __float_as_uint(pb.ub));
    if (pb.lb > fminf(ub, pb.ub)) continue;
    int flags = 0;
    if (pb.lb <= 0.f) {
      const int r = tri_isect_filter_s(fa, fb);
      if (r == ISECT_YES) {
        atomicExch(&h->done, 1);
        atomicMin(&h->ub, 0u);
        return;
      }
      if (r == ISECT_UNSURE) flags = CAND_NEEDS_EXACT;
    }
    const int k = atomicAdd(&h->ncand, 1);
    if (k < kNoAllocMaxCand) cand[k] = make_int4((int)i, (int)j, __float_as_int(pb.lb), flags);
  }
}

__global__ void __launch_bounds__(128) k_noalloc_finalize(const float* __restrict__ A, const float* __restrict__ B,
                                                          unsigned char* scratch) {
  NoAllocHeader* h = (NoAllocHeader*)scratch;
  const int4* cand = (const int4*)(scratch + 256);
  if (h->done) return;
  const int n = min(h->ncand, kNoAllocMaxCand);
  const float ub = __uint_as_float(h->ub);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int4 c = cand[k];
    if (__int_as_float(c.z) > ub) continue;
    double fa[9], fb[9];
    for (int t = 0; t < 9; t++) {
      fa[t] = A[9ll * c.x + t];
      fb[t] = B[9ll * c.y + t];
    }
    if (c.w & CAND_NEEDS_EXACT) {
      ExactCounter ctr;
      if (tri_isect_exact(fa, fb, ctr)) {
        atomicExch(&h->hit, 1);
        continue;
      }
    }
    atomicMin(&h->best, (unsigned long long)__double_as_longlong(tri_dist2_f64(fa, fb)));
  }
}

__global__ void k_noalloc_write(const unsigned char* scratch, double* out, int* status) {
  const NoAllocHeader* h = (const NoAllocHeader*)scratch;
  int st = 0;
  double d;
  if (h->done || h->hit) {
    d = 0.0;
  } else if (h->ncand > kNoAllocMaxCand) {
    st = G3D_ERR_CAND_OVERFLOW;
    d = __longlong_as_double(0x7ff8000000000000ll);
  } else {
    d = sqrt(__longlong_as_double((long long)h->best));
  }
  *out = d;
  if (status) *status = st;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the device must be current).
cudaError_t noalloc_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace

}  // namespace g3d

extern "C" int g3d_distance_soup_noalloc(const float* faces_a, int64_t na, const float* faces_b, int64_t nb,
                                         double* out, int32_t* status_out, void* stream) {
  using namespace g3d;
  if (!faces_a || !faces_b || !out || na <= 0 || nb <= 0) return G3D_ERR_INVALID_ARG;
  if (na > kNoAllocMaxPairs / nb) return G3D_ERR_TOO_LARGE;
  if (!on_device(faces_a) || !on_device(faces_b) || !on_device(out) || (status_out && !on_device(status_out)))
    return G3D_ERR_INVALID_ARG;
  void* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return G3D_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* sc = (unsigned char*)scratch;
  const long long np = (long long)na * nb;
  long long blocks = (np + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_noalloc_reset<<<1, 1, 0, s>>>(sc);
  k_noalloc_pairs<<<(unsigned int)blocks, 256, 0, s>>>(faces_a, na, faces_b, nb, sc);
  k_noalloc_finalize<<<64, 128, 0, s>>>(faces_a, faces_b, sc);
  k_noalloc_write<<<1, 1, 0, s>>>(sc, out, (int*)status_out);
  return cudaGetLastError() == cudaSuccess ? G3D_OK : G3D_ERR_CUDA;
}
