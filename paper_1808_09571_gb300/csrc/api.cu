// C ABI of geo3d (declared in include/geo3d.h): context, mesh store, BVH
// build orchestration and query launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "build.cuh"
#include "gemm_tc.cuh"
#include "segments.cuh"
#include "volume.cuh"
#include "internal.cuh"
#include "mlp.cuh"
#include "traverse.cuh"

using namespace g3d;

// Device memory of the meshes loaded (or built) by one call: one block,
// sub-allocated, released when the last mesh using it is freed or rebuilt.
// (One allocation per call instead of several per mesh: calls with tens of
// thousands of small meshes were dominated by allocator calls.)
struct Slab {
  void* base = nullptr;
  long long refs = 0;
};

struct G3dMesh {
  MeshDev dev{};
  Slab* raw_slab = nullptr;  // holds raw_v (+ box) and raw_i
  Slab* bvh_slab = nullptr;  // holds v0 .. m64
  void* raw_v = nullptr;
  uint32_t* raw_i = nullptr;
  int dtype = G3D_F32;
  int64_t nv = 0, nt = 0;
  bool master = false;
  bool has_bvh = false;
  float rho = 0.f;
  // permanent BVH arrays
  float4 *v0 = nullptr, *v1 = nullptr, *v2 = nullptr, *nodes = nullptr, *leaves = nullptr;
  double* m64 = nullptr;
  int2* nrange = nullptr;
  float* cstats = nullptr;
  unsigned int* box = nullptr;  // [6] vertex box from the ingest (in the tail of raw_v)
  bool cstats_valid = false;  // statistics computed for the current BVH (on first use)
};

struct g3d_ctx {
  int device = 0;
  int num_sms = 0;
  int smem_per_sm = 0;       // shared memory per SM at the largest carve-out (bytes)
  int regs_per_sm = 0;
  int max_warps_per_sm = 0, max_ctas_per_sm = 0;
  int trav_carveout = -1;    // carve-out (percent) last set on the traversal kernel
  // level-synchronous traversal: frontier / leaf-list buffers, counters and
  // the cooperative grid (blocks resident at once)
  FrontierArgs fr{};
  int4* fr_items = nullptr;
  unsigned int* fr_cnt = nullptr;
  // first-visit bitmap of the batch being run (count_visits), else null
  unsigned int* visit = nullptr;
  long long* visit_off = nullptr;
  g3d_config cfg{};
  std::unordered_map<int64_t, G3dMesh*> meshes;
  int64_t next_id = 1;
  // traversal buffers
  Queue queue{};
  CandPool cand{};
  unsigned long long* stats = nullptr;
  QueryDev* qdev = nullptr;  // capacity qcap
  QueryState* st = nullptr;
  int qcap = 0;
  double* d_dist = nullptr;
  unsigned char* d_hit = nullptr;
  int* d_status = nullptr;
  int* d_sticky = nullptr;     // first per-query error since the last sync
  int* d_dbg = nullptr;        // first invalid item seen (diagnostics)
  int* h_pinned = nullptr;     // 8 ints of pinned host scratch
  unsigned long long t_limit_ns = 30ull * 1000000000ull;
  // learned proposal used by distance queries (null = off) and its scratch
  struct g3d_mlp* proposal = nullptr;
  float* prop_X = nullptr;
  int* prop_top = nullptr;
  int prop_cap = 0;
  // queries of the next launch the network proposes for (device list and
  // its length; -1: every query): batch calls set it from the mesh sizes
  int* prop_rows = nullptr;
  int prop_rows_cap = 0;
  int prop_nrows = -1;
  const int* cur_prop_rows = nullptr;  // the row list of the proposal being launched
  int cur_prop_nrows = 0;
  struct Stage {
    void* p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
  } stage[2];  // pinned staging of batch uploads, used in turn
  int stage_i = 0;
  bool use_tc_gemm = true;  // proposal network forward on tcgen05 (false: mma.sync)
  // largest leaf size among the meshes of the launch being prepared (the
  // leaf stage width follows it; meshes of one batch may differ)
  int cur_leaf_max = 16;
  // launch accounting and optional per-kernel CUDA-event timing
  unsigned long long launches = 0;
  bool prof_on = false;
  bool capturing = false;  // launches go into a CUDA graph: no profiling events
  std::string prof_filter;
  struct ProfRec { const char* name; cudaEvent_t e0, e1; };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
};

namespace {

// NVTX range for the duration of a call (visible in timeline profilers)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return G3D_OK;
  if (e == cudaErrorMemoryAllocation) return G3D_ERR_OOM;
  return G3D_ERR_CUDA;
}

#define CK(x)                        \
  do {                               \
    cudaError_t _e = (x);            \
    if (_e != cudaSuccess) return cuda_err(_e); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The driver's cuMemGetAddressRange (looked up once through the runtime, no
// link to the driver library): base and size of the allocation holding a
// device address.
typedef int (*AddressRangeFn)(unsigned long long* base, size_t* size, unsigned long long dptr);

AddressRangeFn address_range_fn() {
  static const AddressRangeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return (AddressRangeFn)p;
  }();
  return fn;
}

// Device allocations met by one load call.  An array that lies inside a
// known device allocation needs no pointer-attribute query of its own: such
// a query costs about half a microsecond of host time, and a call loading
// tens of thousands of meshes made two per mesh, while their arrays sit in
// a few allocations (a caching allocator's segments).
class DeviceRanges {
  std::map<uintptr_t, uintptr_t> r_;  // allocation base -> end
 public:
  bool is_device(const void* p, size_t bytes) {
    const uintptr_t a = (uintptr_t)p;
    auto it = r_.upper_bound(a);
    if (it != r_.begin()) {
      --it;
      if (a >= it->first && a + bytes <= it->second) return true;
    }
    if (!is_device_ptr(p)) return false;
    if (AddressRangeFn fn = address_range_fn()) {
      unsigned long long base = 0;
      size_t size = 0;
      if (fn(&base, &size, (unsigned long long)a) == 0 && size > 0) r_[(uintptr_t)base] = (uintptr_t)base + size;
    }
    return true;
  }
};

G3dMesh* get_mesh(g3d_ctx* c, g3d_mesh h) {
  auto it = c->meshes.find(h);
  return it == c->meshes.end() ? nullptr : it->second;
}

template <class T>
cudaError_t amalloc(T** p, size_t n, cudaStream_t s) {
  return cudaMallocAsync((void**)p, n * sizeof(T) + 16, s);
}

void afree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

void slab_release(Slab*& sl, cudaStream_t s) {
  if (!sl) return;
  if (--sl->refs == 0) {
    cudaFreeAsync(sl->base, s);
    delete sl;
  }
  sl = nullptr;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

unsigned int grid_for(long long n, int block, int cap) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned int)g;
}

cudaEvent_t prof_event(g3d_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool prof_wants(g3d_ctx* c, const char* name) {
  return c->prof_on && !c->capturing &&
         (c->prof_filter.empty() || strstr(name, c->prof_filter.c_str()) != nullptr);
}

// Run F (which issues one launch on stream S and returns its error) and,
// while profiling, bracket it with CUDA events on S under NAME.
template <class F>
cudaError_t profiled(g3d_ctx* c, const char* name, cudaStream_t s, F f) {
  const bool p = prof_wants(c, name);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (p) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  const cudaError_t e = f();
  if (p) {
    cudaEventRecord(e1, s);
    c->prof.push_back({name, e0, e1});
  }
  return e;
}

// Launch a kernel on stream S, counting it and, while profiling, bracketing
// it with CUDA events on the same stream.
#define G3D_LAUNCH(C, NAME, KERN, GRID, BLOCK, SMEM, S, ...)                          \
  do {                                                                                \
    bool _p = prof_wants(C, NAME);                                                    \
    cudaEvent_t _e0 = nullptr, _e1 = nullptr;                                         \
    if (_p) {                                                                         \
      _e0 = prof_event(C);                                                            \
      _e1 = prof_event(C);                                                            \
      cudaEventRecord(_e0, S);                                                        \
    }                                                                                 \
    KERN<<<GRID, BLOCK, SMEM, S>>>(__VA_ARGS__);                                      \
    if (_p) {                                                                         \
      cudaEventRecord(_e1, S);                                                        \
      (C)->prof.push_back({NAME, _e0, _e1});                                          \
    }                                                                                 \
    (C)->launches++;                                                                  \
  } while (0)

// The level-synchronous traversal as one cooperative launch (its blocks
// wait on one another at a grid barrier, so all must be resident at once;
// the launch fails instead of starting otherwise).
int launch_frontier(g3d_ctx* c, const TravArgs& a, cudaStream_t s) {
  const bool p = prof_wants(c, "k_frontier");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (p) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  TravArgs ta = a;
  FrontierArgs fa = c->fr;
  void* args[] = {&ta, &fa};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_frontier, dim3(fa.nblocks), dim3(256), args,
                                                    frontier_smem_bytes(), s);
  if (p) {
    cudaEventRecord(e1, s);
    c->prof.push_back({"k_frontier", e0, e1});
  }
  c->launches++;
  return cuda_err(e);
}

__global__ void k_set_query(QueryDev* dst, QueryDev v) { *dst = v; }

int ensure_query_capacity(g3d_ctx* c, int n, cudaStream_t s) {
  if (n <= c->qcap) return G3D_OK;
  int cap = c->qcap ? c->qcap : 64;
  while (cap < n) cap *= 2;
  QueryDev* qd = nullptr;
  QueryState* st = nullptr;
  double* dd = nullptr;
  unsigned char* dh = nullptr;
  int* ds = nullptr;
  CK(cudaStreamSynchronize(s));
  CK(cudaMalloc(&qd, sizeof(QueryDev) * cap));
  CK(cudaMalloc(&st, sizeof(QueryState) * cap));
  CK(cudaMalloc(&dd, sizeof(double) * cap));
  CK(cudaMalloc(&dh, cap));
  CK(cudaMalloc(&ds, sizeof(int) * cap));
  cudaFree(c->qdev); cudaFree(c->st); cudaFree(c->d_dist); cudaFree(c->d_hit); cudaFree(c->d_status);
  c->qdev = qd; c->st = st; c->d_dist = dd; c->d_hit = dh; c->d_status = ds;
  c->qcap = cap;
  return G3D_OK;
}

TravArgs trav_args(g3d_ctx* c, int nq, const QueryDev* qd = nullptr, QueryState* st = nullptr) {
  TravArgs a{};
  a.q = qd ? qd : c->qdev;
  a.st = st ? st : c->st;
  a.nq = nq;
  a.queue = c->queue;
  a.cand = c->cand;
  a.stats = c->stats;
  a.t_limit_ns = c->t_limit_ns;
  a.total_warps = c->num_sms * c->cfg.ctas_per_sm * c->cfg.warps_per_cta;
  a.pass = 1;
  a.sticky = c->d_sticky;
  a.dbg = c->d_dbg;
  a.leaf_w = c->cur_leaf_max <= 8 ? 16 : 32;
  a.visit = c->visit;
  a.visit_off = c->visit_off;
  return a;
}

QueryDev make_query(const G3dMesh* A, const G3dMesh* B, int op) {
  QueryDev q{};
  q.A = A->dev;
  q.B = B->dev;
  q.op = op;
  float s = 0.f;
  if (A->rho > 0.f || B->rho > 0.f) {
    // sqrt(3) * (rho_A + rho_B), rounded up generously
    s = (float)(1.7320508075688774 * ((double)A->rho + (double)B->rho) * (1.0 + 1e-6));
  }
  q.slack = s;
  q.link = -1;
  q.dlink = -1;
  return q;
}

// seed -> traverse -> (pass 2) -> finalize -> results, all on `s`
// ---------------------------------------------------------------------------
// learned proposal network (host side of mlp.cu)
// ---------------------------------------------------------------------------
}  // namespace

struct g3d_mlp {
  float* params = nullptr;  // FP32 master weights [kNumParams]
  // tensor-core forward: BF16 transposed weights (current when bf16_version
  // == version; version counts parameter changes) and BF16 activations
  __nv_bfloat16* wt16 = nullptr;  // W1t [256 x 1536], W2t, W3t [256 x 256], W4t [4096 x 256]
  __nv_bfloat16* act16 = nullptr; // X [cap x 1536], h1, h2, h3 [cap x 256]
  int act16_cap = 0;
  long long version = 1, bf16_version = 0;
  float* grads = nullptr;
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  float* loss = nullptr;    // device scalar
  long long t = 0;          // Adam steps taken
  // activations: h1, h2, h3 [cap x 256], z [cap x 4096], dh [2 x cap x 256]
  float* ws = nullptr;
  int cap = 0;
};

namespace {

int mlp_reserve(g3d_mlp* p, int B, cudaStream_t s) {
  if (B <= p->cap) return G3D_OK;
  int cap = p->cap ? p->cap : 256;
  while (cap < B) cap *= 2;
  if (p->ws) cudaFreeAsync(p->ws, s);
  p->ws = nullptr;
  CK(cudaMallocAsync((void**)&p->ws, sizeof(float) * (size_t)cap * (5 * kHidden + kFeatOut), s));
  p->cap = cap;
  return G3D_OK;
}

void gemm(g3d_ctx* c, cudaStream_t s, const float* A, long long as0, long long as1, const float* B, long long bs0,
          long long bs1, float* C, long long ldc, const float* bias, int relu, int M, int N, int K) {
  GemmArgs g{A, as0, as1, B, bs0, bs1, C, ldc, bias, relu, M, N, K};
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  G3D_LAUNCH(c, "k_gemm_bf16", k_gemm_bf16, grid, 128, 0, s, g);
}

// The forward pass on the tcgen05 tensor cores (gemm_tc.cu): BF16 copies of
// the transposed weights (remade after a parameter change) and of the
// activations, FP32 accumulation, bias and ReLU in the epilogue; the FP32
// activations are kept for a backward pass as on the other path.
int mlp_forward_tc(g3d_ctx* c, g3d_mlp* p, const float* X, int B, float* z, float* h1, float* h2, float* h3,
                   cudaStream_t s) {
  const float* W = p->params;
  if (!p->wt16) CK(cudaMalloc(&p->wt16, sizeof(__nv_bfloat16) * (size_t)(kNumParams)));
  if (p->act16_cap < B) {
    int cap = std::max(256, p->act16_cap);
    while (cap < B) cap *= 2;
    if (p->act16) cudaFreeAsync(p->act16, s);
    p->act16 = nullptr;
    CK(cudaMallocAsync((void**)&p->act16, sizeof(__nv_bfloat16) * (size_t)cap * (kFeatIn + 3 * kHidden), s));
    p->act16_cap = cap;
  }
  __nv_bfloat16* w1 = p->wt16;
  __nv_bfloat16* w2 = w1 + (size_t)kFeatIn * kHidden;
  __nv_bfloat16* w3 = w2 + (size_t)kHidden * kHidden;
  __nv_bfloat16* w4 = w3 + (size_t)kHidden * kHidden;
  if (p->bf16_version != p->version) {
    transpose_bf16(W + kOffW1, w1, kFeatIn, kHidden, s);
    transpose_bf16(W + kOffW2, w2, kHidden, kHidden, s);
    transpose_bf16(W + kOffW3, w3, kHidden, kHidden, s);
    transpose_bf16(W + kOffW4, w4, kHidden, kFeatOut, s);
    c->launches += 4;
    p->bf16_version = p->version;
  }
  __nv_bfloat16* x16 = p->act16;
  __nv_bfloat16* a1 = x16 + (size_t)p->act16_cap * kFeatIn;
  __nv_bfloat16* a2 = a1 + (size_t)p->act16_cap * kHidden;
  __nv_bfloat16* a3 = a2 + (size_t)p->act16_cap * kHidden;
  cudaError_t e = profiled(c, "k_to_bf16", s, [&] { return to_bf16(X, x16, (long long)B * kFeatIn, s); });
  c->launches++;
  if (e != cudaSuccess) return cuda_err(e);
  const unsigned long long lim = c->t_limit_ns;
  struct Layer { const __nv_bfloat16* A; const __nv_bfloat16* Wt; int N, K; const float* b; int relu; float* C; __nv_bfloat16* C16; };
  const Layer L[4] = {{x16, w1, kHidden, kFeatIn, W + kOffB1, 1, h1, a1},
                      {a1, w2, kHidden, kHidden, W + kOffB2, 1, h2, a2},
                      {a2, w3, kHidden, kHidden, W + kOffB3, 1, h3, a3},
                      {a3, w4, kFeatOut, kHidden, W + kOffB4, 0, z, nullptr}};
  for (const Layer& l : L) {
    TcGemmArgs g{B, l.N, l.K, l.b, l.relu, l.C, l.C16, l.N, c->d_sticky, lim};
    e = profiled(c, "k_gemm_tc", s, [&] { return tc_gemm(l.A, l.Wt, g, s); });
    c->launches++;
    if (e != cudaSuccess) return cuda_err(e);
  }
  return G3D_OK;
}

// logits z [B x 4096] of X [B x 1536]; activations kept in p->ws
int mlp_forward(g3d_ctx* c, g3d_mlp* p, const float* X, int B, float* z, cudaStream_t s) {
  int rc = mlp_reserve(p, B, s);
  if (rc) return rc;
  const float* W = p->params;
  float* h1 = p->ws;
  float* h2 = h1 + (size_t)p->cap * kHidden;
  float* h3 = h2 + (size_t)p->cap * kHidden;
  if (c->use_tc_gemm && tc_gemm_setup() == 1) return mlp_forward_tc(c, p, X, B, z, h1, h2, h3, s);
  gemm(c, s, X, kFeatIn, 1, W + kOffW1, kHidden, 1, h1, kHidden, W + kOffB1, 1, B, kHidden, kFeatIn);
  gemm(c, s, h1, kHidden, 1, W + kOffW2, kHidden, 1, h2, kHidden, W + kOffB2, 1, B, kHidden, kHidden);
  gemm(c, s, h2, kHidden, 1, W + kOffW3, kHidden, 1, h3, kHidden, W + kOffB3, 1, B, kHidden, kHidden);
  gemm(c, s, h3, kHidden, 1, W + kOffW4, kFeatOut, 1, z, kFeatOut, W + kOffB4, 0, B, kFeatOut, kHidden);
  return cuda_err(cudaGetLastError());
}

// gradients of the mean softmax cross-entropy into p->grads, loss into p->loss
int mlp_backward(g3d_ctx* c, g3d_mlp* p, const float* X, const int* labels, int B, cudaStream_t s) {
  int rc = mlp_reserve(p, B, s);  // before taking pointers into the workspace
  if (rc) return rc;
  float* h1 = p->ws;
  float* h2 = h1 + (size_t)p->cap * kHidden;
  float* h3 = h2 + (size_t)p->cap * kHidden;
  float* z = h3 + (size_t)p->cap * kHidden;
  float* dA = z + (size_t)p->cap * kFeatOut;
  float* dB = dA + (size_t)p->cap * kHidden;
  rc = mlp_forward(c, p, X, B, z, s);
  if (rc) return rc;
  const float* W = p->params;
  float* G = p->grads;
  CK(cudaMemsetAsync(p->loss, 0, sizeof(float), s));
  G3D_LAUNCH(c, "k_softmax_ce", k_softmax_ce, B, 256, 0, s, z, labels, kFeatOut, B, p->loss);
  // layer 4: z = h3 W4 + b4
  gemm(c, s, h3, 1, kHidden, z, kFeatOut, 1, G + kOffW4, kFeatOut, nullptr, 0, kHidden, kFeatOut, B);
  G3D_LAUNCH(c, "k_colsum", k_colsum, (kFeatOut + 255) / 256, 256, 0, s, z, B, kFeatOut, G + kOffB4);
  gemm(c, s, z, kFeatOut, 1, W + kOffW4, 1, kFeatOut, dA, kHidden, nullptr, 0, B, kHidden, kFeatOut);
  G3D_LAUNCH(c, "k_relu_bwd", k_relu_bwd, grid_for((long long)B * kHidden, 256, 1 << 30), 256, 0, s, dA, h3,
             (long long)B * kHidden);
  // layer 3
  gemm(c, s, h2, 1, kHidden, dA, kHidden, 1, G + kOffW3, kHidden, nullptr, 0, kHidden, kHidden, B);
  G3D_LAUNCH(c, "k_colsum", k_colsum, 1, 256, 0, s, dA, B, kHidden, G + kOffB3);
  gemm(c, s, dA, kHidden, 1, W + kOffW3, 1, kHidden, dB, kHidden, nullptr, 0, B, kHidden, kHidden);
  G3D_LAUNCH(c, "k_relu_bwd", k_relu_bwd, grid_for((long long)B * kHidden, 256, 1 << 30), 256, 0, s, dB, h2,
             (long long)B * kHidden);
  // layer 2
  gemm(c, s, h1, 1, kHidden, dB, kHidden, 1, G + kOffW2, kHidden, nullptr, 0, kHidden, kHidden, B);
  G3D_LAUNCH(c, "k_colsum", k_colsum, 1, 256, 0, s, dB, B, kHidden, G + kOffB2);
  gemm(c, s, dB, kHidden, 1, W + kOffW2, 1, kHidden, dA, kHidden, nullptr, 0, B, kHidden, kHidden);
  G3D_LAUNCH(c, "k_relu_bwd", k_relu_bwd, grid_for((long long)B * kHidden, 256, 1 << 30), 256, 0, s, dA, h1,
             (long long)B * kHidden);
  // layer 1
  gemm(c, s, X, 1, kFeatIn, dA, kHidden, 1, G + kOffW1, kHidden, nullptr, 0, kFeatIn, kHidden, B);
  G3D_LAUNCH(c, "k_colsum", k_colsum, 1, 256, 0, s, dA, B, kHidden, G + kOffB1);
  return cuda_err(cudaGetLastError());
}

int ensure_prop_capacity(g3d_ctx* c, int n, cudaStream_t s) {
  if (n <= c->prop_cap) return G3D_OK;
  int cap = c->prop_cap ? c->prop_cap : 256;
  while (cap < n) cap *= 2;
  if (c->prop_X) cudaFreeAsync(c->prop_X, s);
  if (c->prop_top) cudaFreeAsync(c->prop_top, s);
  c->prop_X = nullptr;
  c->prop_top = nullptr;
  CK(cudaMallocAsync((void**)&c->prop_X, sizeof(float) * (size_t)cap * (kFeatIn + kFeatOut), s));
  CK(cudaMallocAsync((void**)&c->prop_top, sizeof(int) * (size_t)cap * kMaxProposals, s));
  c->prop_cap = cap;
  return G3D_OK;
}

// The queries of a launch the learned network proposes for: those whose
// two meshes both have at least cfg.proposal_min_faces faces (default 8192;
// the network is trained
// on meshes of 10k-100k faces; a query of small meshes ends within a few
// levels, where a seeded bound saves less than the features, the forward
// pass, the top-k and the extra dives cost).  Sets c->prop_rows /
// c->prop_nrows for the next run_queries (-1: every query); results never
// depend on it.
int select_proposal_rows(g3d_ctx* c, const QueryDev* hq, int64_t m, int* rows, cudaStream_t s) {
  c->prop_nrows = -1;
  if (!c->proposal) return G3D_OK;
  int nr = 0;  // rows: host memory for m entries (pinned: the copy does not wait)
  for (int64_t i = 0; i < m; i++)
    if (std::min(hq[i].A.ntri, hq[i].B.ntri) >= c->cfg.proposal_min_faces) rows[nr++] = (int)i;
  if (nr == m) return G3D_OK;
  if (nr > c->prop_rows_cap) {
    int cap = std::max(256, c->prop_rows_cap);
    while (cap < nr) cap *= 2;
    if (c->prop_rows) cudaFreeAsync(c->prop_rows, s);
    c->prop_rows = nullptr;
    c->prop_rows_cap = 0;
    CK(cudaMallocAsync((void**)&c->prop_rows, sizeof(int) * (size_t)cap, s));
    c->prop_rows_cap = cap;
  }
  if (nr) CK(cudaMemcpyAsync(c->prop_rows, rows, sizeof(int) * nr, cudaMemcpyHostToDevice, s));
  c->prop_nrows = nr;
  return G3D_OK;
}

// Per-cluster statistics of the learned proposal are computed on first use
// (one launch for all meshes of the call that lack them), not at every build.
int cstats_for(g3d_ctx* c, std::vector<G3dMesh*>& need, cudaStream_t s);

// the meshes of the queries, looked up by handle
int ensure_cstats(g3d_ctx* c, const g3d_query* q, int64_t n, cudaStream_t s) {
  std::vector<G3dMesh*> need;
  for (int64_t i = 0; i < n; i++)
    for (g3d_mesh h : {q[i].a, q[i].b}) {
      G3dMesh* m = get_mesh(c, h);
      if (m && m->has_bvh && !m->cstats_valid) {
        m->cstats_valid = true;  // also marks it taken for this call
        need.push_back(m);
      }
    }
  return cstats_for(c, need, s);
}

// the meshes of a batch, as build_queries resolved them (2 per query): no
// handle lookups on the batch path
int ensure_cstats_meshes(g3d_ctx* c, const std::vector<G3dMesh*>& ms, cudaStream_t s) {
  std::vector<G3dMesh*> need;
  for (G3dMesh* m : ms)
    if (m && m->has_bvh && !m->cstats_valid) {
      m->cstats_valid = true;
      need.push_back(m);
    }
  return cstats_for(c, need, s);
}

int cstats_for(g3d_ctx* c, std::vector<G3dMesh*>& need, cudaStream_t s) {
  if (need.empty()) return G3D_OK;
  std::vector<ClusterMesh> cm(need.size());
  for (size_t i = 0; i < need.size(); i++) cm[i] = {need[i]->v0, need[i]->v1, need[i]->v2, need[i]->nt, need[i]->cstats};
  ClusterMesh* dcm = nullptr;
  CK(cudaMallocAsync((void**)&dcm, sizeof(ClusterMesh) * cm.size(), s));
  CK(cudaMemcpyAsync(dcm, cm.data(), sizeof(ClusterMesh) * cm.size(), cudaMemcpyHostToDevice, s));
  G3D_LAUNCH(c, "k_cluster_stats", k_cluster_stats, (unsigned int)(cm.size() * kClusters), 128, 0, s, dcm,
             (int)cm.size());
  CK(cudaGetLastError());
  // the host table must outlive its upload
  CK(cudaStreamSynchronize(s));
  cudaFreeAsync(dcm, s);
  return G3D_OK;
}

// a configuration with every zero field replaced by its default
g3d_config complete_config(const g3d_config* cfg) {
  g3d_config d{};
  if (cfg) d = *cfg;
  if (d.leaf_size == 0) d.leaf_size = 16;
  if (d.warps_per_cta == 0) d.warps_per_cta = 4;
  if (d.ctas_per_sm == 0) d.ctas_per_sm = 1;
  if (d.stack_depth == 0) d.stack_depth = 256;
  if (d.cand_capacity == 0) d.cand_capacity = 1 << 24;
  if (d.queue_capacity == 0) d.queue_capacity = 1 << 20;
  if (d.time_limit_ms == 0) d.time_limit_ms = 30000;
  if (d.isect_first == 0) d.isect_first = 1;
  if (d.morton_bits == 0) d.morton_bits = 10;
  if (d.traversal == 0) d.traversal = 1;
  if (d.frontier_capacity == 0) d.frontier_capacity = 1 << 23;
  if (d.dives == 0) d.dives = 16;
  if (d.chunk_mfaces == 0) d.chunk_mfaces = 2048;
  if (d.proposal_min_faces == 0) d.proposal_min_faces = 8192;
  return d;
}

bool config_ok(const g3d_config& d) {
  return (d.leaf_size == 2 || d.leaf_size == 4 || d.leaf_size == 8 || d.leaf_size == 16) &&
         d.warps_per_cta >= 1 && d.warps_per_cta <= 4 && d.ctas_per_sm >= 1 && d.ctas_per_sm <= 16 &&
         d.stack_depth >= 64 && d.stack_depth <= 1024 && (d.stack_depth & (d.stack_depth - 1)) == 0 &&
         d.cand_capacity >= 1024 && d.queue_capacity >= 8192 && (d.queue_capacity & (d.queue_capacity - 1)) == 0 &&
         d.time_limit_ms >= 10 && d.time_limit_ms <= 600000 && (d.isect_first == 1 || d.isect_first == 2) &&
         d.morton_bits >= 8 && d.morton_bits <= 10 && (d.traversal == 1 || d.traversal == 2) &&
         (d.count_visits == 0 || d.count_visits == 1) && d.frontier_capacity >= 1024 &&
         (d.frontier_capacity & (d.frontier_capacity - 1)) == 0 && d.dives >= 1 && d.dives <= 32 &&
         d.chunk_mfaces >= 1 && d.chunk_mfaces <= (1 << 20) && d.proposal_min_faces >= 1 &&
         d.proposal_min_faces <= (1 << 30);
}

// CTAs of the persistent traversal per SM: the configured count, capped by
// what the SM holds at once (registers, shared memory, warps, CTAs), so that
// every CTA of the launch is resident.  The kernel's shared-memory carve-out
// is set to what those CTAs need: the rest of the unified L1 / shared storage
// stays L1 cache for the node and face reads.  (A carve-out preference of 0
// alone would hold one CTA per SM and leave the others of the grid to run
// after it.)
int trav_ctas(g3d_ctx* c, int W, size_t dyn_smem) {
  cudaFuncAttributes fa{};
  int fit = c->cfg.ctas_per_sm;
  if (cudaFuncGetAttributes(&fa, k_traverse) == cudaSuccess) {
    // registers are allocated per warp in units of 256
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_warp > 0 ? (c->regs_per_sm / regs_warp) / W : fit;
    const size_t cta_smem = dyn_smem + fa.sharedSizeBytes + 1024;  // 1 KB per CTA is reserved
    const int by_smem = (int)((size_t)c->smem_per_sm / cta_smem);
    const int by_warps = c->max_warps_per_sm / W;
    fit = std::max(1, std::min({fit, by_regs, by_smem, by_warps, c->max_ctas_per_sm}));
    const double need = (double)fit * (double)cta_smem;
    const int pct = std::min(100, (int)ceil(100.0 * need / (double)c->smem_per_sm));
    if (pct != c->trav_carveout) {
      if (cudaFuncSetAttribute(k_traverse, cudaFuncAttributePreferredSharedMemoryCarveout, pct) == cudaSuccess)
        c->trav_carveout = pct;
    }
  }
  cudaGetLastError();
  return fit;
}

#ifndef G3D_PROPOSALS
#define G3D_PROPOSALS 4  // cluster pairs the network proposes per query (its top-k), at most kMaxProposals
#endif
static_assert(G3D_PROPOSALS >= 1 && G3D_PROPOSALS <= kMaxProposals, "proposals per query");

// The proposed cluster pairs of every query (caller hints: one per query; or
// the learned network: pair features -> MLP forward -> its G3D_PROPOSALS
// highest logits, for the queries c->prop_rows lists, or all when
// c->prop_nrows < 0), recorded as leaf ranges for the restricted dives; null
// when there is no proposal.
const int* compute_proposal(g3d_ctx* c, const TravArgs& a, int nq, const int* hint, cudaStream_t s, int* rc) {
  *rc = G3D_OK;
  const int* top = hint;
  const int* rows = nullptr;
  int k = 1, nrows = nq;
  if (!top && c->proposal) {
    if (c->prop_nrows >= 0) {
      rows = c->prop_rows;
      nrows = std::min(c->prop_nrows, nq);
    }
    if (nrows == 0) return nullptr;  // no query large enough for the network
    if ((*rc = ensure_prop_capacity(c, nrows, s))) return nullptr;
    float* X = c->prop_X;
    float* z = X + (size_t)c->prop_cap * kFeatIn;
    PairFeatArgs pf{a.q, X, rows};
    G3D_LAUNCH(c, "k_pair_features", k_pair_features, nrows, 128, 0, s, pf);
    if ((*rc = mlp_forward(c, c->proposal, X, nrows, z, s))) return nullptr;
    k = G3D_PROPOSALS;
    G3D_LAUNCH(c, "k_topk", k_topk, nrows, 256, 0, s, z, kFeatOut, k, c->prop_top);
    top = c->prop_top;
  }
  if (top)
    G3D_LAUNCH(c, "k_set_proposal", k_set_proposal, grid_for(nrows, 128, 1 << 20), 128, 0, s, a, top, k, rows,
               nrows);
  c->cur_prop_rows = rows;  // the restricted dives cover these queries only
  c->cur_prop_nrows = nrows;
  return top;
}

// greedy dives of the queries of operator `op` (bound seeding for distance,
// a first certified intersection for intersects), then, with a proposal, 4
// dives restricted to each query's proposed cluster pairs
void dives(g3d_ctx* c, const TravArgs& a, int nq, int op, const int* top, cudaStream_t s) {
  const int D = c->cfg.dives;
  G3D_LAUNCH(c, "k_dive", k_dive, grid_for((long long)nq * D * 32, 128, 1 << 30), 128, 0, s, a, D, 0, op, nullptr,
             nq);
  if (top)  // only the queries holding a proposal
    G3D_LAUNCH(c, "k_dive", k_dive, grid_for((long long)c->cur_prop_nrows * 4 * 32, 128, 1 << 30), 128, 0, s, a, 4,
               1, op, c->cur_prop_rows, c->cur_prop_nrows);
}

// proposal (if any) and distance dives: the persistent form's seeding step
int seed_bounds(g3d_ctx* c, const TravArgs& a, int nq, const int* hint, cudaStream_t s) {
  int rc;
  const int* top = compute_proposal(c, a, nq, hint, s, &rc);
  if (rc) return rc;
  dives(c, a, nq, G3D_OP_DISTANCE, top, s);
  return G3D_OK;
}

// Level-synchronous form of the query sequence: per-query state reset,
// [intersects phase], bounds seeding, distance (or combined) phase; items
// that did not fit a frontier buffer are finished by the persistent kernel;
// a candidate-pool overflow re-runs the unfinished queries (pass 2).
int run_queries_frontier(g3d_ctx* c, int nq, double* dist, unsigned char* hit, int* status, cudaStream_t s,
                         const QueryDev* qd, QueryState* st, long long* witness, int* cluster, const int* hint) {
  TravArgs a = trav_args(c, nq, qd, st);
  const int W = c->cfg.warps_per_cta, S = c->cfg.stack_depth;
  size_t smem = (size_t)W * S * sizeof(int4) + (size_t)W * kLeafStageBytes;
  dim3 grid(c->num_sms * trav_ctas(c, W, smem)), block(32 * W);
  FrontierArgs f = c->fr;
  int rc;
  G3D_LAUNCH(c, "k_reset_state", k_reset_state, grid_for(nq, 256, 1024), 256, 0, s, a);
  // a proposal seeds both operators: intersects queries test the proposed
  // cluster pair first (a certified hit there ends them before the
  // traversal), distance queries start from the bound found there
  const int* top = compute_proposal(c, a, nq, hint, s, &rc);
  if (rc) return rc;
  dives(c, a, nq, G3D_OP_INTERSECTS, top, s);
  const unsigned int top_items = 2048;  // narrow levels run in one block (k_frontier_top)
  if (c->cfg.isect_first == 1) {
    G3D_LAUNCH(c, "k_frontier_zero", k_frontier_zero, 1, 32, 0, s, f);
    G3D_LAUNCH(c, "k_frontier_seed", k_frontier_seed, grid_for(nq, 256, 1 << 20), 256, 0, s, a, f, 0, 1);
    G3D_LAUNCH(c, "k_frontier_top", k_frontier_top, 1, 1024, 0, s, a, f, top_items);
    if ((rc = launch_frontier(c, a, s))) return rc;
    G3D_LAUNCH(c, "k_traverse", k_traverse, grid, block, smem, s, a, S);
    dives(c, a, nq, G3D_OP_DISTANCE, top, s);
    G3D_LAUNCH(c, "k_frontier_zero", k_frontier_zero, 1, 32, 0, s, f);
    G3D_LAUNCH(c, "k_frontier_seed", k_frontier_seed, grid_for(nq, 256, 1 << 20), 256, 0, s, a, f, 1, 0);
  } else {
    dives(c, a, nq, G3D_OP_DISTANCE, top, s);
    G3D_LAUNCH(c, "k_frontier_zero", k_frontier_zero, 1, 32, 0, s, f);
    G3D_LAUNCH(c, "k_frontier_seed", k_frontier_seed, grid_for(nq, 256, 1 << 20), 256, 0, s, a, f, 2, 0);
  }
  G3D_LAUNCH(c, "k_frontier_top", k_frontier_top, 1, 1024, 0, s, a, f, top_items);
  if ((rc = launch_frontier(c, a, s))) return rc;
  G3D_LAUNCH(c, "k_traverse", k_traverse, grid, block, smem, s, a, S);
  G3D_LAUNCH(c, "k_prepare_pass2", k_prepare_pass2, 1, 256, 0, s, a);
  G3D_LAUNCH(c, "k_traverse", k_traverse, grid, block, smem, s, a, S);
  G3D_LAUNCH(c, "k_finalize", k_finalize, c->num_sms * 4, 128, 0, s, a);
  if (witness || cluster) G3D_LAUNCH(c, "k_witness", k_witness, c->num_sms * 4, 128, 0, s, a);
  if (cluster) G3D_LAUNCH(c, "k_witness_label", k_witness_label, c->num_sms * 4, 128, 0, s, a);
  G3D_LAUNCH(c, "k_write_results", k_write_results, grid_for(nq, 128, 1 << 20), 128, 0, s, a, dist, hit, status,
             witness, cluster);
  return cuda_err(cudaGetLastError());
}

int run_queries(g3d_ctx* c, int nq, double* dist, unsigned char* hit, int* status, cudaStream_t s,
                const QueryDev* qd = nullptr, QueryState* st = nullptr, long long* witness = nullptr,
                int* cluster = nullptr, const int* hint = nullptr) {
  NvtxRange nvtx_range("g3d queries");
  if (c->cfg.traversal == 1)
    return run_queries_frontier(c, nq, dist, hit, status, s, qd, st, witness, cluster, hint);
  TravArgs a = trav_args(c, nq, qd, st);
  const int W = c->cfg.warps_per_cta, S = c->cfg.stack_depth;
  size_t smem = (size_t)W * S * sizeof(int4) + (size_t)W * kLeafStageBytes;
  dim3 grid(c->num_sms * trav_ctas(c, W, smem)), block(32 * W);
  // phase 0: intersects traversal of every intersects query and, unless
  // configured otherwise, of every distance query
  G3D_LAUNCH(c, "k_seed", k_seed, 1, 256, 0, s, a, c->cfg.isect_first == 1 ? 1 : 0);
  G3D_LAUNCH(c, "k_traverse", k_traverse, grid, block, smem, s, a, S);
  // greedy dives seed each distance query's upper bound; with a proposal
  // (caller-supplied hint or learned network) more dives follow, kept to the
  // proposed cluster pairs
  int rc;
  const int* top = compute_proposal(c, a, nq, hint, s, &rc);
  if (rc) return rc;
  const unsigned int dive_grid = grid_for((long long)nq * c->cfg.dives * 32, 128, 1 << 30);
  G3D_LAUNCH(c, "k_dive", k_dive, dive_grid, 128, 0, s, a, c->cfg.dives, 0, G3D_OP_DISTANCE, nullptr, nq);
  if (top) {
    const unsigned int rgrid = grid_for((long long)c->cur_prop_nrows * 4 * 32, 128, 1 << 30);
    G3D_LAUNCH(c, "k_dive", k_dive, rgrid, 128, 0, s, a, 4, 1, G3D_OP_DISTANCE, c->cur_prop_rows,
               c->cur_prop_nrows);
  }
  G3D_LAUNCH(c, "k_seed_phase1", k_seed_phase1, 1, 256, 0, s, a);
  G3D_LAUNCH(c, "k_traverse", k_traverse, grid, block, smem, s, a, S);
  G3D_LAUNCH(c, "k_prepare_pass2", k_prepare_pass2, 1, 256, 0, s, a);
  G3D_LAUNCH(c, "k_traverse", k_traverse, grid, block, smem, s, a, S);
  G3D_LAUNCH(c, "k_finalize", k_finalize, c->num_sms * 4, 128, 0, s, a);
  if (witness || cluster) G3D_LAUNCH(c, "k_witness", k_witness, c->num_sms * 4, 128, 0, s, a);
  if (cluster) G3D_LAUNCH(c, "k_witness_label", k_witness_label, c->num_sms * 4, 128, 0, s, a);
  G3D_LAUNCH(c, "k_write_results", k_write_results, grid_for(nq, 128, 1 << 20), 128, 0, s, a, dist, hit, status,
             witness, cluster);
  return cuda_err(cudaGetLastError());
}

}  // namespace

extern "C" {

const char* g3d_strerror(int code) {
  switch (code) {
    case G3D_OK: return "ok";
    case G3D_ERR_INVALID_ARG: return "invalid argument";
    case G3D_ERR_NAN_INPUT: return "NaN or infinite coordinate";
    case G3D_ERR_INDEX_OOB: return "face index out of range";
    case G3D_ERR_EMPTY_MESH: return "empty mesh";
    case G3D_ERR_OOM: return "device out of memory";
    case G3D_ERR_CAND_OVERFLOW: return "candidate list overflow";
    case G3D_ERR_TIMEOUT: return "device wait timed out";
    case G3D_ERR_CUDA: return "CUDA error";
    case G3D_ERR_RANGE: return "coordinate out of supported range";
    case G3D_ERR_NO_BVH: return "mesh has no BVH";
    case G3D_ERR_TOO_LARGE: return "input exceeds a fixed-size scratch area";
    case G3D_ERR_IO: return "file could not be read or written";
    default: return "unknown error";
  }
}

int g3d_create(g3d_ctx** out, int device, const g3d_config* cfg) {
  if (!out) return G3D_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return G3D_ERR_INVALID_ARG;
  }
  CK(cudaSetDevice(device));
  g3d_ctx* c = new g3d_ctx();
  c->device = device;
  CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  CK(cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  CK(cudaDeviceGetAttribute(&c->regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, device));
  CK(cudaDeviceGetAttribute(&c->max_warps_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device));
  c->max_warps_per_sm /= 32;
  CK(cudaDeviceGetAttribute(&c->max_ctas_per_sm, cudaDevAttrMaxBlocksPerMultiprocessor, device));
  g3d_config d = complete_config(cfg);
  if (!config_ok(d)) { delete c; return G3D_ERR_INVALID_ARG; }
  c->cfg = d;
  c->t_limit_ns = (unsigned long long)d.time_limit_ms * 1000000ull;
  // the largest traversal shape the configuration allows (4 warps, 1024-deep stacks)
  if (cudaFuncSetAttribute(k_traverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(4 * (1024 * sizeof(int4) + kLeafStageBytes))) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return G3D_ERR_CUDA;
  }
  // The segment kernel uses no shared memory: all of the unified L1 /
  // shared storage goes to L1 (the traversal's carve-out is set per launch
  // shape, trav_ctas).  A preference only: failure to set it is not an error.
  cudaFuncSetAttribute(k_segments, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaGetLastError();
  // memory pool keeps freed blocks for reuse
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  Queue& Q = c->queue;
  Q.cap = (unsigned int)d.queue_capacity;
  int rc = G3D_OK;
  if (cudaMalloc(&Q.items, sizeof(int4) * Q.cap) != cudaSuccess ||
      cudaMalloc(&Q.seq, sizeof(int) * Q.cap) != cudaSuccess ||
      cudaMalloc(&Q.head, 64) != cudaSuccess || cudaMalloc(&Q.tail, 64) != cudaSuccess ||
      cudaMalloc(&Q.pending, 64) != cudaSuccess || cudaMalloc(&Q.error, 64) != cudaSuccess ||
      cudaMalloc(&c->cand.items, sizeof(int4) * (size_t)d.cand_capacity) != cudaSuccess ||
      cudaMalloc(&c->cand.count, 64) != cudaSuccess ||
      cudaMalloc(&c->stats, sizeof(unsigned long long) * ST_COUNT) != cudaSuccess ||
      cudaMalloc(&c->d_sticky, 64) != cudaSuccess || cudaMalloc(&c->d_dbg, 64) != cudaSuccess ||
      cudaMallocHost(&c->h_pinned, 64) != cudaSuccess)
    rc = G3D_ERR_OOM;
  if (rc) { g3d_destroy(c); return rc; }
  c->cand.cap = d.cand_capacity;
  {
    // level-synchronous traversal: 2 frontiers of frontier_capacity node
    // pairs, 2 leaf lists of half as many, a face-pair list as large as a
    // frontier (512 MiB by default: batches of thousands of queries on
    // 100k-face meshes overflow 2^21-entry lists into the persistent
    // finisher, which is several times slower per item), the
    // cooperative grid = every block the SMs hold at once
    int coop = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (!coop ||
        cudaFuncSetAttribute(k_frontier, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)frontier_smem_bytes()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_frontier, 256, frontier_smem_bytes()) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      g3d_destroy(c);
      return G3D_ERR_CUDA;
    }
    FrontierArgs& f = c->fr;
    f.fcap = d.frontier_capacity;
    f.lcap = d.frontier_capacity / 2;
    f.nblocks = per_sm * c->num_sms;
    f.trace_cap = 1024;
    f.fpcap = d.frontier_capacity;
    if (cudaMalloc(&c->fr_items, sizeof(int4) * (2 * (size_t)f.fcap + 2 * (size_t)f.lcap + (size_t)f.fpcap)) !=
            cudaSuccess ||
        cudaMalloc(&c->fr_cnt, 128 + 48 * (size_t)f.trace_cap) != cudaSuccess) {
      g3d_destroy(c);
      return G3D_ERR_OOM;
    }
    f.trace_next = c->fr_cnt + 31;
    f.trace = (unsigned long long*)(c->fr_cnt + 32);
    f.F[0] = c->fr_items;
    f.F[1] = f.F[0] + f.fcap;
    f.L[0] = f.F[1] + f.fcap;
    f.L[1] = f.L[0] + f.lcap;
    f.FP = f.L[1] + f.lcap;
    f.cnt = c->fr_cnt;
    f.bar = c->fr_cnt + 28;
    cudaMemset(c->fr_cnt, 0, 128 + 48 * (size_t)f.trace_cap);
  }

  cudaMemset(c->stats, 0, sizeof(unsigned long long) * ST_COUNT);
  cudaMemset(c->d_sticky, 0, 64);
  cudaMemset(c->d_dbg, 0, 64);
  cudaMemset(c->cand.count, 0, 64);
  G3D_LAUNCH(c, "k_queue_init", k_queue_init, 256, 256, 0, 0, Q);
  rc = ensure_query_capacity(c, 64, 0);
  if (rc == G3D_OK) rc = cuda_err(cudaDeviceSynchronize());
  if (rc) { g3d_destroy(c); return rc; }
  *out = c;
  return G3D_OK;
}

int g3d_mesh_free(g3d_ctx* c, g3d_mesh h) {
  if (!c) return G3D_ERR_INVALID_ARG;
  G3dMesh* m = get_mesh(c, h);
  if (!m) return G3D_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();  // no queued work may still use the mesh
  slab_release(m->raw_slab, 0);
  slab_release(m->bvh_slab, 0);
  c->meshes.erase(h);
  delete m;
  return G3D_OK;
}

int g3d_mesh_free_many(g3d_ctx* c, int64_t n, const g3d_mesh* hs) {
  if (!c || n < 0 || (n > 0 && !hs)) return G3D_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; i++)
    if (!get_mesh(c, hs[i])) return G3D_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();  // no queued work may still use the meshes
  for (int64_t i = 0; i < n; i++) {
    G3dMesh* m = get_mesh(c, hs[i]);
    if (!m) continue;  // listed twice
    slab_release(m->raw_slab, 0);
    slab_release(m->bvh_slab, 0);
    c->meshes.erase(hs[i]);
    delete m;
  }
  return G3D_OK;
}

int g3d_mesh_free_many_async(g3d_ctx* c, int64_t n, const g3d_mesh* hs, void* stream) {
  if (!c || n < 0 || (n > 0 && !hs)) return G3D_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; i++)
    if (!get_mesh(c, hs[i])) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t i = 0; i < n; i++) {
    G3dMesh* m = get_mesh(c, hs[i]);
    if (!m) continue;  // listed twice
    slab_release(m->raw_slab, s);  // device memory released in stream order
    slab_release(m->bvh_slab, s);
    c->meshes.erase(hs[i]);
    delete m;
  }
  return G3D_OK;
}

int g3d_destroy(g3d_ctx* c) {
  if (!c) return G3D_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  std::vector<int64_t> ids;
  for (auto& kv : c->meshes) ids.push_back(kv.first);
  for (int64_t h : ids) g3d_mesh_free(c, h);
  for (void* p : {(void*)c->queue.items, (void*)c->queue.seq, (void*)c->queue.head, (void*)c->queue.tail,
                  (void*)c->queue.pending, (void*)c->queue.error, (void*)c->cand.items, (void*)c->cand.count,
                  (void*)c->stats, (void*)c->qdev, (void*)c->st, (void*)c->d_dist, (void*)c->d_hit,
                  (void*)c->d_status, (void*)c->d_sticky, (void*)c->d_dbg, (void*)c->fr_items,
                  (void*)c->fr_cnt})
    if (p) cudaFree(p);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  for (void* p : {(void*)c->prop_X, (void*)c->prop_top, (void*)c->prop_rows})
    if (p) cudaFree(p);
  for (auto& st : c->stage) {
    if (st.p) cudaFreeHost(st.p);
    if (st.ev) cudaEventDestroy(st.ev);
  }
  if (c->prop_X) cudaFree(c->prop_X);
  if (c->prop_top) cudaFree(c->prop_top);
  for (auto& r : c->prof) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return G3D_OK;
}

int g3d_get_config(g3d_ctx* c, g3d_config* out) {
  if (!c || !out) return G3D_ERR_INVALID_ARG;
  *out = c->cfg;
  return G3D_OK;
}

int g3d_set_config(g3d_ctx* c, const g3d_config* cfg) {
  if (!c || !cfg) return G3D_ERR_INVALID_ARG;
  g3d_config d = complete_config(cfg);
  if (!config_ok(d)) return G3D_ERR_INVALID_ARG;
  // the pool sizes were allocated at creation
  if ((cfg->cand_capacity && cfg->cand_capacity != c->cfg.cand_capacity) ||
      (cfg->queue_capacity && cfg->queue_capacity != c->cfg.queue_capacity) ||
      (cfg->frontier_capacity && cfg->frontier_capacity != c->cfg.frontier_capacity))
    return G3D_ERR_INVALID_ARG;
  d.cand_capacity = c->cfg.cand_capacity;
  d.queue_capacity = c->cfg.queue_capacity;
  d.frontier_capacity = c->cfg.frontier_capacity;
  c->cfg = d;
  c->t_limit_ns = (unsigned long long)d.time_limit_ms * 1000000ull;
  return G3D_OK;
}

int g3d_mesh_load_many(g3d_ctx* c, int64_t n, const void* const* verts, const int32_t* vdtype,
                       const int64_t* nv, const uint32_t* const* idx, const int64_t* nt, int copy_fp64_master,
                       g3d_mesh* out, int32_t* status_out, void* stream) {
  NvtxRange nvtx_range("g3d_mesh_load_many");
  if (!c || n < 0 || (n > 0 && (!verts || !vdtype || !nv || !idx || !nt || !out))) return G3D_ERR_INVALID_ARG;
  if (n == 0) return G3D_OK;
  for (int64_t i = 0; i < n; i++) {
    if (!verts[i] || !idx[i] || (vdtype[i] != G3D_F32 && vdtype[i] != G3D_F64) || nv[i] < 0 || nt[i] < 0)
      return G3D_ERR_INVALID_ARG;
    if (nt[i] == 0 || nv[i] == 0) return G3D_ERR_EMPTY_MESH;
    if (nt[i] > (1ll << 28) || nv[i] > (1ll << 31)) return G3D_ERR_INVALID_ARG;
  }
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<G3dMesh*> ms((size_t)n, nullptr);
  int* flags = nullptr;  // [2 n]: error bits, rho bits
  int rc = cuda_err(cudaMallocAsync((void**)&flags, sizeof(int) * 2 * n + 16, s));
  if (!rc) rc = cuda_err(cudaMemsetAsync(flags, 0, sizeof(int) * 2 * n, s));
  std::vector<IngestItem> items;
  items.reserve(2 * (size_t)n);
  // one block for the raw copies of all meshes of the call
  size_t total = 0;
  for (int64_t i = 0; i < n; i++) {
    const size_t vbytes = (size_t)nv[i] * 3 * (vdtype[i] == G3D_F32 ? 4 : 8);
    total += up256(((vbytes + 15) & ~(size_t)15) + 32) + up256((size_t)nt[i] * 12);
  }
  Slab* slab = new Slab();
  if (!rc) rc = cuda_err(cudaMallocAsync(&slab->base, total, s));
  size_t at = 0;
  DeviceRanges dev_ranges;
  // a host source repeated within the call (e.g. one index array shared by
  // many meshes of the same tessellation) crosses to the device once; the
  // later meshes ingest from that copy, which its own mesh only reads
  std::map<std::pair<uintptr_t, size_t>, const char*> host_copies;
  for (int64_t i = 0; i < n && !rc; i++) {
    G3dMesh* m = new G3dMesh();
    ms[i] = m;
    m->dtype = vdtype[i];
    m->nv = nv[i];
    m->nt = nt[i];
    m->master = vdtype[i] == G3D_F64 && copy_fp64_master;
    const size_t esize = vdtype[i] == G3D_F32 ? 4 : 8;
    const size_t vbytes = (size_t)nv[i] * 3 * esize;
    const size_t vpad = (vbytes + 15) & ~(size_t)15;
    m->raw_v = (char*)slab->base + at;  // vertices, then the vertex box
    at += up256(vpad + 32);
    m->raw_i = (uint32_t*)((char*)slab->base + at);
    at += up256((size_t)nt[i] * 12);
    m->box = (unsigned int*)((char*)m->raw_v + vpad);
    // device sources aligned to their element are read by the ingest kernel
    // directly; others go through the copy engine first and are then
    // validated in place
    const void* src[2] = {verts[i], idx[i]};
    void* dst[2] = {m->raw_v, m->raw_i};
    const size_t bytes[2] = {vbytes, (size_t)nt[i] * 12};
    const size_t align[2] = {esize, 4};
    const char* from[2];
    for (int k = 0; k < 2 && !rc; k++) {
      if (((uintptr_t)src[k] % align[k]) == 0 && dev_ranges.is_device(src[k], bytes[k])) {
        from[k] = (const char*)src[k];
      } else {
        const std::pair<uintptr_t, size_t> key((uintptr_t)src[k], bytes[k]);
        auto hit = host_copies.find(key);
        if (hit != host_copies.end()) {
          from[k] = hit->second;
        } else {
          rc = cuda_err(cudaMemcpyAsync(dst[k], src[k], bytes[k], cudaMemcpyDefault, s));
          from[k] = (const char*)dst[k];
          host_copies.emplace(key, from[k]);
        }
      }
    }
    const int vec_v = ((uintptr_t)from[0] % 16 == 0) && ((uintptr_t)dst[0] % 16 == 0);
    const int vec_i = ((uintptr_t)from[1] % 16 == 0) && ((uintptr_t)dst[1] % 16 == 0);
    items.push_back({from[0], (char*)dst[0], nv[i] * 3, nv[i], vdtype[i] == G3D_F32 ? ING_F32 : ING_F64, vec_v,
                     flags + 2 * i, m->box});
    items.push_back({from[1], (char*)dst[1], nt[i] * 3, nv[i], ING_IDX, vec_i, flags + 2 * i, nullptr});
  }
  if (!rc) {
    const int ni = (int)items.size();
    std::vector<long long> coff(ni + 1, 0);
    for (int k = 0; k < ni; k++) coff[k + 1] = coff[k] + (items[k].n + kIngestChunk - 1) / kIngestChunk;
    char* tab = nullptr;
    const size_t tb = sizeof(IngestItem) * ni + sizeof(long long) * (ni + 1);
    rc = cuda_err(cudaMallocAsync((void**)&tab, tb + 16, s));
    std::vector<char> ht(tb);
    memcpy(ht.data(), items.data(), sizeof(IngestItem) * ni);
    memcpy(ht.data() + sizeof(IngestItem) * ni, coff.data(), sizeof(long long) * (ni + 1));
    if (!rc) rc = cuda_err(cudaMemcpyAsync(tab, ht.data(), tb, cudaMemcpyHostToDevice, s));
    if (!rc) {
      G3D_LAUNCH(c, "k_ingest_init", k_ingest_init, grid_for(ni, 128, 1 << 30), 128, 0, s, (const IngestItem*)tab,
                 ni);
      G3D_LAUNCH(c, "k_ingest_many", k_ingest_many, (unsigned int)coff[ni], 256, 0, s, (const IngestItem*)tab,
                 (const long long*)(tab + sizeof(IngestItem) * ni), ni);
    }
    if (tab) cudaFreeAsync(tab, s);
  }
  std::vector<int> hf((size_t)(2 * n), 0);
  if (!rc) rc = cuda_err(cudaMemcpyAsync(hf.data(), flags, sizeof(int) * 2 * n, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  int first_err = rc;
  for (int64_t i = 0; i < n; i++) {
    int e = rc;
    if (!rc) {
      int f = hf[2 * i];
      if (f & VAL_NAN) e = G3D_ERR_NAN_INPUT;
      else if (f & VAL_OOB) e = G3D_ERR_INDEX_OOB;
      else if (f & VAL_RANGE) e = G3D_ERR_RANGE;
      unsigned int rb = (unsigned int)hf[2 * i + 1];
      if (ms[i]) memcpy(&ms[i]->rho, &rb, 4);
    }
    if (status_out) status_out[i] = e;
    if (e && !first_err) first_err = e;
  }
  if (flags) cudaFreeAsync(flags, s);
  if (first_err) {
    for (G3dMesh* m : ms) delete m;
    if (slab->base) cudaFreeAsync(slab->base, s);
    delete slab;
    cudaStreamSynchronize(s);
    for (int64_t i = 0; i < n; i++) out[i] = 0;
    return first_err;
  }
  slab->refs = n;
  for (int64_t i = 0; i < n; i++) {
    ms[i]->raw_slab = slab;
    int64_t h = c->next_id++;
    c->meshes[h] = ms[i];
    out[i] = h;
  }
  return G3D_OK;
}

int g3d_mesh_load(g3d_ctx* c, const void* verts, int vdtype, int64_t nv, const uint32_t* idx, int64_t nt,
                  int copy_fp64_master, g3d_mesh* out, void* stream) {
  if (!out) return G3D_ERR_INVALID_ARG;
  int32_t dt = vdtype;
  return g3d_mesh_load_many(c, 1, &verts, &dt, &nv, &idx, &nt, copy_fp64_master, out, nullptr, stream);
}

int g3d_mesh_export(g3d_ctx* c, g3d_mesh h, int32_t* face_ids, float* leaves, float* nodes, int64_t* nleaf_out) {
  if (!c) return G3D_ERR_INVALID_ARG;
  G3dMesh* m = get_mesh(c, h);
  if (!m) return G3D_ERR_INVALID_ARG;
  if (!m->has_bvh) return G3D_ERR_NO_BVH;
  CK(cudaSetDevice(c->device));
  CK(cudaDeviceSynchronize());
  const int64_t nt = m->nt, nleaf = m->dev.nleaf;
  if (nleaf_out) *nleaf_out = nleaf;
  if (face_ids) {
    std::vector<float4> v0((size_t)nt);
    CK(cudaMemcpy(v0.data(), m->v0, sizeof(float4) * nt, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < nt; i++) memcpy(&face_ids[i], &v0[i].w, 4);
  }
  if (leaves) CK(cudaMemcpy(leaves, m->leaves, sizeof(float4) * 2 * nleaf, cudaMemcpyDeviceToHost));
  if (nodes && nleaf > 1) CK(cudaMemcpy(nodes, m->nodes, sizeof(float4) * 4 * (nleaf - 1), cudaMemcpyDeviceToHost));
  return G3D_OK;
}

int g3d_mesh_size(g3d_ctx* c, g3d_mesh h, int64_t* nt) {
  if (!c || !nt) return G3D_ERR_INVALID_ARG;
  G3dMesh* m = get_mesh(c, h);
  if (!m) return G3D_ERR_INVALID_ARG;
  *nt = m->nt;
  return G3D_OK;
}

int g3d_mesh_build_bvh_many(g3d_ctx* c, int64_t n, const g3d_mesh* hs, void* stream) {
  NvtxRange nvtx_range("g3d_mesh_build_bvh_many");
  if (!c || n < 0 || (n > 0 && !hs)) return G3D_ERR_INVALID_ARG;
  if (n == 0) return G3D_OK;
  if (n > 65535) return G3D_ERR_INVALID_ARG;  // the mesh index is 16 bits of the sort key
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int L = c->cfg.leaf_size;
  std::vector<G3dMesh*> M((size_t)n);
  {
    std::unordered_set<g3d_mesh> seen;
    seen.reserve((size_t)n);
    for (int64_t i = 0; i < n; i++) {
      M[i] = get_mesh(c, hs[i]);
      if (!M[i] || !seen.insert(hs[i]).second) return G3D_ERR_INVALID_ARG;  // unknown or listed twice
    }
  }
  // host tables: BuildMesh[n], then face / leaf / node / sort-tile offsets [n+1]
  std::vector<BuildMesh> bm((size_t)n);
  std::vector<long long> off(4 * (size_t)(n + 1), 0);
  long long* face_off = off.data();
  long long* leaf_off = face_off + (n + 1);
  long long* node_off = leaf_off + (n + 1);
  long long* tile_off = node_off + (n + 1);
  {  // the flattened face index is an int: check before allocating anything
    long long nf = 0;
    for (int64_t i = 0; i < n; i++) nf += ((M[i]->nt + 31) / 32) * 32;
    if (nf > (1ll << 31) - 2 * kSortTile) return G3D_ERR_INVALID_ARG;
  }
  // one block for the permanent arrays of all meshes of the call
  size_t total = 0;
  for (int64_t i = 0; i < n; i++) {
    const size_t nt = (size_t)M[i]->nt, nleaf = (nt + L - 1) / L, nint = nleaf > 1 ? nleaf - 1 : 1;
    total += 3 * up256(16 * nt) + up256(64 * nint) + up256(32 * nleaf) + up256(8 * nint) +
             up256(sizeof(float) * kClusters * kClusterStride) + (M[i]->master ? up256(72 * nt) : 0);
  }
  Slab* slab = new Slab();
  if (cudaMallocAsync(&slab->base, total, s) != cudaSuccess) {
    cudaGetLastError();
    delete slab;
    return G3D_ERR_OOM;
  }
  size_t at = 0;
  auto take = [&](size_t bytes) {
    void* p = (char*)slab->base + at;
    at += up256(bytes);
    return p;
  };
  for (int64_t i = 0; i < n; i++) {
    G3dMesh* m = M[i];
    const int nt = (int)m->nt, nleaf = (nt + L - 1) / L, nint = nleaf - 1;
    if (m->has_bvh) {  // rebuild: let go of the previous arrays
      slab_release(m->bvh_slab, s);
      m->has_bvh = false;
    }
    m->bvh_slab = slab;
    slab->refs++;
    m->v0 = (float4*)take(16 * (size_t)nt);
    m->v1 = (float4*)take(16 * (size_t)nt);
    m->v2 = (float4*)take(16 * (size_t)nt);
    m->nodes = (float4*)take(64 * (size_t)(nint > 0 ? nint : 1));
    m->leaves = (float4*)take(32 * (size_t)nleaf);
    m->nrange = (int2*)take(8 * (size_t)(nint > 0 ? nint : 1));
    m->cstats = (float*)take(sizeof(float) * kClusters * kClusterStride);
    m->m64 = m->master ? (double*)take(72 * (size_t)nt) : nullptr;
    BuildMesh& b = bm[i];
    b.V = m->raw_v; b.I = m->raw_i; b.dtype = m->dtype; b.nt = nt; b.L = L; b.nleaf = nleaf;
    b.v0 = m->v0; b.v1 = m->v1; b.v2 = m->v2; b.m64 = m->m64; b.nodes = m->nodes; b.leaves = m->leaves;
    b.nrange = m->nrange;
    b.box = m->box;
    face_off[i + 1] = face_off[i] + ((nt + 31) / 32) * 32;  // padded: warps never straddle meshes
    leaf_off[i + 1] = leaf_off[i] + nleaf;
    node_off[i + 1] = node_off[i] + nint;
    tile_off[i + 1] = tile_off[i] + (nt + kSortTile - 1) / kSortTile;
  }
  const long long NF = face_off[n], NL = leaf_off[n], NN = node_off[n], NT = tile_off[n];
  if (NF > (1ll << 31) - 2 * kSortTile) return G3D_ERR_INVALID_ARG;
  // device copies of the tables
  char* d_tab = nullptr;
  size_t tab_bytes = sizeof(BuildMesh) * n + sizeof(long long) * off.size();
  CK(cudaMallocAsync((void**)&d_tab, tab_bytes + 16, s));
  std::vector<char> h_tab(tab_bytes);
  memcpy(h_tab.data(), bm.data(), sizeof(BuildMesh) * n);
  memcpy(h_tab.data() + sizeof(BuildMesh) * n, off.data(), sizeof(long long) * off.size());
  CK(cudaMemcpyAsync(d_tab, h_tab.data(), tab_bytes, cudaMemcpyHostToDevice, s));
  BuildArgs a{};
  a.m = (const BuildMesh*)d_tab;
  a.n = (int)n;
  const long long* d_off = (const long long*)(d_tab + sizeof(BuildMesh) * n);
  a.face_off = d_off;
  a.leaf_off = d_off + (n + 1);
  a.node_off = d_off + 2 * (n + 1);
  a.tile_off = d_off + 3 * (n + 1);
  a.total_faces = NF; a.total_leaves = NL; a.total_nodes = NN;
  a.cells = (float)((1 << c->cfg.morton_bits) - 1);
  // scratch
  unsigned int *keys1 = nullptr, *vals1 = nullptr, *hist = nullptr, *dtot = nullptr;
  CK(amalloc(&a.bounds, 8 * (size_t)n, s));
  CK(amalloc(&a.keys0, NF, s));
  CK(amalloc(&keys1, NF, s));
  CK(amalloc(&a.vals0, NF, s));
  CK(amalloc(&vals1, NF, s));
  CK(amalloc(&hist, 256 * (size_t)NT, s));
  CK(amalloc(&dtot, 256 * (size_t)n, s));
  CK(amalloc(&a.lkeys, NL, s));
  CK(amalloc(&a.child, 2 * (size_t)(NN > 0 ? NN : 1), s));
  CK(amalloc(&a.ccount, 2 * (size_t)(NN > 0 ? NN : 1), s));
  CK(amalloc(&a.pnode, (size_t)(NN > 0 ? NN : 1), s));
  CK(amalloc(&a.visit, (size_t)(NN > 0 ? NN : 1), s));
  CK(amalloc(&a.pleaf, NL, s));

  G3D_LAUNCH(c, "k_bounds_from_ingest", k_bounds_from_ingest, grid_for(n, 256, 1 << 30), 256, 0, s, a);
  // keys, values and the first pass's digit counts in one launch
  G3D_LAUNCH(c, "k_morton_tiles", k_morton_tiles, (unsigned int)NT, 256, 0, s, a, hist);
  unsigned int *kin = a.keys0, *kout = keys1, *vin = a.vals0, *vout = vals1;
  for (int shift = 0; shift < 3 * c->cfg.morton_bits; shift += 8) {
    if (shift > 0) G3D_LAUNCH(c, "k_seg_hist", k_seg_hist, (unsigned int)NT, 256, 0, s, a, kin, shift, hist);
    G3D_LAUNCH(c, "k_seg_scan_rows", k_seg_scan_rows, grid_for(256ll * n * 32, 256, 1 << 30), 256, 0, s, a, hist,
               dtot);
    G3D_LAUNCH(c, "k_seg_scan_digits", k_seg_scan_digits, grid_for(n * 32, 256, 1 << 30), 256, 0, s, a, dtot);
    G3D_LAUNCH(c, "k_seg_scatter", k_seg_scatter, (unsigned int)NT, 256, 0, s, a, kin, vin, kout, vout, shift, hist,
               dtot);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  G3D_LAUNCH(c, "k_gather_many", k_gather_many, grid_for(NF, 256, 1 << 30), 256, 0, s, a, kin, vin);
  if (NN > 0) {
    G3D_LAUNCH(c, "k_radix_tree_many", k_radix_tree_many, grid_for(NN, 256, 1 << 30), 256, 0, s, a);
    G3D_LAUNCH(c, "k_check_tree_many", k_check_tree_many, grid_for(NN, 256, 1 << 30), 256, 0, s, a, c->d_sticky);
    CK(cudaMemsetAsync(a.visit, 0, sizeof(int) * NN, s));
    G3D_LAUNCH(c, "k_refit_many", k_refit_many, grid_for(NL, 256, 1 << 30), 256, 0, s, a);
  }
  for (void* p : {(void*)a.bounds, (void*)a.keys0, (void*)keys1, (void*)a.vals0, (void*)vals1, (void*)hist, (void*)dtot,
                  (void*)a.lkeys, (void*)a.child, (void*)a.ccount, (void*)a.pnode, (void*)a.visit,
                  (void*)a.pleaf, (void*)d_tab})
    afree(p, s);
  CK(cudaGetLastError());
  for (int64_t i = 0; i < n; i++) {
    G3dMesh* m = M[i];
    MeshDev& d = m->dev;
    const int nleaf = bm[i].nleaf;
    d.v0 = m->v0; d.v1 = m->v1; d.v2 = m->v2;
    d.m64 = m->m64;
    d.nodes = m->nodes;
    d.leaves = m->leaves;
    d.root = nleaf > 1 ? 0 : ~0;
    d.nleaf = nleaf;
    d.ntri = (int)m->nt;
    d.rho = m->rho;
    d.L = L;
    d.nrange = m->nrange;
    d.cstats = m->cstats;
    m->cstats_valid = false;
    m->has_bvh = true;
  }
  return G3D_OK;
}

int g3d_mesh_build_bvh(g3d_ctx* c, g3d_mesh h, void* stream) {
  return g3d_mesh_build_bvh_many(c, 1, &h, stream);
}

static int single_query(g3d_ctx* c, g3d_mesh ha, g3d_mesh hb, int op, double* dout, uint8_t* hout,
                        void* stream) {
  if (!c) return G3D_ERR_INVALID_ARG;
  G3dMesh *A = get_mesh(c, ha), *B = get_mesh(c, hb);
  if (!A || !B) return G3D_ERR_INVALID_ARG;
  if (!A->has_bvh || !B->has_bvh) return G3D_ERR_NO_BVH;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->proposal) {
    const g3d_query one{ha, hb, op, 0};
    int r = ensure_cstats(c, &one, 1, s);
    if (r) return r;
  }
  QueryDev q = make_query(A, B, op);
  c->cur_leaf_max = A->dev.L > B->dev.L ? A->dev.L : B->dev.L;
  G3D_LAUNCH(c, "k_set_query", k_set_query, 1, 1, 0, s, c->qdev, q);
  double* dd = (dout && is_device_ptr(dout)) ? dout : c->d_dist;
  unsigned char* hd = (hout && is_device_ptr(hout)) ? hout : c->d_hit;
  int rc = run_queries(c, 1, op == G3D_OP_DISTANCE ? dd : nullptr, hd, c->d_status, s);
  if (rc) return rc;
  if (op == G3D_OP_DISTANCE && dout && dd != dout) CK(cudaMemcpyAsync(dout, dd, 8, cudaMemcpyDeviceToHost, s));
  if (hout && hd != hout) CK(cudaMemcpyAsync(hout, hd, 1, cudaMemcpyDeviceToHost, s));
  return G3D_OK;
}

int g3d_distance(g3d_ctx* c, g3d_mesh a, g3d_mesh b, double* out, void* stream) {
  if (!out) return G3D_ERR_INVALID_ARG;
  return single_query(c, a, b, G3D_OP_DISTANCE, out, nullptr, stream);
}

int g3d_intersects(g3d_ctx* c, g3d_mesh a, g3d_mesh b, uint8_t* out, void* stream) {
  if (!out) return G3D_ERR_INVALID_ARG;
  return single_query(c, a, b, G3D_OP_INTERSECTS, nullptr, out, stream);
}

// Device query records of a batch, with each distance query linked to an
// intersects query of the same mesh pair when the batch holds one.
// meshes (optional): the meshes of the queries the learned proposal covers
// (both meshes with at least cfg.proposal_min_faces faces), whose cluster
// statistics the network's features read
static int build_queries(g3d_ctx* c, const g3d_query* q, int64_t n, QueryDev* hq,
                         std::vector<G3dMesh*>* meshes = nullptr) {
  if (meshes) meshes->clear();
  int lmax = 2;
  std::unordered_map<uint64_t, int64_t> isect_of;  // unordered mesh pair -> an intersects query
  isect_of.reserve((size_t)n);
  auto pair_key = [](g3d_mesh x, g3d_mesh y) {
    uint64_t lo = (uint64_t)(x < y ? x : y), hi = (uint64_t)(x < y ? y : x);
    return (hi << 32) ^ lo;
  };
  for (int64_t i = 0; i < n; i++) {
    G3dMesh *A = get_mesh(c, q[i].a), *B = get_mesh(c, q[i].b);
    if (!A || !B || (q[i].op != G3D_OP_DISTANCE && q[i].op != G3D_OP_INTERSECTS)) return G3D_ERR_INVALID_ARG;
    if (!A->has_bvh || !B->has_bvh) return G3D_ERR_NO_BVH;
    hq[i] = make_query(A, B, q[i].op);
    if (meshes && std::min(A->dev.ntri, B->dev.ntri) >= c->cfg.proposal_min_faces) {
      meshes->push_back(A);
      meshes->push_back(B);
    }
    if (q[i].op == G3D_OP_INTERSECTS) isect_of.emplace(pair_key(q[i].a, q[i].b), i);
    lmax = std::max(lmax, std::max(A->dev.L, B->dev.L));
  }
  c->cur_leaf_max = lmax;
  // distance == 0 iff the meshes intersect: a distance query shares the
  // intersects phase of an intersects query of the same pair
  for (int64_t i = 0; i < n; i++) {
    if (q[i].op != G3D_OP_DISTANCE) continue;
    auto it = isect_of.find(pair_key(q[i].a, q[i].b));
    if (it != isect_of.end()) {
      const int64_t j = it->second;
      if ((q[j].a == q[i].a && q[j].b == q[i].b) || (q[j].a == q[i].b && q[j].b == q[i].a)) {
        hq[i].link = (int)j;
        if (hq[j].dlink < 0) hq[j].dlink = (int)i;
      }
    }
  }
  return G3D_OK;
}

static int build_queries_v(g3d_ctx* c, const g3d_query* q, int64_t n, std::vector<QueryDev>& hq,
                           std::vector<G3dMesh*>* meshes = nullptr) {
  hq.resize((size_t)n);
  return build_queries(c, q, n, hq.data(), meshes);
}

// Pinned host staging for a batch's query records and proposal rows, two
// buffers used in turn: a copy from pinned memory does not wait for the
// stream's earlier work (one from pageable memory does), so the host can
// prepare the next batch while the device runs this one.  Before a buffer is
// refilled, the copy that last read it is waited for.
void* stage_acquire(g3d_ctx* c, size_t bytes) {
  g3d_ctx::Stage& st = c->stage[c->stage_i];
  if (st.ev) cudaEventSynchronize(st.ev);
  if (st.cap < bytes) {
    if (st.p) cudaFreeHost(st.p);
    st.p = nullptr;
    st.cap = 0;
    size_t cap = std::max<size_t>(bytes, (size_t)1 << 20);
    if (cudaMallocHost(&st.p, cap) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    st.cap = cap;
  }
  return st.p;
}

void stage_release(g3d_ctx* c, cudaStream_t s) {
  g3d_ctx::Stage& st = c->stage[c->stage_i];
  if (!st.ev) cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming);
  if (st.ev) cudaEventRecord(st.ev, s);
  c->stage_i ^= 1;
}

int g3d_batch_ex(g3d_ctx* c, const g3d_query* q, int64_t n, double* dist_out, uint8_t* hit_out,
                 int32_t* status_out, int64_t* witness_out, int32_t* cluster_out, void* stream);

int g3d_batch(g3d_ctx* c, const g3d_query* q, int64_t n, double* dist_out, uint8_t* hit_out, int32_t* status_out,
              void* stream) {
  return g3d_batch_ex(c, q, n, dist_out, hit_out, status_out, nullptr, nullptr, stream);
}

static int batch_impl(g3d_ctx* c, const g3d_query* q, int64_t n, const int32_t* hint, double* dist_out,
                      uint8_t* hit_out, int32_t* status_out, int64_t* witness_out, int32_t* cluster_out,
                      void* stream) {
  if (!c || (!q && n > 0) || n < 0) return G3D_ERR_INVALID_ARG;
  if (n == 0) return G3D_OK;
  if (n > (int64_t)c->queue.cap / 4) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  // query records built in pinned staging (rows of the proposal after them)
  const size_t qbytes = up256(sizeof(QueryDev) * (size_t)n);
  QueryDev* hq = (QueryDev*)stage_acquire(c, qbytes + sizeof(int) * (size_t)n);
  if (!hq) return G3D_ERR_OOM;
  // every return below: the buffer is marked in use by the copies issued
  // from it so far
  struct StageGuard {
    g3d_ctx* c;
    cudaStream_t s;
    bool done = false;
    void release() {  // after the last copy that reads the buffer
      if (!done) stage_release(c, s);
      done = true;
    }
    ~StageGuard() { release(); }
  } stage_guard{c, s};
  int* hrows = (int*)((char*)hq + qbytes);
  std::vector<G3dMesh*> qmeshes;
  int rc = build_queries(c, q, n, hq, c->proposal && !hint ? &qmeshes : nullptr);
  if (rc) return rc;
  rc = ensure_query_capacity(c, (int)n, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->qdev, hq, sizeof(QueryDev) * n, cudaMemcpyHostToDevice, s));
  double* dd = (dist_out && is_device_ptr(dist_out)) ? dist_out : c->d_dist;
  unsigned char* hd = (hit_out && is_device_ptr(hit_out)) ? hit_out : c->d_hit;
  int* sd = (status_out && is_device_ptr(status_out)) ? status_out : c->d_status;
  long long* wd = nullptr;
  if (witness_out) {
    if (!is_device_ptr(witness_out)) return G3D_ERR_INVALID_ARG;
    wd = (long long*)witness_out;
  }
  if (cluster_out && !is_device_ptr(cluster_out)) return G3D_ERR_INVALID_ARG;
  if (c->proposal && !hint) {
    rc = ensure_cstats_meshes(c, qmeshes, s);
    if (rc) return rc;
  }
  const int* hd_hint = nullptr;
  if (hint) {
    if (is_device_ptr(hint)) {
      hd_hint = (const int*)hint;
    } else {
      rc = ensure_prop_capacity(c, (int)n, s);
      if (rc) return rc;
      CK(cudaMemcpyAsync(c->prop_top, hint, sizeof(int) * n, cudaMemcpyHostToDevice, s));
      hd_hint = c->prop_top;
    }
  }
  // count_visits: a first-visit bit per node and leaf of both meshes of
  // every query (stream-ordered scratch, released after the launch)
  void* vis = nullptr;
  if (c->cfg.count_visits) {
    std::vector<long long> off((size_t)n);
    long long bits = 0;
    for (int64_t i = 0; i < n; i++) {
      off[i] = bits;
      bits += 2ll * hq[i].A.nleaf - 1 + 2ll * hq[i].B.nleaf - 1;
    }
    const size_t words = (size_t)((bits + 31) / 32);
    const size_t ob = up256(sizeof(long long) * n);
    rc = cuda_err(cudaMallocAsync(&vis, ob + 4 * words + 4, s));
    if (!rc) rc = cuda_err(cudaMemcpyAsync(vis, off.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, s));
    if (!rc) rc = cuda_err(cudaMemsetAsync((char*)vis + ob, 0, 4 * words + 4, s));
    if (!rc) rc = cuda_err(cudaStreamSynchronize(s));  // the host offsets go out of scope
    if (rc) {
      if (vis) cudaFreeAsync(vis, s);
      return rc;
    }
    c->visit_off = (long long*)vis;
    c->visit = (unsigned int*)((char*)vis + ob);
  }
  // The level-synchronous form keeps a whole batch's frontier in fixed
  // lists: a batch of thousands of queries on meshes of up to a million
  // faces can outgrow them, and the work that then goes to the global queue
  // and the second pass is several times slower.  A batch whose queries
  // reference more than chunk_mfaces Mi faces (both meshes of every query
  // counted) runs as consecutive chunks of at most that many, each with its
  // own links between distance and intersects queries of the same mesh
  // pair.  (How wide a frontier gets depends on the geometry more than on
  // the face count -- pairs far apart relative to their size are the wide
  // ones -- so the default limit is generous and callers that form batches,
  // like a server's rounds, bound them themselves.)
  const long long kChunkFaces = (long long)c->cfg.chunk_mfaces << 20;
  std::vector<std::pair<int64_t, int64_t>> chunks;
  if (c->cfg.traversal == 1 && !c->cfg.count_visits) {
    int64_t i0 = 0;
    long long sum = 0;
    for (int64_t i = 0; i < n; i++) {
      const long long f = (long long)hq[i].A.ntri + hq[i].B.ntri;
      if (i > i0 && sum + f > kChunkFaces) {
        chunks.emplace_back(i0, i);
        i0 = i;
        sum = 0;
      }
      sum += f;
    }
    chunks.emplace_back(i0, n);
  }
  if (chunks.size() > 1) {
    for (const auto& ch : chunks) {
      const int64_t i0 = ch.first, m = ch.second - ch.first;
      std::vector<QueryDev> hc;
      rc = build_queries_v(c, q + i0, m, hc);
      if (!rc) rc = cuda_err(cudaMemcpyAsync(c->qdev, hc.data(), sizeof(QueryDev) * m, cudaMemcpyHostToDevice, s));
      if (!rc && !hd_hint) rc = select_proposal_rows(c, hc.data(), m, hrows + i0, s);
      if (!rc)
        rc = run_queries(c, (int)m, dd + i0, hd + i0, sd + i0, s, nullptr, nullptr, wd ? wd + i0 : nullptr,
                         cluster_out ? (int*)cluster_out + i0 : nullptr, hd_hint ? hd_hint + i0 : nullptr);
      if (rc) break;
    }
  } else {
    if (!hd_hint) rc = select_proposal_rows(c, hq, n, hrows, s);
    stage_guard.release();  // the staging buffer's copies are all issued
    if (!rc) rc = run_queries(c, (int)n, dd, hd, sd, s, nullptr, nullptr, wd, (int*)cluster_out, hd_hint);
  }
  c->prop_nrows = -1;
  c->visit = nullptr;
  c->visit_off = nullptr;
  if (vis) cudaFreeAsync(vis, s);
  if (rc) return rc;
  if (dist_out && dd != dist_out) CK(cudaMemcpyAsync(dist_out, dd, 8 * n, cudaMemcpyDeviceToHost, s));
  if (hit_out && hd != hit_out) CK(cudaMemcpyAsync(hit_out, hd, n, cudaMemcpyDeviceToHost, s));
  if (status_out && sd != status_out) CK(cudaMemcpyAsync(status_out, sd, 4 * n, cudaMemcpyDeviceToHost, s));
  return G3D_OK;
}

int g3d_batch_ex(g3d_ctx* c, const g3d_query* q, int64_t n, double* dist_out, uint8_t* hit_out,
                 int32_t* status_out, int64_t* witness_out, int32_t* cluster_out, void* stream) {
  return batch_impl(c, q, n, nullptr, dist_out, hit_out, status_out, witness_out, cluster_out, stream);
}

int g3d_batch_hint(g3d_ctx* c, const g3d_query* q, int64_t n, const int32_t* hint, double* dist_out,
                   uint8_t* hit_out, int32_t* status_out, int64_t* witness_out, int32_t* cluster_out,
                   void* stream) {
  if (!hint) return G3D_ERR_INVALID_ARG;
  return batch_impl(c, q, n, hint, dist_out, hit_out, status_out, witness_out, cluster_out, stream);
}

struct g3d_plan {
  int64_t n = 0;
  QueryDev* qdev = nullptr;
  QueryState* st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;  // kernel nodes per replay
};

int g3d_plan_create(g3d_ctx* c, const g3d_query* q, int64_t n, double* dist_out, uint8_t* hit_out,
                    int32_t* status_out, g3d_plan** out, void* stream) {
  if (!c || !q || n <= 0 || !out || !dist_out || !hit_out) return G3D_ERR_INVALID_ARG;
  if (n > (int64_t)c->queue.cap / 4) return G3D_ERR_INVALID_ARG;
  if (!is_device_ptr(dist_out) || !is_device_ptr(hit_out) || (status_out && !is_device_ptr(status_out)))
    return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<QueryDev> hq;
  int rc = build_queries_v(c, q, n, hq);
  if (rc) return rc;
  g3d_plan* p = new g3d_plan();
  p->n = n;
  rc = cuda_err(cudaMalloc(&p->qdev, sizeof(QueryDev) * n));
  if (!rc) rc = cuda_err(cudaMalloc(&p->st, sizeof(QueryState) * n));
  if (!rc) rc = cuda_err(cudaMemcpyAsync(p->qdev, hq.data(), sizeof(QueryDev) * n, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  // scratch the captured sequence needs is allocated before the capture
  if (!rc && c->proposal) rc = ensure_cstats(c, q, n, s);
  if (!rc && c->proposal) {
    rc = ensure_prop_capacity(c, (int)n, s);
    if (!rc) rc = mlp_reserve(c->proposal, (int)n, s);
    if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  }
  cudaStream_t cs = nullptr;
  if (!rc) rc = cuda_err(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  if (!rc) {
    const unsigned long long before = c->launches;
    c->capturing = true;
    rc = cuda_err(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    if (!rc) {
      int r2 = run_queries(c, (int)n, dist_out, hit_out, status_out, cs, p->qdev, p->st);
      cudaError_t e = cudaStreamEndCapture(cs, &p->graph);
      rc = r2 ? r2 : cuda_err(e);
    }
    c->capturing = false;
    p->kernels = c->launches - before;
    c->launches = before;
  }
  if (!rc) rc = cuda_err(cudaGraphInstantiate(&p->exec, p->graph, 0));
  if (cs) cudaStreamDestroy(cs);
  if (rc) {
    g3d_plan_destroy(c, p);
    return rc;
  }
  *out = p;
  return G3D_OK;
}

int g3d_plan_launch(g3d_ctx* c, g3d_plan* p, void* stream) {
  if (!c || !p || !p->exec) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  c->launches += p->kernels;
  return G3D_OK;
}

int g3d_plan_destroy(g3d_ctx* c, g3d_plan* p) {
  if (!c || !p) return G3D_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->qdev) cudaFree(p->qdev);
  if (p->st) cudaFree(p->st);
  delete p;
  return G3D_OK;
}

// ---------------------------------------------------------------------------
// mesh volume
// ---------------------------------------------------------------------------
int g3d_volume_many(g3d_ctx* c, int64_t n, const g3d_mesh* hs, double* out, void* stream) {
  NvtxRange nvtx_range("g3d_volume_many");
  if (!c || n < 0 || (n > 0 && (!hs || !out))) return G3D_ERR_INVALID_ARG;
  if (n == 0) return G3D_OK;
  if (n > (1ll << 30)) return G3D_ERR_INVALID_ARG;
  std::vector<VolMesh> vm((size_t)n);
  std::vector<long long> chunk0((size_t)n + 1, 0), vchunk0((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; i++) {
    G3dMesh* m = get_mesh(c, hs[i]);
    if (!m) return G3D_ERR_INVALID_ARG;
    vm[i] = VolMesh{m->raw_v, m->raw_i, (long long)m->nt, (long long)m->nv, m->dtype, 0};
    chunk0[i + 1] = chunk0[i] + (m->nt + kVolChunk - 1) / kVolChunk;
    // the range pass covers float32 meshes only
    vchunk0[i + 1] = vchunk0[i] + (m->dtype == G3D_F32 ? (m->nv + kVolRangeVerts - 1) / kVolRangeVerts : 0);
  }
  const long long nch = chunk0[n], nvch = vchunk0[n];
  if (nch > 0x7fffffffll || nvch > 0x7fffffffll) return G3D_ERR_INVALID_ARG;
  std::vector<int> cmesh((size_t)nch), vcmesh((size_t)nvch);
  std::vector<long long> cfirst((size_t)nch), vcfirst((size_t)nvch);
  for (int64_t i = 0; i < n; i++) {
    for (long long k = chunk0[i]; k < chunk0[i + 1]; k++) {
      cmesh[k] = (int)i;
      cfirst[k] = (k - chunk0[i]) * kVolChunk;
    }
    for (long long k = vchunk0[i]; k < vchunk0[i + 1]; k++) {
      vcmesh[k] = (int)i;
      vcfirst[k] = (k - vchunk0[i]) * kVolRangeVerts;
    }
  }
  std::vector<unsigned int> range0(2 * (size_t)n);
  for (int64_t i = 0; i < n; i++) {
    range0[2 * i] = 0x7f800000u;
    range0[2 * i + 1] = 0u;
  }
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  // one stream-ordered scratch block: tables, coordinate ranges, partial
  // sums, device result
  const size_t b_mesh = sizeof(VolMesh) * n, b_c0 = sizeof(long long) * (n + 1), b_cm = sizeof(int) * nch,
               b_cf = sizeof(long long) * nch, b_vm = sizeof(int) * nvch, b_vf = sizeof(long long) * nvch,
               b_rg = sizeof(unsigned int) * 2 * n, b_part = sizeof(VolPartial) * nch, b_out = sizeof(double) * n;
  auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t o_c0 = up16(b_mesh), o_cm = o_c0 + up16(b_c0), o_cf = o_cm + up16(b_cm), o_vm = o_cf + up16(b_cf),
               o_vf = o_vm + up16(b_vm), o_rg = o_vf + up16(b_vf), o_part = o_rg + up16(b_rg),
               o_out = o_part + up16(b_part), total = o_out + up16(b_out);
  char* d = nullptr;
  CK(cudaMallocAsync((void**)&d, total, s));
  std::vector<char> h(o_part);
  memcpy(h.data(), vm.data(), b_mesh);
  memcpy(h.data() + o_c0, chunk0.data(), b_c0);
  memcpy(h.data() + o_cm, cmesh.data(), b_cm);
  memcpy(h.data() + o_cf, cfirst.data(), b_cf);
  memcpy(h.data() + o_vm, vcmesh.data(), b_vm);
  memcpy(h.data() + o_vf, vcfirst.data(), b_vf);
  memcpy(h.data() + o_rg, range0.data(), b_rg);
  int rc = cuda_err(cudaMemcpyAsync(d, h.data(), o_part, cudaMemcpyHostToDevice, s));
  const bool out_dev = is_device_ptr(out);
  double* dout = out_dev ? out : (double*)(d + o_out);
  if (!rc && nvch > 0) {
    G3D_LAUNCH(c, "k_volume_range", k_volume_range, (unsigned int)nvch, 256, 0, s, (const VolMesh*)d,
               (const int*)(d + o_vm), (const long long*)(d + o_vf), (unsigned int*)(d + o_rg));
  }
  if (!rc && nch > 0) {
    G3D_LAUNCH(c, "k_volume_chunks", k_volume_chunks, (unsigned int)nch, kVolThreads, 0, s, (const VolMesh*)d,
               (const int*)(d + o_cm), (const long long*)(d + o_cf), (const unsigned int*)(d + o_rg),
               (VolPartial*)(d + o_part));
  }
  if (!rc) {
    G3D_LAUNCH(c, "k_volume_finish", k_volume_finish, grid_for(32ll * n, 128, 1 << 30), 128, 0, s, (int)n,
               (const long long*)(d + o_c0), (const VolPartial*)(d + o_part), (const unsigned int*)(d + o_rg), dout);
    rc = cuda_err(cudaGetLastError());
  }
  if (!rc && !out_dev) rc = cuda_err(cudaMemcpyAsync(out, dout, b_out, cudaMemcpyDeviceToHost, s));
  // the host tables must outlive their upload
  if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  cudaFreeAsync(d, s);
  return rc;
}

int g3d_volume(g3d_ctx* c, g3d_mesh h, double* out, void* stream) { return g3d_volume_many(c, 1, &h, out, stream); }

// ---------------------------------------------------------------------------
// line segments / points against one mesh
// ---------------------------------------------------------------------------
int g3d_segments(g3d_ctx* c, g3d_mesh mesh, const float* segs, int64_t n, int32_t op, double* dist_out,
                 uint8_t* hit_out, int32_t* status_out, void* stream) {
  NvtxRange nvtx_range("g3d_segments");
  if (!c || n < 0 || (n > 0 && !segs)) return G3D_ERR_INVALID_ARG;
  if (op != G3D_OP_DISTANCE && op != G3D_OP_INTERSECTS) return G3D_ERR_INVALID_ARG;
  if ((op == G3D_OP_DISTANCE && !dist_out) || (op == G3D_OP_INTERSECTS && !hit_out)) return G3D_ERR_INVALID_ARG;
  G3dMesh* m = get_mesh(c, mesh);
  if (!m) return G3D_ERR_INVALID_ARG;
  if (!m->has_bvh) return G3D_ERR_NO_BVH;
  if (n == 0) return G3D_OK;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  // host inputs / outputs go through stream-ordered device temporaries
  const bool seg_dev = is_device_ptr(segs);
  const bool d_dev = dist_out && is_device_ptr(dist_out);
  const bool h_dev = hit_out && is_device_ptr(hit_out);
  const bool s_dev = status_out && is_device_ptr(status_out);
  float* dsegs = seg_dev ? (float*)segs : nullptr;
  double* dd = d_dev ? dist_out : nullptr;
  unsigned char* dh = h_dev ? hit_out : nullptr;
  int* ds = s_dev ? (int*)status_out : nullptr;
  int rc = G3D_OK;
  if (!seg_dev) rc = cuda_err(cudaMallocAsync((void**)&dsegs, sizeof(float) * 6 * (size_t)n, s));
  if (!rc && dist_out && !d_dev) rc = cuda_err(cudaMallocAsync((void**)&dd, sizeof(double) * (size_t)n, s));
  if (!rc && hit_out && !h_dev) rc = cuda_err(cudaMallocAsync((void**)&dh, (size_t)n, s));
  if (!rc && status_out && !s_dev) rc = cuda_err(cudaMallocAsync((void**)&ds, sizeof(int) * (size_t)n, s));
  if (!rc && !seg_dev)
    rc = cuda_err(cudaMemcpyAsync(dsegs, segs, sizeof(float) * 6 * (size_t)n, cudaMemcpyHostToDevice, s));
  if (!rc) {
    SegArgs a{};
    a.M = m->dev;
    a.segs = dsegs;
    a.n = n;
    a.op = op;
    a.slack = m->rho > 0.f ? (float)(1.7320508075688774 * (double)m->rho * (1.0 + 1e-6)) : 0.f;
    a.dist = dd;
    a.hit = dh;
    a.status = ds;
    a.stats = c->stats;
    a.sticky = c->d_sticky;
    G3D_LAUNCH(c, "k_segments", k_segments, (unsigned int)((n + 127) / 128), 128, 0, s, a);
    rc = cuda_err(cudaGetLastError());
  }
  if (!rc && dist_out && !d_dev)
    rc = cuda_err(cudaMemcpyAsync(dist_out, dd, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
  if (!rc && hit_out && !h_dev) rc = cuda_err(cudaMemcpyAsync(hit_out, dh, (size_t)n, cudaMemcpyDeviceToHost, s));
  if (!rc && status_out && !s_dev)
    rc = cuda_err(cudaMemcpyAsync(status_out, ds, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, s));
  if (!seg_dev && dsegs) cudaFreeAsync(dsegs, s);
  if (dist_out && !d_dev && dd) cudaFreeAsync(dd, s);
  if (hit_out && !h_dev && dh) cudaFreeAsync(dh, s);
  if (status_out && !s_dev && ds) cudaFreeAsync(ds, s);
  return rc;
}

// ---------------------------------------------------------------------------
// autotuner: coordinate search over the launch parameters on a sample batch
// ---------------------------------------------------------------------------
namespace {

// median CUDA-event time (ms) of `reps` runs of the uploaded sample after
// one untimed run; negative on error
float time_sample(g3d_ctx* c, int n, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  std::vector<float> t;
  for (int r = 0; r <= reps; r++) {
    if (cudaEventRecord(e0, s) != cudaSuccess) return -1.f;
    if (run_queries(c, n, c->d_dist, c->d_hit, c->d_status, s)) return -1.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r) t.push_back(ms);
  }
  int err = 0;
  cudaMemcpy(&err, c->d_sticky, sizeof(int), cudaMemcpyDeviceToHost);
  if (err) return -1.f;
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

}  // namespace

int g3d_autotune(g3d_ctx* c, const g3d_query* q, int64_t n, int32_t flags, int32_t reps, g3d_config* chosen,
                 void* stream) {
  NvtxRange nvtx_range("g3d_autotune");
  if (!c || !q || n <= 0 || reps < 1 || reps > 100 || (flags & ~(G3D_TUNE_LEAF_SIZE | G3D_TUNE_COUNT_BUILD)))
    return G3D_ERR_INVALID_ARG;
  if (n > (int64_t)c->queue.cap / 4) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  // the distinct meshes of the sample (rebuilt when leaf sizes are tuned)
  std::vector<g3d_mesh> uniq;
  {
    std::unordered_map<g3d_mesh, int> seen;
    for (int64_t i = 0; i < n; i++)
      for (g3d_mesh h : {q[i].a, q[i].b})
        if (seen.emplace(h, 0).second) uniq.push_back(h);
  }
  auto upload = [&]() -> int {
    std::vector<QueryDev> hq;
    int rc = build_queries_v(c, q, n, hq);
    if (rc) return rc;
    rc = ensure_query_capacity(c, (int)n, s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->qdev, hq.data(), sizeof(QueryDev) * n, cudaMemcpyHostToDevice, s));
    return G3D_OK;
  };
  auto rebuild = [&](int L) -> int {
    c->cfg.leaf_size = L;
    for (size_t i = 0; i < uniq.size(); i += 60000) {
      const int64_t m = (int64_t)std::min<size_t>(60000, uniq.size() - i);
      int rc = g3d_mesh_build_bvh_many(c, m, uniq.data() + i, s);
      if (rc) return rc;
    }
    return upload();
  };
  int rc = upload();
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return G3D_ERR_CUDA; }
  const bool prof = c->prof_on;
  c->prof_on = false;  // the tuner's own runs are not profiled
  g3d_config best = c->cfg;
  float best_ms = time_sample(c, (int)n, reps, s, e0, e1);
  if (best_ms < 0.f) rc = G3D_ERR_CUDA;
  // one sweep per parameter, holding the others at the best values so far
  struct Axis { int32_t g3d_config::*field; std::vector<int> values; };
  const std::vector<Axis> axes = {
      {&g3d_config::traversal, {1, 2}},
      {&g3d_config::isect_first, {1, 2}},
      {&g3d_config::dives, {4, 16, 32}},
      {&g3d_config::ctas_per_sm, {1, 2, 3, 4, 6}},
      {&g3d_config::warps_per_cta, {1, 2, 4}},
      {&g3d_config::stack_depth, {128, 256, 512}},
  };
  for (const Axis& ax : axes) {
    for (int v : ax.values) {
      if (rc || best.*(ax.field) == v) continue;
      c->cfg = best;
      c->cfg.*(ax.field) = v;
      float ms = time_sample(c, (int)n, reps, s, e0, e1);
      if (ms < 0.f) { rc = G3D_ERR_CUDA; break; }
      if (ms < best_ms) { best_ms = ms; best = c->cfg; }
    }
  }
  if (!rc && (flags & G3D_TUNE_LEAF_SIZE)) {
    // wall time of rebuilding the sample's meshes (host work included)
    auto timed_rebuild = [&](int L, float* ms) -> int {
      int r = rebuild(L);  // first build at this size also settles the allocations
      if (r) return r;
      CK(cudaStreamSynchronize(s));
      const auto t0 = std::chrono::steady_clock::now();
      r = rebuild(L);
      if (r) return r;
      CK(cudaStreamSynchronize(s));
      *ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
      return G3D_OK;
    };
    const bool count_build = (flags & G3D_TUNE_COUNT_BUILD) != 0;
    const int L0 = best.leaf_size;
    if (count_build) {
      float bms = 0.f;
      c->cfg = best;
      rc = timed_rebuild(L0, &bms);
      best_ms += bms;
    }
    const int B0 = best.morton_bits;
    for (int L : {4, 8, 16})
      for (int bits : {8, 10}) {
        if (rc || (L == L0 && bits == B0)) continue;
        c->cfg = best;
        c->cfg.morton_bits = bits;
        float bms = 0.f;
        rc = count_build ? timed_rebuild(L, &bms) : rebuild(L);
        if (rc) break;
        float ms = time_sample(c, (int)n, reps, s, e0, e1);
        if (ms < 0.f) { rc = G3D_ERR_CUDA; break; }
        if (ms + bms < best_ms) { best_ms = ms + bms; best = c->cfg; }
      }
    if (!rc) {
      c->cfg = best;
      rc = rebuild(best.leaf_size);  // leave the sample's meshes at the chosen size
    }
  }
  c->cfg = best;
  c->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  if (!rc && chosen) *chosen = best;
  return rc;
}

int64_t g3d_mlp_num_params(void) { return kNumParams; }

int g3d_mlp_create(g3d_ctx* c, g3d_mlp** out) {
  if (!c || !out) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  g3d_mlp* p = new g3d_mlp();
  int rc = G3D_OK;
  for (float** b : {&p->params, &p->grads, &p->m, &p->v})
    if (!rc) rc = cuda_err(cudaMalloc(b, sizeof(float) * kNumParams));
  if (!rc) rc = cuda_err(cudaMalloc(&p->loss, 64));
  for (float* b : {p->params, p->grads, p->m, p->v})
    if (!rc && b) rc = cuda_err(cudaMemset(b, 0, sizeof(float) * kNumParams));
  if (rc) { g3d_mlp_destroy(c, p); return rc; }
  *out = p;
  return G3D_OK;
}

int g3d_mlp_destroy(g3d_ctx* c, g3d_mlp* p) {
  if (!c || !p) return G3D_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->proposal == p) c->proposal = nullptr;
  for (void* b : {(void*)p->params, (void*)p->grads, (void*)p->m, (void*)p->v, (void*)p->loss})
    if (b) cudaFree(b);
  if (p->ws) cudaFree(p->ws);
  if (p->wt16) cudaFree(p->wt16);
  if (p->act16) cudaFree(p->act16);
  delete p;
  return G3D_OK;
}

int g3d_mlp_set_params(g3d_ctx* c, g3d_mlp* p, const float* params) {
  if (!c || !p || !params) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaMemcpy(p->params, params, sizeof(float) * kNumParams, cudaMemcpyDefault));
  CK(cudaMemset(p->m, 0, sizeof(float) * kNumParams));
  CK(cudaMemset(p->v, 0, sizeof(float) * kNumParams));
  p->t = 0;
  p->version++;
  return G3D_OK;
}

int g3d_mlp_get_params(g3d_ctx* c, g3d_mlp* p, float* params) {
  if (!c || !p || !params) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(params, p->params, sizeof(float) * kNumParams, cudaMemcpyDefault));
  return G3D_OK;
}

// Checkpoint file: 8-byte magic, int64 parameter count, int64 Adam step
// count, then the float32 parameters and Adam's first and second moments
// (training resumes exactly).  Files with the parameters only (magic
// ...01, no step count) load with Adam reset.
static const char kMlpMagic1[8] = {'G', '3', 'D', 'M', 'L', 'P', '0', '1'};
static const char kMlpMagic2[8] = {'G', '3', 'D', 'M', 'L', 'P', '0', '2'};

int g3d_mlp_save(g3d_ctx* c, g3d_mlp* p, const char* path) {
  if (!c || !p || !path) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaDeviceSynchronize());
  std::vector<float> h(3 * (size_t)kNumParams);
  CK(cudaMemcpy(h.data(), p->params, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(h.data() + kNumParams, p->m, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(h.data() + 2 * kNumParams, p->v, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return G3D_ERR_IO;
  const int64_t n = kNumParams, t = p->t;
  bool ok = fwrite(kMlpMagic2, 1, 8, f) == 8 && fwrite(&n, sizeof(n), 1, f) == 1 &&
            fwrite(&t, sizeof(t), 1, f) == 1 && fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? G3D_OK : G3D_ERR_IO;
}

int g3d_mlp_load(g3d_ctx* c, g3d_mlp* p, const char* path) {
  if (!c || !p || !path) return G3D_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return G3D_ERR_IO;
  char magic[8];
  int64_t n = 0, t = 0;
  int rc = G3D_OK;
  bool full = false;
  if (fread(magic, 1, 8, f) != 8 || fread(&n, sizeof(n), 1, f) != 1) rc = G3D_ERR_IO;
  else if (n != kNumParams) rc = G3D_ERR_INVALID_ARG;
  else if (memcmp(magic, kMlpMagic2, 8) == 0) full = true;
  else if (memcmp(magic, kMlpMagic1, 8) != 0) rc = G3D_ERR_INVALID_ARG;
  if (!rc && full && (fread(&t, sizeof(t), 1, f) != 1 || t < 0)) rc = G3D_ERR_IO;
  std::vector<float> h((full ? 3 : 1) * (size_t)kNumParams);
  if (!rc && fread(h.data(), sizeof(float), h.size(), f) != h.size()) rc = G3D_ERR_IO;
  if (!rc && fgetc(f) != EOF) rc = G3D_ERR_INVALID_ARG;  // trailing bytes: not this format
  fclose(f);
  if (rc) return rc;
  rc = g3d_mlp_set_params(c, p, h.data());  // also resets Adam
  if (rc || !full) return rc;
  CK(cudaMemcpy(p->m, h.data() + kNumParams, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->v, h.data() + 2 * kNumParams, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
  p->t = t;
  return G3D_OK;
}

int g3d_mlp_forward(g3d_ctx* c, g3d_mlp* p, const float* X, int64_t B, float* logits, void* stream) {
  if (!c || !p || !X || !logits || B <= 0 || B > (1 << 24)) return G3D_ERR_INVALID_ARG;
  if (!is_device_ptr(X) || !is_device_ptr(logits)) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  return mlp_forward(c, p, X, (int)B, logits, (cudaStream_t)stream);
}

int g3d_mlp_gradients(g3d_ctx* c, g3d_mlp* p, const float* X, const int32_t* labels, int64_t B, float* grads_out,
                      float* loss_out, void* stream) {
  if (!c || !p || !X || !labels || B <= 0 || B > (1 << 24)) return G3D_ERR_INVALID_ARG;
  if (!is_device_ptr(X) || !is_device_ptr(labels)) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  int rc = mlp_backward(c, p, X, labels, (int)B, s);
  if (rc) return rc;
  if (grads_out) CK(cudaMemcpyAsync(grads_out, p->grads, sizeof(float) * kNumParams, cudaMemcpyDefault, s));
  if (loss_out) CK(cudaMemcpyAsync(loss_out, p->loss, sizeof(float), cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return G3D_OK;
}

int g3d_mlp_train_step(g3d_ctx* c, g3d_mlp* p, const float* X, const int32_t* labels, int64_t B, float lr,
                       float* loss_out, void* stream) {
  if (!c || !p || !X || !labels || B <= 0 || B > (1 << 24) || !(lr > 0.f)) return G3D_ERR_INVALID_ARG;
  if (!is_device_ptr(X) || !is_device_ptr(labels)) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  int rc = mlp_backward(c, p, X, labels, (int)B, s);
  if (rc) return rc;
  p->t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)p->t), c2 = 1.f - powf(b2, (float)p->t);
  G3D_LAUNCH(c, "k_adam", k_adam, grid_for(kNumParams, 256, 1 << 30), 256, 0, s, p->params, p->grads, p->m, p->v,
             kNumParams, lr, b1, b2, 1e-8f, c1, c2);
  p->version++;
  if (loss_out) CK(cudaMemcpyAsync(loss_out, p->loss, sizeof(float), cudaMemcpyDefault, s));
  return cuda_err(cudaGetLastError());
}

int g3d_mlp_train(g3d_ctx* c, g3d_mlp* p, const float* X, const int32_t* labels, int64_t n, int64_t steps,
                  int32_t batch, float lr, uint64_t seed, float* loss_out, void* stream) {
  NvtxRange nvtx_range("g3d_mlp_train");
  if (!c || !p || !X || !labels || n <= 0 || steps < 0 || batch <= 0 || batch > (1 << 16) || !(lr > 0.f))
    return G3D_ERR_INVALID_ARG;
  if (!is_device_ptr(X) || !is_device_ptr(labels)) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  float* Xb = nullptr;
  CK(cudaMallocAsync((void**)&Xb, sizeof(float) * (size_t)batch * kFeatIn + sizeof(int) * (size_t)batch + 16, s));
  int* Yb = (int*)(Xb + (size_t)batch * kFeatIn);
  int rc = G3D_OK;
  for (int64_t t = 0; t < steps && !rc; t++) {
    G3D_LAUNCH(c, "k_sample_batch", k_sample_batch, (unsigned int)batch, 256, 0, s, X, labels, (long long)n,
               (unsigned long long)seed, (long long)t, Xb, Yb);
    rc = g3d_mlp_train_step(c, p, Xb, Yb, batch, lr, (t + 1 == steps) ? loss_out : nullptr, stream);
  }
  cudaFreeAsync(Xb, s);
  return rc ? rc : cuda_err(cudaGetLastError());
}

int g3d_pair_features(g3d_ctx* c, const g3d_query* q, int64_t n, float* X, void* stream) {
  if (!c || !q || n <= 0 || !X || !is_device_ptr(X)) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<QueryDev> hq;
  int rc = build_queries_v(c, q, n, hq);
  if (rc) return rc;
  rc = ensure_cstats(c, q, n, s);
  if (rc) return rc;
  QueryDev* dq = nullptr;
  CK(cudaMallocAsync((void**)&dq, sizeof(QueryDev) * n, s));
  CK(cudaMemcpyAsync(dq, hq.data(), sizeof(QueryDev) * n, cudaMemcpyHostToDevice, s));
  PairFeatArgs pf{dq, X, nullptr};
  G3D_LAUNCH(c, "k_pair_features", k_pair_features, (unsigned int)n, 128, 0, s, pf);
  afree(dq, s);
  return cuda_err(cudaGetLastError());
}

int g3d_level_trace(g3d_ctx* c, uint64_t* out, int cap, int* n_out, void* stream) {
  if (!c || !n_out || cap < 0 || (cap > 0 && !out)) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  const FrontierArgs& f = c->fr;
  unsigned int next = 0;
  CK(cudaMemcpy(&next, f.trace_next, 4, cudaMemcpyDeviceToHost));
  std::vector<unsigned long long> ring(6 * (size_t)f.trace_cap);
  CK(cudaMemcpy(ring.data(), f.trace, 48 * (size_t)f.trace_cap, cudaMemcpyDeviceToHost));
  const unsigned int have = std::min(next, (unsigned int)f.trace_cap);
  const int n = std::min((int)have, cap);
  for (int i = 0; i < n; i++) {  // the n most recent entries, oldest first
    const unsigned int slot = (next - (unsigned int)n + (unsigned int)i) & (unsigned int)(f.trace_cap - 1);
    for (int k = 0; k < 6; k++) out[6 * i + k] = ring[6 * (size_t)slot + k];
  }
  *n_out = n;
  return G3D_OK;
}

int g3d_proposal_topk(g3d_ctx* c, const float* logits, int64_t B, int32_t N, int32_t k, int32_t* out,
                      void* stream) {
  if (!c || !logits || !out || B <= 0 || B > (1ll << 31) - 1 || N < 1 || N > (1 << 24) || k < 1 || k > 8 ||
      k > N || !is_device_ptr(logits) || !is_device_ptr(out))
    return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  G3D_LAUNCH(c, "k_topk", k_topk, (unsigned int)B, 256, 0, (cudaStream_t)stream, logits, N, k, (int*)out);
  return cuda_err(cudaGetLastError());
}

int g3d_set_proposal(g3d_ctx* c, g3d_mlp* p) {
  if (!c) return G3D_ERR_INVALID_ARG;
  c->proposal = p;
  return G3D_OK;
}

int g3d_sync(g3d_ctx* c, void* stream) {
  if (!c) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  int h[2];
  CK(cudaMemcpy(&h[0], c->queue.error, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&h[1], c->d_sticky, 4, cudaMemcpyDeviceToHost));
  int rc = h[0] ? h[0] : h[1];
  if (h[0]) {  // the queue state is unknown after a device-side failure
    G3D_LAUNCH(c, "k_queue_init", k_queue_init, 256, 256, 0, s, c->queue);
  }
  if (h[1]) CK(cudaMemsetAsync(c->d_sticky, 0, 4, s));
  CK(cudaStreamSynchronize(s));
  return rc;
}

int g3d_stats_get(g3d_ctx* c, g3d_stats* out, void* stream) {
  if (!c || !out) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned long long h[ST_COUNT];
  CK(cudaMemcpy(h, c->stats, sizeof(h), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->node_pairs = h[ST_NODE_PAIRS];
  out->leaf_pairs = h[ST_LEAF_PAIRS];
  out->tri_prefilter = h[ST_TRI_PREFILTER];
  out->tri_tests = h[ST_TRI_TESTS];
  out->candidates = h[ST_CANDIDATES];
  out->fp64_tests = h[ST_FP64_TESTS];
  out->exact_tests = h[ST_EXACT_TESTS];
  out->exact_orients = h[ST_EXACT_ORIENTS];
  out->queue_pushes = h[ST_QUEUE_PUSHES];
  out->second_passes = h[ST_SECOND_PASSES];
  out->frontier_blocks = (uint64_t)c->fr.nblocks;
  out->seed_excess_ppm = h[ST_SEED_EXCESS];
  out->seed_queries = h[ST_SEED_QUERIES];
  out->distinct_nodes = h[ST_DISTINCT_NODES];
  out->distinct_faces = h[ST_DISTINCT_FACES];
  out->levels = h[ST_LEVELS];
  out->launches = c->launches;
  out->warp_busy_ns = h[ST_BUSY_NS];
  out->warp_idle_ns = h[ST_IDLE_NS];
  return G3D_OK;
}

int g3d_profile_begin(g3d_ctx* c, const char* filter) {
  if (!c) return G3D_ERR_INVALID_ARG;
  c->prof_filter = filter ? filter : "";
  c->prof_on = true;
  return G3D_OK;
}

int g3d_profile_end(g3d_ctx* c, g3d_kernel_time* out, int cap, int* n_out) {
  if (!c || (!out && cap > 0) || !n_out) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  c->prof_on = false;
  CK(cudaDeviceSynchronize());
  std::map<std::string, std::pair<unsigned long long, std::pair<double, double>>> agg;
  for (auto& r : c->prof) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    auto& e = agg[r.name];
    e.first++;
    e.second.first += ms;
    if (ms > e.second.second) e.second.second = ms;
    c->ev_pool.push_back(r.e0);
    c->ev_pool.push_back(r.e1);
  }
  c->prof.clear();
  int n = 0;
  for (auto& kv : agg) {
    if (n < cap) {
      memset(&out[n], 0, sizeof(out[n]));
      strncpy(out[n].name, kv.first.c_str(), sizeof(out[n].name) - 1);
      out[n].launches = kv.second.first;
      out[n].total_ms = kv.second.second.first;
      out[n].max_ms = kv.second.second.second;
    }
    n++;
  }
  *n_out = n < cap ? n : cap;
  return cuda_err(cudaGetLastError());
}

int g3d_debug_words(g3d_ctx* c, int* out8) {
  if (!c || !out8) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out8, c->d_dbg, 32, cudaMemcpyDeviceToHost));
  return G3D_OK;
}

int g3d_stats_reset(g3d_ctx* c, void* stream) {
  if (!c) return G3D_ERR_INVALID_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaMemsetAsync(c->stats, 0, sizeof(unsigned long long) * ST_COUNT, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return G3D_OK;
}

}  // extern "C"
