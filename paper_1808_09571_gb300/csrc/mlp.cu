// Learned proposal: per-cluster mesh features and a small MLP (forward,
// softmax cross-entropy, backward, Adam) on BF16 tensor cores with FP32
// accumulation.  The network maps a mesh pair to logits over its 64 x 64
// cluster pairs; its top cluster pair only seeds the certified upper bound of
// the distance traversal, so results never depend on it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp.cuh"

namespace g3d {

// ---------------------------------------------------------------------------
// GEMM: C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]) (ReLU), with
// A(i,k) = A[i*as0 + k*as1], B(k,j) = B[k*bs0 + j*bs1] (any transposition),
// FP32 operands rounded to BF16 on their way into shared memory, FP32
// accumulation in mma.sync.m16n8k16 tiles.  Block tile 64 x 64 x 32, 4 warps
// of 32 x 32.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
  __shared__ __nv_bfloat16 As[GBM][GBK + GPAD];  // [m][k]
  __shared__ __nv_bfloat16 Bt[GBN][GBK + GPAD];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  const long long i0 = (long long)blockIdx.y * GBM, j0 = (long long)blockIdx.x * GBN;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 4; b++)
#pragma unroll
      for (int c = 0; c < 4; c++) acc[a][b][c] = 0.f;

  for (int k0 = 0; k0 < g.K; k0 += GBK) {
    for (int e = tid; e < GBM * GBK; e += 128) {
      const int r = e / GBK, k = e % GBK;
      const long long gi = i0 + r, gk = k0 + k;
      float v = (gi < g.M && gk < g.K) ? g.A[gi * g.as0 + gk * g.as1] : 0.f;
      As[r][k] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < GBN * GBK; e += 128) {
      const int n = e / GBK, k = e % GBK;
      const long long gj = j0 + n, gk = k0 + k;
      float v = (gj < g.N && gk < g.K) ? g.B[gk * g.bs0 + gj * g.bs1] : 0.f;
      Bt[n][k] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; mi++) {
        const int r = wm + mi * 16 + gid;
        af[mi][0] = pack_bf16(As[r][kk + 2 * tig], As[r][kk + 2 * tig + 1]);
        af[mi][1] = pack_bf16(As[r + 8][kk + 2 * tig], As[r + 8][kk + 2 * tig + 1]);
        af[mi][2] = pack_bf16(As[r][kk + 2 * tig + 8], As[r][kk + 2 * tig + 9]);
        af[mi][3] = pack_bf16(As[r + 8][kk + 2 * tig + 8], As[r + 8][kk + 2 * tig + 9]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ni++) {
        const int n = wn + ni * 8 + gid;
        bf[ni][0] = pack_bf16(Bt[n][kk + 2 * tig], Bt[n][kk + 2 * tig + 1]);
        bf[ni][1] = pack_bf16(Bt[n][kk + 2 * tig + 8], Bt[n][kk + 2 * tig + 9]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++) mma_bf16(acc[mi][ni], af[mi], bf[ni]);
    }
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int mi = 0; mi < 2; mi++)
#pragma unroll
    for (int ni = 0; ni < 4; ni++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const long long gi = i0 + wm + mi * 16 + gid + 8 * h;
#pragma unroll
        for (int c = 0; c < 2; c++) {
          const long long gj = j0 + wn + ni * 8 + 2 * tig + c;
          if (gi < g.M && gj < g.N) {
            float v = acc[mi][ni][2 * h + c];
            if (g.bias) v += g.bias[gj];
            if (g.relu) v = fmaxf(v, 0.f);
            g.C[gi * g.ldc + gj] = v;
          }
        }
      }
}

// ---------------------------------------------------------------------------
// elementwise / reductions of the training step
// ---------------------------------------------------------------------------
// dpre = dpost * (post > 0)
__global__ void k_relu_bwd(float* __restrict__ d, const float* __restrict__ post, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && !(post[i] > 0.f)) d[i] = 0.f;
}

// db[j] = sum_i dY[i][j]
__global__ void k_colsum(const float* __restrict__ dY, int M, int N, float* __restrict__ db) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int i = 0; i < M; i++) s += dY[(long long)i * N + j];
  db[j] = s;
}

// one block per row: softmax of the logits, loss -log p[label], gradient
// (p - onehot) / B written in place of the logits
__global__ void __launch_bounds__(256) k_softmax_ce(float* __restrict__ logits, const int* __restrict__ labels,
                                                    int N, int B, float* __restrict__ loss) {
  __shared__ float red[8];
  __shared__ float s_max, s_sum;
  float* z = logits + (long long)blockIdx.x * N;
  const int tid = threadIdx.x;
  float m = -INFINITY;
  for (int j = tid; j < N; j += blockDim.x) m = fmaxf(m, z[j]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  if (tid == 0) {
    float v = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) v = fmaxf(v, red[w]);
    s_max = v;
  }
  __syncthreads();
  float s = 0.f;
  for (int j = tid; j < N; j += blockDim.x) s += expf(z[j] - s_max);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[w];
    s_sum = v;
  }
  __syncthreads();
  const int lab = labels[blockIdx.x];
  const bool ok = lab >= 0 && lab < N;  // a label out of range is ignored (zero gradient row)
  if (tid == 0 && loss && ok) atomicAdd(loss, (logf(s_sum) + s_max - z[lab]) / (float)B);
  __syncthreads();
  const float inv = 1.f / s_sum;
  for (int j = tid; j < N; j += blockDim.x) {
    float p = expf(z[j] - s_max) * inv;
    z[j] = ok ? (p - (j == lab ? 1.f : 0.f)) / (float)B : 0.f;
  }
}

// One minibatch drawn uniformly with replacement from n rows: row r of the
// batch is row splitmix64(seed, step, r) mod n of (X, labels).  One block per
// batch row.  (splitmix64: Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", 2014.)
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

__global__ void k_sample_batch(const float* __restrict__ X, const int* __restrict__ labels, long long n,
                               unsigned long long seed, long long step, float* __restrict__ Xb,
                               int* __restrict__ Yb) {
  const int r = blockIdx.x;
  const unsigned long long h = splitmix64(seed ^ splitmix64((unsigned long long)step * 0x100000001b3ull + r));
  const long long src = (long long)(h % (unsigned long long)n);
  for (int k = threadIdx.x; k < kFeatIn; k += blockDim.x) Xb[(long long)r * kFeatIn + k] = X[src * kFeatIn + k];
  if (threadIdx.x == 0) Yb[r] = labels[src];
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// one block per row: the k largest logits (ties: lowest index), k <= 8
__global__ void __launch_bounds__(256) k_topk(const float* __restrict__ logits, int N, int k,
                                              int* __restrict__ out) {
  __shared__ float sv[8];
  __shared__ int si[8];
  __shared__ int chosen[8];
  const float* z = logits + (long long)blockIdx.x * N;
  const int tid = threadIdx.x;
  for (int r = 0; r < k; r++) {
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int j = tid; j < N; j += blockDim.x) {
      bool taken = false;
      for (int q = 0; q < r; q++) taken |= chosen[q] == j;
      float x = z[j];
      if (!taken && (x > bv || (x == bv && j < bi))) { bv = x; bi = j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { sv[tid >> 5] = bv; si[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      float v = sv[0];
      int ix = si[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); w++)
        if (sv[w] > v || (sv[w] == v && si[w] < ix)) { v = sv[w]; ix = si[w]; }
      chosen[r] = ix;
      out[(long long)blockIdx.x * k + r] = ix;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// cluster statistics and pair features
// ---------------------------------------------------------------------------
// one block per (mesh, cluster): faces f with f * 64 / nt == c, i.e.
// [ceil(c nt / 64), ceil((c+1) nt / 64)); box, centroid sum, area-weighted
// normal sum, area, count
__global__ void __launch_bounds__(128) k_cluster_stats(const ClusterMesh* __restrict__ ms, int n) {
  __shared__ float red[16][4];
  const int m = blockIdx.x / kClusters, c = blockIdx.x % kClusters;
  if (m >= n) return;
  const ClusterMesh M = ms[m];
  const long long f0 = ((long long)c * M.nt + kClusters - 1) / kClusters;
  const long long f1 = ((long long)(c + 1) * M.nt + kClusters - 1) / kClusters;
  float v[14] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long f = f0 + threadIdx.x; f < f1; f += blockDim.x) {
    float4 a = M.v0[f], b = M.v1[f], d = M.v2[f];
    v[0] = fminf(v[0], fminf(a.x, fminf(b.x, d.x)));
    v[1] = fminf(v[1], fminf(a.y, fminf(b.y, d.y)));
    v[2] = fminf(v[2], fminf(a.z, fminf(b.z, d.z)));
    v[3] = fmaxf(v[3], fmaxf(a.x, fmaxf(b.x, d.x)));
    v[4] = fmaxf(v[4], fmaxf(a.y, fmaxf(b.y, d.y)));
    v[5] = fmaxf(v[5], fmaxf(a.z, fmaxf(b.z, d.z)));
    v[6] += (a.x + b.x + d.x) * (1.f / 3.f);
    v[7] += (a.y + b.y + d.y) * (1.f / 3.f);
    v[8] += (a.z + b.z + d.z) * (1.f / 3.f);
    const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
    const float fx = d.x - a.x, fy = d.y - a.y, fz = d.z - a.z;
    const float nx = ey * fz - ez * fy, ny = ez * fx - ex * fz, nz = ex * fy - ey * fx;
    v[9] += 0.5f * nx;
    v[10] += 0.5f * ny;
    v[11] += 0.5f * nz;
    v[12] += 0.5f * sqrtf(nx * nx + ny * ny + nz * nz);
    v[13] += 1.f;
  }
  for (int k = 0; k < 14; k++)
    for (int o = 16; o > 0; o >>= 1) {
      float u = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = k < 3 ? fminf(v[k], u) : (k < 6 ? fmaxf(v[k], u) : v[k] + u);
    }
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 14; k++) red[k][threadIdx.x >> 5] = v[k];
  __syncthreads();
  if (threadIdx.x < 14) {
    const int k = threadIdx.x;
    float r = red[k][0];
    for (int w = 1; w < 4; w++) r = k < 3 ? fminf(r, red[k][w]) : (k < 6 ? fmaxf(r, red[k][w]) : r + red[k][w]);
    M.out[c * kClusterStride + k] = r;
  }
}

// one block per feature row (the query a.rows names, or query r): the
// 2 x 64 x 12 features of the pair, in the frame
// centred on the joint box of both meshes and scaled by its half diagonal;
// empty clusters are zero
__global__ void __launch_bounds__(128) k_pair_features(const PairFeatArgs a) {
  static_assert(2 * kClusters == 128, "one thread per cluster of the pair");
  __shared__ float red[6][4];
  __shared__ float ctr[3], inv_s;
  const int q = a.rows ? a.rows[blockIdx.x] : blockIdx.x;
  const float* SA = a.q[q].A.cstats;
  const float* SB = a.q[q].B.cstats;
  {  // joint box of the non-empty clusters: thread e reads cluster e
    const int e = threadIdx.x;
    const float* t = (e < kClusters ? SA : SB) + (e % kClusters) * kClusterStride;
    const bool use = t[13] != 0.f;
    float v[6];
    for (int k = 0; k < 3; k++) {
      v[k] = use ? t[k] : INFINITY;
      v[3 + k] = use ? t[3 + k] : -INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1)
      for (int k = 0; k < 6; k++) {
        const float u = __shfl_xor_sync(0xffffffffu, v[k], o);
        v[k] = k < 3 ? fminf(v[k], u) : fmaxf(v[k], u);
      }
    if ((threadIdx.x & 31) == 0)
      for (int k = 0; k < 6; k++) red[k][threadIdx.x >> 5] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
      float d2 = 0.f;
      for (int k = 0; k < 3; k++) {
        float lo = red[k][0], hi = red[3 + k][0];
        for (int w = 1; w < 4; w++) { lo = fminf(lo, red[k][w]); hi = fmaxf(hi, red[3 + k][w]); }
        ctr[k] = 0.5f * (lo + hi);
        d2 += (hi - lo) * (hi - lo);
      }
      const float sc = 0.5f * sqrtf(d2);
      inv_s = sc > 0.f ? 1.f / sc : 1.f;
    }
  }
  __syncthreads();
  float* X = a.X + (long long)blockIdx.x * kFeatIn;
  for (int e = threadIdx.x; e < 2 * kClusters; e += blockDim.x) {
    const float* t = (e < kClusters ? SA : SB) + (e % kClusters) * kClusterStride;
    float* o = X + e * kFeatPerCluster;
    const float cnt = t[13];
    if (cnt == 0.f) {
      for (int k = 0; k < kFeatPerCluster; k++) o[k] = 0.f;
      continue;
    }
    for (int k = 0; k < 3; k++) {
      o[k] = (t[k] - ctr[k]) * inv_s;
      o[3 + k] = (t[3 + k] - ctr[k]) * inv_s;
      o[6 + k] = (t[6 + k] / cnt - ctr[k]) * inv_s;
    }
    const float area = t[12];
    for (int k = 0; k < 3; k++) o[9 + k] = area > 0.f ? t[9 + k] / area : 0.f;
  }
}

}  // namespace g3d
