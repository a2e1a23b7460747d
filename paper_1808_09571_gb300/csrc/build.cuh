// Declarations of the ingest / BVH-build kernels (build.cu).
#pragma once
#include "internal.cuh"

namespace g3d {

enum { VAL_NAN = 1, VAL_RANGE = 2, VAL_OOB = 4 };

__global__ void k_validate_verts(const void* V, int dtype, long long n3, int* flags, unsigned int* rho_bits);
__global__ void k_validate_idx(const uint32_t* I, long long n3, long long nv, int* flags);
__global__ void k_centroid_bounds(const void* V, int dtype, const uint32_t* I, int nt, unsigned int* bounds);
__global__ void k_morton(const void* V, int dtype, const uint32_t* I, int nt, const unsigned int* bounds,
                         unsigned long long* keys, unsigned int* vals);
__global__ void k_sort_hist(const unsigned long long* keys, int n, int shift, unsigned int* hist, int ntiles);
__global__ void k_sort_scan_rows(unsigned int* hist, int ntiles, unsigned int* totals);
__global__ void k_sort_scatter(const unsigned long long* kin, const unsigned int* vin, unsigned long long* kout,
                               unsigned int* vout, int n, int shift, const unsigned int* hist,
                               const unsigned int* totals, int ntiles);
__global__ void k_gather_sorted(const void* V, int dtype, const uint32_t* I, int nt, const unsigned int* order,
                                float4* v0, float4* v1, float4* v2, double* m64);
__global__ void k_leaves(const float4* v0, const float4* v1, const float4* v2, int nt, int L, int nleaf,
                         const unsigned long long* skeys, float4* leaves, unsigned long long* lkeys);
__global__ void k_radix_tree(const unsigned long long* lk, int m, int* child, int* ccount, int* parent_node,
                             int* parent_leaf);
__global__ void k_check_tree(const int* child, int m, int* err);
__global__ void k_refit(const float4* leaves, int m, const int* child, const int* ccount, const int* parent_node,
                        const int* parent_leaf, int* visit, float4* nodes);

constexpr int kSortTile = 2048;

}  // namespace g3d
