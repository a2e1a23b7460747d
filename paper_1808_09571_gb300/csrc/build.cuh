// Declarations of the ingest / BVH-build kernels (build.cu).
#pragma once
#include "internal.cuh"

namespace g3d {

enum { VAL_NAN = 1, VAL_RANGE = 2, VAL_OOB = 4 };

#ifndef G3D_SORT_TILE
#define G3D_SORT_TILE 2048
#endif
constexpr int kSortTile = G3D_SORT_TILE;  // keys per radix-sort tile

constexpr int kBoundsChunk = 8192;   // faces per block of the bounds kernel

// One mesh of a batched build.
struct BuildMesh {
  const void* V;        // raw vertices (f32 or f64), device
  const uint32_t* I;    // raw indices, device
  int dtype;
  int nt;
  int L;                // faces per leaf
  int nleaf;
  float4 *v0, *v1, *v2; // outputs (faces in Morton order)
  double* m64;          // optional FP64 master output
  float4* nodes;
  float4* leaves;
  int2* nrange;         // [nleaf - 1] first / last leaf of each internal node
  const unsigned int* box;  // [6] ordered-int vertex box from the ingest
};

// Flattened view of a batched build: mesh i owns the face slots
// [face_off[i], face_off[i] + nt) (face_off is padded to multiples of 32, so a
// warp of the gather never straddles two meshes), leaves [leaf_off[i], ...), internal nodes
// [node_off[i], ...) of the shared scratch arrays, and bounds chunks
// [chunk_off[i], ...) of the bounds kernel's grid.
struct BuildArgs {
  const BuildMesh* m;
  int n;
  const long long* face_off;
  const long long* leaf_off;
  const long long* node_off;
  const long long* chunk_off;
  const long long* tile_off;  // [n+1] radix-sort tiles of each mesh
  unsigned int* bounds;  // [8 n] Morton quantisation per mesh: lo[3], pad, cells / extent[3], pad (float bits)
  unsigned int* keys0;   // [total_faces] 30-bit Morton keys
  unsigned int* vals0;   // [total_faces] face index within the mesh
  unsigned int* lkeys;   // [total_leaves] leaf keys (Morton of first face)
  int* child;                 // [2 total_nodes] local child refs
  int* ccount;                // [2 total_nodes] leaves below each child
  int* pnode;                 // [total_nodes] parent << 1 | slot (local)
  int* pleaf;                 // [total_leaves]
  int* visit;                 // [total_nodes] refit arrival counters
  long long total_faces, total_leaves, total_nodes;
  float cells;  // Morton cells per axis - 1 (2^bits - 1, bits = 8..10)
};

// Batched ingest: one item per array (vertices or indices) of a mesh.
enum { ING_F32 = 0, ING_F64 = 1, ING_IDX = 2 };
struct IngestItem {
  const char* src;     // device source (== dst when the copy engine already copied it)
  char* dst;           // the library's buffer
  long long n;         // elements (coordinates or indices)
  long long nv;        // vertices of the mesh (index bound)
  int kind;            // ING_*
  int vec;             // 1: src and dst start on 16-byte boundaries (16-byte loads and stores)
  int* flags;          // [2] of the mesh: error bits, rho bits (float)
  unsigned int* box;   // [6] of the mesh: ordered-int vertex box (vertex items)
};
constexpr long long kIngestChunk = 1 << 14;  // elements per block of k_ingest_many
__global__ void k_ingest_init(const IngestItem* items, int n);
__global__ void k_ingest_many(const IngestItem* items, const long long* chunk_off, int n);

__global__ void k_bounds_from_ingest(BuildArgs a);
__global__ void k_morton_tiles(BuildArgs a, unsigned int* hist);
__global__ void k_seg_hist(BuildArgs a, const unsigned int* keys, int shift, unsigned int* hist);
__global__ void k_seg_scan_rows(BuildArgs a, unsigned int* hist, unsigned int* totals);
__global__ void k_seg_scan_digits(BuildArgs a, unsigned int* totals);
__global__ void k_seg_scatter(BuildArgs a, const unsigned int* kin, const unsigned int* vin, unsigned int* kout,
                              unsigned int* vout, int shift, const unsigned int* hist, const unsigned int* dbase);
__global__ void k_gather_many(BuildArgs a, const unsigned int* skeys, const unsigned int* svals);
__global__ void k_radix_tree_many(BuildArgs a);
__global__ void k_check_tree_many(BuildArgs a, int* err);
__global__ void k_refit_many(BuildArgs a);

}  // namespace g3d
