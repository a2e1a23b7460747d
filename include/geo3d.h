/*
 * geo3d: exact 3D distance and 3D intersection between triangle meshes on
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Operators (arxiv 1808.09571):
 *  - 3D distance, Sec. 3.2.2: the minimum over all face pairs of the distance
 *    between the closed faces; the face-face distance is the minimum of the
 *    squared distance Q(u, v, t) of Eq. 3 extended to two parametric faces.
 *    It is 0 when the meshes share a point.
 *  - 3D intersection, Sec. 3.2.3 / Eq. 4: whether some pair of closed faces
 *    shares a point (segment cut with the face plane, then barycentric
 *    inclusion, decided exactly; touching counts).
 *  - Geometry model, Sec. 2.2 and Sec. 3.2.1: a TIN / polyhedral surface given
 *    as a set of triangles A_i; it is a surface, not a solid.
 *
 * Conventions for every entry point:
 *  - Return 0 (G3D_OK) or a negative G3D_ERR_* code.  Errors found on the
 *    device while work runs asynchronously (candidate overflow, timeout) are
 *    recorded in the context and returned by g3d_sync(); results of such a
 *    query are NaN (distance) or 0xFF (intersects).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; results are valid once it completes.
 *  - Pointers may be host or device memory unless stated otherwise; the
 *    library detects which.  The library owns every device copy it makes;
 *    the caller keeps ownership of its own buffers and may reuse them as soon
 *    as the call that reads them returns (host input) or the stream reaches
 *    the call (device input).
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef GEO3D_H
#define GEO3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define G3D_OK 0
#define G3D_ERR_INVALID_ARG (-1)   /* bad handle, pointer, size or flag       */
#define G3D_ERR_NAN_INPUT (-2)     /* a vertex coordinate is NaN or infinite  */
#define G3D_ERR_INDEX_OOB (-3)     /* a face index is >= the vertex count     */
#define G3D_ERR_EMPTY_MESH (-4)    /* zero faces                              */
#define G3D_ERR_OOM (-5)           /* device allocation failed                */
#define G3D_ERR_CAND_OVERFLOW (-6) /* candidate list overflowed twice         */
#define G3D_ERR_TIMEOUT (-7)       /* a device wait exceeded its time limit   */
#define G3D_ERR_CUDA (-8)          /* other CUDA runtime error                */
#define G3D_ERR_RANGE (-9)         /* |coordinate| > 2^60, or a nonzero f64   */
                                   /* coordinate below 2^-200                 */
#define G3D_ERR_NO_BVH (-10)       /* query on a mesh without a built BVH     */
#define G3D_ERR_TOO_LARGE (-11)    /* input exceeds a fixed-size scratch area */
#define G3D_ERR_IO (-12)           /* file could not be read or written */

#define G3D_F32 0
#define G3D_F64 1

#define G3D_OP_DISTANCE 0
#define G3D_OP_INTERSECTS 1

typedef struct g3d_ctx g3d_ctx;
typedef int64_t g3d_mesh; /* opaque handle, > 0 */

/* Tuning knobs; zero fields take the defaults given. */
typedef struct g3d_config {
  int32_t leaf_size;       /* faces per BVH leaf: 2, 4, 8 or 16 (default)   */
  int32_t warps_per_cta;   /* traversal warps per CTA (1-4), default 4      */
  int32_t ctas_per_sm;     /* traversal CTAs per SM, default 1; capped at   */
                           /* what one SM holds at once (registers, shared  */
                           /* memory), so every CTA of the launch is resident */
  int32_t stack_depth;     /* per-warp node-pair stack entries, default 256 */
  int32_t cand_capacity;   /* candidate pool entries shared by a launch, default 2^24 */
  int32_t queue_capacity;  /* global work queue entries (power of 2), 2^20  */
  int32_t time_limit_ms;   /* limit of every device-side wait and of each   */
                           /* traversal launch, default 30000               */
  int32_t isect_first;     /* distance queries: 1 (default) run an          */
                           /* intersects traversal before the distance one, */
                           /* 2 go straight to the distance traversal (it   */
                           /* decides intersecting face pairs itself); the  */
                           /* results are the same either way               */
  int32_t morton_bits;     /* Morton key bits per axis of the BVH build,    */
                           /* 8..10 (default 10): 8 sorts in 3 passes       */
                           /* instead of 4, a coarser order                 */
  int32_t traversal;       /* 1 (default): level-synchronous traversal (all */
                           /* queries of a launch descend one level of node */
                           /* pairs per grid-wide step); 2: persistent      */
                           /* per-warp depth-first traversal with a shared  */
                           /* work queue; the results are the same          */
  int32_t count_visits;    /* 1: batches also count the distinct BVH nodes  */
                           /* and faces each query reads (g3d_stats         */
                           /* distinct_nodes / distinct_faces; costs one    */
                           /* bit per node and leaf per query and an atomic */
                           /* per visit); 0 (default) off                   */
  int32_t frontier_capacity; /* node pairs per frontier of the level-       */
                           /* synchronous traversal (power of 2, >= 1024),  */
                           /* default 2^23 (512 MiB of lists); leaf lists   */
                           /* hold half; pairs that do not fit are finished */
                           /* by the persistent kernel (fixed at            */
                           /* g3d_create)                                   */
  int32_t dives;           /* greedy dives per query that seed the bound    */
                           /* (distance) or look for a first intersection   */
                           /* (intersects) before the traversal, 1..32,     */
                           /* default 16 (a query of small meshes gets      */
                           /* fewer); the results do not depend on it       */
  int32_t chunk_mfaces;    /* a level-synchronous batch whose queries       */
                           /* reference more than this many Mi (2^20) faces */
                           /* (both meshes of every query counted) runs as  */
                           /* consecutive chunks of at most that many,      */
                           /* 1..2^20, default 2048; the results are the    */
                           /* same                                          */
  int32_t proposal_min_faces; /* with a learned proposal (g3d_set_proposal): */
                           /* the queries whose two meshes both have at     */
                           /* least this many faces get the network's       */
                           /* proposals, the others only the greedy dives,  */
                           /* 1..2^30, default 8192; the results are the    */
                           /* same                                          */
  int32_t reserved;
} g3d_config;

/* One query of a batch. */
typedef struct g3d_query {
  g3d_mesh a, b;
  int32_t op;  /* G3D_OP_DISTANCE or G3D_OP_INTERSECTS */
  int32_t pad;
} g3d_query;

/* Device work counters, accumulated since g3d_create or g3d_stats_reset. */
typedef struct g3d_stats {
  uint64_t node_pairs;     /* node pairs expanded by the traversal          */
  uint64_t leaf_pairs;     /* leaf pairs whose faces were examined          */
  uint64_t tri_prefilter;  /* face pairs put through the box pre-filter     */
  uint64_t tri_tests;      /* face pairs put through the full FP32 test     */
  uint64_t candidates;     /* face pairs kept for the FP64 recomputation    */
  uint64_t fp64_tests;     /* FP64 face-pair distances computed             */
  uint64_t exact_tests;    /* face pairs decided by the FP64/exact test     */
  uint64_t exact_orients;  /* orientation signs taken in expansion arith.   */
  uint64_t queue_pushes;   /* items donated to the global work queue        */
  uint64_t second_passes;  /* queries re-run after a candidate overflow     */
  uint64_t launches;       /* kernels this context launched (host count)    */
  uint64_t warp_busy_ns;   /* traversal warp-time spent with work           */
  uint64_t warp_idle_ns;   /* traversal warp-time spent waiting for work    */
  uint64_t seed_excess_ppm;  /* sum over separated distance queries of     */
                             /* (bound after the dives / distance - 1) in  */
                             /* millionths: how tight the seeding was      */
  uint64_t seed_queries;     /* queries counted in seed_excess_ppm         */
  uint64_t distinct_nodes;   /* internal BVH nodes read, each counted once */
                             /* per query (with count_visits)              */
  uint64_t distinct_faces;   /* faces of the leaves tested, each counted   */
                             /* once per query (with count_visits)         */
  uint64_t levels;           /* grid-wide steps of level-synchronous       */
                             /* traversals                                 */
  uint64_t frontier_blocks;  /* blocks of the level-synchronous kernel's   */
                             /* cooperative grid (all the SMs hold at once;*/
                             /* fixed at g3d_create)                       */
} g3d_stats;

/* Accumulated CUDA-event time of one kernel while profiling. */
typedef struct g3d_kernel_time {
  char name[40];
  uint64_t launches;
  double total_ms;
  double max_ms;
} g3d_kernel_time;

/* Create a context on CUDA device `device`.  cfg may be NULL. */
int g3d_create(g3d_ctx **out, int device, const g3d_config *cfg);

/* Destroy a context, freeing every mesh and buffer it owns.  Synchronises
 * the device first. */
int g3d_destroy(g3d_ctx *ctx);

/* Load an indexed triangle mesh (Sec. 3.2.1: faces A_i with vertices
 * (u_i, v_i, w_i)).
 *   verts: nv x 3 coordinates, row-major, float (vdtype G3D_F32) or double
 *          (G3D_F64); host or device memory.
 *   idx:   nt x 3 uint32 vertex indices, row-major; host or device memory.
 *   copy_fp64_master: with G3D_F64 input, keep the double coordinates so the
 *          FP64 recomputation and the exact tests use them (results are then
 *          exact for the double input); ignored for G3D_F32.
 * Faces are stored as float32; double input is rounded to nearest and the
 * rounding is accounted for by the certified filters.  Validation (indices,
 * NaN/Inf, range) runs on the device; this call waits for it on `stream` and
 * returns its error.  *out receives a handle.  The BVH is built separately. */
int g3d_mesh_load(g3d_ctx *ctx, const void *verts, int vdtype, int64_t nv,
                  const uint32_t *idx, int64_t nt, int copy_fp64_master,
                  g3d_mesh *out, void *stream);

/* Load n meshes at once (arrays of the g3d_mesh_load arguments).  Device
 * sources (4-byte aligned) are copied by one kernel for the whole call, the
 * validation of all meshes is one kernel, and it is waited for once.  Host
 * sources cross to the device in stream order; a host array passed for
 * several meshes of the call (the same address and size, e.g. one index
 * array shared by copies of a tessellation) crosses once.  status_out (may
 * be NULL) receives each mesh's validation code; if any fails, none is kept,
 * out[] is zeroed and the first error is returned. */
int g3d_mesh_load_many(g3d_ctx *ctx, int64_t n, const void *const *verts, const int32_t *vdtype,
                       const int64_t *nv, const uint32_t *const *idx, const int64_t *nt,
                       int copy_fp64_master, g3d_mesh *out, int32_t *status_out, void *stream);

/* Build the BVHs of n distinct meshes (n <= 65535, at most 2^31 - 8192 faces
 * in total) together: every build kernel runs once over all their faces, and
 * the sort key carries the mesh index above the Morton code.  Asynchronous. */
int g3d_mesh_build_bvh_many(g3d_ctx *ctx, int64_t n, const g3d_mesh *meshes, void *stream);

/* Build the mesh's BVH on `stream`: Morton codes of face centroids over the
 * centroid box (48 bits), LSD radix sort, faces regrouped in that order into
 * leaves of leaf_size consecutive faces, binary radix tree over the leaves,
 * bottom-up box refit.  Asynchronous. */
int g3d_mesh_build_bvh(g3d_ctx *ctx, g3d_mesh m, void *stream);

/* Free a mesh (after the work using it has completed). */
int g3d_mesh_free(g3d_ctx *ctx, g3d_mesh m);

/* Free n meshes (one device synchronisation for all). */
int g3d_mesh_free_many(g3d_ctx *ctx, int64_t n, const g3d_mesh *meshes);
/* Stream-ordered release of meshes: the handles are invalid at once and the
 * device memory goes back in stream order on `stream`, after the work
 * already queued there (no device-wide synchronisation, so a pipeline can
 * keep copies and kernels of other steps in flight).  Work on other streams
 * that uses the meshes must be complete, or ordered before `stream`, when
 * this is called. */
int g3d_mesh_free_many_async(g3d_ctx *ctx, int64_t n, const g3d_mesh *meshes, void *stream);

/* Number of faces of a loaded mesh. */
int g3d_mesh_size(g3d_ctx *ctx, g3d_mesh m, int64_t *nt);
/* Host copies of a built mesh's BVH, for inspection and tests (synchronises
 * the device).  face_ids[nt]: input face id of each face in BVH (Morton)
 * order; leaves[nleaf][8]: box lo x, y, z, first face (int32 bits), box hi
 * x, y, z, face count (int32 bits); nodes[nleaf - 1][16]: per internal node
 * (node 0 is the root when nleaf > 1) its two children, each lo x, y, z,
 * child reference (int32 bits: >= 0 internal node, < 0 leaf ~ref), hi x, y,
 * z, leaves below (int32 bits).  Any output may be NULL; *nleaf_out (may be
 * NULL) gets the leaf count. */
int g3d_mesh_export(g3d_ctx *ctx, g3d_mesh mesh, int32_t *face_ids, float *leaves, float *nodes,
                    int64_t *nleaf_out);

/* 3D distance between meshes a and b (Sec. 3.2.2, Eq. 3): writes one
 * double to *out (host or device memory).  Asynchronous. */
int g3d_distance(g3d_ctx *ctx, g3d_mesh a, g3d_mesh b, double *out, void *stream);

/* 3D intersection of meshes a and b (Sec. 3.2.3, Eq. 4): writes 1 or 0 to
 * *out (host or device memory).  Asynchronous. */
int g3d_intersects(g3d_ctx *ctx, g3d_mesh a, g3d_mesh b, uint8_t *out, void *stream);

/* n independent queries evaluated together by one persistent traversal
 * (the whole-column evaluation of Sec. 3.1 applied to a list of pairs).
 * dist_out[i] is written for distance queries (NaN for intersects ones),
 * hit_out[i] for intersects queries (and 1 for a distance of 0); status_out
 * (may be NULL) receives 0 or a G3D_ERR_* code per query.  Output pointers
 * may be host or device memory.  Asynchronous. */
int g3d_batch(g3d_ctx *ctx, const g3d_query *q, int64_t n, double *dist_out,
              uint8_t *hit_out, int32_t *status_out, void *stream);

/* g3d_batch with, for distance queries, the witness of the result:
 * witness_out[i] = (a << 32) | b, a and b the input face ids (positions in
 * the index buffer given at load) of the face pair attaining the minimum,
 * the lowest (a, b) among ties; cluster_out[i] = cA * 64 + cB, the clusters
 * (see the learned proposal below) holding that pair, the label the
 * proposal is trained on.  Both -1 for intersects queries, intersecting
 * pairs and errors.  Either may be NULL; given, they must be device memory. */
int g3d_batch_ex(g3d_ctx *ctx, const g3d_query *q, int64_t n, double *dist_out, uint8_t *hit_out,
                 int32_t *status_out, int64_t *witness_out, int32_t *cluster_out, void *stream);

/* ---------------------------------------------------------------------------
 * Learned proposal.  Each mesh's faces, in BVH (Morton) order, are split into
 * 64 clusters (cluster c = faces [ceil(c nt / 64), ceil((c+1) nt / 64)));
 * per cluster the box, centroid and area-weighted normal are kept (computed
 * with the BVH).  A pair's 1536 features are those 2 x 64 x 12 numbers in
 * the frame of the pair's joint box (centre, half diagonal).  An MLP
 * 1536 -> 256 -> 256 -> 256 -> 4096 (ReLU) scores the 64 x 64 cluster pairs;
 * BF16 tensor-core GEMMs with FP32 accumulation (the forward pass on the
 * tcgen05 tensor cores), FP32 master weights, Adam.  With a proposal set, a
 * batch's queries whose two meshes both have at least 8,192 faces get the
 * network's 4 highest-scoring cluster pairs, and after the global dives 4
 * more greedy dives, dive d keeping to the leaves of proposed pair d mod 4:
 * a distance query starts its search from the certified upper bound found
 * there, an intersects query is done when a dive certifies an intersection.
 * Both are exact whatever the network predicts.
 * Parameter layout (FP32): W1 [1536 x 256], b1 [256], W2 [256 x 256], b2,
 * W3 [256 x 256], b3, W4 [256 x 4096], b4 [4096] (row-major, y = x W + b).
 * ------------------------------------------------------------------------- */
typedef struct g3d_mlp g3d_mlp;
int64_t g3d_mlp_num_params(void);
int g3d_mlp_create(g3d_ctx *ctx, g3d_mlp **out);            /* parameters zero */
int g3d_mlp_destroy(g3d_ctx *ctx, g3d_mlp *mlp);
/* copy g3d_mlp_num_params() floats in / out (host or device); set resets Adam */
int g3d_mlp_set_params(g3d_ctx *ctx, g3d_mlp *mlp, const float *params);
int g3d_mlp_get_params(g3d_ctx *ctx, g3d_mlp *mlp, float *params);
/* Checkpoints: the 8 bytes "G3DMLP02", the parameter count and Adam's step
 * count as int64, then the float32 parameters and Adam's first and second
 * moments (host byte order), so training resumes exactly.  Load also takes
 * parameter-only files ("G3DMLP01", count, parameters) and then resets Adam.
 * It checks the header and the length (G3D_ERR_INVALID_ARG when they do not
 * match, G3D_ERR_IO when the file cannot be read). */
int g3d_mlp_save(g3d_ctx *ctx, g3d_mlp *mlp, const char *path);
int g3d_mlp_load(g3d_ctx *ctx, g3d_mlp *mlp, const char *path);
/* logits [B x 4096] of features X [B x 1536]; both device memory */
int g3d_mlp_forward(g3d_ctx *ctx, g3d_mlp *mlp, const float *X, int64_t B, float *logits, void *stream);
/* gradients of the mean softmax cross-entropy over B rows with labels in
 * [0, 4096) (device); grads_out (g3d_mlp_num_params floats) and loss_out may
 * be host or device memory or NULL.  Synchronises the stream. */
int g3d_mlp_gradients(g3d_ctx *ctx, g3d_mlp *mlp, const float *X, const int32_t *labels, int64_t B,
                      float *grads_out, float *loss_out, void *stream);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on the same loss */
int g3d_mlp_train_step(g3d_ctx *ctx, g3d_mlp *mlp, const float *X, const int32_t *labels, int64_t B, float lr,
                       float *loss_out, void *stream);
/* `steps` Adam steps (as g3d_mlp_train_step) on minibatches of `batch` rows
 * drawn uniformly with replacement from X [n x 1536] / labels [n] (device
 * memory): row r of step t is row splitmix64(seed, t, r) mod n, so a run is
 * reproducible for a given seed.  loss_out (host or device, may be NULL)
 * gets the last step's loss.  Asynchronous on `stream`. */
int g3d_mlp_train(g3d_ctx *ctx, g3d_mlp *mlp, const float *X, const int32_t *labels, int64_t n, int64_t steps,
                  int32_t batch, float lr, uint64_t seed, float *loss_out, void *stream);
/* features [n x 1536] (device) of the pairs (a, b) of q (op ignored) */
int g3d_pair_features(g3d_ctx *ctx, const g3d_query *q, int64_t n, float *X, void *stream);
/* The proposal's selection: for each of the B rows of logits [B x N]
 * (device memory, row-major), the indices of its k largest values, largest
 * first, ties to the lowest index, into out [B x k] (device memory).
 * 1 <= k <= 8, 1 <= N <= 2^24.  This is the step that turns the network's
 * 64 x 64 cluster-pair logits into the cluster pairs the restricted dives
 * keep to (the paper has no learned component; the proposal only seeds the
 * certified bound).  Asynchronous on `stream`. */
int g3d_proposal_topk(g3d_ctx *ctx, const float *logits, int64_t B, int32_t N, int32_t k, int32_t *out,
                      void *stream);
/* use mlp (NULL = none) for the queries of this context's batches (see the
 * learned proposal above; the context does not own mlp) */
int g3d_set_proposal(g3d_ctx *ctx, g3d_mlp *mlp);

/* g3d_batch_ex with caller-supplied proposals: hint[i] = cA * 64 + cB names
 * the cluster pair (clusters as for the learned proposal above) that query i
 * searches first, or -1 for none; host or device memory of n int32.
 * A typical source is the cluster_out of an earlier call on the same meshes
 * (a moving object queried frame after frame).  The result is exact whatever
 * the hints; the context's learned proposal is not used by this call.  The
 * paper has no counterpart (it computes every face pair). */
int g3d_batch_hint(g3d_ctx *ctx, const g3d_query *q, int64_t n, const int32_t *hint, double *dist_out,
                   uint8_t *hit_out, int32_t *status_out, int64_t *witness_out, int32_t *cluster_out,
                   void *stream);

/* Volume of meshes (Sec. 3.2.1, Eq. 2): out[i] = 1/6 sum over the faces
 * (u, v, w) of mesh hs[i] of u . ((v - u) x (w - u)), the divergence
 * theorem on a closed mesh whose faces are counter-clockwise seen from
 * outside (clockwise faces give the negative volume; an open mesh gets the
 * formula's value, which depends on the origin).  Evaluated in FP64 from the
 * loaded vertices with compensated summation in a fixed order: the result
 * does not depend on scheduling.  No BVH is needed.  out: n doubles, host or
 * device memory.  Blocks until the result is written. */
int g3d_volume(g3d_ctx *ctx, g3d_mesh mesh, double *out, void *stream);
int g3d_volume_many(g3d_ctx *ctx, int64_t n, const g3d_mesh *meshes, double *out, void *stream);

/* Line segments and points against one polyhedral surface (Sec. 3.2.2:
 * line segment / polyhedral surface and point / polyhedral surface).
 * segs: n segments as float32 [n][6] = (P0, P1), host or device memory; a
 * point is a segment with P0 == P1.  Each segment is a closed set, the mesh
 * the union of its closed faces.  op = G3D_OP_DISTANCE: dist_out[i] = the
 * exact distance (0 when they meet; hit_out, if given, 1 when they meet);
 * op = G3D_OP_INTERSECTS: hit_out[i] = 1 when the segment meets a face
 * (dist_out, if given, NaN).  Outputs host or device memory; status_out (may
 * be NULL) gets 0 or G3D_ERR_NAN_INPUT / G3D_ERR_RANGE per segment (that
 * segment's outputs are then NaN / 0xff); without status_out the first such
 * error is also recorded for the next g3d_sync.  One GPU thread per segment walks
 * the mesh's BVH; asynchronous on `stream` (host outputs are valid after a
 * g3d_sync).  The mesh must have a BVH and stay loaded until the call ends. */
int g3d_segments(g3d_ctx *ctx, g3d_mesh mesh, const float *segs, int64_t n, int32_t op, double *dist_out,
                 uint8_t *hit_out, int32_t *status_out, void *stream);

/* Autotuner.  Runs the sample batch q[0..n) under each value of one launch
 * parameter at a time (coordinate search: isect_first, CTAs per SM, warps
 * per CTA, stack depth, in that order), timing `reps` runs (after one
 * untimed run) with CUDA events on `stream` and keeping the median-fastest
 * value before moving to the next parameter.  With G3D_TUNE_LEAF_SIZE the
 * sample's meshes are also rebuilt with leaf sizes 4, 8 and 16 and Morton
 * widths 8 and 10 bits per axis, and left built with the fastest; meshes built later use it too, other meshes keep theirs
 * (one batch may mix leaf sizes); with G3D_TUNE_COUNT_BUILD as well, each
 * leaf size is charged the wall time of rebuilding the sample's meshes on top
 * of the query time (for workloads that build as often as they query).  The
 * chosen values become the context's
 * configuration and are copied to *chosen (may be NULL).  No parameter
 * changes any result.  Plans created before a leaf-size rebuild must be
 * recreated.  Blocks until done.  The paper has no counterpart. */
#define G3D_TUNE_LEAF_SIZE 1
#define G3D_TUNE_COUNT_BUILD 2
int g3d_autotune(g3d_ctx *ctx, const g3d_query *q, int64_t n, int32_t flags, int32_t reps, g3d_config *chosen,
                 void *stream);

/* A prepared batch: the query list is uploaded once and the whole launch
 * sequence of g3d_batch (seed, traversal phases, finalisation, results) is
 * captured in a CUDA graph; each g3d_plan_launch replays it with one graph
 * launch.  dist_out and hit_out must be device memory (status_out device
 * memory or NULL); they are written on every replay.  The meshes must stay
 * loaded and unchanged while the plan is used; plans of one context must not
 * run concurrently (they share its work queue and candidate pool). */
typedef struct g3d_plan g3d_plan;
int g3d_plan_create(g3d_ctx *ctx, const g3d_query *q, int64_t n, double *dist_out, uint8_t *hit_out,
                    int32_t *status_out, g3d_plan **out, void *stream);
int g3d_plan_launch(g3d_ctx *ctx, g3d_plan *plan, void *stream);
int g3d_plan_destroy(g3d_ctx *ctx, g3d_plan *plan);

/* Wait for `stream` and return the first device-side error recorded since
 * the previous g3d_sync (0 if none), clearing it. */
int g3d_sync(g3d_ctx *ctx, void *stream);

/* Read / reset the device work counters (synchronises `stream`). */
int g3d_stats_get(g3d_ctx *ctx, g3d_stats *out, void *stream);
int g3d_stats_reset(g3d_ctx *ctx, void *stream);

/* Level trace of the level-synchronous traversal (diagnostics): the `cap`
 * (at most 1,024) most recent levels, oldest first, as 6 uint64 each into
 * out [cap x 6]: ns since that launch started, the level, its frontier node
 * pairs, its leaf pairs, and the ns block 0 spent on its share of the
 * expansion and until it finished its leaf tests; *n_out gets the entries
 * written.  Host memory.  Synchronises `stream`. */
int g3d_level_trace(g3d_ctx *ctx, uint64_t *out, int cap, int *n_out, void *stream);

/* Diagnostics: copies 8 ints describing the first invalid work item or
 * candidate any kernel of this context met and skipped (all zero if none):
 * {where (1 stack item, 2 leaf pair, 3 candidate), x, y, z, w, 0, 0, 0}.
 * Synchronises the device. */
int g3d_debug_words(g3d_ctx *ctx, int *out8);

/* Per-kernel timing: between g3d_profile_begin and g3d_profile_end every
 * kernel launch whose name contains `name_filter` (NULL or "" = all) is
 * bracketed by CUDA events on its own stream.  g3d_profile_end synchronises
 * the device and writes up to `cap` entries (one per kernel name) to `out`,
 * the count to *n_out. */
int g3d_profile_begin(g3d_ctx *ctx, const char *name_filter);
int g3d_profile_end(g3d_ctx *ctx, g3d_kernel_time *out, int cap, int *n_out);

/* Current configuration (after defaults). */
int g3d_get_config(g3d_ctx *ctx, g3d_config *out);
/* Change the configuration of a context (zero fields take their defaults).
 * cand_capacity and queue_capacity must be 0 or their current values; a new
 * leaf_size applies to meshes built afterwards (built meshes keep theirs).
 * Must not be called while work of the context is in flight. */
int g3d_set_config(g3d_ctx *ctx, const g3d_config *cfg);

/* Distance between two triangle soups with no device allocation at all.
 * The paper has no counterpart: this is for callers that cannot allocate
 * device memory, e.g. a host application whose device memory is owned by its
 * own allocator or budgeted up front (a database engine or a simulation that
 * loads this library as a plug-in), or a real-time pipeline that must not
 * call cudaMalloc once it runs (an allocation may synchronise the device and
 * take unbounded time).
 *   faces_a: na x 9 floats (x0 y0 z0 x1 y1 z1 x2 y2 z2 per face), faces_b:
 *            nb x 9 floats, out: one double, status_out: one int32 (required);
 *            all in memory the current device can read and write (its own
 *            device memory or managed memory), owned by the caller.
 *   Every face pair is tested (no BVH), so na * nb must not exceed 2^26;
 *   larger inputs are rejected with G3D_ERR_TOO_LARGE before any work.  Two
 *   passes over the face pairs: the first finds the smallest certified upper
 *   bound (or a certified intersection), the second recomputes in FP64, and
 *   decides exactly where needed, every pair whose certified lower bound does
 *   not exceed it; nothing is buffered, so no size of the surviving set
 *   fails.  *status_out receives 0, or G3D_ERR_NAN_INPUT / G3D_ERR_RANGE
 *   (a NaN / Inf coordinate, or |coordinate| > 2^60) with *out NaN.
 * Returns G3D_ERR_INVALID_ARG for a NULL pointer, a non-positive count or a
 * buffer the current device cannot access (another GPU's memory, host
 * memory), G3D_ERR_CUDA if a launch fails.
 * Same definitions and exactness as g3d_distance (0 if the soups intersect).
 * The working memory is one __device__ array of 256 bytes inside the library
 * (bound, flags, FP64 minimum), held on every GPU that loads the library
 * until the process exits.  The first call on a device looks up that array's
 * device address and the device's SM count (with that device current); make
 * that first call before any stream capture.  All calls share the array, and
 * each call clears it before use, so calls whose work overlaps on the GPU
 * (different streams, or different host threads) race and must be serialised
 * by the caller.  Asynchronous on `stream`.  No context is needed and none is
 * used. */
int g3d_distance_soup_noalloc(const float *faces_a, int64_t na, const float *faces_b, int64_t nb,
                              double *out, int32_t *status_out, void *stream);

/* Human-readable name of an error code. */
const char *g3d_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GEO3D_H */
