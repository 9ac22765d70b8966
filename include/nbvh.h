/*
 * nbvh.h - C ABI of the B300 (sm_103a) neural ray query library.
 *
 * Implements the neural ray query of N-BVH (Weier et al., "N-BVH: Neural ray
 * queries with bounding volume hierarchies", SIGGRAPH 2024) and its training
 * step. The paper states the problem as: given geometric elements and their
 * bounding box, train a neural model that answers intersection queries for
 * rays crossing the box (Sec. 4); a shallow BVH of hollow leaf boxes supplies
 * the ray-box intervals in which the model is probed (Sec. 3, Sec. 5), and a
 * neural query returns the same intersection record as a classical one
 * (Sec. 7).
 *
 * Conventions (all entry points):
 *  - Every buffer is owned by the caller. Device buffers are plain device
 *    pointers; host buffers are plain host pointers. The library allocates no
 *    memory: scratch space is a caller-provided workspace whose size the
 *    matching *_workspace_size call returns.
 *  - Device work is enqueued on the caller's stream (a cudaStream_t passed as
 *    void*; NULL = the legacy default stream) and the call returns without
 *    synchronising, except where a function says otherwise.
 *  - Every call returns an nbvh_status. Arguments are validated on the host
 *    before any launch; an invalid argument launches nothing. No exception and
 *    no process exit crosses this ABI.
 *  - Conditions found on the device (segment-list overflow, a wait that gave
 *    up) are recorded in a per-process device status word, read and cleared by
 *    nbvh_get_device_status. Kernels never trap.
 *  - Directions need not be unit length; t is measured in units of |d|.
 *
 * Precision: slab tests, clipping, sample positions, trilinear weights and
 * depth reconstruction are FP32. Hash-table entries are stored in
 * FP32/FP16/BF16. The MLP runs either on CUDA cores in FP32
 * (mlp_prec = NBVH_FP32) or on the tensor cores (tcgen05) with FP16/BF16
 * operands and FP32 accumulation (mlp_prec = NBVH_FP16 / NBVH_BF16).
 */
#ifndef NBVH_H_
#define NBVH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NBVH_MAX_LEVELS 32
#define NBVH_MAX_SAMPLES 64
#define NBVH_MAX_INPUTS 2048   /* n_samples * n_levels * n_features (queries; training: see nbvh_train_workspace_size) */

typedef enum {
  NBVH_OK = 0,
  NBVH_ERR_INVALID_ARG = 1,           /* null pointer, negative size, out-of-range field */
  NBVH_ERR_CUDA = 2,                  /* a CUDA runtime call failed (launch, copy, attribute) */
  NBVH_ERR_OOM = 3,                   /* reserved: the library itself never allocates */
  NBVH_ERR_WORKSPACE_TOO_SMALL = 4,   /* ws_bytes below the *_workspace_size result */
  NBVH_ERR_SEGMENT_OVERFLOW = 5,      /* device: a ray crossed more than max_segs leaves */
  NBVH_ERR_TIMEOUT = 6,               /* device: a bounded wait gave up */
  NBVH_ERR_UNSUPPORTED = 7            /* valid but not implemented for this shape/precision */
} nbvh_status;

typedef enum { NBVH_FP32 = 0, NBVH_FP16 = 1, NBVH_BF16 = 2 } nbvh_precision;

/* Neural model shape (Sec. 4 Fig. 3: samples along the ray-box interval,
 * multi-resolution hash-grid features concatenated in ray order, MLP decoder;
 * Sec. 6 "Neural model & training": ReLU hidden layers).
 * Level l has resolution N_l = floor(base_res * growth^l); it is indexed
 * densely while (N_l+1)^3 <= 2^log2_table and through the spatial hash
 * otherwise (nbvh_level_layout). Grid coordinates of a point p are
 * xhat = (p - frame_centre) / frame_extent + 1/2, clamped to [0,1]^3. */
typedef struct {
  int32_t n_levels;      /* L, 1..NBVH_MAX_LEVELS */
  int32_t n_features;    /* F per level: 1, 2, 4 or 8 */
  int32_t log2_table;    /* log2 of the hashed-level table size T, 4..26 */
  int32_t base_res;      /* N_min >= 1 */
  float growth;          /* b >= 1 */
  int32_t n_samples;     /* N samples per segment, 1..NBVH_MAX_SAMPLES */
  int32_t n_hidden;      /* hidden layers, 1..8 */
  int32_t width;         /* hidden width: 16, 32, 64 or 128 */
  int32_t n_out;         /* outputs: 5 = hit logit, depth logit, normal xyz;
                            8 = the same plus albedo logits rgb (5..8 accepted) */
  nbvh_precision table_prec;  /* storage type of the hash-table entries */
  nbvh_precision mlp_prec;    /* FP32: CUDA-core MLP; FP16/BF16: tensor-core MLP */
  float frame_centre[3];
  float frame_extent;
  int32_t flags;         /* NBVH_FLAG_*; 0 = the default query */
} nbvh_model_desc;

/* Query option (the paper's Sec. 6 text on depth from within a node,
 * commented out in its source): a ray whose origin lies inside a leaf box
 * (the box's entry t is below tmin) queries that leaf over its whole chord
 * with the samples concatenated in reverse order, from the exit point back
 * towards the entry, as a ray entering the box at its exit would see it. The
 * predicted hit is t = exit - sigmoid(o_d) (exit - entry) and counts only if
 * tmin < t <= tmax. Such a segment is listed with its endpoints swapped
 * (t0 = exit > t1 = entry) and ordered by its entry. */
#define NBVH_FLAG_REVERSE_INSIDE 1

/* Rays, device structure-of-arrays, n entries each. */
typedef struct {
  const float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
  int64_t n;
} nbvh_rays;

/* Query result per ray, device structure-of-arrays. Rays without a predicted
 * hit get hit = 0, t = +inf, leaf = -1, normal = 0, albedo 0. The albedo
 * arrays are optional (all three NULL, or all three set): the hit's albedo,
 * sigmoid of outputs 5-7 for a model with n_out = 8 (Sec. 5.2, auxiliary
 * intersection data), the triangle's albedo for a triangle BLAS that has one,
 * else 0. */
typedef struct {
  uint8_t *hit;
  float *t, *nx, *ny, *nz;
  int32_t *leaf;
  float *ar, *ag, *ab;
} nbvh_hits;

/* One N-BVH node, 64 bytes: the boxes of both children (lo xyz, hi xyz) and
 * their indices; child >= 0 is an internal node, child < 0 is leaf ~child.
 * Node 0 is the root. A tree of L leaves has max(1, L-1) nodes. */
typedef struct {
  float lo0[3], hi0[3];
  float lo1[3], hi1[3];
  int32_t child0, child1;
  int32_t pad[2];
} nbvh_node;

/* Scene frame derived from the triangles (host output of the leaf build). */
typedef struct {
  float lo[3], hi[3];        /* triangles' AABB */
  float centre[3];           /* (lo + hi)/2 rounded to float */
  float extent;              /* largest AABB side */
  float sphere_radius;       /* 1.01 * half diagonal (training chords) */
} nbvh_scene_info;

const char* nbvh_status_string(nbvh_status s);

/* Library version and the compute capability it was built for (1030). */
int32_t nbvh_version(void);
int32_t nbvh_built_arch(void);

/* Host. Per-level resolution, density flag, entry count and entry offset of
 * the hash table described by desc (Sec. 3, Sec. 6). Arrays hold
 * NBVH_MAX_LEVELS entries; *total = sum of sizes. Pure host computation. */
nbvh_status nbvh_level_layout(const nbvh_model_desc* desc, int32_t* res, int32_t* dense,
                              int64_t* size, int64_t* offset, int64_t* total);

/* Host. Number of float parameters of the MLP: per layer W [out][in] row-major
 * then b [out], layers in order input -> hidden ... -> output. */
nbvh_status nbvh_mlp_param_count(const nbvh_model_desc* desc, int64_t* count);

/* Host. S0 leaf build (Sec. 5: leaves are hollow boxes over geometric
 * clusters; Sec. 6: nodes are inflated slightly). Median split over triangle
 * centroids: the leaf with the most triangles (ties: lowest node id) splits
 * on the axis of largest centroid extent (ties x<y<z), sorting by centroid
 * then triangle index, the first floor(n/2) going left, until n_leaves exist.
 * Leaves are numbered left to right; leaf i owns
 * tri_perm[leaf_range[2i] .. leaf_range[2i+1]) in ascending triangle order.
 * Leaf boxes are the triangles' AABB pushed out by inflate_rel * extent on
 * every face, rounded outward to float.
 *   tris        host, [n_tris][3][3] float (vertex-major xyz)
 *   nodes       host, node_cap entries (>= max(1, n_leaves-1)); *out_n_nodes set
 *   tri_perm    host, n_tris int32; leaf_range host, 2*n_leaves int32
 *   leaf_box    host, [n_leaves][6] float (lo xyz, hi xyz)
 *   info        host, scene frame
 * Errors: INVALID_ARG for n_leaves outside [1, n_tris] or node_cap too small. */
nbvh_status nbvh_build_leaves(const float* tris, int64_t n_tris, int32_t n_leaves, double inflate_rel,
                              nbvh_node* nodes, int32_t node_cap, int32_t* out_n_nodes,
                              int32_t* tri_perm, int32_t* leaf_range, float* leaf_box,
                              nbvh_scene_info* info);

/* Device. S1 traversal + slab test + clip (Sec. 3: probe only inside ray-box
 * intervals; Sec. 5: traverse the N-BVH and query each leaf reached).
 * For every ray, every leaf whose box gives a non-empty clip
 * [max(entry, tmin), min(exit, tmax)] (t0 <= t1 kept), sorted by (t0, leaf).
 * Output is slot-major: entry s of ray r at [s * n + r], s < seg_count[r].
 * A ray with more than max_segs segments keeps its first max_segs, and the
 * device status records NBVH_ERR_SEGMENT_OVERFLOW.
 *   nodes: device, n_nodes nbvh_node; outputs: device int32/float arrays. */
nbvh_status nbvh_traverse(const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays, int32_t max_segs,
                          int32_t* seg_count, int32_t* seg_leaf, float* seg_t0, float* seg_t1,
                          void* stream);

/* Device. S2+S3 (Sec. 4 "Sampling & reconstruction quality", Fig. 3):
 * features of n_seg segments (ray index seg_ray[i], interval [t0[i], t1[i]]):
 * N stratum-midpoint samples t_k = t0 + (k+1/2)/N (t1-t0), each encoded on
 * every level by trilinear interpolation of the 8 vertices' entries; written
 * FP32 to feat[i * K + k*L*F + l*F + f], K = N*L*F. table: device, layout of
 * nbvh_level_layout, type desc->table_prec. */
nbvh_status nbvh_encode(const nbvh_model_desc* desc, const void* table, nbvh_rays rays,
                        const int32_t* seg_ray, const float* t0, const float* t1, int64_t n_seg,
                        float* feat, void* stream);

/* Evaluation options of a query (S6; Sec. 5: the number of neural queries
 * per ray equals the leaves met before an intersection, so rays need uneven
 * amounts of work). Every choice gives the same hit records; they only change
 * how the work is scheduled and shaped on the GPU. Passed per call (NULL =
 * nbvh_query_options_default); the library keeps no schedule state.
 *  schedule         NBVH_SCHEDULE_WAVES: one launch per segment slot w
 *                   evaluates slot w of every ray still active (compacted
 *                   queue per wave). NBVH_SCHEDULE_PERSISTENT (FP16/BF16 only;
 *                   the FP32 form always runs waves): one launch whose CTAs
 *                   claim tiles of up to 128 (ray, segment) items from a queue
 *                   that each resolve refills with the ray's next segment, so
 *                   rays with many segments leave no wave tail per slot. A
 *                   queue wait that gives up (about a second) records
 *                   NBVH_ERR_TIMEOUT.
 *  patience_cycles  persistent schedule: SM cycles a CTA waits for a full
 *                   tile before it takes fewer items (0 .. 2^40).
 *  traverse_block   threads per traversal CTA: 64, 128 or 256.
 *  eval_threads     FP16/BF16 evaluation CTA: 256 (two CTAs per SM, hidden
 *                   width <= 64), 512 (one CTA per SM), 0 = automatic (512).
 *  w1_mode          FP16/BF16 evaluation: where the first layer's weights
 *                   live. Both forms convert them once per call into a 16-bit
 *                   image in the workspace. NBVH_W1_RESIDENT: each CTA copies
 *                   the whole image into shared memory at its start;
 *                   NBVH_W1_STREAMED: streamed through two shared-memory
 *                   buffers, 128 inputs at a time, by bulk copies;
 *                   NBVH_W1_AUTO: resident when the layer's image is at
 *                   most 64 KB (N * L * F <= 512 at width 64), else streamed:
 *                   resident weights take their size out of the SM's
 *                   unified L1 / shared memory, which the gather uses (128 KB
 *                   resident made the mixed scene 11 % slower; 64 KB resident
 *                   made the queries 1-5 % faster). The training forward
 *                   keeps them resident whenever they fit.
 *  eval_pipeline    persistent FP16/BF16 schedule: NBVH_PIPELINE_PHASES runs
 *                   each tile in CTA-wide phases (all warps gather, then the
 *                   MLP, resolve and claim); NBVH_PIPELINE_WARP_SPECIALISED
 *                   gives four warps the claims, MMAs, epilogues and resolves
 *                   and twelve the gather, handing work over through
 *                   mbarriers, so the next tile is gathered while the last
 *                   one is finished (hidden width 32 or 64, first layer
 *                   resident, L * F a multiple of 16; else UNSUPPORTED);
 *                   NBVH_PIPELINE_AUTO: the phase kernel (the faster one on
 *                   the displaced-icosphere workload; the autotuner times
 *                   both).
 *  wait_spins       persistent schedule: polling rounds (each with a short
 *                   sleep) before a queue wait gives up and records
 *                   NBVH_ERR_TIMEOUT; 0 = the default (about a second).
 *  test_phantom_items  test hook, 0 otherwise: the persistent queue announces
 *                   this many extra items (0 .. 1024) that nothing ever
 *                   writes, so the waits for them run out; the query then
 *                   returns with NBVH_ERR_TIMEOUT in the device status (it
 *                   never traps or spins unbounded) and the records of the
 *                   rays are not defined.
 *  segments_out     statistics, nullptr = none: device int64 array to which
 *                   the call adds, on its stream and without synchronising,
 *                   the segments it evaluated (nbvh_query_rays: entry 0;
 *                   nbvh_hybrid_trace: entry i for neural instance i). One
 *                   extra one-block launch per evaluation.
 *  instance_streams nbvh_hybrid_trace: 1 = the neural instances one after
 *                   another in index order, each merged into the record;
 *                   0 or >= 2 = evaluated concurrently on the library's two
 *                   side streams (forked from and joined back into the
 *                   caller's stream, also under graph capture), each into its
 *                   own staging record, then merged per ray in instance order
 *                   (the same record bit for bit); the persistent
 *                   evaluations' idle CTAs then leave early so that the
 *                   other stream's kernels get their SMs. nbvh_query_rays
 *                   ignores it.
 *  partial_items    persistent schedule: the most queued items a partial
 *                   tile claims (1 .. 128; 0 = the default, 16). The tile's
 *                   other rows evaluate those rays' next segments
 *                   (lookahead), so with a shallow queue several CTAs share
 *                   it and each ray advances up to 128 / items segments per
 *                   tile. Results do not depend on it. The concurrent hybrid
 *                   form defaults to 128 (beside the other stream's kernels,
 *                   smaller partial tiles measured slower). A query whose
 *                   traversal queues fewer than 128 items per evaluation CTA
 *                   spreads them over all CTAs at once: each claim takes at
 *                   most max(32, queued / CTAs) items, the tile's other rows
 *                   holding lookahead segments. */
#define NBVH_SCHEDULE_WAVES 0
#define NBVH_SCHEDULE_PERSISTENT 1
#define NBVH_W1_AUTO 0
#define NBVH_W1_RESIDENT 1
#define NBVH_W1_STREAMED 2
#define NBVH_PIPELINE_AUTO 0
#define NBVH_PIPELINE_PHASES 1
#define NBVH_PIPELINE_WARP_SPECIALISED 2
typedef struct {
  int32_t schedule;
  int64_t patience_cycles;
  int32_t traverse_block;
  int32_t eval_threads;
  int32_t w1_mode;
  int32_t eval_pipeline;
  int64_t wait_spins;
  int32_t test_phantom_items;
  int64_t* segments_out;
  int32_t instance_streams;
  int32_t partial_items;
} nbvh_query_options;

/* Host. The defaults: persistent schedule, patience 4000 cycles, traversal
 * CTAs of 128 threads, automatic evaluation CTA shape and weight placement. */
nbvh_status nbvh_query_options_default(nbvh_query_options* opt);

/* Host. The query evaluation's launch plan for desc under opt (NULL = the
 * defaults): threads per CTA, whether the first layer's weights are streamed
 * (1) or resident (0), dynamic shared memory bytes and TMEM columns per CTA
 * (0 for the FP32 form, whose CTAs use no TMEM; for it *threads is the CTA
 * size and *w1_streamed says whether the first layer is taken in chunks), and
 * the pipeline (NBVH_PIPELINE_PHASES or NBVH_PIPELINE_WARP_SPECIALISED).
 * NBVH_ERR_UNSUPPORTED when the kernels cannot run this combination. */
nbvh_status nbvh_eval_plan(const nbvh_model_desc* desc, const nbvh_query_options* opt, int32_t* threads,
                           int32_t* w1_streamed, int32_t* smem_bytes, int32_t* tmem_cols, int32_t* pipeline);

/* Host. Workspace bytes of nbvh_eval_segments for desc (the streamed
 * first-layer image of the FP16/BF16 form; may be 0). */
nbvh_status nbvh_eval_workspace_size(const nbvh_model_desc* desc, size_t* bytes);

/* Device. S2..S4 fused: raw MLP outputs out[i * n_out + j] of n_seg segments
 * (as nbvh_encode), through the MLP selected by desc->mlp_prec. mlp: device
 * float parameters (nbvh_mlp_param_count). The FP32 form uses CUDA cores;
 * the FP16/BF16 form uses tcgen05 tensor-core MMAs with FP32 accumulation.
 * Both take the first layer in chunks of inputs, so every descriptor up to
 * NBVH_MAX_INPUTS inputs runs. opt: NULL or the evaluation shape (schedule,
 * patience and traverse_block are ignored). workspace: device, 256-byte
 * aligned, >= nbvh_eval_workspace_size bytes (NULL when that is 0). */
nbvh_status nbvh_eval_segments(const nbvh_model_desc* desc, const void* table, const float* mlp,
                               nbvh_rays rays, const int32_t* seg_ray, const float* t0,
                               const float* t1, int64_t n_seg, float* out, const nbvh_query_options* opt,
                               void* workspace, size_t ws_bytes, void* stream);

/* Host. Workspace bytes of nbvh_query_rays for n_rays rays and at most
 * max_segs segments per ray. */
nbvh_status nbvh_query_workspace_size(const nbvh_model_desc* desc, int64_t n_rays, int32_t max_segs,
                                      size_t* bytes);

/* Device. The neural ray query, S1..S5 (Sec. 5: the number of neural
 * queries per ray equals the leaves met before an intersection is found).
 * nbvh_query_rays runs with nbvh_query_options_default; nbvh_query_rays_opt
 * takes the options (NULL = the defaults).
 * Traversal lists each ray's segments in (t0, leaf) order; each ray's
 * segments are then evaluated in that order, keeping the closest predicted
 * hit (hit iff hit logit > 0; t = t0 + sigmoid(depth)(t1 - t0); normal =
 * normalised normal head) and dropping the ray once its next segment starts
 * at or beyond its best t. The result equals the closest predicted hit over
 * all segments, ties to the earlier segment. The evaluation runs as waves
 * (one launch per segment slot) or, for FP16/BF16, as one persistent launch
 * (nbvh_query_options).
 * workspace: device, >= nbvh_query_workspace_size bytes, 256-byte aligned.
 * A descriptor or option the kernels cannot run returns NBVH_ERR_UNSUPPORTED
 * before anything is enqueued. */
nbvh_status nbvh_query_rays(const nbvh_model_desc* desc, const void* table, const float* mlp,
                            const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays, int32_t max_segs,
                            nbvh_hits out, void* workspace, size_t ws_bytes, void* stream);
nbvh_status nbvh_query_rays_opt(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays, int32_t max_segs,
                                nbvh_hits out, void* workspace, size_t ws_bytes, const nbvh_query_options* opt,
                                void* stream);

/* Writable rays, device structure-of-arrays, n entries each. */
typedef struct {
  float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
  int64_t n;
} nbvh_rays_out;

/* Device. One secondary bounce per ray (Sec. 7: at the intersection a neural
 * query returns, the path tracer samples the next direction). For a hit:
 * origin o + t d + 1e-4 n' with n' the predicted normal turned to face -d;
 * direction cosine-weighted about n' from Philox4x32-10 keyed by seed (low,
 * high word) with counter (ray low word, ray high word, 0, 2):
 * r = sqrt(u1), phi = 2 pi u2, u = top 24 bits * 2^-24, in the orthonormal
 * basis of Duff et al. (JCGT 2017); tmin 0, tmax +inf. A miss gets the primary
 * ray with the empty interval tmin 0, tmax -1 (no segments).
 * rays, hits: device inputs of n entries; out: device outputs, out.n == rays.n. */
nbvh_status nbvh_bounce_rays(nbvh_rays rays, nbvh_hits hits, uint64_t seed, nbvh_rays_out out, void* stream);

/* One configuration of the query and its median time. */
typedef struct {
  nbvh_query_options opt;
  float ms;                  /* median of the timed runs */
} nbvh_tune_result;

/* Device (synchronises). S6 autotuner: times nbvh_query_rays_opt on the
 * caller's own inputs under candidate options and returns the fastest in
 * *best (nothing is stored in the library). The search runs in stages, each
 * keeping the best so far: (1) waves, and for FP16/BF16 the persistent
 * schedule with patience 0, 1000, 4000, 16000 and 64000 cycles (automatic
 * pipeline and shape); (2) for FP16/BF16 the other evaluation pipeline and
 * the phase kernel's CTA shapes, 256 and 512 threads (256 only for width
 * <= 64) times resident and streamed first-layer weights, where the model
 * stages them; (3) from the fastest persistent phase-kernel candidate,
 * partial tiles of 4, 8, 32 and 128 items (16 is the default); (4)
 * traversal CTAs of 64, 128 and 256 threads. Each
 * candidate runs once untimed and reps times timed (CUDA events on the
 * stream, median). The first all_cap candidates with their times go to
 * all[], their count to *n_all. Every candidate gives the same hit records
 * (out holds the last run's). */
nbvh_status nbvh_autotune_query(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays, int32_t max_segs,
                                nbvh_hits out, void* workspace, size_t ws_bytes, int32_t reps,
                                nbvh_tune_result* best, nbvh_tune_result* all, int32_t all_cap, int32_t* n_all,
                                void* stream);

/* Device. Reads from a query workspace (after nbvh_query_rays on the same
 * stream) the number of segments evaluated and the number of evaluation
 * launches that had work (waves: one per segment slot; the persistent
 * schedule reports 1). Synchronises the stream. */
nbvh_status nbvh_query_stats(const void* workspace, int64_t n_rays, int32_t max_segs, int64_t* segments,
                             int32_t* waves, void* stream);

/* Host. Kernel-class timing: while enabled, every enqueueing call records a
 * CUDA event pair on the caller's stream around each group of launches of
 * one class (a query's traversal; its evaluation: image, queue set-up and the
 * persistent launch or every wave; a triangle trace; ...), except while the
 * stream is being captured into a graph. nbvh_get_kernel_times synchronises
 * on the events recorded since its previous call and returns, per class
 * (index NBVH_KERNEL_*, n_kinds entries, at most NBVH_KERNEL_KINDS used),
 * the summed milliseconds, the number of timed groups and the kernels they
 * launched (counted by this process, so exact when one host thread
 * enqueues). Timing adds two event records per group and no
 * synchronisation to the enqueueing calls. */
#define NBVH_KERNEL_TRAVERSE 0        /* S1 traversal */
#define NBVH_KERNEL_EVAL 1            /* S2..S5 query evaluation (encode + MLP + resolve) */
#define NBVH_KERNEL_TRI_TRACE 2       /* triangle BLAS closest hit */
#define NBVH_KERNEL_TLAS_CULL 3       /* hybrid top-level ray lists */
#define NBVH_KERNEL_BOUNCE 4          /* cosine-weighted bounce rays */
#define NBVH_KERNEL_TRAIN_RAYS 5      /* training rays, leaf selection and grouping */
#define NBVH_KERNEL_LABELS 6          /* brute-force ray-triangle labels */
#define NBVH_KERNEL_TRAIN_FORWARD 7   /* training forward and loss terms */
#define NBVH_KERNEL_TRAIN_BACKWARD 8  /* MLP adjoint + table-gradient scatter */
#define NBVH_KERNEL_WEIGHT_GRAD 9     /* MLP weight gradients */
#define NBVH_KERNEL_ADAM 10           /* gradient check, Adam, loss scale */
#define NBVH_KERNEL_OTHER 11          /* clears, loss reduction, statistics */
#define NBVH_KERNEL_KINDS 12
nbvh_status nbvh_set_timing(int32_t enable);
nbvh_status nbvh_get_kernel_times(double* ms, int64_t* sections, int64_t* launches, int32_t n_kinds);

/* Host. Number of kernels this library has launched in this process. */
int64_t nbvh_launch_count(void);

/* ------------------------------------------------------------------------
 * Training (S7, S8): Sec. 4 "Encoding, inference & training", Sec. 5.2
 * (ray distribution, visibility / distance / normal losses, combined loss),
 * Sec. 6 "Neural model & training" (batches of rays, Adam, lr 1e-2).
 * ------------------------------------------------------------------------ */

typedef enum {
  NBVH_TRAIN_PROBED_MIX = 0, /* even rays: leaf chosen uniformly, point uniform in its box, uniform
                                direction, origin on the bounding sphere, trains that leaf; odd rays:
                                bounding-sphere chords, train the first leaf met */
  NBVH_TRAIN_PAPER = 1       /* origin uniform in the 50%-inflated scene box, uniform direction,
                                trains the first leaf met (Sec. 4, Sec. 5.2) */
} nbvh_train_mode;

/* Device geometry the training step reads. */
typedef struct {
  const nbvh_node* nodes;
  int32_t n_nodes;
  const float* leaf_box;     /* device [n_leaves][6] lo xyz, hi xyz */
  int32_t n_leaves;
  const float* tris;         /* device [n_tris][9] */
  const int32_t* tri_perm;   /* device, as nbvh_build_leaves */
  const int32_t* leaf_range; /* device [n_leaves][2] */
  const float* leaf_tris;    /* optional device [n_tris][9]: the triangles in tri_perm order (each
                                leaf's triangles contiguous); the labels read them when set */
  nbvh_scene_info info;      /* by value */
  const float* tri_albedo;   /* optional device [n_tris][3] RGB in [0, 1] by triangle index, NULL = none */
} nbvh_train_scene;

/* Training labels, device structure-of-arrays. The albedo arrays are optional
 * (all three NULL or all three set); the loss uses them with n_out = 8. */
typedef struct {
  uint8_t* hit;
  float *depth, *nx, *ny, *nz;
  float *ar, *ag, *ab;
} nbvh_labels;

/* Device. S7 rays of one training step. Randomness: Philox4x32-10 keyed by
 * seed (low, high word), counter (ray, step low, step high, block 0 or 1);
 * uniforms are the top 24 bits times 2^-24; a uniform direction is
 * z = 1 - 2u, phi = 2 pi u'. Probed rays: leaf = floor(u32 * n_leaves / 2^32)
 * of the first word, point = lo + u (hi - lo), origin moved back along -d to
 * the bounding sphere (centre = scene centre, radius = info.sphere_radius).
 * Output: rays (tmin 0; tmax +inf, or the chord length), the trained leaf
 * (-1: the ray meets no leaf and does not train), its segment [t0, t1], and
 * *n_valid (device) incremented by the number of training rays. */
nbvh_status nbvh_train_rays(int32_t mode, uint64_t seed, int64_t step, const nbvh_train_scene* scene,
                            nbvh_rays_out rays, int32_t* leaf, float* t0, float* t1, int32_t* n_valid,
                            void* stream);

/* Device. S7 labels: closest Moller-Trumbore intersection (edges inclusive,
 * det == 0 a miss) among the trained leaf's own triangles with t in
 * [t0, t1]; hit, local depth (t - t0)/(t1 - t0), geometric normal turned to
 * face -d; with scene->tri_albedo and out.ar set, the hit triangle's albedo
 * (0 on a miss). Rays with leaf < 0 get hit 0. */
nbvh_status nbvh_train_labels(nbvh_rays rays, const int32_t* leaf, const float* t0, const float* t1,
                              const nbvh_train_scene* scene, nbvh_labels out, void* stream);

/* Host. Workspace of nbvh_forward_train / nbvh_backward / nbvh_train_step for
 * batches of n rays that stores the whole batch's activations; n_leaves = the
 * scene's leaf count for nbvh_train_step (its rays are grouped by leaf), 0 for
 * forward/backward only.
 * Recompute mode: a workspace smaller than this (but at least the budget
 * call's minimum) holds the per-ray outputs of the whole batch and the
 * activations of one chunk of rays only. The forward then runs chunk by chunk
 * keeping the raw outputs, dL/d(raw) and loss terms, and the backward runs each
 * chunk's forward again to rebuild its activations before differentiating it
 * (the same gradients up to FP32 summation order). The calls choose the mode
 * from ws_bytes, so a forward and its backward must get the same ws_bytes.
 * Training supports N * L * F up to 2048 at width 64 in FP16/BF16 (the
 * forward chunks the first layer as the query does; the backward copies W0^T
 * 128 features at a time when it does not fit shared memory whole). The FP32
 * training kernels stage the first layer whole, which caps N * L * F at
 * about 550 at width 64. Larger models return NBVH_ERR_UNSUPPORTED before
 * anything is enqueued. */
nbvh_status nbvh_train_workspace_size(const nbvh_model_desc* desc, int64_t n, int32_t n_leaves, size_t* bytes);

/* Host. Memory budget of a training workspace: *bytes = the stored-mode size
 * when it is at most max_bytes (*chunk = n), else the recompute-mode size of
 * the largest activation chunk (a multiple of 128 rays, *chunk) that fits.
 * NBVH_ERR_WORKSPACE_TOO_SMALL when not even a 128-ray chunk fits. */
nbvh_status nbvh_train_workspace_budget(const nbvh_model_desc* desc, int64_t n, int32_t n_leaves, size_t max_bytes,
                                        size_t* bytes, int64_t* chunk);

/* Device. Forward of n training segments (segment i belongs to ray i and to
 * leaf[i]; leaf < 0 does not train) storing the activations in the workspace.
 * raw_out: device [n][n_out] raw MLP outputs. With labels (labels.hit != NULL)
 * it also evaluates the combined loss L = mean over training segments of
 * 2 BCE(sigmoid(o_hit), y) + y (2 |sigmoid(o_d) - d| + (1/3) sum_j |o_nj - n_j|)
 * (Sec. 5.2), plus, for n_out = 8 with albedo labels, the relative L2 term
 * y (1/3) sum_c (s_c - a_c)^2 / (s_c^2 + 0.01), s_c = sigmoid(o_{5+c}), the
 * denominator held constant; keeps dL/d(raw) times the loss scale for nbvh_backward, and
 * writes L to *loss_out (device, may be NULL): an FP32 sum of the per-segment
 * terms, compensated per thread and pairwise across threads, without atomics.
 * n_valid: device count of training segments (nbvh_train_rays). The loss
 * scale is *loss_scale_dev when that is not NULL, else loss_scale. */
nbvh_status nbvh_forward_train(const nbvh_model_desc* desc, const void* table, const float* mlp,
                               nbvh_rays rays, const int32_t* leaf, const float* t0, const float* t1,
                               nbvh_labels labels, const int32_t* n_valid, float loss_scale,
                               const float* loss_scale_dev, float* raw_out, float* loss_out, void* workspace,
                               size_t ws_bytes, void* stream);

/* Device. The loss of the last nbvh_forward_train on this workspace (n rays,
 * the same ws_bytes) summed with FP64 accumulation into *loss_out (device).
 * For finite-difference gradient checks only: central differences subtract
 * two nearly equal losses. */
nbvh_status nbvh_loss_fp64(const nbvh_model_desc* desc, int64_t n, const int32_t* n_valid, const void* workspace,
                           size_t ws_bytes, double* loss_out, void* stream);

/* Device. Backward of the last nbvh_forward_train on the same workspace:
 * from grad_out (device [n][n_out], dL/d(raw); NULL = the loss gradient the
 * forward kept) through the MLP into grad_mlp (FP32, parameter order of
 * nbvh_mlp_param_count) and through the encoding into grad_table (FP32,
 * [entries][F]): every (sample, level, corner) adds its trilinear weight times
 * dL/dfeature (Sec. 3, Sec. 4). Both gradients accumulate (callers zero them). */
nbvh_status nbvh_backward(const nbvh_model_desc* desc, const void* table, const float* mlp, nbvh_rays rays,
                          const int32_t* leaf, const float* t0, const float* t1, const float* grad_out,
                          float* grad_table, float* grad_mlp, void* workspace, size_t ws_bytes, void* stream);

/* Optimiser state, all device. The table is optimised in FP32 (table_master);
 * table_work is the copy the kernels read in desc->table_prec (NULL when
 * that is FP32 and the master is read directly). */
typedef struct {
  float* table_master;
  void* table_work;
  float *table_m, *table_v, *grad_table;
  float* mlp;
  float *mlp_m, *mlp_v, *grad_mlp;
  float* loss_scale;   /* device scalar */
  int32_t* counters;   /* device [4]: good steps, bad flag, applied flag, spare */
} nbvh_optim;

/* Device. Adam (bias-corrected; step counts from 1) on the FP32 masters with
 * the gradients divided by the loss scale, then the gradients are zeroed. A
 * step whose gradients are not all finite is skipped; with dynamic_scale the
 * scale halves on such a step and doubles after 2000 clean ones. */
nbvh_status nbvh_adam(const nbvh_model_desc* desc, const nbvh_optim* opt, int64_t step, float lr, float beta1,
                      float beta2, float eps, int32_t dynamic_scale, void* stream);

/* Device. One whole training step: rays (nbvh_train_rays), labels, forward
 * with loss, backward, Adam (lr, beta 0.9 / 0.999, eps 1e-8, Sec. 6). FP16 /
 * BF16 MLPs use dynamic loss scaling. *loss_out (device) receives the loss. */
nbvh_status nbvh_train_step(const nbvh_model_desc* desc, const nbvh_optim* opt, const nbvh_train_scene* scene,
                            int32_t mode, int64_t batch, uint64_t seed, int64_t step, float lr, float* loss_out,
                            void* workspace, size_t ws_bytes, void* stream);

/* Per-leaf statistics of training steps (Sec. 5.1 "Node error": a node's error
 * is its training loss q times the probability p that a training ray hits
 * it, p estimated by the fraction of training rays that hit it). Device
 * arrays of n_leaves entries that the steps accumulate into (callers zero
 * them): hits = rays whose first leaf (the leaf they would train) is the
 * leaf; trained = those that trained it; loss = the sum of their combined
 * loss terms (per-ray, before the mean over the batch; FP32, each step's
 * per-leaf sum compensated). */
typedef struct {
  uint32_t* hits;
  uint32_t* trained;
  float* loss;
} nbvh_leaf_stats;

/* Device. nbvh_train_step with error-driven ray selection (Sec. 5.2 "Ray
 * distribution": a ray trains the first leaf it meets only with that leaf's
 * probability). leaf_prob: device [n_leaves] probabilities in [0, 1] or NULL
 * (every ray trains); a ray with first leaf l trains iff u < leaf_prob[l],
 * u from Philox4x32-10 keyed by seed (low, high word) with counter
 * (ray, step-1 low, step-1 high, 3), top 24 bits * 2^-24. stats: host struct
 * of device arrays accumulated as nbvh_leaf_stats describes, or NULL. The
 * loss mean runs over the rays that train. */
nbvh_status nbvh_train_step_weighted(const nbvh_model_desc* desc, const nbvh_optim* opt,
                                     const nbvh_train_scene* scene, int32_t mode, int64_t batch, uint64_t seed,
                                     int64_t step, float lr, const float* leaf_prob, const nbvh_leaf_stats* stats,
                                     float* loss_out, void* workspace, size_t ws_bytes, void* stream);

/* Host. N-BVH from a cut through a base BVH (Sec. 5.1 "Base-BVH cut
 * optimization": the nodes along the cut become the N-BVH leaves, inflated
 * as in nbvh_build_leaves). base_nodes/base_leaf_range: a base BVH in the
 * format of nbvh_build_tri_blas (host). cut: n_cut base references, ref in
 * [0, n_base_nodes) = the subtree of that base node (0 = the whole tree),
 * ref < 0 = base leaf ~ref; every root-to-leaf path must cross exactly one.
 * Outputs (host): nodes (node_cap >= max(1, n_cut - 1)), *out_n_nodes;
 * leaf_range [n_cut][2] into the base BVH's triangle order; leaf_box
 * [n_cut][6], the reference's box pushed out by inflate_rel * extent and
 * rounded outward; leaf_ref [n_cut], the reference of each N-BVH leaf. Leaves
 * are numbered depth-first, first child first. Errors: INVALID_ARG for an
 * invalid base tree or cut. */
nbvh_status nbvh_build_cut(const nbvh_node* base_nodes, int32_t n_base_nodes, const int32_t* base_leaf_range,
                           int32_t n_base_leaves, const int32_t* cut, int32_t n_cut, double inflate_rel,
                           float extent, nbvh_node* nodes, int32_t node_cap, int32_t* out_n_nodes,
                           int32_t* leaf_range, float* leaf_box, int32_t* leaf_ref);

/* Host. Sec. 5.1 "Node error" for the leaves of a cut, from the per-leaf
 * statistics of training steps (nbvh_leaf_stats, copied to the host):
 * q = loss / trained, the leaf's mean training loss (a leaf hit but never
 * trained takes the mean q of the trained leaves, 1 if none trained);
 * p = hits / n_rays, the fraction of training rays that hit it; ranking
 * r = 2 ln q + ln p (-inf when hits = 0 or q <= 0, never split). Training
 * probability of Sec. 5.2, read as the ranking's linear-domain ratio:
 * prob = max(exp(r - r_max), 0.005) (0.005 for r = -inf), r_max the largest
 * finite r. All arrays host, n_leaves entries; q, p, r FP64 (host). */
nbvh_status nbvh_rank_leaves(const uint32_t* hits, const uint32_t* trained, const float* loss, int32_t n_leaves,
                             int64_t n_rays, double* q, double* p, double* r, float* prob);

/* Host. Sec. 5.1 split step: among the cut's references that are internal
 * base nodes (cut[i] >= 0) with a finite ranking r[i], the k_splits of
 * largest r (ties to the lower leaf index) are replaced by their base
 * children in place (first child first); the leaf order is kept otherwise.
 * new_prob: prob[i] for a kept leaf, 1 for a new child (no statistics yet).
 * base_nodes: the base BVH (nbvh_build_tri_blas format), host. new_cut,
 * new_prob: host, cap entries; *n_new = the new cut's length
 * (NBVH_ERR_WORKSPACE_TOO_SMALL if above cap). */
nbvh_status nbvh_refine_cut(const nbvh_node* base_nodes, int32_t n_base_nodes, const int32_t* cut, int32_t n_cut,
                            const double* r, const float* prob, int32_t k_splits, int32_t* new_cut, float* new_prob,
                            int32_t cap, int32_t* n_new);

/* Size of the library's built-in query scratch (32 MiB), see
 * nbvh_query_rays_static. */
#define NBVH_STATIC_SCRATCH_BYTES 33554432

/* Device. The same neural ray query as nbvh_query_rays, for callers that must
 * not allocate device memory themselves: for example a renderer or plug-in
 * whose GPU memory is owned by a host application's fixed-budget arena, or a
 * frame loop that cannot afford the implicit synchronisation of cudaMalloc.
 * This entry point has no counterpart in the paper; it only changes where the
 * query's scratch lives.
 *
 * The scratch is a 256-byte aligned array of NBVH_STATIC_SCRATCH_BYTES bytes
 * built into the library: every GPU that loads the library holds it until the
 * process exits. A request whose workspace (nbvh_query_workspace_size for
 * rays.n and max_segs) is larger returns NBVH_ERR_WORKSPACE_TOO_SMALL and
 * launches nothing; for max_segs = 16 that is about 160,000 rays per call.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine). Leave stage timing (nbvh_set_timing) off here: it creates CUDA
 * events.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it with the
 * current context; a call in another context of the device (one created after
 * cudaDeviceReset, for example) looks it up again. Make the first call of each
 * context before any stream capture on the device. Every call on a device
 * shares the one array and finds the previous call's data in it (the query
 * clears what must start at zero itself), so calls whose GPU work overlaps,
 * on different streams or from different threads, race on the scratch:
 * serialise them. Inputs and outputs are caller buffers as in
 * nbvh_query_rays. */
nbvh_status nbvh_query_rays_static(const nbvh_model_desc* desc, const void* table, const float* mlp,
                                   const nbvh_node* nodes, int32_t n_nodes, nbvh_rays rays, int32_t max_segs,
                                   nbvh_hits out, void* stream);

/* ------------------------------------------------------------------------
 * CUDA graphs: record a sequence of this library's calls (for example a
 * whole query step: query, bounce rays, query) once and replay it with one
 * launch. Capture needs a created stream (not the legacy default stream);
 * between nbvh_graph_begin and nbvh_graph_end only enqueueing calls may be
 * made (no nbvh_get_device_status, nbvh_query_stats or host allocations), and
 * stage timing is not recorded. The graph replays the recorded pointers and
 * sizes: rerecord when they change. Empty query waves stay in the graph and
 * exit after reading their queue length.
 * ------------------------------------------------------------------------ */
typedef struct nbvh_graph_s* nbvh_graph;

nbvh_status nbvh_graph_begin(void* stream);
nbvh_status nbvh_graph_end(void* stream, nbvh_graph* out);
nbvh_status nbvh_graph_launch(nbvh_graph graph, void* stream);
nbvh_status nbvh_graph_destroy(nbvh_graph graph);

/* ------------------------------------------------------------------------
 * Hybrid two-level hierarchy (S9; Sec. 7 "Application: Hybrid path
 * tracing"): a top level holds several bottom-level structures, each either a
 * classical BVH over triangles or an N-BVH; reaching a BLAS leaf runs a
 * classical or a neural intersection query, and both return the same hit
 * record, from which the path tracer samples the next direction.
 * ------------------------------------------------------------------------ */

/* Host. Classical triangle BLAS: binned surface-area-heuristic BVH over
 * triangle centroids (32 bins per axis; the base BVH the paper builds on the
 * CPU is an SAH tree, Sec. 6 "BVH construction"). A node splits where
 * area(left) n_left + area(right) n_right is smallest; it stays a leaf when it
 * holds at most max_leaf triangles and no split beats area(node) n (one node
 * visit counted as one triangle test). Node boxes are the exact float AABBs
 * of their triangles (no inflation). Nodes use the nbvh_node format (child < 0
 * is leaf ~child; a single leaf is node 0 with child1 = 0x7fffffff).
 *   tris        host, [n_tris][3][3] float
 *   nodes       host, node_cap >= max(1, n_tris - 1) entries; *out_n_nodes set
 *   tri_perm    host, n_tris int32: the triangles in leaf order (caller indices)
 *   leaf_range  host, 2 * leaf_cap int32 (leaf_cap >= n_tris): leaf i owns
 *               tri_perm[leaf_range[2i] .. leaf_range[2i+1]); *out_n_leaves set
 * Errors: INVALID_ARG for a null pointer, n_tris < 1, max_leaf outside
 * [1, 64], a non-finite vertex or a capacity below the bounds above. */
nbvh_status nbvh_build_tri_blas(const float* tris, int64_t n_tris, int32_t max_leaf, nbvh_node* nodes,
                                int32_t node_cap, int32_t* out_n_nodes, int32_t* tri_perm, int32_t* leaf_range,
                                int32_t leaf_cap, int32_t* out_n_leaves);

/* A triangle BLAS on the device (all pointers device memory). */
typedef struct {
  const nbvh_node* nodes;
  int32_t n_nodes;
  const float* tris;          /* [n_tris][9] vertices in leaf order (tris[tri_perm[i]]) */
  const int32_t* leaf_range;  /* [n_leaves][2] as nbvh_build_tri_blas */
  const int32_t* tri_id;      /* [n_tris] tri_perm: caller index of each leaf-order triangle */
  const float* albedo;        /* optional [n_tris][3] RGB by caller index, NULL = none */
} nbvh_tri_blas;

/* Device. Closest triangle hit of every ray with t in [tmin, tmax]
 * (Moller-Trumbore, edges inclusive, det == 0 a miss, FP32); equal t goes to
 * the lower caller index. hits: hit 1, t, the geometric normal (unit, turned
 * to face -d), leaf = the triangle's caller index; a miss gets hit 0,
 * t +inf, normal 0, leaf -1. rays/hits: device SoA of rays.n entries. */
nbvh_status nbvh_trace_triangles(const nbvh_tri_blas* blas, nbvh_rays rays, nbvh_hits hits, void* stream);

typedef enum { NBVH_BLAS_TRIANGLES = 0, NBVH_BLAS_NEURAL = 1 } nbvh_blas_kind;

/* One top-level instance (host struct; the pointers inside are device memory).
 * Instances are placed in world space (no transform). */
typedef struct {
  int32_t kind;             /* nbvh_blas_kind */
  nbvh_tri_blas tri;        /* kind == NBVH_BLAS_TRIANGLES */
  nbvh_model_desc desc;     /* kind == NBVH_BLAS_NEURAL: the asset's model, */
  const void* table;        /*   hash table (desc.table_prec), */
  const float* mlp;         /*   MLP parameters (nbvh_mlp_param_count order), */
  const nbvh_node* nodes;   /*   N-BVH nodes (nbvh_build_leaves) */
  int32_t n_nodes;
  int32_t max_segs;         /*   segment slots per ray for this asset */
} nbvh_instance;

/* Host. Workspace bytes of nbvh_hybrid_trace for n_rays rays, for either
 * form (instance_streams): two query workspaces of the deepest instance, the
 * per-instance ray lists, and per neural instance a staging hit record
 * (about 21 bytes per ray, 33 with an albedo head). */
nbvh_status nbvh_hybrid_workspace_size(const nbvh_instance* inst, int32_t n_inst, int64_t n_rays, size_t* bytes);

/* Device. Closest hit over every instance of the two-level hierarchy. Each
 * triangle instance answers as nbvh_trace_triangles; each neural instance
 * answers as nbvh_query_rays on its own N-BVH over the ray's full
 * [tmin, tmax]. The result is the smallest t over the instances; equal t goes
 * to the lower instance index. out.leaf is the triangle index or the N-BVH
 * leaf; out_inst (device, rays.n int32) the instance index, -1 on a miss.
 * The result is the closest hit over all instances, equal t to the lower
 * instance index. Sequential form (instance_streams = 1): instances are
 * processed in index order as wavefront passes, each keeping the record
 * unless it finds a strictly closer hit. Before the first neural instance,
 * one top-level pass tests every ray against the root boxes of all remaining
 * neural instances and lists, per instance, the rays that meet them before
 * the record; each neural pass then traverses only its list and skips the
 * leaves whose segment starts at or beyond the record (their hits cannot be
 * closer), which leaves the result unchanged. Concurrent form (the default):
 * the triangle instances first, then the top-level pass, then the neural
 * instances on two side streams, each searching from the triangles' answer
 * into its own staging record, then one per-ray merge in instance order; the
 * record equals the sequential form's bit for bit.
 * inst: host array of n_inst (1..64) instances; workspace: device, 256-byte
 * aligned, >= nbvh_hybrid_workspace_size bytes. opt: the evaluation options
 * of the neural passes (NULL = nbvh_query_options_default). Segment overflow
 * of a neural pass is reported as in nbvh_query_rays. */
nbvh_status nbvh_hybrid_trace(const nbvh_instance* inst, int32_t n_inst, nbvh_rays rays, nbvh_hits out,
                              int32_t* out_inst, void* workspace, size_t ws_bytes, const nbvh_query_options* opt,
                              void* stream);

/* Device (synchronises). Measurement utility, no counterpart in the paper:
 * the L2 random-gather ceiling that bounds the hash-table gather when the
 * table is L2-resident. One CTA of 1,024 threads per SM issues independent
 * 4-byte loads at pseudo-random positions of table (n_entries 4-byte
 * entries, a power of two in [1024, 2^31]; device memory the caller owns,
 * any contents; pick 16-64 MB so it stays in L2), 16 in flight per thread.
 * *gsectors_per_s receives the best of three timed launches in 1e9 loads per
 * second (each load a distinct 32-byte sector). sink: one device uint32 the
 * kernel may write. */
nbvh_status nbvh_probe_l2_gather(const void* table, int64_t n_entries, uint32_t* sink, double* gsectors_per_s,
                                 void* stream);

/* Device (synchronises). Measurement utility, no counterpart in the paper:
 * the L2 reduction ceiling that bounds the training backward's table-
 * gradient scatter when the gradient buffer is L2-resident. One CTA of 1,024
 * threads per SM issues fire-and-forget float2 atomic adds (8 bytes each,
 * the scatter's update at F = 2) at pseudo-random entries of grad
 * (n_entries float2 entries, a power of two in [1024, 2^30]; device memory
 * the caller owns; each add puts 1e-30 into both floats of an entry), 16 per
 * thread per round. *gops_per_s receives the best of three timed launches
 * in 1e9 atomic adds per second. */
nbvh_status nbvh_probe_l2_reduce(float* grad, int64_t n_entries, double* gops_per_s, void* stream);

/* Device. Reads and clears the device status word (synchronises the stream). */
nbvh_status nbvh_get_device_status(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NBVH_H_ */
