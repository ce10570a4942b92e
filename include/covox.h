/*
 * covox.h -- C ABI of the GB300 TSDF integration library (libcovox.so).
 *
 * Projective TSDF integration of range scans into block-hashed voxel submaps,
 * as coVoxSLAM describes it:
 *   - submaps are sparse sets of dense 8^3-voxel blocks indexed by their
 *     integer 3-D position through a GPU open-addressing hash table, voxel
 *     fields stored as separate arrays (Sec. III-A data layout, Sec. III-B
 *     hash table with "activate", Sec. III-C two-level representation);
 *   - a scan is integrated by ray casting every point, updating the voxels the
 *     ray crosses within the truncation band around the point (Sec. III-C,
 *     ray-casting paragraph), in a count / allocate / process sequence whose
 *     per-voxel sums are reduced before they are merged (Sec. III-D).
 *
 * Conventions shared by every entry point:
 *   - All calls are asynchronous on the caller's CUDA stream (`stream`, a
 *     cudaStream_t; NULL = legacy default stream) unless stated otherwise.
 *   - Device pointers are borrowed: they must stay valid until the stream has
 *     executed the call.  The library never frees caller memory.
 *   - Invalid arguments are detected on the host and returned at once
 *     (CVX_ERR_INVALID_ARG); nothing is launched then.
 *   - Errors found on the device (hash table full, block pool exhausted,
 *     key out of range, a bounded wait that gave up) set a per-scan error
 *     word: the voxel-update (merge) phase of that scan is skipped, so stored
 *     distances and weights are unchanged, while blocks allocated by the scan
 *     stay allocated with zero weight.  The error is also OR-ed into a sticky
 *     word read by cvx_submap_status().
 *   - A submap is not thread safe: calls on one submap must be serialised.
 *   - Voxel (i,j,k) of a submap holds the cube [i,i+1) x [j,j+1) x [k,k+1)
 *     times the voxel size; its block key is (i>>3, j>>3, k>>3) (arithmetic
 *     shift, i.e. floor division) and its local index lx + 8 ly + 64 lz with
 *     lx = i & 7 etc.  Keys must stay within [-2^20, 2^20) per axis.
 */
#ifndef COVOX_H
#define COVOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CVX_OK = 0,
  CVX_ERR_INVALID_ARG = -1,
  CVX_ERR_OOM = -2,        /* an allocation of the submap failed */
  CVX_ERR_CAPACITY = -3,   /* hash table or block pool full */
  CVX_ERR_KEY_RANGE = -4,  /* a band endpoint left the +-2^23 voxel index range */
  CVX_ERR_TIMEOUT = -5,    /* a bounded wait inside a persistent launch gave up */
  CVX_ERR_CUDA = -6        /* a CUDA runtime call failed */
} cvx_status;

typedef enum { CVX_STORE_F32 = 0, CVX_STORE_F16 = 1 } cvx_storage;

/* Integration weight of one observation (Sec. III-C, weighting paragraph):
 * constant 1, quadratic 1/z^2 (z = optical-axis depth for a pinhole sensor,
 * range for a spherical one), or a caller-supplied value per point. */
typedef enum { CVX_W_CONST = 0, CVX_W_QUADRATIC = 1, CVX_W_PER_POINT = 2 } cvx_weight_mode;

/* Behind-surface drop-off: for signed distance d < -vs the weight is scaled by
 * f = (trunc + d) / (trunc - vs) (LINEAR) or f^2 (QUADRATIC); f reaches 0 at
 * d = -trunc.  Requires trunc > voxel_size. */
typedef enum { CVX_DROP_NONE = 0, CVX_DROP_LINEAR = 1, CVX_DROP_QUADRATIC = 2 } cvx_dropoff;

typedef enum { CVX_SENSOR_PINHOLE = 0, CVX_SENSOR_SPHERICAL = 1 } cvx_sensor;

/* Device-memory allocator hooks.  alloc returns NULL on failure; free receives
 * the pointer and the size it was allocated with.  Both may be NULL, in which
 * case the library uses cudaMalloc / cudaFree. */
typedef void* (*cvx_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*cvx_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

/* A pipelined submap holds a second set of per-scan sums and touched-block
 * list, so that the merge of one scan overlaps the accumulation of the next
 * (same results; twice the per-scan memory).  In a batched launch the merges
 * of wave k overlap the tiles of wave k + 1.  On the per-scan path each
 * cvx_integrate_scan() launches one kernel that accumulates its scan and
 * merges the scan of the previous call; the last scan stays pending until
 * cvx_flush_submap(), cvx_extract_blocks(), cvx_submap_counters(),
 * cvx_reset_submap() (which drops it) or a batched launch merges it.  Which
 * set is in use lives on the device, so recorded CUDA graphs replay
 * correctly. */
#define CVX_SUBMAP_PIPELINED 1
/* Four sets of per-scan sums and touch epochs (implies CVX_SUBMAP_PIPELINED):
 * in a batched launch scan k accumulates into set k mod 4, so its tiles wait
 * only for the merge of scan k - 4, and several consecutive scans of one
 * submap are in flight at once (same results; four times the per-scan
 * memory, 4 KB per block per set).  The per-scan path uses the first two. */
#define CVX_SUBMAP_FOUR_SETS 2
/* Colour submap (the "TSDF + Color" integration of Sec. IV): every voxel also
 * holds a fused RGB colour, three float32 planes per block, and every
 * per-scan set holds colour sums (16 bytes per voxel).  Every scan integrated
 * into it must carry per-point colours (cvx_integrate_scan_color, or
 * colors_rgb of a batched scan); each voxel's colour is the weighted mean of
 * its observations' colours under the observation weights of the TSDF:
 * C <- (C W + sum w c) / (W + sum w) in the same merge as D (W the stored
 * weight before the merge).  A point with a non-finite colour channel is
 * invalid (skipped, not counted).  Colours are fused in float32 in both
 * storage modes. */
#define CVX_SUBMAP_COLOR 4

typedef struct {
  float voxel_size;      /* metres, > 0 */
  float trunc;           /* truncation distance, metres, > 0 */
  float max_weight;      /* cap on the stored weight, > 0 */
  int32_t storage;       /* cvx_storage */
  int64_t max_blocks;    /* block pool capacity (blocks of 512 voxels) */
  int64_t hash_slots;    /* hash table slots, a power of two >= 2 * max_blocks advised */
  int64_t flags;         /* 0 or CVX_SUBMAP_PIPELINED or CVX_SUBMAP_FOUR_SETS, each optionally
                            with CVX_SUBMAP_COLOR */
  cvx_alloc_fn alloc;
  cvx_free_fn free;
  void* alloc_ctx;
  void* stream;          /* stream used for the creation-time clears */
} cvx_submap_params;

typedef struct {
  int32_t weight_mode;   /* cvx_weight_mode */
  int32_t dropoff;       /* cvx_dropoff */
  float min_range;       /* points with |p - o| outside [min_range, max_range] are skipped */
  float max_range;
  int32_t height, width; /* organised scan layout (0, 0 = unorganised) */
  int32_t sensor;        /* cvx_sensor: defines z of the quadratic weight */
  int32_t pts_per_cta;   /* tuning: points per CTA tile (0 = default; organised scans use
                            32-pixel-wide tiles of pts_per_cta / 32 rows) */
  int32_t local_blocks;  /* tuning: shared-memory block slots per CTA: 0 = default (8), a
                            power of two <= 16, or -1 = no shared slots (global atomics) */
  int32_t flags;         /* 0, or CVX_INTEGRATE_CARVE */
} cvx_integrate_params;

/* Free-space carving (the paper's ray casting from the optical centre,
 * Sec. III-C): each ray is traversed from the sensor origin to
 * p + trunc u instead of over the band [p - trunc u, p + trunc u]; voxels in
 * front of the band receive d = +trunc.  A = origin / voxel_size replaces
 * (p - trunc u) / voxel_size in the traversal; everything else is unchanged. */
#define CVX_INTEGRATE_CARVE 1

typedef struct {
  int64_t n_blocks;         /* allocated blocks */
  int64_t frames;           /* scans integrated */
  int64_t valid_points;     /* points that passed the validity test */
  int64_t observations;     /* (point, voxel) pairs of the band traversals */
  int64_t voxels_merged;    /* per-scan unique voxels whose D/W were updated, summed */
  int64_t blocks_touched;   /* per-scan distinct blocks, summed */
} cvx_counters;

typedef struct cvx_submap cvx_submap;

/* Create an empty submap (hash table, block pool with D and W per voxel,
 * per-scan scratch).  Synchronous.  *out receives the handle. */
cvx_status cvx_create_submap(const cvx_submap_params* params, cvx_submap** out);

/* Integrate one scan as one frame (Sec. III-C ray casting; Sec. III-D count,
 * allocate, process).  points_xyz: device float32 [n,3], sensor frame, NaN or
 * out-of-range points skipped.  T_sub_sensor: HOST float32[12], 3x4 row-major
 * rigid transform submap <- sensor (its translation is the sensor origin).
 * point_weights: device float32 [n] for CVX_W_PER_POINT, else NULL; a point
 * whose weight is not finite or is negative is invalid (skipped, not counted).
 * For every valid point p with unit ray direction u from the origin o, each
 * voxel v crossed by the segment [p - trunc u, p + trunc u] receives the
 * observation d = clamp((p - c_v).u, -trunc, trunc) (c_v = voxel centre) with
 * weight w; then, per voxel, D <- (D W + sum w d) / (W + sum w) and
 * W <- min(W + sum w, max_weight) when W + sum w > 0. */
cvx_status cvx_integrate_scan(cvx_submap* map, const float* points_xyz, int64_t n,
                              const float T_sub_sensor[12], const float* point_weights,
                              const cvx_integrate_params* params, void* stream);

/* cvx_integrate_scan with per-point colours (colour submaps, which require
 * them; any other submap returns CVX_ERR_INVALID_ARG).  colors_rgb: device
 * float32 [n,3], any units (typically [0,1]).  Colour scans run the general
 * tile form with L2 vector reductions (params->local_blocks is ignored). */
cvx_status cvx_integrate_scan_color(cvx_submap* map, const float* points_xyz, int64_t n,
                                    const float T_sub_sensor[12], const float* point_weights,
                                    const float* colors_rgb, const cvx_integrate_params* params, void* stream);

/* Copy out the fused colours of a colour submap: rgb float32 [capacity,3,512]
 * (block, channel, voxel), device or host memory, the blocks in the order of
 * cvx_extract_blocks; min(n_blocks, capacity) blocks are copied and counted
 * in *n_out.  With rgb == NULL only *n_out (the number of blocks) is written.
 * CVX_ERR_INVALID_ARG for a submap without colour.  Synchronises `stream`. */
cvx_status cvx_extract_colors(cvx_submap* map, int64_t capacity, float* rgb, int64_t* n_out, void* stream);

/* Copy out the allocated blocks in allocation order.  Two-call convention:
 * with keys == NULL only *n_out (the number of blocks) is written.  Otherwise
 * min(n_blocks, capacity) blocks are copied: keys int32 [cap,3], dist and
 * weight [cap,512] in the storage type (float32, or float16 with dist holding
 * D / trunc).  Pointers may be device or host memory.  Synchronises `stream`. */
cvx_status cvx_extract_blocks(cvx_submap* map, int64_t capacity, int32_t* keys, void* dist,
                              void* weight, int64_t* n_out, void* stream);

/* Clear all blocks and counters (asynchronous, no host synchronisation).  A
 * scan still pending in a pipelined submap is dropped, and so are the
 * per-scan sums a launch that gave up (CVX_ERR_TIMEOUT) left unmerged. */
cvx_status cvx_reset_submap(cvx_submap* map, void* stream);

/* cvx_reset_submap() of n distinct submaps (asynchronous): two kernel
 * launches per 48 submaps instead of a handful of launches and copies per
 * submap, for mappers that keep many submaps (one per stretch of the
 * trajectory, Sec. III-C) and clear them together.  INVALID_ARG if maps is NULL (n > 0) or holds a
 * NULL entry; nothing is launched then. */
cvx_status cvx_reset_submaps(cvx_submap* const* maps, int32_t n, void* stream);

/* Pipelined submap: merge the scan the last cvx_integrate_scan() left
 * pending, asynchronously on `stream` (one kernel; nothing when no scan is
 * pending on the device).  Other submaps: no-op.  Coalescing the per-scan
 * merge with the next scan's accumulation is this library's scheduling; the
 * paper merges every frame before the next one (Sec. III-D), which is the
 * result this reproduces. */
cvx_status cvx_flush_submap(cvx_submap* map, void* stream);

/* Sticky device error word as a status (CVX_OK if no error).  Synchronises the
 * stream of the last call on this submap. */
cvx_status cvx_submap_status(cvx_submap* map);

/* Cumulative counters (synchronises like cvx_submap_status; merges a
 * pending scan first). */
cvx_status cvx_submap_counters(cvx_submap* map, cvx_counters* out);

/* Euclidean distance field of the submap (Sec. III-E builds an ESDF from the
 * TSDF blocks; the paper fixes neither the site rule nor a cap, this is the
 * library's reading).  For every voxel of every allocated block, in the
 * block order of cvx_extract_blocks(): out = voxel_size * the distance, in
 * voxel units, from its centre to the centre of the nearest site voxel,
 * capped at max_dist (max_dist when the submap has no site); sites are the
 * allocated voxels with W > w_min and |D| <= site_band (metres).  Unsigned.
 * out: device float32 [n_blocks, 512]; sq_dist: device int32 [n_blocks, 512]
 * of the exact squared distances in voxel units (-1: no site), or NULL.
 * Computed from scratch over the box spanned by the allocated blocks (a
 * pipelined submap's pending scan is merged first); scratch of 24 B per box
 * voxel comes from the submap's allocator.  CVX_ERR_CAPACITY if the box
 * exceeds 16,384 voxels on an axis, CVX_ERR_OOM if the scratch cannot be
 * allocated.  Synchronises `stream` once (to size the box). */
cvx_status cvx_compute_esdf(cvx_submap* map, float site_band, float w_min, float max_dist, float* out,
                            int32_t* sq_dist, void* stream);

/* Registration points (Sec. III-F: the backend's ICP takes each submap's
 * points by their weights; the selection rule is the library's reading): the
 * centres, in the submap frame (metres, ((i + 1/2) * voxel_size) in FP32),
 * of the allocated voxels with W >= w_min, W > 0 and |D| <= d_band, in no
 * particular order.  xyz: device float32 [capacity,3]; *n_out receives the
 * number of qualifying voxels, of which the first min(*n_out, capacity) are
 * written.  A pipelined submap's pending scan is merged first.  Synchronises
 * `stream`. */
cvx_status cvx_registration_points(cvx_submap* map, float w_min, float d_band, int64_t capacity, float* xyz,
                                   int64_t* n_out, void* stream);

/* Axis-aligned bounds of the allocated blocks in the submap frame, for the
 * backend's overlap test (Sec. III-F): lo_hi = {lo x, y, z, hi x, y, z}
 * (block corners, metres, FP32); lo > hi when the submap is empty.
 * Synchronises `stream`. */
cvx_status cvx_submap_bounds(cvx_submap* map, float lo_hi[6], void* stream);

/* Overlap of posed submaps (Sec. III-F: the backend registers submaps whose
 * boxes overlap).  bounds: device float32 [n,6], each submap's lo_hi from
 * cvx_submap_bounds (submap frame; lo > hi marks an empty submap); poses:
 * device float32 [n,12], 3x4 row-major world <- submap.  For every ordered
 * pair (i, j): each box carried to the world frame (the axis-aligned box of
 * its 8 transformed corners), the two intersected; volume[i*n + j] (device
 * float32 [n,n], m^3) is the intersection's volume, 0 if disjoint or empty;
 * boxes (device float32 [n,n,6] or NULL) receives the intersection lo, hi.
 * Asynchronous on `stream`. */
cvx_status cvx_submap_overlaps(int32_t n, const float* bounds, const float* poses, float* volume, float* boxes,
                               void* stream);

/* Free the submap and everything it allocated (synchronises its stream). */
void cvx_destroy(cvx_submap* map);

/* ---- the block hash on its own (Sec. III-B "activate"; Sec. IV's hash
 * stress test inserts tens of millions of keys) ----
 * The table a submap uses: packed block keys (each coordinate in
 * [-2^20, 2^20)), open addressing with linear probing (at most 4,096 probes),
 * keys claimed by 64-bit CAS.  A new key takes the next pool index (blocks
 * are numbered in allocation order); the new keys of a warp take theirs with
 * one atomic per warp. */
typedef struct cvx_block_hash cvx_block_hash;

/* slots: power of two >= 2 (load factor = keys / slots; the table keeps
 * working up to ~0.85); max_blocks: pool capacity.  Synchronous. */
cvx_status cvx_block_hash_create(int64_t slots, int64_t max_blocks, cvx_block_hash** out);
/* Insert-or-find the n blocks of coords (device int32 [n,3]); pool (device
 * int32 [n]) receives each block's pool index, equal for equal keys, or -1 if
 * the key could not be placed (capacity, key range: recorded, see _info).
 * Asynchronous on `stream`. */
cvx_status cvx_block_hash_insert(cvx_block_hash* hash, const int32_t* coords, int64_t n, int32_t* pool,
                                 void* stream);
/* Lookup only: pool[i] = the block's pool index or -1.  Asynchronous. */
cvx_status cvx_block_hash_find(cvx_block_hash* hash, const int32_t* coords, int64_t n, int32_t* pool,
                               void* stream);
/* Number of blocks and, if block_keys != NULL, the first min(n, capacity)
 * block coordinates in pool order (int32 [.,3], host or device).  Returns the
 * recorded error (CVX_ERR_CAPACITY, CVX_ERR_KEY_RANGE, CVX_ERR_TIMEOUT) or
 * CVX_OK.  Synchronises the stream of the last call. */
cvx_status cvx_block_hash_info(cvx_block_hash* hash, int64_t* n_blocks, int32_t* block_keys, int64_t capacity);
void cvx_block_hash_destroy(cvx_block_hash* hash);

/* Library version string. */
const char* cvx_version(void);

/* ---- batched integration: many submaps, uneven scans, one persistent launch ----
 * A scan of a batch: which submap it goes to (index into the maps array of
 * cvx_integrate_batch), its points (device float32 [n,3], sensor frame), pose
 * (host float32 3x4 submap <- sensor), optional per-point weights (device
 * [n]) and integration parameters, all as for cvx_integrate_scan. */
typedef struct {
  int32_t submap;
  int32_t pad;
  const float* points_xyz;
  int64_t n;
  float T_sub_sensor[12];
  const float* point_weights;
  cvx_integrate_params params;
  const float* colors_rgb;  /* device float32 [n,3] for colour submaps, else NULL */
} cvx_scan_desc;

typedef struct cvx_batch cvx_batch;

/* Descriptor buffers for batches of up to max_submaps submaps (<= 1024) and
 * max_scans scans (device memory and pinned host staging).  Synchronous. */
cvx_status cvx_batch_create(int32_t max_submaps, int32_t max_scans, cvx_batch** out);

/* Integrate a batch of scans into distinct submaps with one persistent
 * kernel (Sec. III-D workload equalisation across scans).  Scans
 * of one submap are integrated as successive frames in array order (exactly
 * as successive cvx_integrate_scan calls); scans of different submaps are
 * independent; empty scans are skipped.  The kernel takes tile and merge
 * work items from one queue in dependency order (a scan's tiles wait for the
 * merge that last used their per-scan set -- with pipelined submaps two
 * sets, with four-set submaps four, so consecutive scans overlap --, a
 * scan's merge for its tiles and for the previous scan's merge: each merge
 * part only for the same part of the previous merge when both have the same
 * part count, since it covers the same blocks), so no grid-wide barrier is
 * needed.  Asynchronous
 * on `stream`; the descriptor upload reads the batch object's pinned staging
 * buffer when the stream executes it, so a CUDA graph that captured this call
 * replays the staging buffer's contents at replay time: do not issue another
 * call on the same batch object between replays.  Every wait inside the
 * kernel is bounded; a wait that gives up is reported by cvx_batch_error() as
 * CVX_ERR_TIMEOUT, after which the batch's submaps must be reset. */
cvx_status cvx_integrate_batch(cvx_batch* batch, cvx_submap* const* maps, int32_t n_maps,
                               const cvx_scan_desc* scans, int32_t n_scans, void* stream);

/* Tuning: the queue takes the scans in rounds (round k: the k-th scan of
 * every submap, its merges in the next round); this cuts every round into
 * chunks of at most max_scans_per_wave scans (0 = no limit), which bounds the
 * submaps in flight.  Results do not depend on it. */
cvx_status cvx_batch_wave_limit(cvx_batch* batch, int32_t max_scans_per_wave);

/* Tuning: the queue of a batched launch takes the submaps in groups of
 * `group` consecutive submaps (by index in the launch's submap array): every
 * scan of one group, round by round of equal frame rank, before the next
 * group's (0 = all submaps in one group, the default).  Small groups keep a
 * group's voxel fields and per-scan sums resident in the L2 between its
 * scans when many large submaps share a launch; one group gives the most
 * scans in flight.  Results do not depend on it. */
cvx_status cvx_batch_submap_group(cvx_batch* batch, int32_t group);

/* Tuning: each scan's merge runs as `parts` work items of the persistent
 * launch (1..256; 0 = chosen per round of the queue, a round being the scans
 * of equal rank in their submaps: the largest power of two in [8, 64] whose
 * product with the round's scan count stays within the launch's resident
 * CTAs).  A round of few scans -- one submap, or the last frames of the
 * longest chains -- is a few merges on the critical path, where more parts
 * shorten each merge; many scans run their merges side by side, where fewer
 * parts cost less queue traffic (Sec. III-D workload equalisation).  Results
 * do not depend on it. */
cvx_status cvx_batch_merge_parts(cvx_batch* batch, int32_t parts);

/* CVX_ERR_TIMEOUT if a wait of the last batch gave up (synchronous). */
int32_t cvx_batch_error(cvx_batch* batch);

/* Test hook for the bounded waits (off by default): while missing_cta >= 0,
 * that CTA of this batch's launches takes one work item and leaves without
 * doing it, and the waits give up after barrier_polls polls (<= 0: the
 * default limit, about one second).  The CTAs waiting for the item run out
 * their limit and the launch drains; cvx_batch_error() reports
 * CVX_ERR_TIMEOUT (also when nothing waited for the item: the last CTA to
 * leave checks that every scan was merged) and the submaps must be reset.
 * missing_cta < 0 restores normal launches.  Nothing faults or hangs: it
 * exercises the timeout path the waits always have. */
cvx_status cvx_batch_test_missing_cta(cvx_batch* batch, int32_t missing_cta, int64_t barrier_polls);

void cvx_batch_destroy(cvx_batch* batch);

/* Tracing of the batched kernel: with timing enabled, the kernel stamps the
 * GPU global timer at its start, when the last tile of each scan finishes and
 * when each scan's merge completes; cvx_batch_phase_times() (synchronous)
 * returns, for each scan of the last batch in queue order (rounds of equal
 * rank), the milliseconds from the launch start to its tiles' end
 * (ms[3 * scan]) and to its merge's end (ms[3 * scan + 1]; ms[3 * scan + 2] =
 * 0).  Returns the scans written (at most max_scans). */
cvx_status cvx_batch_timing(cvx_batch* batch, int32_t enable);
int32_t cvx_batch_phase_times(cvx_batch* batch, double* ms, int32_t max_scans);

/* ---- learned per-point weight (Sec. III-C weighting paragraph) ----
 * Features of an organised scan, one row of three per point (device float32
 * [height*width, 3]): f1 = |P| / max_range; f2 = theta / (pi/2) with theta the
 * angle between the ray and the surface normal from the cross product of the
 * horizontal and vertical neighbour differences (0 when a neighbour is
 * missing); f3 = ln(var + 1e-8) / 10 with var the population variance of the
 * depths (z for a pinhole, range for a spherical sensor) of the valid points
 * of the 5x5 window (0 if fewer than 3).  Invalid points get zeros. */
cvx_status cvx_point_features(const float* points_xyz, int32_t height, int32_t width, int32_t sensor,
                              float max_range, float* features, void* stream);

/* Weight network w = softplus(W3 . h2 + b3), h2 = relu(W2 h1 + b2),
 * h1 = relu(W1 f + b1), 3-32-32-1, GEMM operands rounded to BF16 with FP32
 * accumulation on the tensor cores.  Parameters: float32[CVX_MLP_PARAMS] in
 * the order W1 [32,3] row-major, b1 [32], W2 [32,32], b2 [32], W3 [32], b3. */
#define CVX_MLP_PARAMS 1217
typedef struct cvx_weight_model cvx_weight_model;

/* Device copy of init_params (host or device pointer) plus Adam state. */
cvx_status cvx_weight_model_create(const float* init_params, cvx_weight_model** out);
/* Set (set != NULL) and/or read back (get != NULL, synchronous) the parameters. */
cvx_status cvx_weight_model_params(cvx_weight_model* model, const float* set, float* get, void* stream);
/* weights[i] = network(features[i]) for n points (device arrays). */
cvx_status cvx_weight_model_infer(cvx_weight_model* model, const float* features, int64_t n,
                                  float* weights, void* stream);
/* Per-point weights of an organised scan in one pass: the features of
 * cvx_point_features and the network of cvx_weight_model_infer, computed
 * together (the features never leave the chip).  points_xyz: device float32
 * [height*width, 3]; weights: device float32 [height*width]. */
cvx_status cvx_weight_model_point_weights(cvx_weight_model* model, const float* points_xyz, int32_t height,
                                          int32_t width, int32_t sensor, float max_range, float* weights,
                                          void* stream);
/* The same for n_frames organised scans of one shape in one persistent
 * launch: points_xyz device float32 [n_frames, height*width, 3], weights
 * device float32 [n_frames, height*width] (frame-major). */
cvx_status cvx_weight_model_point_weights_frames(cvx_weight_model* model, const float* points_xyz,
                                                 int32_t n_frames, int32_t height, int32_t width, int32_t sensor,
                                                 float max_range, float* weights, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr; lr = 0 only
 * computes the gradient) on the mean over points with mask != 0 of
 * w e2 - ln w (Gaussian negative log likelihood of precision w).  The
 * per-CTA gradient partials are summed in a fixed order: deterministic. */
cvx_status cvx_weight_model_train_step(cvx_weight_model* model, const float* features, const float* e2,
                                       const float* mask, int64_t n, float lr, void* stream);
/* The last step's mean gradient [CVX_MLP_PARAMS] and loss (synchronous). */
cvx_status cvx_weight_model_last(cvx_weight_model* model, float* grad, float* loss, void* stream);
void cvx_weight_model_destroy(cvx_weight_model* model);

/* Training targets of a noisy scan against a noise-free float32 submap:
 * e2[i] = mean over the point's band voxels with clean W > 0 of
 * (d - D_clean)^2 (d as in cvx_integrate_scan), mask[i] = 1 if there was at
 * least one such voxel, else e2 = mask = 0.  Device arrays of n floats. */
cvx_status cvx_training_targets(cvx_submap* clean, const float* points_xyz, int64_t n,
                                const float T_sub_sensor[12], const cvx_integrate_params* params,
                                float* e2, float* mask, void* stream);

/* Scale of a training set's targets: e2[i] /= mean, mean = sum(e2 mask) /
 * max(sum(mask), 1), in place on the device (fixed-order reduction, so the
 * result does not depend on scheduling); *mean_out (host) receives the mean.
 * The fitted weights are then ~1 for a typical point, the scale of the
 * constant weight, so the stored weight's cap is met no sooner than with the
 * plain weighting.  Synchronises `stream`. */
cvx_status cvx_normalise_targets(float* e2, const float* mask, int64_t n, float* mean_out, void* stream);

/* ---- integration without device allocation ----
 * No counterpart in the paper: an addition for callers that cannot allocate
 * device memory -- a real-time loop that must never allocate after start-up,
 * a host whose memory manager owns all device memory and hands out fixed
 * buffers, or a plugin that may not touch the process's allocator.
 *
 * cvx_integrate_scan_noalloc() integrates one scan, with the same arithmetic
 * and results as cvx_integrate_scan() on float32 storage, into submap storage
 * the caller owns and describes with a cvx_submap_view.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its per-scan scratch
 * (per-voxel sums, the blocks' touch epochs and their voxel groups' touch
 * tags, about 16.5 MiB) is one fixed array in device memory that every GPU
 * loading this library holds until the process exits.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress) and sets a kernel
 *     attribute; make that first call before any stream capture.
 *   - All calls on a device share the array.  Each call clears what must
 *     start at zero, so calls that overlap on the GPU (different streams, or
 *     different views at the same time) race: serialise them.
 *   - view->max_blocks above CVX_NOALLOC_MAX_BLOCKS is rejected with
 *     CVX_ERR_CAPACITY before anything is launched; other invalid arguments
 *     give CVX_ERR_INVALID_ARG.  Device errors behave as in
 *     cvx_integrate_scan() and are recorded in the view's state buffer.
 * Caller initialisation of a view: hash_keys all bits set (0xff bytes),
 * hash_vals -1 (0xff bytes), dist and weight zero, state zero.  Alignment:
 * dist and weight 16 bytes, hash_keys and state 8 bytes, hash_vals and
 * block_keys 4 bytes; a misaligned view gives CVX_ERR_INVALID_ARG.  The
 * number of allocated blocks is min(first int32 of the state buffer,
 * max_blocks): after the pool overflowed the counter can exceed max_blocks,
 * and the sticky error word (the int32 at byte offset 12 of the state) has
 * bit 0 set (capacity; bit 1: key range, bit 2: timeout).  Blocks are in
 * allocation order in block_keys / dist / weight. */
#define CVX_NOALLOC_MAX_BLOCKS 4096
#define CVX_SUBMAP_STATE_BYTES 128

typedef struct {
  unsigned long long* hash_keys; /* device [hash_slots] */
  int32_t* hash_vals;            /* device [hash_slots] */
  int64_t hash_slots;            /* power of two >= 2 */
  int32_t* block_keys;           /* device [max_blocks,3] */
  float* dist;                   /* device [max_blocks,512], D in metres */
  float* weight;                 /* device [max_blocks,512], W */
  void* state;                   /* device, CVX_SUBMAP_STATE_BYTES bytes */
  int64_t max_blocks;            /* <= CVX_NOALLOC_MAX_BLOCKS */
  float voxel_size, trunc, max_weight;
} cvx_submap_view;

cvx_status cvx_integrate_scan_noalloc(const cvx_submap_view* view, const float* points_xyz, int64_t n,
                                      const float T_sub_sensor[12], const float* point_weights,
                                      const cvx_integrate_params* params, void* stream);

/* ---- tracing: launch accounting and per-kernel timing ----
 * Every kernel launch of the library is counted.  While profiling is on, an
 * event pair is recorded on the launching stream around each launch (up to
 * max_launches launches); cvx_profile_read() synchronises on those events and
 * returns, per kernel kind, its name (32 chars each), total milliseconds and
 * number of timed launches, then clears the records.  Not thread safe. */
cvx_status cvx_profile_start(int64_t max_launches);
cvx_status cvx_profile_stop(void);
int32_t cvx_profile_read(int32_t max_kinds, char* names, double* total_ms, int64_t* launches);
int64_t cvx_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* COVOX_H */
