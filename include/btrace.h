/*
 * btrace.h -- C ABI of libbtrace, a GB300 (sm_103a) implementation of the
 * hybrid beam/ray-tracing method of "Beam-tracing domain decomposition method
 * for urban acoustic pollution" (Gbikpi-Benissan & Magoules, arXiv:1912.03998).
 *
 * The problem (Section 2 and Section 4): acoustic beams leave point sources,
 * their energy split by the power per direction; each beam's intersection
 * with a city model is resolved by its guiding (axis) ray only, and a beam is
 * never split; every reflection creates an image (virtual) source and a
 * mirrored beam, up to a maximum order; microphones lying inside a beam
 * receive its energy; the result is a sound level per microphone and band.
 *
 * Conventions shared by every call:
 *   - Return value: BT_OK (0) or a negative BT_E_* code (bt_poll may also
 *     return BT_PENDING).  No call aborts the process.  After an error,
 *     bt_last_error() describes it.
 *   - Pointers: every array argument may be host memory (pageable or pinned)
 *     or device memory of the context's GPU; the library tells them apart by
 *     unified addressing and copies them before the call returns.  The caller
 *     keeps ownership of all its arrays.
 *   - Units: metres (z up, ground at z = 0), watts, dB.  float32 inputs are
 *     promoted exactly where the library computes in higher precision.
 *   - Streams: all device work of a context runs on the context's stream (the
 *     one given to bt_create, or one the context creates).  Calls are
 *     synchronous with respect to that stream: they return once their work has
 *     finished.  A context is not thread-safe; use one per host thread.
 *   - Device memory: scenes, acceleration structures, microphone bins and
 *     energy accumulators stay resident on the device until bt_destroy, or
 *     until a later call on the same scene replaces them.
 */
#ifndef BTRACE_H
#define BTRACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BT_OK 0
#define BT_E_INVALID (-1)    /* bad argument or input value (NaN, index out of range, ...) */
#define BT_E_NOMEM (-2)      /* a device or host allocation failed */
#define BT_E_CUDA (-3)       /* a CUDA runtime call failed */
#define BT_E_STATE (-4)      /* call out of order (e.g. trace before sources are set) */
#define BT_E_QUEUE_FULL (-5) /* a device work queue overflowed */
#define BT_E_TIMEOUT (-6)    /* a bounded device wait gave up (watchdog) */
#define BT_PENDING 1         /* bt_poll: the submitted trace is still running (not an error) */

#define BT_MAX_BANDS 8       /* octave bands 63 Hz .. 8 kHz */
#define BT_MAX_SCENES 64     /* resident scenes per context */
#define BT_MAX_TILES 32      /* per axis */

/* Precision of the trace (Section 2 does not fix one).
 * BT_PREC_FP32: the whole beam lineage (directions, image-source apex, ray
 *   origin, cone planes) in float32; float64 energy accumulation.
 * BT_PREC_MIXED (default): the image-source chain (apex, cone normals, ray
 *   origin and direction) in float pairs (double-float, about 48 bits) on the
 *   float32 pipe; float32 watertight traversal whose ambiguous triangle tests
 *   (ray within 1e-4 relative of an edge) are re-done in float64, near-equal
 *   hit distances settled in float64 (up to 8 such candidates per ray, past
 *   which float32 decides); float32 microphone tests relative to
 *   the apex, re-done in float pairs near the cone and end planes; float64
 *   energy accumulation.
 * BT_PREC_FP64: the image-source chain in float64; every triangle test in
 *   float64 (Moller-Trumbore on the float64 ray; the BVH boxes stay float32,
 *   grown to be conservative); every microphone test and contribution in
 *   float64 (the apex exact, cone normals to about 48 bits); band powers
 *   W_b prod(r_b) in float32; float64 accumulation.  Slower: GB300 issues
 *   float64 at a small fraction of the float32 rate.
 * BT_PREC_MIXED64: float32 traversal and hit tests as in MIXED (ambiguous
 *   tests and near ties settled in float64), the image-source chain in
 *   float64 as in FP64, microphone tests as in MIXED, float64 accumulation:
 *   float64 only where the chain's stability needs it. */
#define BT_PREC_FP32 0
#define BT_PREC_MIXED 1
#define BT_PREC_FP64 2
#define BT_PREC_MIXED64 3

typedef struct bt_ctx bt_ctx;

/* Parameters of one trace.  Start from bt_params_default(). */
typedef struct {
  int32_t max_order;                        /* K: reflections traced, orders 0..K (0..32) */
  float air_atten_db_per_m[BT_MAX_BANDS];   /* air damping per band, dB/m (Section 2); default 0 */
  float energy_threshold_w;                 /* delete a reflected beam whose largest per-band
                                               power W_b*prod(r_b) falls below this; 0 = off */
  float t_eps_m;                            /* self-hit guard, metres; default 1e-3 */
  int32_t tiles_x, tiles_y;                 /* sub-domain grid over the scene's xy box
                                               (Section 3); 1 x 1 = no split; max 32 x 32 */
  int32_t precision;                        /* BT_PREC_* */
  int32_t watchdog_ms;                      /* bound on any device-side wait; default 2000 */
  int32_t chunk_beams;                      /* beam lineages per persistent launch; 0 = automatic
                                               (room for (max_order + 1) segment records of
                                               192 B per lineage within a quarter of the free
                                               device memory, clamped to 1..32 GiB) */
  int32_t count_work;                       /* 1: also count BVH nodes visited and triangles
                                               tested (slower; for roofline accounting) */
  int32_t blocks_per_sm;                    /* resident blocks per SM of the persistent trace
                                               kernels; 0 = as many as fit (tuning knob) */
  int32_t queue_depth;                      /* hand-off queue slots per sub-domain, a power of
                                               two in 32..2^22, or 0 = automatic (at least
                                               twice the lanes of one launch); also the most
                                               lineages in flight at once, so that no queue
                                               can overflow */
  int32_t leaf_size;                        /* most triangles per BVH leaf, 1..4 (0 = 1): a
                                               subtree of the LBVH holding at most this many
                                               triangles is tested as one leaf (tuning knob;
                                               the hits do not depend on it) */
  int32_t beams_per_warp;                   /* beam lineages a warp of the persistent trace
                                               reserves from the launch's lineage counter at a
                                               time and hands to its lanes as they free up: 0
                                               (as many as lanes need) or a multiple of 32 up
                                               to 4096 (tuning knob) */
  int32_t fault_test;                       /* test hook, 0 in normal use.  BT_FAULT_WITHHOLD:
                                               the sub-domain trace withholds the publication
                                               of its first hand-off, so the bounded wait of
                                               its consumer runs out (BT_E_TIMEOUT);
                                               BT_FAULT_SEGMENTS: the segment buffer gets room
                                               for one record (BT_E_QUEUE_FULL) */
} bt_trace_params;
#define BT_FAULT_WITHHOLD 1
#define BT_FAULT_SEGMENTS 2

/* Counters of the last trace of a scene. */
typedef struct {
  int64_t beams;          /* primary beams launched: n_sources * 20 * 4^L */
  int64_t segments;       /* beam segments traced (one per axis-ray query) */
  int64_t hits;           /* segments whose axis ray hit a triangle */
  int64_t escapes;        /* segments whose axis ray left the scene */
  int64_t emitted;        /* segments handed to the microphone scatter (those whose cone can
                             reach the microphones' height range) */
  int64_t candidates;     /* microphones tested against a segment */
  int64_t contributions;  /* (microphone, segment) pairs inside the beam */
  int64_t handoffs;       /* rays passed from one sub-domain to the next through its queue */
  int64_t steals;         /* hand-offs served by a warp whose home is another sub-domain */
  int64_t rounds;         /* persistent sub-domain launches (one per batch of lineages) */
  int64_t nodes_visited;  /* BVH nodes fetched (only with count_work) */
  int64_t tris_tested;    /* triangles tested (only with count_work) */
  int64_t trace_launches; /* launches of the traversal kernel */
  int64_t scatter_launches; /* launches of the microphone scatter kernel */
  double trace_ms;        /* device time of the whole trace (CUDA events) */
  double trace_kernel_ms; /* summed device time of the traversal kernel launches */
  double scatter_kernel_ms; /* summed device time of the scatter kernel launches */
} bt_stats;

/* Fill *p with the defaults: K = 4, no air damping, no threshold, t_eps = 1 mm,
 * 1 x 1 tiles, BT_PREC_MIXED, watchdog 2000 ms, automatic chunking. */
int bt_params_default(bt_trace_params *p);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on, or NULL for a stream owned by the context.  On success *out owns
 * all device memory of the context. */
int bt_create(bt_ctx **out, int device, void *cuda_stream);

/* Free every resource of the context (waits for its stream first).  NULL is a
 * no-op. */
int bt_destroy(bt_ctx *ctx);

/* Load a city model (Section 4: buildings and ground as triangles) and build
 * its acceleration structure on the device (Section 2: the guiding ray is
 * resolved by efficient ray shooting).
 *   verts        [n_verts][3] float32, metres
 *   tris         [n_tris][3] int32 vertex indices, 0 <= index < n_verts
 *   tri_material [n_tris] uint8, < n_materials
 *   refl         [n_materials][n_bands] float32 energy reflection coefficients in [0, 1]
 *   n_bands      1..BT_MAX_BANDS
 * *scene_id_out receives the new scene's id (0..BT_MAX_SCENES-1).  Errors:
 * BT_E_INVALID for NaN/inf coordinates, indices or materials out of range,
 * coefficients outside [0, 1]; BT_E_NOMEM; BT_E_CUDA. */
int bt_load_scene(bt_ctx *ctx, const float *verts, int64_t n_verts, const int32_t *tris,
                  int64_t n_tris, const uint8_t *tri_material, const float *refl,
                  int32_t n_materials, int32_t n_bands, int32_t *scene_id_out);

/* Drop a scene and its device memory. */
int bt_unload_scene(bt_ctx *ctx, int32_t scene_id);

/* Point sources of a scene (Section 4: car traffic sources).
 *   pos     [n_s][3] float32
 *   power_w [n_s][n_bands] float32 acoustic power per band, >= 0
 *   icosa_level L in 0..8: each source emits 20 * 4^L beams, one per face of
 *   a geodesic icosahedron, each carrying power_w * (solid angle / 4 pi)
 *   (Section 2: the source energy is split between beams by direction). */
int bt_set_sources(bt_ctx *ctx, int32_t scene_id, const float *pos, const float *power_w,
                   int64_t n_s, int32_t icosa_level);

/* Directional sources (Section 2: a source's energy is split between the
 * beams by its power in each direction).
 *   patterns   [n_patterns][20 * 4^L] float32 gains >= 0, one per beam of the
 *              scene's icosahedron level L, in the beam order of bt_beam_axes
 *   pattern_of [n_src] int32: each source's pattern, -1 = omnidirectional
 * A beam's band powers are the source's power_w times its pattern's gain for
 * the beam (a pattern whose gains average 1 over the sphere, weighted by the
 * beams' solid angles, keeps the source's total power).  Host or device
 * pointers; copied before the call returns.  n_patterns = 0 (the arrays may
 * then be NULL) makes every source omnidirectional again, and so does every
 * bt_set_sources.  Errors: BT_E_STATE before bt_set_sources; BT_E_INVALID for
 * NULL arrays, a negative or non-finite gain, or a pattern index outside
 * -1..n_patterns-1 (the scene then stays omnidirectional). */
int bt_set_directivity(bt_ctx *ctx, int32_t scene_id, const float *patterns, int32_t n_patterns,
                       const int32_t *pattern_of);

/* Unit axis (float32, [20 * 4^L][3], host or device) of every beam of
 * icosahedron level L in 0..8, in the order bt_set_directivity's gains use:
 * beam i lies in base face i >> 2L and is refined by the base-4 digits of
 * the rest of i (corner-0, corner-1, corner-2, centre child). */
int bt_beam_axes(bt_ctx *ctx, int32_t icosa_level, float *axes);

/* Microphones of a scene (Section 4: a regular grid of receivers, filling a
 * volume or a plane).
 *   pos [n_m][3] float32, n_m <= 2^28.  They are binned on the device into an
 *   xy cell grid with up to 64 height layers (Section 3: microphones are
 *   partitioned with the geometry).  The scene's accumulated result starts
 *   at zero.  Errors: BT_E_INVALID for NaN/inf positions. */
int bt_set_microphones(bt_ctx *ctx, int32_t scene_id, const float *pos, int64_t n_m);

/* Trace every beam of every source of the scene (Section 2, hybrid method)
 * and accumulate per-microphone, per-band intensity.  Replaces the result of
 * any earlier trace of the scene.  Errors: BT_E_STATE when sources or
 * microphones are missing; BT_E_INVALID for bad parameters;
 * BT_E_QUEUE_FULL / BT_E_TIMEOUT from the sub-domain scheduler. */
int bt_trace(bt_ctx *ctx, int32_t scene_id, const bt_trace_params *p);

/* Asynchronous trace: bt_submit enqueues the same work as bt_trace (Section
 * 2's trace; the asynchrony has no counterpart in the paper) on the
 * context's stream and returns without waiting for the GPU, so the caller's
 * thread is free while the scene is traced.  bt_poll returns BT_PENDING while
 * the trace runs and BT_OK once it has finished (its result and stats are then
 * read with bt_read_levels); bt_wait blocks until it has finished.  A failed
 * trace makes both return its error code (BT_E_QUEUE_FULL, BT_E_TIMEOUT,
 * BT_E_CUDA), as bt_trace would have; they keep returning the outcome of the
 * scene's last trace until the next one is submitted, and BT_E_STATE when the
 * scene was never traced.  Submissions on several scenes run one after the
 * other on the stream.  Any other call that names a scene with a trace in
 * flight first waits for that trace, so calls take effect in the order they
 * were made.  bt_submit may itself wait for earlier work on the stream when
 * it builds a scene's sub-domain hierarchy or allocates.  Errors of
 * bt_submit: those of bt_trace that are found before any GPU work (bad
 * parameters, missing sources or microphones, allocation). */
int bt_submit(bt_ctx *ctx, int32_t scene_id, const bt_trace_params *p);
int bt_poll(bt_ctx *ctx, int32_t scene_id);
int bt_wait(bt_ctx *ctx, int32_t scene_id);

/* Read the result of the last trace of the scene.
 *   level_db  [n_m][n_bands] float64: 10 log10(I / 1e-12 W/m^2), -inf where no
 *             beam reached the microphone (Section 4: sound level distribution)
 *   intensity [n_m][n_bands] float64 W/m^2, may be NULL
 *   path_count [n_m] int32 beam segments that contained the microphone, may be NULL
 *   stats     may be NULL
 * level_db may also be NULL when only the other outputs are wanted. */
int bt_read_levels(bt_ctx *ctx, int32_t scene_id, double *level_db, double *intensity,
                   int32_t *path_count, bt_stats *stats);

/* Closest hit of arbitrary rays in the scene's acceleration structure: the
 * axis-ray query of bt_trace on its own (Section 2: only the guiding ray of a
 * beam is tested).
 *   origins, dirs  [n][3] float32 (dirs are normalised by the library)
 *   start_normals  [n][3] float32 or NULL: for a ray leaving a reflector, the
 *                  reflector's normal; hits closer than t_eps_m to that plane
 *                  are then ignored, as in bt_trace
 *   t_out          [n] float32 hit distance (formed in float64 along the
 *                  normalised ray to the hit triangle's plane), +inf on a miss
 *   tri_out        [n] int32 index of the hit triangle in the scene's input
 *                  order, -1 on a miss; equal distances go to the lowest index
 * Hits with distance <= t_eps_m are ignored. */
int bt_cast_rays(bt_ctx *ctx, int32_t scene_id, const float *origins, const float *dirs,
                 const float *start_normals, int64_t n, float t_eps_m, float *t_out,
                 int32_t *tri_out);

/* Trace without allocating (the paper has no counterpart).  For callers that
 * must not call cudaMalloc or cudaFree during a trace: a service running
 * under a device-memory budget fixed up front, where another framework's pool
 * owns the rest of the GPU and a new allocation could fail part-way; or a
 * per-frame update loop, where cudaMalloc and cudaFree synchronise the device
 * and stall every other stream.  The scene, its sources and microphones must
 * already be set (those calls allocate); this call then allocates nothing.
 * It computes what bt_trace followed by bt_read_levels gives, and like
 * bt_trace it replaces the scene's last result (bt_read_levels and the stats
 * then refer to it).
 *   level_db   [n_m][n_bands] float64, DEVICE memory of the context's GPU
 *   path_count [n_m] int32, device memory, or NULL
 * The parameters are checked as bt_trace checks them; in addition only
 * tiles_x = tiles_y = 1 is accepted (this call traces without sub-domains,
 * so queue_depth is not used), and chunk_beams, when > 0, can only lower the
 * lineages per launch below what the scratch holds.  count_work fills the
 * stats' work counters as in bt_trace.
 * Its scratch is one static device array of BT_NOALLOC_SCRATCH_MB MiB inside
 * the library, held on every GPU that loads the library until the process
 * exits.  The icosahedron level must be <= BT_NOALLOC_MAX_LEVEL (the beam table
 * lives in that scratch), and (max_order + 1) segment records must fit in
 * it; larger requests, and tiles other than 1x1, fail with BT_E_INVALID and
 * say so.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call, from any context, shares the one
 * array and clears what must start at zero; calls whose device work overlaps
 * (different streams or host threads) race on it. */
#define BT_NOALLOC_SCRATCH_MB 32
#define BT_NOALLOC_MAX_LEVEL 6
int bt_trace_noalloc(bt_ctx *ctx, int32_t scene_id, const bt_trace_params *p, double *level_db,
                     int32_t *path_count);

/* Hit log of a scene's traces (the paper has no counterpart: a measurement
 * aid for precision studies, which hit decisions differ between variants).
 * Registers the caller's DEVICE array hits[n] (int32, device memory of the
 * context's GPU); every later bt_trace / bt_submit of the scene writes, per
 * segment, hits[lineage * (max_order + 1) + order] = the input index of the
 * triangle the segment's axis ray hit, or -1 if it escaped; entries of orders
 * a lineage does not reach are left as they were.  Lineage = source *
 * 20 * 4^L + beam, beams in the order of bt_beam_axes.  A trace whose
 * lineages x (max_order + 1) exceed n fails with BT_E_INVALID.  Batches,
 * range traces and bt_trace_noalloc do not write it.  hits = NULL clears the
 * log.  The array must outlive the traces that write it. */
int bt_set_hit_log(bt_ctx *ctx, int32_t scene_id, int32_t *hits, int64_t n);

/* Install a trace result computed elsewhere into a scene, replacing its last
 * result: the sum of the partial results of traces of disjoint subsets of the
 * scene's sources (Section 3: processes trace their own beams and their
 * results are gathered; beams of different sources never interact, so the
 * sum over source shards is the result for all sources).  A caller splits
 * the sources over contexts or GPUs, reads each partial with bt_read_levels
 * (intensity, path_count), sums them (e.g. an all-reduce), installs the sum
 * here, and reads the levels with bt_read_levels.
 *   intensity  [n_m][n_bands] float64, W/m^2, input microphone order
 *   path_count [n_m] int32, or NULL for zero counts
 * The scene's microphones must be set (BT_E_STATE otherwise).  Stats of the
 * scene are zeroed. */
int bt_set_result(bt_ctx *ctx, int32_t scene_id, const double *intensity, const int32_t *path_count);

/* Batches (the paper has none: it traces one city at a time).  Several
 * loaded scenes -- cities of uneven size, each with its own sources,
 * microphones and parameters -- traced together: every run issues one
 * persistent trace launch and one scatter launch per group of lineages drawn
 * from all scenes, the whole sequence captured once as a CUDA graph and
 * replayed by every later run.  Each scene's result is then read with
 * bt_read_levels as after bt_trace.
 *   scene_ids  [n_scenes] distinct loaded scenes with sources and microphones
 *   params     [n_scenes] per-scene parameters; tiles must be 1x1, and
 *              precision, count_work, blocks_per_sm and chunk_beams must agree
 * The batch reads the scenes' device buffers in place: after bt_load_scene,
 * bt_set_sources, bt_set_directivity, bt_set_microphones or bt_unload_scene on
 * any of its scenes,
 * bt_batch_run fails with BT_E_STATE (create a new batch).  bt_batch_run
 * synchronises the context's stream; the context's stream must not be in
 * stream capture.  Batches are freed by bt_batch_destroy or with the
 * context. */
typedef struct bt_batch bt_batch;
int bt_batch_create(bt_ctx *ctx, const int32_t *scene_ids, int32_t n_scenes, const bt_trace_params *params,
                    bt_batch **batch_out);
int bt_batch_run(bt_batch *batch);
/* Totals of the last run (per-scene stats hold only `beams`); trace_ms is
 * the device time of the whole run. */
int bt_batch_stats(const bt_batch *batch, bt_stats *stats);
int bt_batch_destroy(bt_batch *batch);

/* A new scene that shares the geometry (triangles, BVH, materials) of a
 * loaded scene without copying it, for its own sources and microphones: one
 * resident city serves many queries.  The base scene cannot be unloaded
 * while shares remain (BT_E_STATE); unloading a share frees only its own
 * buffers. */
int bt_scene_share(bt_ctx *ctx, int32_t base_scene_id, int32_t *scene_id_out);

/* Trace part of the lineages of several scenes together: for scene i the
 * lineages lineage_begin[i] .. lineage_end[i]-1, numbered source-major
 * (lineage = source * 20 * 4^L + beam), all in the same persistent launches
 * (each lane on its own lineage's scene; Section 2's method for every
 * scene).  With BT_ACCUMULATE the contributions are added to each scene's
 * current result instead of replacing it, so a scene's lineages can be
 * traced over several calls -- the step of a continuous-batching server.
 * params[i] as for bt_trace (tiles 1x1; precision, blocks_per_sm and
 * count_work must agree).  One scene (n = 1) runs the single-scene kernels,
 * several the batch kernels.  Synchronous; totals with bt_ranges_stats. */
#define BT_ACCUMULATE 1
int bt_trace_ranges(bt_ctx *ctx, int32_t n, const int32_t *scene_ids, const int64_t *lineage_begin,
                    const int64_t *lineage_end, const bt_trace_params *params, int32_t flags);
int bt_ranges_stats(const bt_ctx *ctx, bt_stats *stats);

/* Message of the last error of the context ("" if none).  Valid until the
 * next call on the context. */
const char *bt_last_error(const bt_ctx *ctx);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts).  Lets a caller count the kernels inside a timed region. */
int64_t bt_kernel_launches(void);

/* Measured L2 read bandwidth of the context's GPU, GB/s (the paper has no
 * counterpart: a measurement aid).  Reads a `bytes`-byte device buffer
 * (16 MiB..96 MiB, small enough to stay resident in L2) `repeats` times
 * (1..10000) in one kernel, with loads cached in L2 only, on a grid of
 * `blocks_per_sm` blocks of 256 threads per SM (1..8), and returns the bytes
 * read over the kernel's CUDA-event time.  The traversal's node, triangle and
 * plane arrays stay in L2, so this is the roof its L2 traffic is reported
 * against.  Allocates the buffer from the context's pool; synchronous. */
int bt_l2_bandwidth(bt_ctx *ctx, int64_t bytes, int32_t repeats, int32_t blocks_per_sm, double *gbs_out);

/* Measured rate of float64 atomic additions in the L2 of the context's GPU,
 * additions per second (the paper has no counterpart: a measurement aid).
 * Every thread of a grid of `blocks_per_sm` blocks of 256 threads per SM
 * (1..8) adds to the eight consecutive doubles of a 64-byte slot `repeats`
 * times (1..10000), at slots spread over a `bytes`-byte device buffer
 * (16 MiB..96 MiB, a multiple of 64, small enough to stay resident in L2):
 * the pattern of the scatter's band accumulators, which take every
 * contribution as eight float64 atomic additions.  Returns the additions
 * over the kernel's CUDA-event time in *ops_out.  Allocates the buffer from
 * the context's pool; synchronous. */
int bt_l2_atomics(bt_ctx *ctx, int64_t bytes, int32_t repeats, int32_t blocks_per_sm, double *ops_out);

#ifdef __cplusplus
}
#endif

#endif /* BTRACE_H */
