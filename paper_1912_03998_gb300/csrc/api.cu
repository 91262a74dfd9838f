// api.cu -- the C ABI of libbtrace (declared in include/btrace.h).
//
// Host code only arranges memory and launches; every step of the trace runs
// in the kernels of build.cu and trace.cu.  All device work of a context is
// ordered on the context's stream.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <utility>
#include <vector>

#include "bt_internal.cuh"

#define BT_API extern "C" __attribute__((visibility("default")))

#include <nvtx3/nvToolsExt.h>

namespace {
// An NVTX range named after the entry point, open while the call runs, so
// that profilers can attribute kernels and copies to library calls (ncu
// --nvtx, Nsight Systems); without an attached tool it costs one pointer test.
struct ApiRange {
  explicit ApiRange(const char *name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
  ApiRange(const ApiRange &) = delete;
  ApiRange &operator=(const ApiRange &) = delete;
};
}  // namespace
#define BT_RANGE() ApiRange bt_range_(__func__)

namespace bt {
static std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace bt

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

struct SceneState {
  bool used = false;
  int64_t n_tris = 0;
  int n_mat = 0, n_bands = 0;
  int root = -1;
  float box[6] = {0, 0, 0, 0, 0, 0};
  DevBuf nodes, tris, planes, planes64, planes_df, refl;
  // sources
  bool has_src = false;
  int64_t n_src = 0;
  int level = 0;
  DevBuf src, power;
  int n_pat = 0;           // directional sources: patterns in dir_gain (0 = all omnidirectional)
  DevBuf dir_gain, dir_of;
  // microphones
  bool has_mics = false;
  int64_t n_mics = 0;
  int side = 1, nz = 1;
  DevBuf mics, cell_start, grid, energy, count;
  // tiled hierarchy (sub-domains), built on the first trace that asks for it
  int tiled_tx = 0, tiled_ty = 0;
  int64_t n_pairs = 0;
  bt::TileGrid tg;
  DevBuf t_nodes, t_tris, t_planes, t_planes64, t_planes_df, t_roots;
  // result
  bool traced = false;
  bool pending = false;  // a bt_submit trace is in flight
  int trace_error = 0;   // error code of the last trace (0 = none)
  bt_stats stats;
  unsigned long long gen = 0;  // changes whenever the scene's buffers may change (batches check it)
  int geom_of = -1;            // >= 0: the geometry buffers belong to that scene (bt_scene_share)
  int leaf = 1, t_leaf = 1;    // leaf size the flat and the tiled hierarchy are collapsed to
  int32_t *hit_log = nullptr;  // bt_set_hit_log: caller's device array, or null
  int64_t hit_log_n = 0;
  int n_shares = 0;            // scenes sharing this scene's geometry
  DevBuf out_level, out_int, out_cnt;
};

// A scene slot's trace: events around the whole trace and around each kernel
// launch (kind 0 traversal, 1 scatter), launch counts, and the event that
// marks its counters copied to the host.  Kept per slot so that traces of
// several scenes can be in flight on the context's stream (bt_submit).
struct TraceRec {
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, done = nullptr;
  std::vector<cudaEvent_t> kev;
  std::vector<int> kind;  // kind of each pair of events in kev
  int64_t beams = 0, trace_launches = 0, scatter_launches = 0, rounds = 0;
};

}  // namespace

struct bt_batch;

struct bt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_sm = 1;
  SceneState sc[BT_MAX_SCENES];
  char err[512] = {0};
  DevBuf scratch, stage_a, stage_b, stage_c, segs;
  DevBuf seg_order, order_hist;  // scatter in order of place (scenes with many microphones)
  DevBuf beam_table;       // cone normals + axis per beam of one icosahedron level, float pairs
  int beam_table_level = -1;
  bt::Counters *d_ctr = nullptr;
  bt::Counters *h_ctr = nullptr;  // pinned
  bt::Counters *h_sctr = nullptr; // pinned, one per scene slot: counters of the slot's last trace
  TraceRec rec[BT_MAX_SCENES];
  unsigned long long *d_seg_count = nullptr;
  unsigned long long *d_lineage_next = nullptr;
  float *d_box = nullptr;  // scene box of the scene being loaded (6 floats)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<DevBuf> pool;      // released device buffers, reused before any new cudaMalloc
  DevBuf t_ring, t_seq, t_qctl;  // sub-domain trace: queue slots, slot sequence words, queue counters
  unsigned long long gen_counter = 0;
  std::vector<bt_batch *> batches;  // live batches, freed with the context
  DevBuf views;                     // scene views of the last bt_trace_ranges
  DevBuf level_tables[9];           // float-pair beam tables per icosahedron level (bt_trace_ranges)
  bt_stats range_stats;             // totals of the last bt_trace_ranges
};

namespace {

int fail(bt_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

struct DeviceGuard {
  int prev = -1, want;
  explicit DeviceGuard(int d) : want(d) {
    cudaGetDevice(&prev);
    if (prev != want) cudaSetDevice(want);
  }
  ~DeviceGuard() {
    if (prev >= 0 && prev != want) cudaSetDevice(prev);
  }
};

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, e_ == cudaErrorMemoryAllocation ? BT_E_NOMEM : BT_E_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

// Grow-only device buffer.  A buffer that is too small goes back to the
// context's pool; the smallest pooled buffer that fits is taken before any new
// allocation.  Every user of a buffer runs on the context's one stream, so a
// reused buffer is only touched after the work that used it before.
int ensure(bt_ctx *c, DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (b.cap >= bytes) return BT_OK;
  if (b.p) {
    c->pool.push_back(b);
    b = DevBuf();
  }
  int best = -1;
  for (int i = 0; i < (int)c->pool.size(); i++)
    if (c->pool[i].cap >= bytes && (best < 0 || c->pool[i].cap < c->pool[best].cap)) best = i;
  if (best >= 0) {
    b = c->pool[best];
    c->pool.erase(c->pool.begin() + best);
    return BT_OK;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    // give the pool back to the device and retry once
    CK(cudaStreamSynchronize(c->stream));
    for (DevBuf &q : c->pool) cudaFree(q.p);
    c->pool.clear();
    e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b = DevBuf();
      return fail(c, BT_E_NOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  b.cap = bytes;
  return BT_OK;
}

void release(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

// Scene buffers go back to the context's pool (freed by bt_destroy).
void release_scene(bt_ctx *c, SceneState &s) {
  DevBuf *own[] = {&s.t_nodes, &s.t_tris, &s.t_planes, &s.t_planes64, &s.t_planes_df, &s.t_roots, &s.src,
                   &s.power, &s.dir_gain, &s.dir_of, &s.mics, &s.cell_start, &s.grid, &s.energy, &s.count,
                   &s.out_level, &s.out_int, &s.out_cnt};
  DevBuf *geom[] = {&s.nodes, &s.tris, &s.planes, &s.planes64, &s.planes_df, &s.refl};
  for (DevBuf *b : own)
    if (b->p) c->pool.push_back(*b);
  if (s.geom_of >= 0) {
    c->sc[s.geom_of].n_shares--;  // the geometry stays with its owner
  } else {
    for (DevBuf *b : geom)
      if (b->p) c->pool.push_back(*b);
  }
  s = SceneState();
}

#define TRY(x)                 \
  do {                         \
    int r_ = (x);              \
    if (r_ != BT_OK) return r_; \
  } while (0)

int check_ctx(bt_ctx *c) { return c ? BT_OK : BT_E_INVALID; }

// True if p is device (or managed) memory of device `device`.
bool is_device_ptr(const void *p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}


bt::DevScene dev_scene(const SceneState &s) {
  bt::DevScene d;
  memset(&d, 0, sizeof(d));
  d.n_tris = s.n_tris;
  d.root = s.root;
  d.nodes = bt::hier_wide(s.nodes.p, s.n_tris);
  d.tris = (const bt::Tri *)s.tris.p;
  d.planes = (const bt::Plane *)s.planes.p;
  d.planes64 = (const bt::Plane64 *)s.planes64.p;
  d.planes_df = (const bt::PlaneDF *)s.planes_df.p;
  d.refl = (const float *)s.refl.p;
  d.n_mat = s.n_mat;
  d.n_bands = s.n_bands;
  for (int k = 0; k < 3; k++) { d.lo[k] = s.box[k]; d.hi[k] = s.box[3 + k]; }
  return d;
}

// Finish the bt_submit trace of scene slot `id`, if one is in flight: with
// `wait`, block until it is done, else return BT_PENDING while it runs.  A
// finished trace's stats are filled from its events and counters.  With
// `report` a failure is also written to the context's message; without, it is
// only kept in the scene (trace_error) for bt_poll and bt_read_levels.
int collect(bt_ctx *c, int id, bool wait, bool report) {
  SceneState &s = c->sc[id];
  if (!s.pending) return BT_OK;
  TraceRec &r = c->rec[id];
  DeviceGuard g(c->device);
  cudaError_t e = wait ? cudaEventSynchronize(r.done) : cudaEventQuery(r.done);
  if (e == cudaErrorNotReady && !wait) {
    cudaGetLastError();  // not an error: leave no trace in the runtime's last-error state
    return BT_PENDING;
  }
  s.pending = false;
  s.traced = false;
  float ms = 0.0f;
  double trace_kms = 0.0, scatter_kms = 0.0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.ev0, r.ev1);
  for (size_t q = 0; e == cudaSuccess && q + 1 < r.kev.size() && q / 2 < r.kind.size(); q += 2) {
    float a = 0.0f;
    e = cudaEventElapsedTime(&a, r.kev[q], r.kev[q + 1]);
    if (r.kind[q / 2] == 0) trace_kms += a;
    else scatter_kms += a;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    s.trace_error = BT_E_CUDA;
    return report ? fail(c, BT_E_CUDA, "trace of scene %d: %s", id, cudaGetErrorString(e)) : BT_E_CUDA;
  }
  const bt::Counters &h = c->h_sctr[id];
  bt_stats &o = s.stats;
  memset(&o, 0, sizeof(o));
  o.beams = r.beams;
  o.segments = (int64_t)h.segments;
  o.hits = (int64_t)h.hits;
  o.escapes = (int64_t)h.escapes;
  o.emitted = (int64_t)h.emitted;
  o.candidates = (int64_t)h.candidates;
  o.contributions = (int64_t)h.contributions;
  o.handoffs = (int64_t)h.handoffs;
  o.steals = (int64_t)h.steals;
  o.rounds = r.rounds;
  o.nodes_visited = (int64_t)h.nodes_visited;
  o.tris_tested = (int64_t)h.tris_tested;
  o.trace_launches = r.trace_launches;
  o.scatter_launches = r.scatter_launches;
  o.trace_ms = ms;
  o.trace_kernel_ms = trace_kms;
  o.scatter_kernel_ms = scatter_kms;
  if (h.error) {
    s.trace_error = h.error;
    if (!report) return h.error;
    return fail(c, h.error, h.error == BT_E_QUEUE_FULL ? "device queue or traversal stack overflow"
                                                       : "device error %d", h.error);
  }
  s.trace_error = 0;
  s.traced = true;
  return BT_OK;
}

// The scene `id`; a bt_submit trace of it still in flight is waited for first,
// so every call sees the scene as if the submitted trace had been synchronous.
int scene_ref(bt_ctx *c, int32_t id, SceneState **out) {
  if (id < 0 || id >= BT_MAX_SCENES || !c->sc[id].used)
    return fail(c, BT_E_INVALID, "unknown scene id %d", id);
  if (c->sc[id].pending) collect(c, id, true, false);
  *out = &c->sc[id];
  return BT_OK;
}

// Reset the sticky kernel error word and the counters.
int reset_counters(bt_ctx *c) {
  CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(bt::Counters), c->stream));
  return BT_OK;
}

int read_counters(bt_ctx *c) {
  CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(bt::Counters), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return BT_OK;
}

// ---------------------------------------------------------------- packing
__global__ void k_pack_sources(const float *pos, const float *power, int64_t n, int n_bands, float4 *src,
                               float *pw, int *error) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicExch(error, BT_E_INVALID);
  src[i] = make_float4(x, y, z, 0.0f);
  for (int b = 0; b < n_bands; b++) {
    float w = power[i * n_bands + b];
    if (!isfinite(w) || w < 0.0f) atomicExch(error, BT_E_INVALID);
    pw[i * n_bands + b] = w;
  }
}

// Directional source patterns: every gain finite and >= 0, every source's
// pattern index in -1..n_pat-1.
__global__ void k_check_directivity(const float *gain, int64_t n_gain, const int *of, int64_t n_src, int n_pat,
                                    int *error) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n_gain && !(isfinite(gain[i]) && gain[i] >= 0.0f)) atomicExch(error, BT_E_INVALID);
  if (i < n_src && (of[i] < -1 || of[i] >= n_pat)) atomicExch(error, BT_E_INVALID);
}


// Tiled hierarchy of a scene for a tx x ty sub-domain grid (cached until the
// grid changes or the scene is dropped).
int ensure_tiled(bt_ctx *c, SceneState &s, int tx, int ty) {
  if (s.tiled_tx == tx && s.tiled_ty == ty) return BT_OK;
  cudaStream_t st = c->stream;
  bt::TileGrid tg;
  tg.gx0 = s.box[0] - 1.0f;
  tg.gy0 = s.box[1] - 1.0f;
  tg.gx1 = s.box[3] + 1.0f;
  tg.gy1 = s.box[4] + 1.0f;
  tg.wx = (tg.gx1 - tg.gx0) / tx;
  tg.wy = (tg.gy1 - tg.gy0) / ty;
  tg.tx = tx;
  tg.ty = ty;
  const int T = tx * ty;
  s.tiled_tx = s.tiled_ty = 0;
  TRY(ensure(c, s.t_roots, sizeof(int) * T));
  int64_t P = 0;
  if (s.n_tris > 0) {
    CK(cudaMemcpyAsync(c->d_box, s.box, sizeof(float) * 6, cudaMemcpyHostToDevice, st));
    TRY(ensure(c, c->scratch, sizeof(uint32_t) * (size_t)(s.n_tris + 1) + 256));
    CK(bt::tiled_count(st, (const bt::Tri *)s.tris.p, s.n_tris, tg, (uint32_t *)c->scratch.p));
    uint32_t pairs = 0;
    CK(cudaMemcpyAsync(&pairs, (uint32_t *)c->scratch.p + s.n_tris, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    P = pairs;
    // the offsets stay at the start of the scratch; grow it without losing them
    size_t need = bt::build_tiled_scratch_bytes(s.n_tris, P);
    if (c->scratch.cap < need) {
      DevBuf fresh;
      TRY(ensure(c, fresh, need));
      CK(cudaMemcpyAsync(fresh.p, c->scratch.p, sizeof(uint32_t) * (size_t)(s.n_tris + 1), cudaMemcpyDeviceToDevice, st));
      c->pool.push_back(c->scratch);
      c->scratch = fresh;
    }
    TRY(ensure(c, s.t_nodes, bt::hier_bytes(P)));
    TRY(ensure(c, s.t_tris, sizeof(bt::Tri) * (size_t)P));
    TRY(ensure(c, s.t_planes, sizeof(bt::Plane) * (size_t)P));
    TRY(ensure(c, s.t_planes64, sizeof(bt::Plane64) * (size_t)P));
    TRY(ensure(c, s.t_planes_df, sizeof(bt::PlaneDF) * (size_t)P));
    CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(bt::Counters), st));
    CK(bt::tiled_build(st, (const bt::Tri *)s.tris.p, (const bt::Plane *)s.planes.p, (const bt::Plane64 *)s.planes64.p,
                       (const bt::PlaneDF *)s.planes_df.p, s.n_tris, tg, c->d_box, (const uint32_t *)c->scratch.p, P,
                       c->scratch.p, c->scratch.cap, s.t_nodes.p, (bt::Tri *)s.t_tris.p,
                       (bt::Plane *)s.t_planes.p, (bt::Plane64 *)s.t_planes64.p, (bt::PlaneDF *)s.t_planes_df.p,
                       (int *)s.t_roots.p, &c->d_ctr->error));
  } else {
    std::vector<int> empty(T, (int)0x80000000);
    CK(cudaMemcpyAsync(s.t_roots.p, empty.data(), sizeof(int) * T, cudaMemcpyHostToDevice, st));
  }
  TRY(read_counters(c));
  if (c->h_ctr->error) return fail(c, BT_E_CUDA, "tiled hierarchy build failed (device error %d)", c->h_ctr->error);
  s.n_pairs = P;
  s.tg = tg;
  s.tiled_tx = tx;
  s.tiled_ty = ty;
  return BT_OK;
}

}  // namespace

// ====================================================================== ABI
BT_API int bt_params_default(bt_trace_params *p) {
  if (!p) return BT_E_INVALID;
  memset(p, 0, sizeof(*p));
  p->max_order = 4;
  p->t_eps_m = 1e-3f;
  p->tiles_x = 1;
  p->tiles_y = 1;
  p->precision = BT_PREC_MIXED;
  p->watchdog_ms = 2000;
  return BT_OK;
}

BT_API int bt_create(bt_ctx **out, int device, void *cuda_stream) {
  BT_RANGE();
  if (!out) return BT_E_INVALID;
  *out = nullptr;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return BT_E_CUDA;
  }
  bt_ctx *c = new (std::nothrow) bt_ctx();
  if (!c) return BT_E_NOMEM;
  c->device = device;
  DeviceGuard g(device);
  int rc = BT_OK;
  do {
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      rc = BT_E_CUDA;
      break;
    }
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = BT_E_CUDA; break; }
      c->own_stream = true;
    }
    if (cudaMalloc(&c->d_ctr, sizeof(bt::Counters)) != cudaSuccess) { rc = BT_E_NOMEM; break; }
    if (cudaMalloc(&c->d_seg_count, sizeof(unsigned long long)) != cudaSuccess) { rc = BT_E_NOMEM; break; }
    if (cudaMalloc(&c->d_box, 8 * sizeof(float)) != cudaSuccess) { rc = BT_E_NOMEM; break; }
    if (cudaMalloc(&c->d_lineage_next, sizeof(unsigned long long)) != cudaSuccess) { rc = BT_E_NOMEM; break; }
    if (cudaMallocHost(&c->h_ctr, sizeof(bt::Counters)) != cudaSuccess) { rc = BT_E_NOMEM; break; }
    if (cudaMallocHost(&c->h_sctr, sizeof(bt::Counters) * BT_MAX_SCENES) != cudaSuccess) { rc = BT_E_NOMEM; break; }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) { rc = BT_E_CUDA; break; }
  } while (0);
  if (rc != BT_OK) {
    cudaGetLastError();
    bt_destroy(c);
    return rc;
  }
  *out = c;
  return BT_OK;
}

static void free_batch(bt_batch *b);

BT_API int bt_destroy(bt_ctx *c) {
  BT_RANGE();
  if (!c) return BT_OK;
  DeviceGuard g(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (bt_batch *b : c->batches) free_batch(b);
  c->batches.clear();
  release(c->views);
  for (DevBuf &t : c->level_tables) release(t);
  for (auto &s : c->sc) release_scene(c, s);
  for (DevBuf &q : c->pool) release(q);
  c->pool.clear();
  release(c->scratch);
  release(c->stage_a);
  release(c->stage_b);
  release(c->stage_c);
  release(c->segs);
  release(c->seg_order);
  release(c->order_hist);
  release(c->beam_table);
  if (c->d_ctr) cudaFree(c->d_ctr);
  if (c->d_seg_count) cudaFree(c->d_seg_count);
  if (c->d_box) cudaFree(c->d_box);
  if (c->d_lineage_next) cudaFree(c->d_lineage_next);
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_sctr) cudaFreeHost(c->h_sctr);
  for (TraceRec &r : c->rec) {
    for (cudaEvent_t e : {r.ev0, r.ev1, r.done})
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : r.kev) cudaEventDestroy(e);
  }
  release(c->t_ring);
  release(c->t_seq);
  release(c->t_qctl);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
  return BT_OK;
}

BT_API const char *bt_last_error(const bt_ctx *c) { return c ? c->err : "null context"; }

BT_API int64_t bt_kernel_launches(void) { return (int64_t)bt::g_launches.load(); }

BT_API int bt_l2_bandwidth(bt_ctx *c, int64_t bytes, int32_t repeats, int32_t blocks_per_sm, double *gbs_out) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  if (!gbs_out) return fail(c, BT_E_INVALID, "gbs_out is NULL");
  if (bytes < ((int64_t)16 << 20) || bytes > ((int64_t)96 << 20) || bytes % 16 != 0)
    return fail(c, BT_E_INVALID, "bytes must be a multiple of 16 in 16..96 MiB");
  if (repeats < 1 || repeats > 10000) return fail(c, BT_E_INVALID, "repeats must be in 1..10000");
  if (blocks_per_sm < 1 || blocks_per_sm > 8) return fail(c, BT_E_INVALID, "blocks_per_sm must be in 1..8");
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  const int blocks = c->n_sm * blocks_per_sm;
  TRY(ensure(c, c->stage_a, (size_t)bytes));
  TRY(ensure(c, c->stage_b, sizeof(float) * 256 * (size_t)blocks));
  CK(cudaMemsetAsync(c->stage_a.p, 0, (size_t)bytes, st));
  const float4 *buf = (const float4 *)c->stage_a.p;
  float *sink = (float *)c->stage_b.p;
  CK(bt::launch_l2_read(st, buf, bytes / 16, 2, sink, blocks));  // warm: the buffer into L2
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = bt::launch_l2_read(st, buf, bytes / 16, repeats, sink, blocks);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BT_E_CUDA, "L2 probe: %s", cudaGetErrorString(e));
  }
  *gbs_out = (double)bytes * repeats / (ms * 1e-3) / 1e9;
  return BT_OK;
}

BT_API int bt_l2_atomics(bt_ctx *c, int64_t bytes, int32_t repeats, int32_t blocks_per_sm, double *ops_out) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  if (!ops_out) return fail(c, BT_E_INVALID, "ops_out is NULL");
  if (bytes < ((int64_t)16 << 20) || bytes > ((int64_t)96 << 20) || bytes % 64 != 0)
    return fail(c, BT_E_INVALID, "bytes must be a multiple of 64 in 16..96 MiB");
  if (repeats < 1 || repeats > 10000) return fail(c, BT_E_INVALID, "repeats must be in 1..10000");
  if (blocks_per_sm < 1 || blocks_per_sm > 8) return fail(c, BT_E_INVALID, "blocks_per_sm must be in 1..8");
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  const int blocks = c->n_sm * blocks_per_sm;
  TRY(ensure(c, c->stage_a, (size_t)bytes));
  CK(cudaMemsetAsync(c->stage_a.p, 0, (size_t)bytes, st));
  double *buf = (double *)c->stage_a.p;
  const uint32_t n_slots = (uint32_t)(bytes / 64);
  CK(bt::launch_l2_atomics(st, buf, n_slots, 2, blocks));  // warm: the buffer into L2
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = bt::launch_l2_atomics(st, buf, n_slots, repeats, blocks);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, BT_E_CUDA, "L2 atomics probe: %s", cudaGetErrorString(e));
  }
  // every addition must have landed: the buffer sums to their count
  std::vector<double> h((size_t)bytes / 8);
  CK(cudaMemcpy(h.data(), buf, (size_t)bytes, cudaMemcpyDeviceToHost));
  double sum = 0.0;
  for (double x : h) sum += x;
  const double adds = (double)blocks * 256.0 * 8.0;
  if (sum != adds * (2.0 + repeats))
    return fail(c, BT_E_CUDA, "L2 atomics probe: the buffer sums to %.0f, not %.0f", sum, adds * (2.0 + repeats));
  *ops_out = adds * repeats / (ms * 1e-3);
  return BT_OK;
}

BT_API int bt_load_scene(bt_ctx *c, const float *verts, int64_t n_verts, const int32_t *tris,
                         int64_t n_tris, const uint8_t *tri_material, const float *refl,
                         int32_t n_materials, int32_t n_bands, int32_t *scene_id_out) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  if (!scene_id_out) return fail(c, BT_E_INVALID, "scene_id_out is NULL");
  if (n_verts < 0 || n_tris < 0 || n_tris > (1 << 30) || n_verts > ((int64_t)1 << 31))
    return fail(c, BT_E_INVALID, "bad sizes n_verts=%lld n_tris=%lld", (long long)n_verts, (long long)n_tris);
  if (n_bands < 1 || n_bands > BT_MAX_BANDS) return fail(c, BT_E_INVALID, "n_bands %d not in 1..%d", n_bands, BT_MAX_BANDS);
  if (n_materials < 1 || n_materials > 256) return fail(c, BT_E_INVALID, "n_materials %d not in 1..256", n_materials);
  if (n_tris > 0 && (!verts || !tris || !tri_material)) return fail(c, BT_E_INVALID, "NULL geometry array");
  if (!refl) return fail(c, BT_E_INVALID, "NULL reflection table");
  DeviceGuard g(c->device);
  int id = -1;
  for (int i = 0; i < BT_MAX_SCENES; i++)
    if (!c->sc[i].used) { id = i; break; }
  if (id < 0) return fail(c, BT_E_NOMEM, "all %d scene slots are in use", BT_MAX_SCENES);
  // reflection table: small, checked on the host
  float hrefl[256 * BT_MAX_BANDS];
  CK(cudaMemcpy(hrefl, refl, sizeof(float) * n_materials * n_bands, cudaMemcpyDefault));
  for (int i = 0; i < n_materials * n_bands; i++)
    if (!(hrefl[i] >= 0.0f && hrefl[i] <= 1.0f))
      return fail(c, BT_E_INVALID, "reflection coefficient %d = %g not in [0,1]", i, (double)hrefl[i]);
  SceneState &s = c->sc[id];
  s = SceneState();
  s.n_tris = n_tris;
  s.n_mat = n_materials;
  s.n_bands = n_bands;
  int rc = BT_OK;
  do {
    if ((rc = ensure(c, c->stage_a, sizeof(float) * 3 * (size_t)n_verts))) break;
    if ((rc = ensure(c, c->stage_b, sizeof(int32_t) * 3 * (size_t)n_tris))) break;
    if ((rc = ensure(c, c->stage_c, (size_t)n_tris))) break;
    if ((rc = ensure(c, c->scratch, bt::build_scene_scratch_bytes(n_tris)))) break;
    if ((rc = ensure(c, s.nodes, bt::hier_bytes(n_tris)))) break;
    if ((rc = ensure(c, s.tris, sizeof(bt::Tri) * (size_t)n_tris))) break;
    if ((rc = ensure(c, s.planes, sizeof(bt::Plane) * (size_t)n_tris))) break;
    if ((rc = ensure(c, s.planes64, sizeof(bt::Plane64) * (size_t)n_tris))) break;
    if ((rc = ensure(c, s.planes_df, sizeof(bt::PlaneDF) * (size_t)n_tris))) break;
    if ((rc = ensure(c, s.refl, sizeof(float) * n_materials * n_bands))) break;
  } while (0);
  if (rc != BT_OK) { release_scene(c, s); return rc; }
  s.used = true;
  s.gen = ++c->gen_counter;
  cudaStream_t st = c->stream;
  float *box = c->d_box;
#define CKS(call)                      \
  do {                                 \
    cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) {           \
      cudaGetLastError();              \
      release_scene(c, s);                \
      return fail(c, BT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    }                                  \
  } while (0)
  if (n_verts > 0) CKS(cudaMemcpyAsync(c->stage_a.p, verts, sizeof(float) * 3 * n_verts, cudaMemcpyDefault, st));
  if (n_tris > 0) {
    CKS(cudaMemcpyAsync(c->stage_b.p, tris, sizeof(int32_t) * 3 * n_tris, cudaMemcpyDefault, st));
    CKS(cudaMemcpyAsync(c->stage_c.p, tri_material, (size_t)n_tris, cudaMemcpyDefault, st));
  }
  CKS(cudaMemcpyAsync(s.refl.p, hrefl, sizeof(float) * n_materials * n_bands, cudaMemcpyHostToDevice, st));
  CKS(cudaMemsetAsync(c->d_ctr, 0, sizeof(bt::Counters), st));
  CKS(bt::validate_scene(st, (const float *)c->stage_a.p, n_verts, (const int32_t *)c->stage_b.p, n_tris,
                         (const uint8_t *)c->stage_c.p, n_materials, box, &c->d_ctr->error));
  CKS(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(bt::Counters), cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(s.box, box, sizeof(float) * 6, cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  if (c->h_ctr->error) {
    release_scene(c, s);
    return fail(c, BT_E_INVALID, "scene rejected: vertex index, material or coordinate out of range");
  }
  CKS(bt::build_scene(st, (const float *)c->stage_a.p, (const int32_t *)c->stage_b.p, n_tris,
                      (const uint8_t *)c->stage_c.p, s.nodes.p, (bt::Tri *)s.tris.p,
                      (bt::Plane *)s.planes.p, (bt::Plane64 *)s.planes64.p, (bt::PlaneDF *)s.planes_df.p,
                      c->scratch.p, c->scratch.cap, box, &c->d_ctr->error));
  CKS(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(bt::Counters), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
#undef CKS
  if (c->h_ctr->error) {
    int e = c->h_ctr->error;
    release_scene(c, s);
    return fail(c, BT_E_CUDA, "acceleration structure build failed (device error %d)", e);
  }
  s.root = n_tris == 1 ? ~0 : 0;
  *scene_id_out = id;
  return BT_OK;
}

BT_API int bt_unload_scene(bt_ctx *c, int32_t scene_id) {
  BT_RANGE();
  TRY(check_ctx(c));
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (s->n_shares > 0)
    return fail(c, BT_E_STATE, "scene %d: %d scenes still share its geometry", scene_id, s->n_shares);
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  release_scene(c, *s);
  s->gen = ++c->gen_counter;
  return BT_OK;
}

BT_API int bt_scene_share(bt_ctx *c, int32_t base_id, int32_t *scene_id_out) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *b;
  TRY(scene_ref(c, base_id, &b));
  if (!scene_id_out) return fail(c, BT_E_INVALID, "NULL scene id output");
  if (b->geom_of >= 0) return fail(c, BT_E_INVALID, "scene %d itself shares another scene's geometry", base_id);
  int id = -1;
  for (int i = 0; i < BT_MAX_SCENES; i++)
    if (!c->sc[i].used) {
      id = i;
      break;
    }
  if (id < 0) return fail(c, BT_E_NOMEM, "all %d scene slots are in use", BT_MAX_SCENES);
  SceneState &s = c->sc[id];
  s = SceneState();
  s.used = true;
  s.n_tris = b->n_tris;
  s.n_mat = b->n_mat;
  s.n_bands = b->n_bands;
  s.root = b->root;
  for (int q = 0; q < 6; q++) s.box[q] = b->box[q];
  s.nodes = b->nodes;
  s.tris = b->tris;
  s.planes = b->planes;
  s.planes64 = b->planes64;
  s.planes_df = b->planes_df;
  s.refl = b->refl;
  s.geom_of = base_id;
  s.gen = ++c->gen_counter;
  b->n_shares++;
  *scene_id_out = id;
  return BT_OK;
}

BT_API int bt_set_sources(bt_ctx *c, int32_t scene_id, const float *pos, const float *power_w,
                          int64_t n_s, int32_t icosa_level) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (n_s < 0 || n_s > (1 << 24)) return fail(c, BT_E_INVALID, "bad source count %lld", (long long)n_s);
  if (icosa_level < 0 || icosa_level > 8) return fail(c, BT_E_INVALID, "icosa_level %d not in 0..8", icosa_level);
  if (n_s > 0 && (!pos || !power_w)) return fail(c, BT_E_INVALID, "NULL source array");
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  TRY(ensure(c, c->stage_a, sizeof(float) * 3 * (size_t)n_s));
  TRY(ensure(c, c->stage_b, sizeof(float) * s->n_bands * (size_t)n_s));
  TRY(ensure(c, s->src, sizeof(float4) * (size_t)n_s));
  TRY(ensure(c, s->power, sizeof(float) * s->n_bands * (size_t)n_s));
  TRY(reset_counters(c));
  if (n_s > 0) {
    CK(cudaMemcpyAsync(c->stage_a.p, pos, sizeof(float) * 3 * n_s, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(c->stage_b.p, power_w, sizeof(float) * s->n_bands * n_s, cudaMemcpyDefault, st));
    k_pack_sources<<<(int)((n_s + 255) / 256), 256, 0, st>>>((const float *)c->stage_a.p,
                                                            (const float *)c->stage_b.p, n_s, s->n_bands,
                                                            (float4 *)s->src.p, (float *)s->power.p,
                                                            &c->d_ctr->error);
    bt::note_launches(1);
    CK(cudaGetLastError());
  }
  TRY(read_counters(c));
  if (c->h_ctr->error) {
    s->has_src = false;
    return fail(c, BT_E_INVALID, "source position not finite or power negative/not finite");
  }
  s->n_src = n_s;
  s->level = icosa_level;
  s->n_pat = 0;  // new sources are omnidirectional until bt_set_directivity
  s->has_src = true;
  s->traced = false;
  s->trace_error = 0;
  s->gen = ++c->gen_counter;
  return BT_OK;
}

BT_API int bt_set_directivity(bt_ctx *c, int32_t scene_id, const float *patterns, int32_t n_patterns,
                              const int32_t *pattern_of) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (!s->has_src) return fail(c, BT_E_STATE, "bt_set_directivity needs the scene's sources");
  if (n_patterns < 0) return fail(c, BT_E_INVALID, "n_patterns must be >= 0");
  const int64_t n_beams = (int64_t)20 << (2 * s->level);
  if (n_patterns > 0 && (int64_t)n_patterns * n_beams > ((int64_t)1 << 31))
    return fail(c, BT_E_INVALID, "%d patterns of %lld beams are too many", n_patterns, (long long)n_beams);
  if (n_patterns > 0 && (!patterns || !pattern_of)) return fail(c, BT_E_INVALID, "NULL directivity array");
  if (n_patterns == 0) {
    s->n_pat = 0;
    s->traced = false;
    s->trace_error = 0;
    s->gen = ++c->gen_counter;
    return BT_OK;
  }
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  const int64_t n_gain = (int64_t)n_patterns * n_beams;
  TRY(ensure(c, s->dir_gain, sizeof(float) * (size_t)n_gain));
  TRY(ensure(c, s->dir_of, sizeof(int) * (size_t)(s->n_src > 0 ? s->n_src : 1)));
  TRY(reset_counters(c));
  CK(cudaMemcpyAsync(s->dir_gain.p, patterns, sizeof(float) * (size_t)n_gain, cudaMemcpyDefault, st));
  if (s->n_src > 0)
    CK(cudaMemcpyAsync(s->dir_of.p, pattern_of, sizeof(int) * (size_t)s->n_src, cudaMemcpyDefault, st));
  const int64_t n_check = n_gain > s->n_src ? n_gain : s->n_src;
  k_check_directivity<<<(int)((n_check + 255) / 256), 256, 0, st>>>((const float *)s->dir_gain.p, n_gain,
                                                                    (const int *)s->dir_of.p, s->n_src,
                                                                    n_patterns, &c->d_ctr->error);
  bt::note_launches(1);
  CK(cudaGetLastError());
  TRY(read_counters(c));
  if (c->h_ctr->error) {
    s->n_pat = 0;
    return fail(c, BT_E_INVALID, "directivity gain negative or not finite, or pattern index out of range");
  }
  s->n_pat = n_patterns;
  s->traced = false;
  s->trace_error = 0;
  s->gen = ++c->gen_counter;
  return BT_OK;
}

BT_API int bt_beam_axes(bt_ctx *c, int32_t icosa_level, float *axes) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  if (icosa_level < 0 || icosa_level > 8) return fail(c, BT_E_INVALID, "icosa_level %d not in 0..8", icosa_level);
  if (!axes) return fail(c, BT_E_INVALID, "NULL axes array");
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  const int64_t n = (int64_t)20 << (2 * icosa_level);
  TRY(ensure(c, c->stage_a, sizeof(float) * 3 * (size_t)n));
  CK(bt::launch_beam_axes(st, icosa_level, (float *)c->stage_a.p));
  CK(cudaMemcpyAsync(axes, c->stage_a.p, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return BT_OK;
}

BT_API int bt_set_microphones(bt_ctx *c, int32_t scene_id, const float *pos, int64_t n_m) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (n_m < 0 || n_m > (1 << 28)) return fail(c, BT_E_INVALID, "bad microphone count %lld", (long long)n_m);
  if (n_m > 0 && !pos) return fail(c, BT_E_INVALID, "NULL microphone array");
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  TRY(ensure(c, c->stage_a, sizeof(float) * 3 * (size_t)n_m));
  TRY(ensure(c, c->scratch, bt::build_mics_scratch_bytes(n_m)));
  TRY(ensure(c, s->mics, sizeof(float4) * (size_t)n_m));
  TRY(ensure(c, s->grid, sizeof(bt::MicGrid)));
  TRY(ensure(c, s->energy, sizeof(double) * bt::kMaxBands * (size_t)n_m));
  TRY(ensure(c, s->count, sizeof(int) * (size_t)n_m));
  // the result accumulators start at zero (bt_trace_ranges may add to them)
  CK(cudaMemsetAsync(s->energy.p, 0, sizeof(double) * bt::kMaxBands * (size_t)n_m, c->stream));
  CK(cudaMemsetAsync(s->count.p, 0, sizeof(int) * (size_t)n_m, c->stream));
  TRY(reset_counters(c));
  if (n_m > 0) CK(cudaMemcpyAsync(c->stage_a.p, pos, sizeof(float) * 3 * n_m, cudaMemcpyDefault, st));
  CK(bt::mic_box(st, (const float *)c->stage_a.p, n_m, c->d_box, &c->d_ctr->error));
  float box[6] = {0, 0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(box, c->d_box, sizeof(box), cudaMemcpyDeviceToHost, st));
  TRY(read_counters(c));
  if (c->h_ctr->error) {
    s->has_mics = false;
    return fail(c, BT_E_INVALID, "microphone position not finite");
  }
  // Grid: about four microphones per cell.  Microphones at (nearly) one
  // height get square xy cells and one layer; a volumetric set gets cubic
  // cells, at most 64 layers (the scatter clips every segment per layer, so
  // thinner layers mean tighter footprints: on 13.75 M microphones through
  // the district's height, 34 layers against 16 cut the candidates by 35 %
  // and the scatter by 6 %; layers half the cell's size lost it again).
  int nx = 1, ny = 1, nz = 1;
  if (n_m > 0) {
    const double ex = box[3] - box[0], ey = box[4] - box[1], ez = box[5] - box[2];
    if (ez <= 1.0) {
      nx = ny = (int)ceil(sqrt((double)n_m / 4.0));
    } else {
      const double h = cbrt(fmax(ex, 1.0) * fmax(ey, 1.0) * ez / fmax(1.0, (double)n_m / 4.0));
      nx = (int)fmin(4096.0, fmax(1.0, ceil(ex / h)));
      ny = (int)fmin(4096.0, fmax(1.0, ceil(ey / h)));
      nz = (int)fmin(64.0, fmax(1.0, ceil(ez / h)));
    }
  }
  const size_t n_cells = (size_t)nx * ny * nz;
  TRY(ensure(c, s->cell_start, sizeof(int) * (n_cells + 1)));
  CK(bt::build_mics(st, (const float *)c->stage_a.p, n_m, nx, ny, nz, c->d_box, (bt::MicGrid *)s->grid.p,
                    (float4 *)s->mics.p, (int *)s->cell_start.p, c->scratch.p, c->scratch.cap));
  CK(cudaStreamSynchronize(st));
  const int side = nx;
  s->n_mics = n_m;
  s->side = side;
  s->nz = nz;
  s->has_mics = true;
  s->traced = false;
  s->trace_error = 0;
  s->gen = ++c->gen_counter;
  return BT_OK;
}

// The kernels' view of scene s traced with parameters p (alpha_log2 and
// has_alpha already derived from p; the beam table is set by the caller).
static void fill_view(bt::SceneView &v, SceneState &s, const bt_trace_params *p, const float *alpha_log2,
                      int has_alpha) {
  memset(&v, 0, sizeof(v));
  v.sc = dev_scene(s);
  v.src = (const float4 *)s.src.p;
  v.power = (const float *)s.power.p;
  v.n_src = s.n_src;
  v.level = s.level;
  v.max_order = p->max_order;
  v.n_beams = (int64_t)20 << (2 * s.level);
  v.lineage_base = 0;
  v.t_eps = p->t_eps_m;
  v.energy_threshold = p->energy_threshold_w;
  for (int b = 0; b < BT_MAX_BANDS; b++) v.alpha_log2[b] = alpha_log2[b];
  v.has_alpha = has_alpha;
  v.grid = (const bt::MicGrid *)s.grid.p;
  v.beam_table = nullptr;
  v.mics = (const float4 *)s.mics.p;
  v.cell_start = (const int *)s.cell_start.p;
  v.energy = (double *)s.energy.p;
  v.count = (int *)s.count.p;
  v.dir_gain = s.n_pat > 0 ? (const float *)s.dir_gain.p : nullptr;
  v.dir_of = s.n_pat > 0 ? (const int *)s.dir_of.p : nullptr;
}

// Above this many microphones (80 bytes of accumulators and position each:
// 80 MB, against a 129 MB L2 shared with the geometry) a trace orders its
// scatter by place.
constexpr int64_t kOrderMics = (int64_t)1 << 20;

// Lineages per persistent launch when the caller leaves it to the library:
// segment records of at most a quarter of the free device memory and at most
// 32 GiB (fewer, larger launches have fewer launch tails), at least 1 GiB.
static int64_t default_chunk(int max_order) {
  size_t free_b = 0, total_b = 0;
  int64_t budget = (int64_t)8 << 30;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
    budget = (int64_t)(free_b / 4);
    if (budget > ((int64_t)32 << 30)) budget = (int64_t)32 << 30;
  }
  cudaGetLastError();
  if (budget < ((int64_t)1 << 30)) budget = (int64_t)1 << 30;
  return budget / ((int64_t)sizeof(bt::Seg) * (max_order + 1));
}

// Lineages per launch: the caller's chunk_beams, else default_chunk, at most
// the whole batch, and small enough that a launch's segment records are
// indexed by int32 (the scatter keeps record indices in 32 bits).
static int64_t launch_chunk(int32_t chunk_beams, int64_t total, int max_order) {
  int64_t chunk = chunk_beams > 0 ? chunk_beams : default_chunk(max_order);
  const int64_t max_chunk = (int64_t)INT32_MAX / (max_order + 1);
  if (chunk > max_chunk) chunk = max_chunk;
  if (chunk > total) chunk = total;
  if (chunk < 1) chunk = 1;
  return chunk;
}

// Check the trace parameters p for scene s; derive the air damping exponents.
static int check_params(bt_ctx *c, SceneState *s, const bt_trace_params *p, float *alpha_log2, int *has_alpha) {
  if (!p) return fail(c, BT_E_INVALID, "NULL params");
  if (!s->has_src || !s->has_mics) return fail(c, BT_E_STATE, "sources and microphones must be set before tracing");
  if (p->max_order < 0 || p->max_order > 32) return fail(c, BT_E_INVALID, "max_order %d not in 0..32", p->max_order);
  if (!(p->t_eps_m > 0.0f) || !isfinite(p->t_eps_m)) return fail(c, BT_E_INVALID, "t_eps_m must be > 0");
  if (!(p->energy_threshold_w >= 0.0f)) return fail(c, BT_E_INVALID, "energy_threshold_w must be >= 0");
  if (p->precision != BT_PREC_MIXED && p->precision != BT_PREC_FP32 && p->precision != BT_PREC_FP64 &&
      p->precision != BT_PREC_MIXED64)
    return fail(c, BT_E_INVALID, "unknown precision %d", p->precision);
  if (p->tiles_x < 1 || p->tiles_y < 1 || p->tiles_x > BT_MAX_TILES || p->tiles_y > BT_MAX_TILES)
    return fail(c, BT_E_INVALID, "tiles %dx%d not in 1..%d per axis", p->tiles_x, p->tiles_y, BT_MAX_TILES);
  if (p->chunk_beams < 0) return fail(c, BT_E_INVALID, "chunk_beams must be >= 0");
  if (p->blocks_per_sm < 0 || p->blocks_per_sm > 32) return fail(c, BT_E_INVALID, "blocks_per_sm must be in 0..32");
  if (p->queue_depth != 0 && (p->queue_depth < 32 || p->queue_depth > (1 << 22) ||
                              (p->queue_depth & (p->queue_depth - 1)) != 0))
    return fail(c, BT_E_INVALID, "queue_depth must be 0 or a power of two in 32..2^22");
  if (p->leaf_size < 0 || p->leaf_size > bt::kMaxLeafSize)
    return fail(c, BT_E_INVALID, "leaf_size %d not in 0..%d", p->leaf_size, bt::kMaxLeafSize);
  if (p->beams_per_warp < 0 || p->beams_per_warp > 4096 || p->beams_per_warp % 32 != 0)
    return fail(c, BT_E_INVALID, "beams_per_warp must be 0 or a multiple of 32 up to 4096");
  if (p->fault_test < 0 || p->fault_test > BT_FAULT_SEGMENTS) return fail(c, BT_E_INVALID, "unknown fault_test %d", p->fault_test);
  *has_alpha = 0;
  for (int b = 0; b < BT_MAX_BANDS; b++) {
    float a = p->air_atten_db_per_m[b];
    if (!(a >= 0.0f) || !isfinite(a)) return fail(c, BT_E_INVALID, "air attenuation must be finite and >= 0");
    alpha_log2[b] = -a * 3.32192809488736f / 10.0f;  // 10^(-a d/10) = 2^(-a d log2(10)/10)
    if (b < s->n_bands && a != 0.0f) *has_alpha = 1;
  }
  return BT_OK;
}

// Collapse the flat (or, with `tiled`, the sub-domain) hierarchy of scene s
// to the leaf size p asks for, unless it already has it.  The hits do not
// depend on the leaf size, so every scene sharing the geometry may see the
// change.
static int apply_leaf_size(bt_ctx *c, SceneState &s, const bt_trace_params *p, bool tiled) {
  const int want = p->leaf_size > 0 ? p->leaf_size : 1;
  SceneState &g = s.geom_of >= 0 ? c->sc[s.geom_of] : s;
  int &have = tiled ? s.t_leaf : g.leaf;
  if (have == want) return BT_OK;
  const int64_t n = tiled ? s.n_pairs : g.n_tris;
  if (want > 1 && n >= ((int64_t)1 << bt::kLeafShift))
    return fail(c, BT_E_INVALID, "leaf_size > 1 needs fewer than 2^%d leaves (the hierarchy has %lld)", bt::kLeafShift,
                (long long)n);
  CK(bt::collapse_leaves(c->stream, tiled ? s.t_nodes.p : g.nodes.p, n, want));
  have = want;
  return BT_OK;
}

// Enqueue a whole trace of scene slot `id` on the context's stream: chunks of
// lineages, each a persistent traversal launch and a scatter launch, events
// around every launch, and the counters' copy to the slot's pinned record.
// The scene is then pending until collect().
static int enqueue_trace(bt_ctx *c, int32_t id, const bt_trace_params *p) {
  SceneState *s = &c->sc[id];
  int has_alpha = 0;
  float alpha_log2[BT_MAX_BANDS];
  TRY(check_params(c, s, p, alpha_log2, &has_alpha));
  DeviceGuard g(c->device);
  s->traced = false;
  s->trace_error = 0;
  TraceRec &r = c->rec[id];
  for (cudaEvent_t *e : {&r.ev0, &r.ev1, &r.done})
    if (!*e) CK(cudaEventCreate(e));
  r.kind.clear();
  cudaStream_t st = c->stream;
  const int64_t n_beams = (int64_t)20 << (2 * s->level);
  const int64_t total = s->n_src * n_beams;
  const bool tiled = p->tiles_x * p->tiles_y > 1;
  const int T = p->tiles_x * p->tiles_y;
  // One persistent launch per group of lineages: fewer, larger groups mean
  // fewer launch tails.
  const int64_t chunk = launch_chunk(p->chunk_beams, total, p->max_order);
  const unsigned long long cap = (unsigned long long)chunk * (p->max_order + 1);
  TRY(ensure(c, c->segs, sizeof(bt::Seg) * cap));
  // Microphones whose accumulators and positions are several times the L2
  // (a receiver volume) are scattered to in order of place.
  const bool by_place = s->n_mics > kOrderMics;
  if (by_place) {
    TRY(ensure(c, c->seg_order, sizeof(uint32_t) * cap));
    TRY(ensure(c, c->order_hist, sizeof(uint32_t) * bt::kOrderBins));
  }
  // Hand-off queues: at most qcap lineages are in flight (traced or queued),
  // so no tile's ring of qcap slots can overflow.  Automatic: at least twice
  // the lanes of one launch, so that the cap rarely holds a lane back.
  unsigned qcap = 1024;
  if (tiled) {
    TRY(ensure_tiled(c, *s, p->tiles_x, p->tiles_y));
    TRY(apply_leaf_size(c, *s, p, true));
    if (p->queue_depth > 0) {
      qcap = (unsigned)p->queue_depth;
    } else {
      const int64_t lanes = bt::tiled_resident_lanes(c->n_sm);
      while ((int64_t)qcap < 2 * lanes && qcap < (1u << 22)) qcap <<= 1;
      while (qcap > 1024 && (int64_t)T * qcap * (bt::kStateRows * 4 + 4) > ((int64_t)4 << 30)) qcap >>= 1;
    }
    TRY(ensure(c, c->t_ring, sizeof(uint32_t) * bt::kStateRows * (size_t)T * qcap));
    TRY(ensure(c, c->t_seq, sizeof(unsigned) * (size_t)T * qcap));
    TRY(ensure(c, c->t_qctl, sizeof(int) * (3 * (size_t)T + 3)));
  } else {
    TRY(apply_leaf_size(c, *s, p, false));
  }
  TRY(reset_counters(c));
  CK(cudaMemsetAsync(s->energy.p, 0, sizeof(double) * bt::kMaxBands * (size_t)s->n_mics, st));
  CK(cudaMemsetAsync(s->count.p, 0, sizeof(int) * (size_t)s->n_mics, st));
  bt::TraceArgs ta;
  memset(&ta, 0, sizeof(ta));
  fill_view(ta.v, *s, p, alpha_log2, has_alpha);
  ta.v.seg_key = by_place ? 1 : 0;
  if (tiled) {
    ta.v.sc.n_tris = s->n_pairs;
    ta.v.sc.nodes = bt::hier_wide(s->t_nodes.p, s->n_pairs);
    ta.v.sc.tris = (const bt::Tri *)s->t_tris.p;
    ta.v.sc.planes = (const bt::Plane *)s->t_planes.p;
    ta.v.sc.planes64 = (const bt::Plane64 *)s->t_planes64.p;
    ta.v.sc.planes_df = (const bt::PlaneDF *)s->t_planes_df.p;
    ta.v.sc.root = 0;
  }
  ta.segs = (bt::Seg *)c->segs.p;
  ta.seg_count = c->d_seg_count;
  // (test hook: room for one segment record, so that the trace overflows)
  ta.seg_capacity = p->fault_test == BT_FAULT_SEGMENTS ? 1 : cap;
  ta.lineage_next = c->d_lineage_next;
  ta.ctr = c->d_ctr;
  ta.count_work = p->count_work ? 1 : 0;
  ta.prec = p->precision;
  ta.blocks_per_sm = p->blocks_per_sm;
  ta.beams_per_warp = p->beams_per_warp;
  ta.leaf_size = p->leaf_size > 1 ? p->leaf_size : 1;
  if (s->hit_log) {
    if (s->hit_log_n < total * (p->max_order + 1))
      return fail(c, BT_E_INVALID, "hit log of %lld entries is smaller than %lld lineages x %d orders",
                  (long long)s->hit_log_n, (long long)total, p->max_order + 1);
    ta.hit_log = s->hit_log;
    ta.hit_log_stride = p->max_order + 1;
  }
  if (ta.prec == BT_PREC_MIXED && total > 0) {
    if (c->beam_table_level != s->level) {
      TRY(ensure(c, c->beam_table, sizeof(float) * 24 * (size_t)n_beams));
      CK(bt::launch_beam_table(st, s->level, (float *)c->beam_table.p));
      c->beam_table_level = s->level;
    }
    ta.v.beam_table = (const float *)c->beam_table.p;
  }
  bt::ScatterArgs sa;
  memset(&sa, 0, sizeof(sa));
  sa.v = ta.v;
  sa.fp64 = p->precision == BT_PREC_FP64 ? 1 : 0;
  sa.max_nz = s->nz;
  sa.segs = ta.segs;
  sa.seg_count = c->d_seg_count;
  sa.seg_capacity = ta.seg_capacity;
  sa.ctr = c->d_ctr;
  sa.order = by_place ? (const uint32_t *)c->seg_order.p : nullptr;
  bt::TiledArgs tga;
  memset(&tga, 0, sizeof(tga));
  if (tiled) {
    tga.tg = s->tg;
    tga.n_tiles = T;
    tga.roots = (const int *)s->t_roots.p;
    tga.bin = (const bt::Node *)s->t_nodes.p;
    tga.qcap = qcap;
    tga.ring = (uint32_t *)c->t_ring.p;
    tga.seq = (unsigned *)c->t_seq.p;
    tga.ctl = (int *)c->t_qctl.p;
    tga.watchdog_ns = (unsigned long long)(p->watchdog_ms > 0 ? p->watchdog_ms : 2000) * 1000000ull;
    tga.withhold = p->fault_test == BT_FAULT_WITHHOLD ? 1 : 0;
  }
  // Events bracket every launch: a pair per launch, its kind in r.kind.
  int n_ev = 0;
  auto mark = [&](int kind) -> int {
    while ((int)r.kev.size() < n_ev + 1) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      r.kev.push_back(e);
    }
    CK(cudaEventRecord(r.kev[n_ev], st));
    if (n_ev % 2 == 0) r.kind.push_back(kind);
    n_ev++;
    return BT_OK;
  };
  auto scatter_round = [&]() -> int {
    if (s->n_mics <= 0) return BT_OK;
    TRY(mark(1));
    if (by_place)
      CK(bt::launch_seg_order(st, ta.segs, c->d_seg_count, ta.seg_capacity, ta.v.grid,
                              (uint32_t *)c->order_hist.p, (uint32_t *)c->seg_order.p, c->n_sm));
    CK(bt::launch_scatter(st, sa, c->n_sm));
    return mark(1);
  };
  const int64_t n_chunks = total > 0 ? (total + chunk - 1) / chunk : 0;
  int64_t n_trace_launches = 0, n_scatter_launches = 0, n_rounds = 0;
  CK(cudaEventRecord(r.ev0, st));
  for (int64_t ci = 0; ci < n_chunks; ci++) {
    int64_t b0 = ci * chunk;
    ta.lineage_begin = b0;
    ta.lineage_end = b0 + chunk < total ? b0 + chunk : total;
    CK(cudaMemsetAsync(c->d_seg_count, 0, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(c->d_lineage_next, 0, sizeof(unsigned long long), st));
    if (tiled) {
      CK(cudaMemsetAsync(c->t_seq.p, 0, sizeof(unsigned) * (size_t)T * qcap, st));
      CK(cudaMemsetAsync(c->t_qctl.p, 0, sizeof(int) * (3 * (size_t)T + 3), st));
    }
    TRY(mark(0));
    if (tiled) {
      CK(bt::launch_trace_tiled(st, ta, tga, c->n_sm));
      n_rounds++;
    } else {
      CK(bt::launch_trace(st, ta, c->n_sm));
    }
    TRY(mark(0));
    n_trace_launches++;
    TRY(scatter_round());
    n_scatter_launches += s->n_mics > 0;
  }
  CK(cudaEventRecord(r.ev1, st));
  CK(cudaMemcpyAsync(&c->h_sctr[id], c->d_ctr, sizeof(bt::Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(r.done, st));
  r.beams = total;
  r.trace_launches = n_trace_launches;
  r.scatter_launches = n_scatter_launches;
  r.rounds = n_rounds;
  s->pending = true;
  return BT_OK;
}

BT_API int bt_set_hit_log(bt_ctx *c, int32_t scene_id, int32_t *hits, int64_t n) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (!hits) {
    s->hit_log = nullptr;
    s->hit_log_n = 0;
    return BT_OK;
  }
  if (n < 0) return fail(c, BT_E_INVALID, "negative hit log size");
  if (!is_device_ptr(hits, c->device)) return fail(c, BT_E_INVALID, "the hit log must be device memory of device %d", c->device);
  s->hit_log = hits;
  s->hit_log_n = n;
  return BT_OK;
}

BT_API int bt_trace(bt_ctx *c, int32_t scene_id, const bt_trace_params *p) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  TRY(enqueue_trace(c, scene_id, p));
  return collect(c, scene_id, true, true);
}

BT_API int bt_submit(bt_ctx *c, int32_t scene_id, const bt_trace_params *p) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  return enqueue_trace(c, scene_id, p);
}

// bt_poll (wait = false) and bt_wait (wait = true).
static int finish(bt_ctx *c, int32_t scene_id, bool wait) {
  TRY(check_ctx(c));
  c->err[0] = 0;
  if (scene_id < 0 || scene_id >= BT_MAX_SCENES || !c->sc[scene_id].used)
    return fail(c, BT_E_INVALID, "unknown scene id %d", scene_id);
  SceneState &s = c->sc[scene_id];
  if (s.pending) return collect(c, scene_id, wait, true);
  if (s.traced) return BT_OK;
  if (s.trace_error) return fail(c, s.trace_error, "the last trace of scene %d failed (code %d)", scene_id, s.trace_error);
  return fail(c, BT_E_STATE, "scene %d has no trace submitted", scene_id);
}

BT_API int bt_poll(bt_ctx *c, int32_t scene_id) { BT_RANGE(); return finish(c, scene_id, false); }

BT_API int bt_wait(bt_ctx *c, int32_t scene_id) { BT_RANGE(); return finish(c, scene_id, true); }

BT_API int bt_read_levels(bt_ctx *c, int32_t scene_id, double *level_db, double *intensity,
                          int32_t *path_count, bt_stats *stats) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (!s->traced) {
    if (s->trace_error) return fail(c, s->trace_error, "the last trace of scene %d failed (code %d)", scene_id, s->trace_error);
    return fail(c, BT_E_STATE, "scene %d has no trace result", scene_id);
  }
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  const size_t nv = (size_t)s->n_mics * s->n_bands;
  TRY(ensure(c, s->out_level, sizeof(double) * nv));
  TRY(ensure(c, s->out_int, sizeof(double) * nv));
  TRY(ensure(c, s->out_cnt, sizeof(int) * (size_t)s->n_mics));
  CK(bt::launch_levels(st, (const double *)s->energy.p, (const int *)s->count.p, (const float4 *)s->mics.p,
                       s->n_mics, s->n_bands, (double *)s->out_level.p, (double *)s->out_int.p,
                       (int *)s->out_cnt.p));
  if (level_db && nv) CK(cudaMemcpyAsync(level_db, s->out_level.p, sizeof(double) * nv, cudaMemcpyDefault, st));
  if (intensity && nv) CK(cudaMemcpyAsync(intensity, s->out_int.p, sizeof(double) * nv, cudaMemcpyDefault, st));
  if (path_count && s->n_mics)
    CK(cudaMemcpyAsync(path_count, s->out_cnt.p, sizeof(int) * (size_t)s->n_mics, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  if (stats) *stats = s->stats;
  return BT_OK;
}

BT_API int bt_set_result(bt_ctx *c, int32_t scene_id, const double *intensity, const int32_t *path_count) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (!s->has_mics) return fail(c, BT_E_STATE, "scene %d has no microphones", scene_id);
  if (s->n_mics > 0 && !intensity) return fail(c, BT_E_INVALID, "NULL intensity");
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  const size_t nv = (size_t)s->n_mics * s->n_bands;
  TRY(ensure(c, s->out_int, sizeof(double) * (nv ? nv : 1)));
  TRY(ensure(c, s->out_cnt, sizeof(int) * (size_t)(s->n_mics ? s->n_mics : 1)));
  if (nv) CK(cudaMemcpyAsync(s->out_int.p, intensity, sizeof(double) * nv, cudaMemcpyDefault, st));
  if (path_count && s->n_mics)
    CK(cudaMemcpyAsync(s->out_cnt.p, path_count, sizeof(int) * (size_t)s->n_mics, cudaMemcpyDefault, st));
  CK(bt::launch_set_result(st, (const double *)s->out_int.p, path_count ? (const int *)s->out_cnt.p : nullptr,
                           (const float4 *)s->mics.p, s->n_mics, s->n_bands, (double *)s->energy.p,
                           (int *)s->count.p));
  CK(cudaStreamSynchronize(st));
  memset(&s->stats, 0, sizeof(s->stats));
  s->traced = true;
  s->trace_error = 0;
  return BT_OK;
}

// ===================================================================== batches
// Many scenes traced together: one persistent trace launch and one scatter
// launch per batch of lineages drawn from all scenes (every lane finds its
// lineage's scene), the whole launch sequence captured once as a CUDA graph
// and replayed by every run.
struct bt_batch {
  bt_ctx *c = nullptr;
  std::vector<int> ids;
  std::vector<unsigned long long> gens;
  std::vector<int64_t> beams;  // lineages per scene
  int prec = BT_PREC_MIXED;
  int count_work = 0, blocks_per_sm = 0, beams_per_warp = 0, leaf_size = 1;
  int max_order = 0, max_nz = 1;
  int64_t total = 0, chunk = 1;
  DevBuf views, segs, beam_tables[9];
  bt::Counters *d_ctr = nullptr, *h_ctr = nullptr;
  unsigned long long *d_cursors = nullptr;  // seg_count, lineage_next
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  long long kernels_per_run = 0;
  bt_stats stats;
};

static void free_batch(bt_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  release(b->views);
  release(b->segs);
  for (DevBuf &t : b->beam_tables) release(t);
  if (b->d_ctr) cudaFree(b->d_ctr);
  if (b->h_ctr) cudaFreeHost(b->h_ctr);
  if (b->d_cursors) cudaFree(b->d_cursors);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  cudaGetLastError();
  delete b;
}

BT_API int bt_batch_create(bt_ctx *c, const int32_t *scene_ids, int32_t n_scenes, const bt_trace_params *params,
                           bt_batch **out) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  if (!out) return fail(c, BT_E_INVALID, "NULL output handle");
  *out = nullptr;
  if (n_scenes < 1 || n_scenes > BT_MAX_SCENES || !scene_ids || !params)
    return fail(c, BT_E_INVALID, "a batch needs 1..%d scenes and their parameters", BT_MAX_SCENES);
  std::vector<bt::SceneView> hv((size_t)n_scenes);
  const int prec = params[0].precision;
  for (int i = 0; i < n_scenes; i++) {
    SceneState *s;
    TRY(scene_ref(c, scene_ids[i], &s));
    for (int j = 0; j < i; j++)
      if (scene_ids[j] == scene_ids[i]) return fail(c, BT_E_INVALID, "scene %d listed twice", scene_ids[i]);
    const bt_trace_params *p = &params[i];
    float alpha_log2[BT_MAX_BANDS];
    int has_alpha = 0;
    TRY(check_params(c, s, p, alpha_log2, &has_alpha));
    if (p->tiles_x != 1 || p->tiles_y != 1)
      return fail(c, BT_E_INVALID, "a batch traces every scene unsplit (tiles 1x1)");
    if (p->precision != prec || p->count_work != params[0].count_work ||
        p->blocks_per_sm != params[0].blocks_per_sm || p->chunk_beams != params[0].chunk_beams ||
        p->beams_per_warp != params[0].beams_per_warp)
      return fail(c, BT_E_INVALID,
                  "precision, count_work, blocks_per_sm, beams_per_warp and chunk_beams must agree across a batch");
    TRY(apply_leaf_size(c, *s, p, false));
    fill_view(hv[i], *s, p, alpha_log2, has_alpha);
  }
  bt_batch *b = new bt_batch();
  b->c = c;
  b->prec = prec;
  b->count_work = params[0].count_work ? 1 : 0;
  b->blocks_per_sm = params[0].blocks_per_sm;
  b->beams_per_warp = params[0].beams_per_warp;
  for (int i = 0; i < n_scenes; i++)
    if (params[i].leaf_size > b->leaf_size) b->leaf_size = params[i].leaf_size;
  memset(&b->stats, 0, sizeof(b->stats));
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  int rc = BT_OK;
  do {
    for (int i = 0; i < n_scenes; i++) {
      SceneState &s = c->sc[scene_ids[i]];
      b->ids.push_back(scene_ids[i]);
      b->gens.push_back(s.gen);
      const int64_t nb = (int64_t)20 << (2 * s.level);
      hv[i].lineage_base = b->total;
      b->beams.push_back(s.n_src * nb);
      b->total += s.n_src * nb;
      if (params[i].max_order > b->max_order) b->max_order = params[i].max_order;
      if (s.nz > b->max_nz) b->max_nz = s.nz;
      if (prec == BT_PREC_MIXED && s.n_src > 0) {
        DevBuf &t = b->beam_tables[s.level];
        if (!t.p) {
          if ((rc = ensure(c, t, sizeof(float) * 24 * (size_t)nb))) break;
          if (bt::launch_beam_table(st, s.level, (float *)t.p) != cudaSuccess) { rc = BT_E_CUDA; break; }
        }
        hv[i].beam_table = (const float *)t.p;
      }
    }
    if (rc) break;
    b->chunk = launch_chunk(params[0].chunk_beams, b->total, b->max_order);
    if ((rc = ensure(c, b->views, sizeof(bt::SceneView) * (size_t)n_scenes))) break;
    if ((rc = ensure(c, b->segs, sizeof(bt::Seg) * (size_t)b->chunk * (b->max_order + 1)))) break;
    if (cudaMalloc(&b->d_ctr, sizeof(bt::Counters)) != cudaSuccess ||
        cudaMallocHost(&b->h_ctr, sizeof(bt::Counters)) != cudaSuccess ||
        cudaMalloc(&b->d_cursors, 2 * sizeof(unsigned long long)) != cudaSuccess) {
      rc = BT_E_NOMEM;
      break;
    }
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) { rc = BT_E_CUDA; break; }
    if (cudaMemcpyAsync(b->views.p, hv.data(), sizeof(bt::SceneView) * (size_t)n_scenes, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = BT_E_CUDA;
      break;
    }
  } while (0);
  if (rc) {
    free_batch(b);
    cudaGetLastError();
    return fail(c, rc, "batch set-up failed (%d)", rc);
  }
  c->batches.push_back(b);
  *out = b;
  return BT_OK;
}

// Record the whole launch sequence of one batch run on the context's stream.
static int record_batch(bt_batch *b) {
  bt_ctx *c = b->c;
  cudaStream_t st = c->stream;
  const int n = (int)b->ids.size();
  CK(cudaMemsetAsync(b->d_ctr, 0, sizeof(bt::Counters), st));
  for (int i = 0; i < n; i++) {
    SceneState &s = c->sc[b->ids[i]];
    if (s.n_mics > 0) {
      CK(cudaMemsetAsync(s.energy.p, 0, sizeof(double) * bt::kMaxBands * (size_t)s.n_mics, st));
      CK(cudaMemsetAsync(s.count.p, 0, sizeof(int) * (size_t)s.n_mics, st));
    }
  }
  bt::TraceArgs ta;
  memset(&ta, 0, sizeof(ta));
  ta.views = (const bt::SceneView *)b->views.p;
  ta.n_views = n;
  ta.segs = (bt::Seg *)b->segs.p;
  ta.seg_count = b->d_cursors;
  ta.lineage_next = b->d_cursors + 1;
  ta.seg_capacity = (unsigned long long)b->chunk * (b->max_order + 1);
  ta.ctr = b->d_ctr;
  ta.count_work = b->count_work;
  ta.prec = b->prec;
  ta.blocks_per_sm = b->blocks_per_sm;
  ta.beams_per_warp = b->beams_per_warp;
  ta.leaf_size = b->leaf_size;
  bt::ScatterArgs sa;
  memset(&sa, 0, sizeof(sa));
  sa.views = ta.views;
  sa.n_views = n;
  sa.fp64 = b->prec == BT_PREC_FP64 ? 1 : 0;
  sa.max_nz = b->max_nz;
  sa.segs = ta.segs;
  sa.seg_count = ta.seg_count;
  sa.seg_capacity = ta.seg_capacity;
  sa.ctr = b->d_ctr;
  const int64_t n_chunks = b->total > 0 ? (b->total + b->chunk - 1) / b->chunk : 0;
  for (int64_t ci = 0; ci < n_chunks; ci++) {
    ta.lineage_begin = ci * b->chunk;
    ta.lineage_end = ta.lineage_begin + b->chunk < b->total ? ta.lineage_begin + b->chunk : b->total;
    CK(cudaMemsetAsync(b->d_cursors, 0, 2 * sizeof(unsigned long long), st));
    CK(bt::launch_trace(st, ta, c->n_sm));
    CK(bt::launch_scatter(st, sa, c->n_sm));
  }
  return BT_OK;
}

BT_API int bt_batch_run(bt_batch *b) {
  BT_RANGE();
  if (!b) return BT_E_INVALID;
  bt_ctx *c = b->c;
  c->err[0] = 0;
  for (size_t i = 0; i < b->ids.size(); i++) {
    if (c->sc[b->ids[i]].gen != b->gens[i])
      return fail(c, BT_E_STATE, "scene %d changed since the batch was created", b->ids[i]);
    if (c->sc[b->ids[i]].pending) collect(c, b->ids[i], true, false);  // a submitted trace finishes first
  }
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  if (!b->exec) {
    // capture the launch sequence once; every run replays it
    const long long k0 = bt_kernel_launches();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = record_batch(b);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    b->kernels_per_run = bt_kernel_launches() - k0;
    bt::note_launches((int)-b->kernels_per_run);  // counted when they run
    if (rc != BT_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(c, rc != BT_OK ? rc : BT_E_CUDA, "batch graph capture failed");
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return fail(c, BT_E_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e));
    }
  }
  CK(cudaEventRecord(b->ev0, st));
  CK(cudaGraphLaunch(b->exec, st));
  CK(cudaEventRecord(b->ev1, st));
  bt::note_launches((int)b->kernels_per_run);
  CK(cudaMemcpyAsync(b->h_ctr, b->d_ctr, sizeof(bt::Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  const bt::Counters &h = *b->h_ctr;
  bt_stats &o = b->stats;
  memset(&o, 0, sizeof(o));
  o.beams = b->total;
  o.segments = (int64_t)h.segments;
  o.hits = (int64_t)h.hits;
  o.escapes = (int64_t)h.escapes;
  o.emitted = (int64_t)h.emitted;
  o.candidates = (int64_t)h.candidates;
  o.contributions = (int64_t)h.contributions;
  o.nodes_visited = (int64_t)h.nodes_visited;
  o.tris_tested = (int64_t)h.tris_tested;
  const int64_t n_chunks = b->total > 0 ? (b->total + b->chunk - 1) / b->chunk : 0;
  o.trace_launches = n_chunks;
  o.scatter_launches = n_chunks;
  o.trace_ms = ms;
  for (size_t i = 0; i < b->ids.size(); i++) {
    SceneState &s = c->sc[b->ids[i]];
    memset(&s.stats, 0, sizeof(s.stats));
    s.stats.beams = b->beams[i];
    s.traced = h.error == 0;
    s.trace_error = h.error;
  }
  if (h.error)
    return fail(c, h.error, h.error == BT_E_QUEUE_FULL ? "device queue or traversal stack overflow"
                                                        : "device error %d", h.error);
  return BT_OK;
}

BT_API int bt_batch_stats(const bt_batch *b, bt_stats *stats) {
  BT_RANGE();
  if (!b || !stats) return BT_E_INVALID;
  *stats = b->stats;
  return BT_OK;
}

BT_API int bt_batch_destroy(bt_batch *b) {
  BT_RANGE();
  if (!b) return BT_OK;
  bt_ctx *c = b->c;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  for (size_t i = 0; i < c->batches.size(); i++)
    if (c->batches[i] == b) {
      c->batches.erase(c->batches.begin() + (long)i);
      break;
    }
  free_batch(b);
  return BT_OK;
}

BT_API int bt_trace_ranges(bt_ctx *c, int32_t n, const int32_t *scene_ids, const int64_t *lineage_begin,
                           const int64_t *lineage_end, const bt_trace_params *params, int32_t flags) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  if (n < 0 || n > BT_MAX_SCENES) return fail(c, BT_E_INVALID, "n must be in 0..%d", BT_MAX_SCENES);
  if (n > 0 && (!scene_ids || !lineage_begin || !lineage_end || !params))
    return fail(c, BT_E_INVALID, "NULL argument");
  if (flags & ~BT_ACCUMULATE) return fail(c, BT_E_INVALID, "unknown flags 0x%x", flags);
  memset(&c->range_stats, 0, sizeof(c->range_stats));
  if (n == 0) return BT_OK;
  std::vector<bt::SceneView> hv((size_t)n);
  const int prec = params[0].precision;
  int kmax = 0, max_nz = 1;
  int64_t total = 0;
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  for (int i = 0; i < n; i++) {
    SceneState *s;
    TRY(scene_ref(c, scene_ids[i], &s));
    for (int j = 0; j < i; j++)
      if (scene_ids[j] == scene_ids[i]) return fail(c, BT_E_INVALID, "scene %d listed twice", scene_ids[i]);
    const bt_trace_params *p = &params[i];
    float alpha_log2[BT_MAX_BANDS];
    int has_alpha = 0;
    TRY(check_params(c, s, p, alpha_log2, &has_alpha));
    if (p->tiles_x != 1 || p->tiles_y != 1) return fail(c, BT_E_INVALID, "bt_trace_ranges traces unsplit (tiles 1x1)");
    if (p->precision != prec || p->blocks_per_sm != params[0].blocks_per_sm || p->count_work != params[0].count_work ||
        p->beams_per_warp != params[0].beams_per_warp)
      return fail(c, BT_E_INVALID, "precision, blocks_per_sm, beams_per_warp and count_work must agree across the scenes");
    TRY(apply_leaf_size(c, *s, p, false));
    const int64_t nl = s->n_src * ((int64_t)20 << (2 * s->level));
    if (lineage_begin[i] < 0 || lineage_end[i] < lineage_begin[i] || lineage_end[i] > nl)
      return fail(c, BT_E_INVALID, "scene %d: lineage range [%lld, %lld) outside [0, %lld)", scene_ids[i],
                  (long long)lineage_begin[i], (long long)lineage_end[i], (long long)nl);
    fill_view(hv[i], *s, p, alpha_log2, has_alpha);
    hv[i].lineage_base = total;
    hv[i].lineage_first = lineage_begin[i];
    total += lineage_end[i] - lineage_begin[i];
    if (p->max_order > kmax) kmax = p->max_order;
    if (s->nz > max_nz) max_nz = s->nz;
    if (prec == BT_PREC_MIXED && nl > 0) {
      DevBuf &t = c->level_tables[s->level];
      if (!t.p) {
        TRY(ensure(c, t, sizeof(float) * 24 * (size_t)((int64_t)20 << (2 * s->level))));
        CK(bt::launch_beam_table(st, s->level, (float *)t.p));
      }
      hv[i].beam_table = (const float *)t.p;
    }
  }
  const int64_t chunk = launch_chunk(params[0].chunk_beams, total, kmax);
  const unsigned long long cap = (unsigned long long)chunk * (kmax + 1);
  TRY(ensure(c, c->segs, sizeof(bt::Seg) * cap));
  TRY(ensure(c, c->views, sizeof(bt::SceneView) * (size_t)n));
  CK(cudaMemcpyAsync(c->views.p, hv.data(), sizeof(bt::SceneView) * (size_t)n, cudaMemcpyHostToDevice, st));
  TRY(reset_counters(c));
  for (int i = 0; i < n; i++) {
    SceneState &s = c->sc[scene_ids[i]];
    if (!(flags & BT_ACCUMULATE) && s.n_mics > 0) {
      CK(cudaMemsetAsync(s.energy.p, 0, sizeof(double) * bt::kMaxBands * (size_t)s.n_mics, st));
      CK(cudaMemsetAsync(s.count.p, 0, sizeof(int) * (size_t)s.n_mics, st));
    }
  }
  // One scene: the single-scene kernels, with the view in kernel parameters
  // and the scene's own lineage indices; several: the batch kernels over the
  // ranges laid end to end.
  const bool single = n == 1;
  const int64_t first = single ? lineage_begin[0] : 0;
  bt::TraceArgs ta;
  memset(&ta, 0, sizeof(ta));
  if (single) {
    ta.v = hv[0];
    ta.v.lineage_first = 0;
  } else {
    ta.views = (const bt::SceneView *)c->views.p;
    ta.n_views = n;
  }
  ta.segs = (bt::Seg *)c->segs.p;
  ta.seg_count = c->d_seg_count;
  ta.lineage_next = c->d_lineage_next;
  ta.seg_capacity = cap;
  ta.ctr = c->d_ctr;
  ta.count_work = params[0].count_work ? 1 : 0;
  ta.prec = prec;
  ta.blocks_per_sm = params[0].blocks_per_sm;
  ta.beams_per_warp = params[0].beams_per_warp;
  ta.leaf_size = 1;
  for (int i = 0; i < n; i++)
    if (params[i].leaf_size > ta.leaf_size) ta.leaf_size = params[i].leaf_size;
  bt::ScatterArgs sa;
  memset(&sa, 0, sizeof(sa));
  sa.v = ta.v;
  sa.views = ta.views;
  sa.n_views = ta.n_views;
  sa.fp64 = prec == BT_PREC_FP64 ? 1 : 0;
  sa.max_nz = max_nz;
  sa.segs = ta.segs;
  sa.seg_count = ta.seg_count;
  sa.seg_capacity = cap;
  sa.ctr = c->d_ctr;
  CK(cudaEventRecord(c->ev0, st));
  const int64_t n_chunks = total > 0 ? (total + chunk - 1) / chunk : 0;
  for (int64_t ci = 0; ci < n_chunks; ci++) {
    ta.lineage_begin = first + ci * chunk;
    ta.lineage_end = ci * chunk + chunk < total ? ta.lineage_begin + chunk : first + total;
    CK(cudaMemsetAsync(c->d_seg_count, 0, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(c->d_lineage_next, 0, sizeof(unsigned long long), st));
    CK(bt::launch_trace(st, ta, c->n_sm));
    CK(bt::launch_scatter(st, sa, c->n_sm));
  }
  CK(cudaEventRecord(c->ev1, st));
  TRY(read_counters(c));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  const bt::Counters &h = *c->h_ctr;
  bt_stats &o = c->range_stats;
  o.beams = total;
  o.segments = (int64_t)h.segments;
  o.hits = (int64_t)h.hits;
  o.escapes = (int64_t)h.escapes;
  o.emitted = (int64_t)h.emitted;
  o.candidates = (int64_t)h.candidates;
  o.contributions = (int64_t)h.contributions;
  o.nodes_visited = (int64_t)h.nodes_visited;
  o.tris_tested = (int64_t)h.tris_tested;
  o.trace_launches = n_chunks;
  o.scatter_launches = n_chunks;
  o.trace_ms = ms;
  for (int i = 0; i < n; i++) {
    SceneState &s = c->sc[scene_ids[i]];
    memset(&s.stats, 0, sizeof(s.stats));
    s.traced = h.error == 0;
    s.trace_error = h.error;
  }
  if (h.error)
    return fail(c, h.error, h.error == BT_E_QUEUE_FULL ? "device queue or traversal stack overflow"
                                                        : "device error %d", h.error);
  return BT_OK;
}

BT_API int bt_ranges_stats(const bt_ctx *c, bt_stats *stats) {
  BT_RANGE();
  if (!c || !stats) return BT_E_INVALID;
  *stats = c->range_stats;
  return BT_OK;
}

BT_API int bt_cast_rays(bt_ctx *c, int32_t scene_id, const float *origins, const float *dirs,
                        const float *start_normals, int64_t n, float t_eps_m, float *t_out,
                        int32_t *tri_out) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  if (n < 0 || n > (1 << 28)) return fail(c, BT_E_INVALID, "bad ray count %lld", (long long)n);
  if (n > 0 && (!origins || !dirs || !t_out || !tri_out)) return fail(c, BT_E_INVALID, "NULL ray array");
  if (!(t_eps_m >= 0.0f)) return fail(c, BT_E_INVALID, "t_eps_m must be >= 0");
  if (n == 0) return BT_OK;
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  size_t v = sizeof(float) * 3 * (size_t)n;
  TRY(ensure(c, c->stage_a, 3 * v));
  TRY(ensure(c, c->stage_b, sizeof(float) * (size_t)n + sizeof(int) * (size_t)n + 256));
  float *d_o = (float *)c->stage_a.p, *d_d = d_o + 3 * n, *d_ns = start_normals ? d_d + 3 * n : nullptr;
  float *d_t = (float *)c->stage_b.p;
  int *d_id = (int *)(d_t + n);
  TRY(reset_counters(c));
  CK(cudaMemcpyAsync(d_o, origins, v, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(d_d, dirs, v, cudaMemcpyDefault, st));
  if (start_normals) CK(cudaMemcpyAsync(d_ns, start_normals, v, cudaMemcpyDefault, st));
  CK(bt::launch_cast(st, dev_scene(*s), d_o, d_d, d_ns, n, t_eps_m, d_t, d_id, &c->d_ctr->error));
  CK(cudaMemcpyAsync(t_out, d_t, sizeof(float) * n, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(tri_out, d_id, sizeof(int) * n, cudaMemcpyDefault, st));
  TRY(read_counters(c));
  if (c->h_ctr->error) return fail(c, c->h_ctr->error, "device error %d in ray query", c->h_ctr->error);
  return BT_OK;
}

// ============================================================ no allocation
// A trace that calls no cudaMalloc/cudaFree: its scratch (counters, beam
// table, segment records) lives in one file-scope device array of fixed size,
// and its results go straight into device arrays the caller owns.
namespace {

constexpr size_t kNoAllocBytes = (size_t)BT_NOALLOC_SCRATCH_MB << 20;
// Reserved on every GPU that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up on the
// first no-allocation call made with that device current.  Atomic, so that
// first calls from several host threads at once are well defined (they all
// store the same address).
std::atomic<void *> g_noalloc_ptr[256];

__global__ void k_levels_noalloc(const double *energy, const int *count, const float4 *mics, int64_t n_m,
                                 int n_bands, double *level_db, int *path_count) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_m) return;
  int64_t orig = __float_as_int(mics[p].w);
  for (int b = 0; b < n_bands; b++) {
    double I = energy[p * bt::kMaxBands + b];
    level_db[orig * n_bands + b] = I > 0.0 ? 10.0 * log10(I) + 120.0 : -__builtin_huge_val();
  }
  if (path_count) path_count[orig] = count[p];
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

BT_API int bt_trace_noalloc(bt_ctx *c, int32_t scene_id, const bt_trace_params *p, double *level_db,
                            int32_t *path_count) {
  BT_RANGE();
  TRY(check_ctx(c));
  c->err[0] = 0;
  SceneState *s;
  TRY(scene_ref(c, scene_id, &s));
  int has_alpha = 0;
  float alpha_log2[BT_MAX_BANDS];
  TRY(check_params(c, s, p, alpha_log2, &has_alpha));
  if (p->tiles_x != 1 || p->tiles_y != 1)
    return fail(c, BT_E_INVALID, "tiles %dx%d: bt_trace_noalloc traces without sub-domains (1x1 only)", p->tiles_x,
                p->tiles_y);
  if (s->level > BT_NOALLOC_MAX_LEVEL)
    return fail(c, BT_E_INVALID, "bt_trace_noalloc: icosahedron level %d exceeds the limit of %d of its %d MiB scratch",
                s->level, BT_NOALLOC_MAX_LEVEL, BT_NOALLOC_SCRATCH_MB);
  const size_t nv = (size_t)s->n_mics * s->n_bands;
  if (nv > 0 && (!level_db || !is_device_ptr(level_db, c->device)))
    return fail(c, BT_E_INVALID, "bt_trace_noalloc: level_db must be device memory of device %d", c->device);
  if (path_count && !is_device_ptr(path_count, c->device))
    return fail(c, BT_E_INVALID, "bt_trace_noalloc: path_count must be device memory of device %d or NULL", c->device);
  DeviceGuard g(c->device);
  if (c->device < 0 || c->device >= 256) return fail(c, BT_E_INVALID, "device ordinal %d out of range", c->device);
  char *base = (char *)g_noalloc_ptr[c->device].load(std::memory_order_acquire);
  if (!base) {
    // set-up, once per device, with that device current
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return fail(c, BT_E_CUDA, "bt_trace_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    }
    g_noalloc_ptr[c->device].store(ptr, std::memory_order_release);
    base = (char *)ptr;
  }
  // carve the scratch: counters, two cursors, beam table, segment records
  const int64_t n_beams = (int64_t)20 << (2 * s->level);
  const int mixed = p->precision == BT_PREC_MIXED ? 1 : 0;
  size_t off = 0;
  bt::Counters *ctr = (bt::Counters *)(base + off);
  off = align_up(off + sizeof(bt::Counters), 256);
  unsigned long long *seg_count = (unsigned long long *)(base + off);
  unsigned long long *lineage_next = seg_count + 1;
  off = align_up(off + 2 * sizeof(unsigned long long), 256);
  float *beam_table = (float *)(base + off);
  if (mixed) off = align_up(off + sizeof(float) * 24 * (size_t)n_beams, 256);
  bt::Seg *segs = (bt::Seg *)(base + off);
  const unsigned long long seg_room = (kNoAllocBytes - off) / sizeof(bt::Seg);
  const int64_t total = s->n_src * n_beams;
  int64_t chunk = (int64_t)(seg_room / (unsigned long long)(p->max_order + 1));
  if (chunk < 1) return fail(c, BT_E_INVALID, "bt_trace_noalloc: max_order %d too large for its scratch", p->max_order);
  if (p->chunk_beams > 0 && p->chunk_beams < chunk) chunk = p->chunk_beams;
  if (chunk > total) chunk = total > 0 ? total : 1;
  const unsigned long long cap = (unsigned long long)chunk * (p->max_order + 1);
  cudaStream_t st = c->stream;
  CK(cudaMemsetAsync(ctr, 0, sizeof(bt::Counters), st));
  CK(cudaMemsetAsync(s->energy.p, 0, sizeof(double) * bt::kMaxBands * (size_t)s->n_mics, st));
  CK(cudaMemsetAsync(s->count.p, 0, sizeof(int) * (size_t)s->n_mics, st));
  if (mixed && total > 0) CK(bt::launch_beam_table(st, s->level, beam_table));
  TRY(apply_leaf_size(c, *s, p, false));
  bt::TraceArgs ta;
  memset(&ta, 0, sizeof(ta));
  fill_view(ta.v, *s, p, alpha_log2, has_alpha);
  ta.v.beam_table = mixed ? beam_table : nullptr;
  ta.segs = segs;
  ta.seg_count = seg_count;
  ta.seg_capacity = cap;
  ta.lineage_next = lineage_next;
  ta.ctr = ctr;
  ta.count_work = p->count_work ? 1 : 0;
  ta.prec = p->precision;
  ta.blocks_per_sm = p->blocks_per_sm;
  ta.beams_per_warp = p->beams_per_warp;
  ta.leaf_size = p->leaf_size > 1 ? p->leaf_size : 1;
  bt::ScatterArgs sa;
  memset(&sa, 0, sizeof(sa));
  sa.v = ta.v;
  sa.fp64 = p->precision == BT_PREC_FP64 ? 1 : 0;
  sa.max_nz = s->nz;
  sa.segs = segs;
  sa.seg_count = seg_count;
  sa.seg_capacity = cap;
  sa.ctr = ctr;
  const int64_t n_chunks = total > 0 ? (total + chunk - 1) / chunk : 0;
  for (int64_t ci = 0; ci < n_chunks; ci++) {
    ta.lineage_begin = ci * chunk;
    ta.lineage_end = ta.lineage_begin + chunk < total ? ta.lineage_begin + chunk : total;
    CK(cudaMemsetAsync(seg_count, 0, 2 * sizeof(unsigned long long), st));
    CK(bt::launch_trace(st, ta, c->n_sm));
    if (s->n_mics > 0) CK(bt::launch_scatter(st, sa, c->n_sm));
  }
  if (s->n_mics > 0) {
    k_levels_noalloc<<<(int)((s->n_mics + 255) / 256), 256, 0, st>>>(
        (const double *)s->energy.p, (const int *)s->count.p, (const float4 *)s->mics.p, s->n_mics, s->n_bands,
        level_db, path_count);
    bt::note_launches(1);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(c->h_ctr, ctr, sizeof(bt::Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const bt::Counters &h = *c->h_ctr;
  bt_stats &o = s->stats;
  memset(&o, 0, sizeof(o));
  o.beams = total;
  o.segments = (int64_t)h.segments;
  o.hits = (int64_t)h.hits;
  o.escapes = (int64_t)h.escapes;
  o.emitted = (int64_t)h.emitted;
  o.candidates = (int64_t)h.candidates;
  o.contributions = (int64_t)h.contributions;
  o.nodes_visited = (int64_t)h.nodes_visited;
  o.tris_tested = (int64_t)h.tris_tested;
  o.trace_launches = n_chunks;
  o.scatter_launches = s->n_mics > 0 ? n_chunks : 0;
  if (h.error) {
    s->traced = false;
    s->trace_error = h.error;
    return fail(c, h.error, "device error %d in the no-allocation trace", h.error);
  }
  s->traced = true;
  s->trace_error = 0;
  return BT_OK;
}
