// bt_internal.cuh -- device data layouts and device helpers shared by the
// kernels of libbtrace.  Not part of the public ABI (include/btrace.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "btrace.h"

namespace bt {

constexpr int kMaxBands = BT_MAX_BANDS;
// traversal stack: a 4-wide step pushes at most three siblings, and the
// 4-wide hierarchy is at most 32 levels deep (an LBVH over 64-bit keys at most
// 64), plus the rests of multi-triangle leaves
constexpr int kStackDepth = 112;
constexpr float kInf = __builtin_huge_valf();

// ------------------------------------------------------------------ layouts
// Binary LBVH node as built, 64 bytes: both children's boxes.  Child index
// c >= 0: internal node; c < 0: a leaf, v = ~c: the leaf holds leaf_count(v)
// triangles from slot leaf_slot(v) on (a leaf of one triangle is ~slot;
// larger leaves come from collapsing small subtrees).  The traversal reads
// the 4-wide form below; the sub-domain trace's tile walk tests the binary
// root nodes.
struct __align__(16) Node {
  float4 lxy;  // left  lo.x, hi.x, lo.y, hi.y
  float4 rxy;  // right lo.x, hi.x, lo.y, hi.y
  float4 lrz;  // left lo.z, hi.z, right lo.z, hi.z
  int4 child;  // left, right, parent, far end of the node's key range
};

// 4-wide node, 128 bytes (one cache line), what the traversal reads: the
// boxes of up to four children, lane c of each float4 for child c, and their
// codes (as in Node; kNoChild for an unused lane).  Wide node i stands for
// binary node i and lists its grandchildren -- a child that is a leaf stands
// for itself -- so a traversal from any binary node visits the wide nodes of
// every other level below it.
constexpr int kNoChild = (int)0x80000000;
struct __align__(128) Node4 {
  float4 lox, hix, loy, hiy, loz, hiz;
  int4 child;
  int4 unused;
};
static_assert(sizeof(Node4) == 128, "wide node layout");

// A hierarchy's buffer: the binary LBVH (n_leaves - 1 nodes), then its wide
// form at a 256-byte boundary (one Node4 per binary node).
__host__ __device__ inline size_t hier_binary_bytes(int64_t n_leaves) {
  const size_t m = (size_t)(n_leaves > 1 ? n_leaves - 1 : 1);
  return (sizeof(Node) * m + 255) & ~(size_t)255;
}
__host__ __device__ inline size_t hier_bytes(int64_t n_leaves) {
  const size_t m = (size_t)(n_leaves > 1 ? n_leaves - 1 : 1);
  return hier_binary_bytes(n_leaves) + sizeof(Node4) * m;
}
__host__ __device__ inline Node4 *hier_wide(void *base, int64_t n_leaves) {
  return (Node4 *)((char *)base + hier_binary_bytes(n_leaves));
}

constexpr int kLeafShift = 29;  // leaf code: slot in bits 0..28, count - 1 above
constexpr int kMaxLeafSize = 4;
__host__ __device__ __forceinline__ int leaf_slot(int v) { return v & ((1 << kLeafShift) - 1); }
__host__ __device__ __forceinline__ int leaf_count(int v) { return (v >> kLeafShift) + 1; }

// Triangle in leaf order, 48 bytes for the hit test: v0.w = material (int
// bits), v1.w = original triangle id (int bits), v2.w unused.
struct __align__(16) Tri {
  float4 v0, v1, v2;
};

// Plane of a triangle: unit normal (x, y, z) and w = n . v0.
using Plane = float4;
// The same in float64, 32 bytes.
struct __align__(32) Plane64 {
  double x, y, z, w;
};
// The same as float pairs (hi + lo, see double-float below): hi = (n.hi, w.hi),
// lo = (n.lo, w.lo).
struct __align__(16) PlaneDF {
  float4 hi, lo;
};

// Sub-domain grid over the scene's xy box grown by 1 m: tx x ty tiles of
// wx x wy, tile (ix, iy) = [gx0 + ix wx, gx0 + (ix+1) wx) x [...), half-open,
// points outside clamped to the border tiles.
struct TileGrid {
  float gx0, gy0, wx, wy;
  float gx1, gy1;
  int tx, ty;
};

// Everything the sub-domain trace needs besides TraceArgs.  Each tile has a
// ring queue of handed-off lineages: `qcap` slots (a power of two), each
// holding a lineage's whole state as kStateRows words (row r of slot q of
// tile k at ring[(k * kStateRows + r) * qcap + q]).  Positions count up from
// zero per launch: a producer reserves positions by advancing tail[k] and,
// once they are written, adds them to avail[k]; a consumer first takes items
// from avail[k] (a counting semaphore) and then positions from head[k].
// seq[k * qcap + slot], relative to the position's generation
// g = pos & ~(qcap - 1), says whether the slot is free for it (g), filled
// (g + 1), or released to the next generation (g + qcap).  At most qcap
// lineages are in flight (traced or queued) at any time, so a ring never
// holds more than qcap items and a producer never waits for a consumer.
struct TiledArgs {
  TileGrid tg;
  int n_tiles;
  const int *roots;         // [n_tiles] subtree root per tile (INT_MIN: empty tile)
  const Node *bin;          // the binary LBVH the wide nodes come from (the tile walk's root tests)
  unsigned qcap;            // ring slots per tile, a power of two; also the cap on lineages in flight
  uint32_t *ring;           // [n_tiles][kStateRows][qcap]
  unsigned *seq;            // [n_tiles][qcap], zero at launch
  int *ctl;                 // zero at launch: head[n_tiles], tail[n_tiles], avail[n_tiles],
                            // credits in use, lineages finished
  unsigned long long watchdog_ns;  // bound on any wait of a warp that has no work
  int withhold;             // test hook: the launch's first hand-off is never published
};

struct DevScene {
  int64_t n_tris;
  int root;              // root child code: internal index >= 0, or ~leaf for one triangle (unused when n_tris == 0)
  const Node4 *nodes;    // n_tris - 1 wide nodes (hier_wide)
  const Tri *tris;       // n_tris, leaf order
  const Plane *planes;   // n_tris, leaf order
  const Plane64 *planes64;  // n_tris, leaf order: float64 unit normal and n . v0
  const PlaneDF *planes_df; // n_tris, leaf order: the float64 plane split into float pairs
  const float *refl;     // [n_mat][n_bands]
  int n_mat, n_bands;
  float lo[3], hi[3];    // scene box
};

// Microphone bin grid over the microphones' box: nx x ny cells in xy and nz
// layers in z (one layer for microphones at one height; several for a
// volumetric set), cell (layer, row, column) = (iz * ny + iy) * nx + ix.
// [zlo, zhi] is the microphones' height slab.
struct MicGrid {
  float x0, y0, cw, ch, inv_cw, inv_ch, zlo, zhi;
  int nx, ny;
  int n_mics;
  int nz;
  float z0, dz, inv_dz, pad;
};

// One beam segment handed from the trace kernel to the scatter kernel, 192 B.
// The apex and the cone normals are float pairs (hi + lo; lo is zero in
// BT_PREC_FP32).  With v = m - apex, microphone m is inside when
// n_j . v >= 0 (j = 0,1,2), start.xyz . v - start.w > 0 and
// end.xyz . v - end.w >= 0; plane offsets are relative to the apex.  A
// missing plane is (0, 0, 0, -inf).
struct __align__(16) Seg {
  float ahi[3], alo[3];  // apex (source or image source)
  int view;              // index of the scene view (0 in a single-scene trace)
  int key;               // the microphone-grid cell under the segment, x | y << 16, when the scene orders
                         // its scatter by place (SceneView::seg_key), else 0
  float4 n0;             // cone-face normal 0 (hi); w: leaf slot of the start plane's triangle (-1 none)
  float4 n1;             // w: leaf slot of the end plane's triangle (-1 none)
  float4 n2;             // w: reflection order (int bits)
  float4 start;
  float4 end;
  float4 p03;            // per-band power W_b * prod(r_b), bands 0..3
  float4 p47;            // bands 4..7
  float nlo[9];          // lo parts of the three cone normals
  float pad[3];
};
static_assert(sizeof(Seg) == 192, "segment record layout");

// Device counters of one trace, accumulated with atomics.
struct Counters {
  unsigned long long segments, hits, escapes, emitted, candidates, contributions;
  unsigned long long handoffs, steals, rounds, pad2;
  unsigned long long nodes_visited, tris_tested;
  int error;  // sticky error code set by kernels (0 = none)
  int pad;
};

// Everything the trace and scatter kernels need about one scene: geometry,
// sources, microphones, result arrays and trace parameters.  A single-scene
// trace passes one view by value; a batch passes an array of views in device
// memory and every lineage and segment carries its view's index.
struct SceneView {
  DevScene sc;
  const float4 *src;      // [n_s] xyz
  const float *power;     // [n_s][n_bands]
  int64_t n_src;
  int level;              // icosahedron level L
  int max_order;
  int64_t n_beams;        // 20 * 4^L
  int64_t lineage_base;   // batch: first lineage of this scene in the batch's lineage space
  int64_t lineage_first;  // batch: the scene's own lineage index at lineage_base
  float t_eps;
  float energy_threshold;
  float alpha_log2[kMaxBands];  // air damping as a base-2 exponent per metre: -alpha_b * log2(10) / 10
  int has_alpha;
  int seg_key;            // 1: each segment record carries its grid cell (Seg::key)
  const MicGrid *grid;
  const float *beam_table;   // MIXED: per beam 3 cone normals + axis as float pairs: [n_beams][12] hi, then lo
  const float4 *mics;        // sorted by cell: xyz, w = original index (int bits)
  const int *cell_start;     // [nx * ny + 1]
  double *energy;            // [n_mics][kMaxBands], sorted order
  int *count;                // [n_mics], sorted order
  const float *dir_gain;     // directional sources: [n_patterns][n_beams] gains, or null
  const int *dir_of;         // [n_src]: each source's pattern, -1 = omnidirectional; null = all
};

struct TraceArgs {
  SceneView v;                         // the scene (single-scene trace)
  const SceneView *views;              // batch: [n_views] in device memory, else null
  int n_views;
  int64_t lineage_begin, lineage_end;  // chunk of (scene,) source, beam lineages
  unsigned long long *lineage_next;    // lineages of the chunk taken so far (zeroed per chunk)
  Seg *segs;
  unsigned long long *seg_count;
  unsigned long long seg_capacity;
  Counters *ctr;
  int count_work;
  int prec;   // BT_PREC_FP32, BT_PREC_MIXED or BT_PREC_FP64
  int blocks_per_sm;  // persistent grid: resident blocks per SM, 0 = as many as fit
  int beams_per_warp; // lineages a warp reserves at a time (0 = what its lanes need)
  int leaf_size;      // most triangles per BVH leaf (1: the traversal without leaf runs)
  int *hit_log;       // single-scene traces: [lineages][hit_log_stride] hit triangle per segment, or null
  int hit_log_stride; // max_order + 1
};

struct ScatterArgs {
  SceneView v;              // the scene (single-scene trace)
  const SceneView *views;   // batch: [n_views] in device memory, else null
  int n_views;
  int fp64;                 // 1: every microphone test in float64 (BT_PREC_FP64)
  int max_nz;               // most microphone layers of any scene traced
  const Seg *segs;
  const unsigned long long *seg_count;
  unsigned long long seg_capacity;
  Counters *ctr;
  const uint32_t *order;    // the emitted segments in order of place (launch_seg_order), or null
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Cross product without contraction into FMA: b x a is then exactly -(a x b),
// so two beams sharing an edge test it with exactly opposite signs.
__device__ __forceinline__ float3 cross_exact(float3 a, float3 b) {
  return make_float3(__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)),
                     __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
                     __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

__device__ __forceinline__ float3 normalize3(float3 a) { return a * rsqrtf(dot3(a, a)); }

__device__ __forceinline__ float pick(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// Ray prepared for the watertight test (Woop, Benthin & Wald, JCGT 2013):
// axes permuted so the dominant direction component is z, plus a shear.
struct Ray {
  float3 o, d, inv;
  int kx, ky, kz;
  float sx, sy, sz;
  float t_eps;
  float dns;  // d . n_start for a reflected ray, 0 for a primary ray
};

__device__ __forceinline__ Ray make_ray(float3 o, float3 d, float t_eps, float dns) {
  Ray r;
  r.o = o;
  r.d = d;
  // zero components become tiny so the slab test never forms 0 * inf
  float dx = fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x);
  float dy = fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y);
  float dz = fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z);
  r.inv = make_float3(1.0f / dx, 1.0f / dy, 1.0f / dz);
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  if (pick(d, kz) < 0.0f) { int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  float dkz = pick(d, kz);
  r.sx = pick(d, kx) / dkz;
  r.sy = pick(d, ky) / dkz;
  r.sz = 1.0f / dkz;
  r.t_eps = t_eps;
  r.dns = dns;
  return r;
}

// Watertight, two-sided ray/triangle test.  Edge functions are formed
// without FMA contraction so a shared edge gets exactly opposite values in
// its two triangles, and recomputed in double when one is exactly zero, as
// the published method prescribes.  Returns the hit distance or +inf.
// `amb` is set when the ray passes within a relative 1e-4 of an edge (or
// nearly parallel to the plane): there a float32 ray that was rounded from a
// float64 one may decide differently, and callers holding the float64 ray
// re-test it in float64.
__device__ __forceinline__ float hit_watertight(const Ray &r, float4 v0, float4 v1, float4 v2, bool &amb) {
  float3 A = f3(v0) - r.o, B = f3(v1) - r.o, C = f3(v2) - r.o;
  float Akz = pick(A, r.kz), Bkz = pick(B, r.kz), Ckz = pick(C, r.kz);
  float ax = pick(A, r.kx) - r.sx * Akz, ay = pick(A, r.ky) - r.sy * Akz;
  float bx = pick(B, r.kx) - r.sx * Bkz, by = pick(B, r.ky) - r.sy * Bkz;
  float cx = pick(C, r.kx) - r.sx * Ckz, cy = pick(C, r.ky) - r.sy * Ckz;
  float u1 = __fmul_rn(cx, by), u2 = __fmul_rn(cy, bx);
  float v1_ = __fmul_rn(ax, cy), v2_ = __fmul_rn(ay, cx);
  float w1 = __fmul_rn(bx, ay), w2 = __fmul_rn(by, ax);
  float U = __fsub_rn(u1, u2), V = __fsub_rn(v1_, v2_), W = __fsub_rn(w1, w2);
  // ambiguous: every edge function that is clearly away from zero agrees in
  // sign (so the decision is not a clear miss) and at least one lies within
  // the rounding band of its terms
  const float tau = 1e-4f;
  float su = fabsf(u1) + fabsf(u2), sv = fabsf(v1_) + fabsf(v2_), sw = fabsf(w1) + fabsf(w2);
  bool zu = fabsf(U) <= tau * su, zv = fabsf(V) <= tau * sv, zw = fabsf(W) <= tau * sw;
  bool pos = (!zu && U > 0.0f) || (!zv && V > 0.0f) || (!zw && W > 0.0f);
  bool neg = (!zu && U < 0.0f) || (!zv && V < 0.0f) || (!zw && W < 0.0f);
  amb = (zu || zv || zw) && !(pos && neg);
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = (float)((double)cx * (double)by - (double)cy * (double)bx);
    V = (float)((double)ax * (double)cy - (double)ay * (double)cx);
    W = (float)((double)bx * (double)ay - (double)by * (double)ax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return kInf;
  float det = U + V + W;
  if (det == 0.0f) return kInf;
  float T = U * (r.sz * Akz) + V * (r.sz * Bkz) + W * (r.sz * Ckz);
  float t = __fdiv_rn(T, det);
  return t;
}

// float64 vectors
__device__ __forceinline__ double3 d3(float4 v) { return make_double3(v.x, v.y, v.z); }
__device__ __forceinline__ double3 operator+(double3 a, double3 b) { return make_double3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ double3 operator-(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double3 operator*(double3 a, double s) { return make_double3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double dot3(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 cross3(double3 a, double3 b) {
  return make_double3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// b x a is exactly -(a x b): no contraction into FMA
__device__ __forceinline__ double3 cross_exact(double3 a, double3 b) {
  return make_double3(__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)),
                      __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
                      __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double3 normalize3(double3 a) { return a * (1.0 / sqrt(dot3(a, a))); }
__device__ __forceinline__ Plane64 ldg_d4(const Plane64 *p) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  Plane64 r;
  r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
  return r;
}

// Moller & Trumbore (1997) in float64, two-sided, edges inclusive: the
// float64 re-test of an ambiguous float32 decision, and the float64 hit
// distance of the chosen triangle.
__device__ __forceinline__ bool hit_mt64(double3 o, double3 d, float4 fa, float4 fb, float4 fc, double &t) {
  double3 a = d3(fa), e1 = d3(fb) - a, e2 = d3(fc) - a;
  double3 p = cross3(d, e2);
  double det = dot3(e1, p);
  if (det == 0.0) return false;
  double inv = 1.0 / det;
  double3 s = o - a;
  double u = dot3(s, p) * inv;
  if (u < 0.0 || u > 1.0) return false;
  double3 q = cross3(s, e1);
  double v = dot3(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  t = dot3(e2, q) * inv;
  return true;
}

// Hit acceptance (same rule as the oracle): beyond t_eps, and for a reflected
// ray more than t_eps away from the plane it left.
__device__ __forceinline__ bool accept_hit(const Ray &r, float t) {
  return t > r.t_eps && (r.dns == 0.0f || t * r.dns > r.t_eps);
}

// Three-input minimum and maximum (one instruction each on sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Slab test with the ray origin pre-scaled: (lo - o) * inv is formed as
// fma(lo, inv, -o * inv), one instruction per bound; oi = o * inv.  The far
// distance is grown by 1 + 2*gamma(3) as in the robust test of Ize (2013), and
// the boxes themselves are grown at build time (1e-6 relative + 0.1 mm), which
// covers the rounding of o * inv (at most |o| * 2^-24 along the ray).
__device__ __forceinline__ bool slab(const Ray &r, float3 oi, float lox, float hix, float loy, float hiy,
                                     float loz, float hiz, float tmax, float &tnear) {
  float tx0 = fmaf(lox, r.inv.x, -oi.x), tx1 = fmaf(hix, r.inv.x, -oi.x);
  float ty0 = fmaf(loy, r.inv.y, -oi.y), ty1 = fmaf(hiy, r.inv.y, -oi.y);
  float tz0 = fmaf(loz, r.inv.z, -oi.z), tz1 = fmaf(hiz, r.inv.z, -oi.z);
  float tn = fmax3(fminf(tx0, tx1), fminf(ty0, ty1), fmaxf(fminf(tz0, tz1), 0.0f));
  float tf = fmin3(fmaxf(tx0, tx1), fmaxf(ty0, ty1), fmaxf(tz0, tz1)) * 1.0000004f;
  tnear = tn;
  return tn <= fminf(tf, tmax);
}
__device__ __forceinline__ float3 origin_scaled(const Ray &r) {
  return make_float3(r.o.x * r.inv.x, r.o.y * r.inv.y, r.o.z * r.inv.z);
}
__device__ __forceinline__ bool slab(const Ray &r, float lox, float hix, float loy, float hiy, float loz, float hiz,
                                     float tmax, float &tnear) {
  return slab(r, origin_scaled(r), lox, hix, loy, hiy, loz, hiz, tmax, tnear);
}

// ------------------------------------------------------------ double-float
// Unevaluated sums hi + lo of two float32 (about 48 significant bits), built
// from the error-free transformations TwoSum (Knuth), Fast2Sum (Dekker) and
// FMA-based TwoProd, in the arrangement of the published double-double
// algorithms (Hida, Li & Bailey).  GB300 runs float32 some 64 times faster
// than float64, so the image-source chain uses these pairs instead of double.
// Every step is written with explicit round-to-nearest intrinsics so the
// compiler cannot contract or reassociate it.
struct df {
  float hi, lo;
};
struct df3 {
  df x, y, z;
};

__device__ __forceinline__ df mkdf(float a) { return df{a, 0.0f}; }
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // needs |a| >= |b| (or a == 0)
  float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
// The "sloppy" pair sum (Dekker's add2; QD's sloppy_add): the high parts by
// TwoSum, the low parts added in float32, one renormalisation.  Its error is
// bounded relative to |a| + |b| rather than to |a + b|, which is the bound the
// geometry needs: every sum here is a coordinate, a plane offset or a
// component of a unit vector, whose absolute error matters on the scale of
// its operands (2^-44 of 2 km is 0.1 nm).  It takes 11 float32 operations
// against 20 for the variant accurate to the result (district split trace
// 44.9 -> 41.5 ms, identical levels and path counts).
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ df df_mulf(df a, float b) {
  df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_sub(a, df_mulf(b, q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = df_sub(r, df_mulf(b, q2));
  float q3 = __fdiv_rn(r.hi, b.hi);
  df q = fast_two_sum(q1, q2);
  return df_add(q, mkdf(q3));
}
__device__ __forceinline__ df3 mkdf3(float3 v) { return df3{mkdf(v.x), mkdf(v.y), mkdf(v.z)}; }
__device__ __forceinline__ df3 df3_add(df3 a, df3 b) { return df3{df_add(a.x, b.x), df_add(a.y, b.y), df_add(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_sub(df3 a, df3 b) { return df3{df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_scale(df3 a, df s) { return df3{df_mul(a.x, s), df_mul(a.y, s), df_mul(a.z, s)}; }
__device__ __forceinline__ df df3_dot(df3 a, df3 b) {
  return df_add(df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_mul(a.z, b.z));
}
// mirror of a direction (or plane normal) v in the plane with unit normal n
__device__ __forceinline__ df3 df3_mirror(df3 v, df3 n) {
  df k = df3_dot(v, n);
  k = df{2.0f * k.hi, 2.0f * k.lo};
  return df3_sub(v, df3_scale(n, k));
}
// Fused forms for the reflection, each about half the operations of the
// same expression built from the pair operations above, with an error of
// the same order relative to the operands' magnitudes.
// a . b: the products of the high parts exact (TwoProd) and summed by
// TwoSum, every low-order term gathered in one float32 (the compensated dot
// product Dot2 of Ogita, Rump and Oishi, with pair operands).
__device__ __forceinline__ df df3_dot2(df3 a, df3 b) {
  df px = two_prod(a.x.hi, b.x.hi), py = two_prod(a.y.hi, b.y.hi), pz = two_prod(a.z.hi, b.z.hi);
  df s = two_sum(px.hi, py.hi);
  df u = two_sum(s.hi, pz.hi);
  float c = __fadd_rn(__fadd_rn(s.lo, u.lo), __fadd_rn(__fadd_rn(px.lo, py.lo), pz.lo));
  c = __fmaf_rn(a.x.hi, b.x.lo, c);
  c = __fmaf_rn(a.x.lo, b.x.hi, c);
  c = __fmaf_rn(a.y.hi, b.y.lo, c);
  c = __fmaf_rn(a.y.lo, b.y.hi, c);
  c = __fmaf_rn(a.z.hi, b.z.lo, c);
  c = __fmaf_rn(a.z.lo, b.z.hi, c);
  return fast_two_sum(u.hi, c);
}
// v - 2 k n (a mirror image once k = v . n): the high product exact, the
// high difference by TwoSum (2 k n is exact scaling), the rest in float32.
__device__ __forceinline__ df df_sub2kn(df v, df k, df n) {
  df q = two_prod(k.hi, n.hi);
  df s = two_sum(v.hi, -2.0f * q.hi);
  float t = __fmaf_rn(k.hi, n.lo, q.lo);
  t = __fmaf_rn(k.lo, n.hi, t);
  return fast_two_sum(s.hi, __fmaf_rn(-2.0f, t, __fadd_rn(s.lo, v.lo)));
}
__device__ __forceinline__ df3 df3_sub2kn(df3 v, df k, df3 n) {
  return df3{df_sub2kn(v.x, k, n.x), df_sub2kn(v.y, k, n.y), df_sub2kn(v.z, k, n.z)};
}
// o + s d, the same way.
__device__ __forceinline__ df df_axpy(df o, df s, df d) {
  df q = two_prod(s.hi, d.hi);
  df u = two_sum(o.hi, q.hi);
  float t = __fmaf_rn(s.hi, d.lo, q.lo);
  t = __fmaf_rn(s.lo, d.hi, t);
  return fast_two_sum(u.hi, __fadd_rn(__fadd_rn(u.lo, o.lo), t));
}
// a / b to two terms: q1 = a.hi / b.hi, the remainder a - q1 b with q1 b.hi
// exact, and its quotient as the low part.
__device__ __forceinline__ df df_div2(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df p = two_prod(q1, b.hi);
  float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), __fsub_rn(a.lo, __fmul_rn(q1, b.lo)));
  return fast_two_sum(q1, __fdiv_rn(r, b.hi));
}
__device__ __forceinline__ float3 df3_hi(df3 a) { return make_float3(a.x.hi, a.y.hi, a.z.hi); }
__device__ __forceinline__ df d_to_df(double x) {
  float hi = (float)x;
  return df{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

}  // namespace bt

// ------------------------------------------------------------ host launchers
namespace bt {
// process-wide count of kernel launches (host side), read by bt_kernel_launches()
void note_launches(int n);
// scene build in two steps: validation (sets *d_error, fills the scene box)
// and, only if validation passed, the BVH build.
cudaError_t validate_scene(cudaStream_t st, const float *d_verts, int64_t n_verts,
                           const int32_t *d_tris, int64_t n_tris, const uint8_t *d_mat, int n_mat,
                           float *d_box /*lo xyz, hi xyz*/, int *d_error);
cudaError_t build_scene(cudaStream_t st, const float *d_verts, const int32_t *d_tris, int64_t n_tris,
                        const uint8_t *d_mat, void *d_hier, Tri *d_tris_out, Plane *d_planes,
                        Plane64 *d_planes64, PlaneDF *d_planes_df, void *d_scratch, size_t scratch_bytes,
                        const float *d_box, int *d_error);
cudaError_t launch_beam_table(cudaStream_t st, int level, float *table);
cudaError_t launch_beam_axes(cudaStream_t st, int level, float *axes);
size_t build_tiled_scratch_bytes(int64_t n_src, int64_t n_pairs);
cudaError_t tiled_count(cudaStream_t st, const Tri *src, int64_t n_src, const TileGrid &tg, uint32_t *offs);
cudaError_t tiled_build(cudaStream_t st, const Tri *src, const Plane *sp, const Plane64 *sp64, const PlaneDF *spdf,
                        int64_t n_src, const TileGrid &tg, const float *d_box, const uint32_t *offs, int64_t n_pairs,
                        void *scratch, size_t scratch_bytes, void *hier, Tri *tris, Plane *planes,
                        Plane64 *planes64, PlaneDF *planes_df, int *roots, int *d_error);
size_t build_scene_scratch_bytes(int64_t n_tris);
// Rewrite the child links of a built LBVH (n_leaves leaves) so that every
// subtree of at most leaf_size triangles is one leaf; any earlier collapse is
// undone first, so the call can change the leaf size back and forth.  The
// wide form is rebuilt after.  `hier`: the hierarchy's buffer (hier_bytes).
cudaError_t collapse_leaves(cudaStream_t st, void *hier, int64_t n_leaves, int leaf_size);
// (Re)build the wide form of the binary LBVH in `hier`.
cudaError_t widen(cudaStream_t st, void *hier, int64_t n_leaves);
cudaError_t mic_box(cudaStream_t st, const float *d_pos, int64_t n_m, float *d_box, int *d_error);
cudaError_t build_mics(cudaStream_t st, const float *d_pos, int64_t n_m, int nx, int ny, int nz,
                       const float *d_box, MicGrid *d_grid, float4 *d_sorted, int *d_cell_start, void *d_scratch,
                       size_t scratch_bytes);
size_t build_mics_scratch_bytes(int64_t n_m);
cudaError_t launch_trace(cudaStream_t st, const TraceArgs &a, int n_sm);
cudaError_t launch_trace_tiled(cudaStream_t st, const TraceArgs &a, const TiledArgs &t, int n_sm);
int tiled_resident_lanes(int n_sm);  // lanes of one full persistent sub-domain launch
constexpr int kStateRows = 56;
cudaError_t launch_cast(cudaStream_t st, const DevScene &sc, const float *o, const float *d, const float *ns,
                        int64_t n, float t_eps, float *t_out, int *tri_out, int *err);
cudaError_t launch_scatter(cudaStream_t st, const ScatterArgs &a, int n_sm);
// Order of the emitted segments by place (the grid cell in each record's
// key, bins along a Morton curve); hist holds kOrderBins counters and is
// zeroed here, order receives min(*seg_count, cap) record indices.
constexpr int kOrderBits = 6, kOrderBins = 1 << (2 * kOrderBits);
cudaError_t launch_seg_order(cudaStream_t st, const Seg *segs, const unsigned long long *seg_count,
                             unsigned long long cap, const MicGrid *grid, uint32_t *hist, uint32_t *order,
                             int n_sm);
cudaError_t launch_set_result(cudaStream_t st, const double *intensity, const int *count_in, const float4 *mics,
                              int64_t n_m, int n_bands, double *energy, int *count);
// L2 read-bandwidth probe: `blocks` blocks of 256 threads read the n4 float4s
// of buf `repeats` times; sink holds blocks * 256 floats.
cudaError_t launch_l2_read(cudaStream_t st, const float4 *buf, int64_t n4, int repeats, float *sink, int blocks);
cudaError_t launch_l2_atomics(cudaStream_t st, double *buf, uint32_t n_slots, int repeats, int blocks);
cudaError_t launch_levels(cudaStream_t st, const double *energy, const int *count, const float4 *mics,
                          int64_t n_m, int n_bands, double *level_db, double *intensity, int *path_count);
}  // namespace bt
