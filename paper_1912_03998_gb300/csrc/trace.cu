// trace.cu -- the tracing half of the hot path of the hybrid beam/ray
// tracer (Section 2 of the paper): beam generation, axis-ray traversal and
// image-source reflection, with and without the sub-domain split (Section 3).
// The microphone-in-beam test, the energy scatter and the level readout are
// in scatter.cu.
//
//   k_trace   persistent warps, one lineage (source, icosahedron face) per
//             lane: for orders 0..K it casts the beam's axis ray through the
//             BVH, writes the segment (apex, cone planes, start/end planes,
//             band power) unless it cannot reach the microphones' height, and
//             reflects the beam about the hit triangle's plane (image source);
//             a lane whose lineage ends takes the next one at once.
//   k_trace_tiled  the same over sub-domains (Section 3): one hierarchy per
//             tile, hand-off queues between tiles and work stealing, all in
//             one persistent launch.
//   k_cast    the axis-ray query on its own (closest hit of given rays).
//
// Precision.  BT_PREC_FP32 carries the lineage in float32.  BT_PREC_MIXED
// carries the image-source chain -- apex, cone normals, ray origin and
// direction -- as float pairs (about 48 bits, on the float32 pipe) from a
// float64 beam table through every reflection, on the triangles' float64
// planes.  Traversal is float32; a triangle whose float32 test is ambiguous
// (the ray within a relative 1e-4 of an edge) is re-tested in float64, near-
// equal hit distances are compared in float64 -- both after the search, from
// a short per-lane list, so that no float64 code sits in the traversal loop.
// The reflection's float-pair arithmetic runs in stages, each reading its
// rows from shared memory and writing them back.  The microphone tests are
// in scatter.cu.
#include <stdio.h>

#include <type_traits>

#include "bt_internal.cuh"

namespace bt {

// precision variants of the trace kernels (BT_PREC_*)
constexpr int kPF32 = 0, kPMixed = 1, kPF64 = 2, kPMixed64 = 3;
// What each variant does: the image-source chain (apex, cone normals, ray
// origin and direction) as float pairs (`pairs`, MIXED) or in float64
// (`chain64`, FP64 and MIXED64), else float32; float32 triangle tests whose
// ambiguous cases and near ties are settled in float64 after the search
// (`defer`, MIXED and MIXED64), or every triangle test in float64 (`all64`,
// FP64).
template <int kP>
struct Prec {
  static constexpr bool pairs = kP == kPMixed;
  static constexpr bool chain64 = kP == kPF64 || kP == kPMixed64;
  static constexpr bool defer = kP == kPMixed || kP == kPMixed64;
  static constexpr bool all64 = kP == kPF64;
};

// Regular icosahedron: unit vertices (the cyclic permutations of
// (0, +-1, +-phi), normalised) and its 20 faces, counter-clockwise seen
// from outside.  Vertex coordinates are 0, +-A or +-B with
// A = 1/sqrt(1+phi^2), B = phi/sqrt(1+phi^2); the table holds 0, +-1 (A),
// +-2 (B).
__constant__ signed char c_ico_s[12][3] = {
    {0, -1, 2}, {0, 1, 2},   {2, 0, 1},   {-2, 0, 1},  {-1, -2, 0}, {1, -2, 0},
    {1, 2, 0},  {-1, 2, 0},  {2, 0, -1},  {-2, 0, -1}, {0, -1, -2}, {0, 1, -2},
};
__constant__ int c_ico_f[20][3] = {
    {0, 2, 1},  {0, 1, 3},  {0, 5, 2},  {0, 3, 4},  {1, 2, 6},   {1, 7, 3},  {0, 4, 5},
    {1, 6, 7},  {2, 5, 8},  {2, 8, 6},  {3, 9, 4},  {3, 7, 9},   {4, 10, 5}, {6, 11, 7},
    {4, 9, 10}, {5, 10, 8}, {6, 8, 11}, {7, 11, 9}, {8, 10, 11}, {9, 11, 10},
};

template <typename T>
struct Vec3;
template <>
struct Vec3<float> { using type = float3; };
template <>
struct Vec3<double> { using type = double3; };

template <typename T>
__device__ __forceinline__ typename Vec3<T>::type ico_vertex(int v) {
  const T phi = (T)0.5 * ((T)1 + sqrt((T)5));
  const T inv = (T)1 / sqrt((T)1 + phi * phi);
  const T A = inv, B = phi * inv;
  T c[3];
  for (int k = 0; k < 3; k++) {
    int s = c_ico_s[v][k];
    c[k] = s == 0 ? (T)0 : (s == 1 ? A : (s == -1 ? -A : (s == 2 ? B : -B)));
  }
  typename Vec3<T>::type r;
  r.x = c[0];
  r.y = c[1];
  r.z = c[2];
  return r;
}

// Edge directions of face `i` of the level-L geodesic icosahedron.  The base
// face is i >> 2L; each further pair of bits picks one of the four children
// (a,ab,ca), (ab,b,bc), (ca,bc,c), (ab,bc,ca), ab = midpoint pushed to the
// sphere.  A vertex shared by two faces is computed from the same operands in
// both, so both faces get the bit-identical direction.
template <typename T>
__device__ __forceinline__ void beam_dirs(int level, int64_t i, typename Vec3<T>::type &a,
                                          typename Vec3<T>::type &b, typename Vec3<T>::type &c) {
  int f = (int)(i >> (2 * level));
  a = ico_vertex<T>(c_ico_f[f][0]);
  b = ico_vertex<T>(c_ico_f[f][1]);
  c = ico_vertex<T>(c_ico_f[f][2]);
  for (int l = level - 1; l >= 0; --l) {
    int ch = (int)((i >> (2 * l)) & 3);
    auto ab = normalize3(a + b), bc = normalize3(b + c), ca = normalize3(c + a);
    if (ch == 0) { b = ab; c = ca; }
    else if (ch == 1) { a = ab; c = bc; }
    else if (ch == 2) { a = ca; b = bc; }
    else { a = ab; b = bc; c = ca; }
  }
}

// Beam table of one icosahedron level, formed in float64 and stored as float
// pairs: per beam the three cone-face normals d_j x d_{j+1} (no FMA, so
// neighbours share exactly opposite normals; the split keeps that) and the
// unit axis -- 12 hi floats, then 12 lo floats.
__global__ void k_beam_table(int level, int64_t n_beams, float *table) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_beams) return;
  double3 d0, d1, d2;
  beam_dirs<double>(level, i, d0, d1, d2);
  double3 v[4] = {cross_exact(d0, d1), cross_exact(d1, d2), cross_exact(d2, d0), normalize3((d0 + d1) + d2)};
  float *o = table + 24 * i;
  for (int k = 0; k < 4; k++) {
    double c[3] = {v[k].x, v[k].y, v[k].z};
    for (int q = 0; q < 3; q++) {
      df h = d_to_df(c[q]);
      o[3 * k + q] = h.hi;
      o[12 + 3 * k + q] = h.lo;
    }
  }
}

cudaError_t launch_beam_table(cudaStream_t st, int level, float *table) {
  int64_t n = (int64_t)20 << (2 * level);
  k_beam_table<<<(int)((n + 127) / 128), 128, 0, st>>>(level, n, table);
  note_launches(1);
  return cudaGetLastError();
}

// Unit axis of every beam of a level, float32 [n_beams][3] (the order of the
// lineages' beam index: a directional source's gains are given in it).
__global__ void k_beam_axes(int level, int64_t n_beams, float *axes) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_beams) return;
  double3 d0, d1, d2;
  beam_dirs<double>(level, i, d0, d1, d2);
  const double3 ax = normalize3((d0 + d1) + d2);
  axes[3 * i] = (float)ax.x;
  axes[3 * i + 1] = (float)ax.y;
  axes[3 * i + 2] = (float)ax.z;
}

cudaError_t launch_beam_axes(cudaStream_t st, int level, float *axes) {
  const int64_t n = (int64_t)20 << (2 * level);
  k_beam_axes<<<(int)((n + 127) / 128), 128, 0, st>>>(level, n, axes);
  note_launches(1);
  return cudaGetLastError();
}

// float64 distance along the ray to the plane of leaf slot `slot`.
__device__ __forceinline__ double plane_t64(const DevScene &sc, int slot, double3 od, double3 dd) {
  Plane64 pl = ldg_d4(&sc.planes64[slot]);
  double3 n = make_double3(pl.x, pl.y, pl.z);
  return (pl.w - dot3(n, od)) / dot3(n, dd);
}

// Best hit so far.  In MIXED mode t64 holds the float64 distance when known.
struct Best {
  float t;
  int slot, id;
  double t64;
  bool has64;
};

// Candidates a MIXED search leaves to float64 (kPend at most per search):
// triangles whose float32 test was ambiguous (slot | kPendAmb) and near ties
// of the best hit (slot).  Past kPend a candidate is decided in float32 like
// any other (a search meets that many only on a ray running along a line of
// triangle edges).
constexpr int kPend = 8;
constexpr int kPendAmb = 0x40000000;

// Ray as float pairs in shared memory: rows 0..5 of `hi` and `lo` hold origin
// xyz and direction xyz, `stride` floats apart.
// In FP64 mode `dv` points at the same rows held as float64.  MIXED: `pend`
// is the lane's column of the pending list (entry 0 the count, entries 1..
// kPend the candidates, `stride` ints apart).
struct RaySrc {
  const float *hi, *lo;
  int stride;
  const double *dv;
  int *pend;
  __device__ __forceinline__ void get(double3 &o, double3 &d) const {
    if (dv) {
      o = make_double3(dv[0], dv[stride], dv[2 * stride]);
      d = make_double3(dv[3 * stride], dv[4 * stride], dv[5 * stride]);
      return;
    }
    o = make_double3((double)hi[0] + lo[0], (double)hi[stride] + lo[stride], (double)hi[2 * stride] + lo[2 * stride]);
    d = make_double3((double)hi[3 * stride] + lo[3 * stride], (double)hi[4 * stride] + lo[4 * stride],
                     (double)hi[5 * stride] + lo[5 * stride]);
  }
};

// Record a candidate for float64 after the search; false if the list is full.
__device__ __forceinline__ bool pend_add(const RaySrc &rs, int entry) {
  const int n = rs.pend[0];
  if (n >= kPend) return false;
  rs.pend[(n + 1) * rs.stride] = entry;
  rs.pend[0] = n + 1;
  return true;
}

// Closest accepted hit of the ray in the BVH; ties in distance go to the
// lowest original triangle id.  In the deferring variants `rs` gives the
// float-pair or float64 ray that the float32 ray `r` rounds, read only on the
// rare float64 paths.
// Returns the leaf slot or -1.

// Candidate triangle `slot` against the best hit so far (ties in distance go
// to the lowest original triangle id).  With MIXED/FP64, `rs` gives the
// float-pair or float64 ray that the float32 ray `r` rounds, read only on the
// float64 paths.  Hits beyond `tlim` are ignored.
// An event count of a warp, in shared memory: every lane that passes an
// increment adds one, the lanes that execute it together with one atomic.
struct WarpCount {
  unsigned *p;
  __device__ __forceinline__ void operator++(int) const {
    const unsigned m = __activemask();
    if ((int)(threadIdx.x & 31u) == __ffs(m) - 1) atomicAdd(p, (unsigned)__popc(m));
  }
};

template <int kP, bool kCount>
__device__ __forceinline__ void consider_tri(const DevScene &sc, const Tri *tris, const Ray &r, const RaySrc &rs,
                                             double dns64, Best &best, int slot, const WarpCount &n_tris, float tlim) {
  constexpr bool kDefer = Prec<kP>::defer, kAll64 = Prec<kP>::all64;
  if (kCount) n_tris++;
  const Tri *tp = tris + slot;
  float4 v0 = __ldg(&tp->v0), v1 = __ldg(&tp->v1), v2 = __ldg(&tp->v2);
  float t;
  double t64 = 0.0;
  bool has64 = false;
  bool amb = false;
  if (kAll64) {
    // FP64: every candidate in float64 Moller-Trumbore on the float64 ray
    double3 o, d;
    rs.get(o, d);
    double tt;
    if (!hit_mt64(o, d, v0, v1, v2, tt)) return;
    if (!(tt > (double)r.t_eps && (dns64 == 0.0 || tt * dns64 > (double)r.t_eps))) return;
    t64 = tt;
    has64 = true;
    t = (float)tt;
  } else {
    t = hit_watertight(r, v0, v1, v2, amb);
  }
  if (kAll64) {
  } else {
    // MIXED: an ambiguous candidate is decided in float64 after the search
    if (kDefer && amb && pend_add(rs, slot | kPendAmb)) return;
    if (!(t < kInf && accept_hit(r, t))) return;
  }
  if (t > tlim) return;  // sub-domain: beyond the tile (see k_trace_tiled)
  int id = __float_as_int(v1.w);
  if (kP == kPF32) {
    if (t < best.t || (t == best.t && id < best.id)) { best.t = t; best.slot = slot; best.id = id; }
    return;
  }
  // MIXED and FP64: a clearly nearer or farther float32 distance decides; a
  // near tie is settled in float64, where distances within 1e-9 relative tie
  // and go to the lowest triangle index (MIXED: after the search)
  float win = 1e-5f * fabsf(best.t) + 1e-4f;
  if (best.slot < 0 || t < best.t - win) {
    best.t = t; best.slot = slot; best.id = id; best.t64 = t64; best.has64 = has64;
    return;
  }
  if (t > best.t + win) return;
  if (kDefer) {
    if (!pend_add(rs, slot) && (t < best.t || (t == best.t && id < best.id))) {
      best.t = t; best.slot = slot; best.id = id; best.t64 = 0.0; best.has64 = false;
    }
    return;
  }
  double tol = 1e-9 * (1.0 + fabs(t64));
  if (t64 < best.t64 - tol || (fabs(t64 - best.t64) <= tol && id < best.id)) {
    best.t = (float)t64; best.slot = slot; best.id = id; best.t64 = t64; best.has64 = true;
  }
}

// MIXED, after a search: the candidates it left to float64.  An ambiguous
// triangle is tested with float64 Moller-Trumbore; a near tie compares the
// float64 plane distances of both triangles.  Each is then weighed against
// the best hit as during the search.
__device__ __forceinline__ void settle_pending(const DevScene &sc, const Ray &r, const RaySrc &rs, double dns64,
                                               Best &best, float tlim);
__device__ __noinline__ void settle_pending_call(const DevScene &sc, const Ray &r, const RaySrc &rs, double dns64,
                                                 Best &best, float tlim) {
  settle_pending(sc, r, rs, dns64, best, tlim);
}
// kOutOfLine: the rarely needed float64 code as a call, out of the caller's
// instruction stream (the sub-domain trace, whose service code measured
// faster the smaller it was: 46.1 -> 45.2 ms on the district)
template <bool kOutOfLine = false>
__device__ __forceinline__ void settle_search(const DevScene &sc, const Ray &r, const RaySrc &rs, double dns64,
                                              Best &best, float tlim) {
  if (rs.pend[0] == 0) return;
  if (kOutOfLine) settle_pending_call(sc, r, rs, dns64, best, tlim);
  else settle_pending(sc, r, rs, dns64, best, tlim);
}
__device__ __forceinline__ void settle_pending(const DevScene &sc, const Ray &r, const RaySrc &rs, double dns64,
                                               Best &best, float tlim) {
  const int n = rs.pend[0];
  const Tri *const tris = sc.tris;
  double3 o, d;
  rs.get(o, d);
#pragma unroll 1
  for (int q = 1; q <= n; q++) {
    const int e = rs.pend[q * rs.stride];
    const int slot = e & ~kPendAmb;
    const Tri *tp = tris + slot;
    const float4 v1 = __ldg(&tp->v1);
    double tt;
    if (e & kPendAmb) {
      if (!hit_mt64(o, d, __ldg(&tp->v0), v1, __ldg(&tp->v2), tt)) continue;
      if (!(tt > (double)r.t_eps && (dns64 == 0.0 || tt * dns64 > (double)r.t_eps))) continue;
    } else {
      tt = plane_t64(sc, slot, o, d);
    }
    const float t = (float)tt;
    if (t > tlim) continue;
    const int id = __float_as_int(v1.w);
    const float win = 1e-5f * fabsf(best.t) + 1e-4f;
    if (best.slot < 0 || t < best.t - win) {
      best.t = t; best.slot = slot; best.id = id; best.t64 = tt; best.has64 = true;
      continue;
    }
    if (t > best.t + win) continue;
    if (!best.has64) {
      best.t64 = plane_t64(sc, best.slot, o, d);
      best.has64 = true;
    }
    const double tol = 1e-9 * (1.0 + fabs(tt));
    if (tt < best.t64 - tol || (fabs(tt - best.t64) <= tol && id < best.id)) {
      best.t = t; best.slot = slot; best.id = id; best.t64 = tt; best.has64 = true;
    }
  }
}

// Order two (distance, child) pairs by distance.
__device__ __forceinline__ void sort_pair(float &ka, int &ca, float &kb, int &cb) {
  const bool sw = kb < ka;
  const float k = sw ? kb : ka;
  const int c = sw ? cb : ca;
  kb = sw ? ka : kb;
  cb = sw ? ca : cb;
  ka = k;
  ca = c;
}

// A closest-hit search that can stop after any node and resume later: its
// state is the current node, the stack (an array the caller keeps) and the
// best hit so far.
struct HitSearch {
  int node, sp, visits;
  Best best;
  __device__ __forceinline__ void start(int root) {
    node = root;
    sp = 0;
    visits = 0;
    best.t = kInf;
    best.slot = -1;
    best.id = 0x7fffffff;
    best.t64 = 0.0;
    best.has64 = false;
  }
  // One wide node of the traversal (the boxes of its up to four children in
  // one 128-byte fetch; the nearest child hit next, the others pushed
  // farthest first) and the leaves it exposes.  False once the search is
  // over.
  template <int kP, bool kCount, bool kLeaves>
  __device__ __forceinline__ bool step(const DevScene &sc, const Node4 *nodes, const Tri *tris, int64_t n_tri,
                                       const Ray &r, const RaySrc &rs, double dns64, int *stack, int *err,
                                       const WarpCount &n_nodes, const WarpCount &n_tris, float tlim) {
    if (n_tri == 0 || node == kNoChild) return false;
    // the leaves this step tests: child codes in `lc`, the lanes in `lm`
    int4 lc = make_int4(node, 0, 0, 0);
    unsigned lm = 0;
    bool more = true;
    if (node < 0) {
      // a leaf: the root of a one-leaf hierarchy, or (kLeaves) the rest of a
      // larger leaf put back on the stack (below)
      lm = 1;
      if (kLeaves && sp > 0) node = stack[--sp];
      else more = false;
    } else {
      // a well-formed BVH is visited at most once per node; the bound only
      // guarantees termination should the structure ever be malformed
      if (++visits > (int)n_tri + 64) {
        atomicExch(err, BT_E_TIMEOUT);
        return false;
      }
      const Node4 *nd = nodes + node;
      if (kCount) n_nodes++;
      const float4 lox = __ldg(&nd->lox), hix = __ldg(&nd->hix), loy = __ldg(&nd->loy), hiy = __ldg(&nd->hiy);
      const float4 loz = __ldg(&nd->loz), hiz = __ldg(&nd->hiz);
      const int4 ch = __ldg(&nd->child);
      // in MIXED and FP64 mode near ties must still be visited
      const float tmax = fminf(kP != kPF32 ? best.t + (1e-5f * fabsf(best.t) + 1e-4f) : best.t, tlim);
      const float3 oi = origin_scaled(r);
      float k0, k1, k2, k3;
      const bool h0 = slab(r, oi, lox.x, hix.x, loy.x, hiy.x, loz.x, hiz.x, tmax, k0) && ch.x != kNoChild;
      const bool h1 = slab(r, oi, lox.y, hix.y, loy.y, hiy.y, loz.y, hiz.y, tmax, k1) && ch.y != kNoChild;
      const bool h2 = slab(r, oi, lox.z, hix.z, loy.z, hiy.z, loz.z, hiz.z, tmax, k2) && ch.z != kNoChild;
      const bool h3 = slab(r, oi, lox.w, hix.w, loy.w, hiy.w, loz.w, hiz.w, tmax, k3) && ch.w != kNoChild;
      lc = ch;
      lm = (unsigned)(h0 && ch.x < 0) | (unsigned)(h1 && ch.y < 0) << 1 | (unsigned)(h2 && ch.z < 0) << 2 |
           (unsigned)(h3 && ch.w < 0) << 3;
      // inner children hit, nearest first (a sorting network on the entry
      // distances; misses sort last)
      int c0 = ch.x, c1 = ch.y, c2 = ch.z, c3 = ch.w;
      k0 = h0 && c0 >= 0 ? k0 : kInf;
      k1 = h1 && c1 >= 0 ? k1 : kInf;
      k2 = h2 && c2 >= 0 ? k2 : kInf;
      k3 = h3 && c3 >= 0 ? k3 : kInf;
      const int ni = (k0 < kInf) + (k1 < kInf) + (k2 < kInf) + (k3 < kInf);
      sort_pair(k0, c0, k1, c1);
      sort_pair(k2, c2, k3, c3);
      sort_pair(k0, c0, k2, c2);
      sort_pair(k1, c1, k3, c3);
      sort_pair(k1, c1, k2, c2);
      if (ni > 0) {
        if (sp + ni - 1 <= kStackDepth) {
          if (ni > 3) stack[sp++] = c3;
          if (ni > 2) stack[sp++] = c2;
          if (ni > 1) stack[sp++] = c1;
        } else {
          atomicExch(err, BT_E_QUEUE_FULL);
        }
        node = c0;
      } else if (sp > 0) {
        node = stack[--sp];
      } else {
        more = false;
      }
    }
#pragma unroll 1
    while (lm) {
      const int c = __ffs(lm) - 1;
      lm &= lm - 1;
      const int v = ~(c == 0 ? lc.x : c == 1 ? lc.y : c == 2 ? lc.z : lc.w);
      if (kLeaves && (v >> kLeafShift)) {
        // a leaf of several triangles: its first now, the rest as a leaf of
        // one triangle fewer at a later step, so that a step still tests at
        // most one triangle per leaf
        const int rest = ~((leaf_slot(v) + 1) | (((v >> kLeafShift) - 1) << kLeafShift));
        if (!more) {
          node = rest;
          more = true;
        } else if (sp < kStackDepth) {
          stack[sp++] = rest;
        } else {
          atomicExch(err, BT_E_QUEUE_FULL);
        }
      }
      consider_tri<kP, kCount>(sc, tris, r, rs, dns64, best, kLeaves ? leaf_slot(v) : v, n_tris, tlim);
    }
    return more;
  }
};

// Closest accepted hit of the ray in the BVH under `root`; the leaf slot or -1.
template <int kP, bool kCount>
__device__ __forceinline__ int closest_hit(const DevScene &sc, const Ray &r, RaySrc rs, double dns64, Best &best,
                                           int *err, const WarpCount &n_nodes, const WarpCount &n_tris,
                                           int root, float tlim = kInf) {
  // the hot fields in registers: in a batch `sc` lives in device memory and
  // would otherwise be re-read on every node
  const int64_t n_tri = sc.n_tris;
  const Node4 *const nodes = sc.nodes;
  const Tri *const tris = sc.tris;
  int stack[kStackDepth];
  HitSearch hs;
  hs.start(root);
  if constexpr (Prec<kP>::defer) rs.pend[0] = 0;
  while (hs.step<kP, kCount, true>(sc, nodes, tris, n_tri, r, rs, dns64, stack, err, n_nodes, n_tris, tlim)) {
  }
  best = hs.best;
  if constexpr (Prec<kP>::defer) settle_search(sc, r, rs, dns64, best, tlim);
  return best.slot;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Cheap rejection of a segment that cannot reach the microphones' height
// slab: the cone lies on one side of its apex height when all three edge
// directions point the same way in z.  Edge j is along n_{j-1} x n_j times
// the sign of det(n0, n1, n2), which a mirror image flips.  Everything else
// goes to the scatter, which clips the footprint exactly.
__device__ __forceinline__ bool may_reach_slab(float3 n0, float3 n1, float3 n2, float az, const MicGrid &g) {
  float det = n0.x * (n1.y * n2.z - n1.z * n2.y) + n0.y * (n1.z * n2.x - n1.x * n2.z) +
              n0.z * (n1.x * n2.y - n1.y * n2.x);
  float sg = det >= 0.0f ? 1.0f : -1.0f;
  float dz0 = sg * (n2.x * n0.y - n2.y * n0.x);
  float dz1 = sg * (n0.x * n1.y - n0.y * n1.x);
  float dz2 = sg * (n1.x * n2.y - n1.y * n2.x);
  float m = 1e-3f;
  if (dz0 < 0.0f && dz1 < 0.0f && dz2 < 0.0f && az < g.zlo - m) return false;
  if (dz0 > 0.0f && dz1 > 0.0f && dz2 > 0.0f && az > g.zhi + m) return false;
  return true;
}

// The microphone-grid cell under the middle of a segment (of its first 200 m
// when it is longer or escapes), x | y << 16: the place the scatter orders
// segments by, so that segments processed together reach the same
// microphones and accumulators.
__device__ __forceinline__ int seg_cell_key(const MicGrid &g, const Ray &r, float t) {
  const float h = 0.5f * fminf(t, 200.0f);
  const int cx = clampi((int)((r.o.x + r.d.x * h - g.x0) * g.inv_cw), 0, g.nx - 1);
  const int cy = clampi((int)((r.o.y + r.d.y * h - g.y0) * g.inv_ch), 0, g.ny - 1);
  return (cx & 0xffff) | cy << 16;
}

// Warp-aggregated append of a segment record.
__device__ __forceinline__ void emit_segment(const TraceArgs &a, const Seg &s, bool emit,
                                             const WarpCount &n_emit) {
  unsigned mask = __activemask();
  unsigned bal = __ballot_sync(mask, emit);
  if (!bal) return;
  int leader = __ffs(bal) - 1;
  unsigned long long base = 0;
  if ((int)lane_id() == leader) {
    base = atomicAdd(a.seg_count, (unsigned long long)__popc(bal));
    atomicAdd(n_emit.p, (unsigned)__popc(bal));
  }
  base = __shfl_sync(mask, base, leader);
  if (emit) {
    unsigned long long idx = base + __popc(bal & ((1u << lane_id()) - 1u));
    if (idx < a.seg_capacity) a.segs[idx] = s;
    else atomicExch(&a.ctr->error, BT_E_QUEUE_FULL);
  }
}

// Lineage state of one thread, in shared memory (one column per thread) so
// that it holds no registers across the traversal.  Rows: apex 0..2, cone
// normals 3..11, ray origin 12..14, ray direction 15..17; `lo` holds the low
// parts of the float pairs (MIXED only).
constexpr int kTraceThreads = 128;

constexpr int kRowA = 0, kRowN = 3, kRowO = 12, kRowD = 15, kRows = 18;
// a sub-domain accepts hits up to this far (m along the ray) past its exit
constexpr float kTileEps = 1e-2f;
// per-lane event counters (rows of LineageSmem::cnt)
enum { kCSeg, kCHit, kCEsc, kCEmit, kCHand, kCSteal, kCNodes, kCTris, kNumCounts };
template <int kP>
struct LineageSmem {
  double dv[Prec<kP>::chain64 ? kRows : 1][kTraceThreads];  // float64 chain; `hi` holds its float32 rounding
  float hi[kRows][kTraceThreads];
  float lo[Prec<kP>::pairs ? kRows : 1][kTraceThreads];
  float p[kMaxBands][kTraceThreads];  // band power W_b prod(r_b)
  float st[4][kTraceThreads];         // start plane (relative to the apex)
  int pend[Prec<kP>::defer ? kPend + 1 : 1][kTraceThreads];  // candidates left to float64
};

template <int kP>
__device__ __forceinline__ df3 ld_df3(const LineageSmem<kP> &sm, int row, int t) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  df3 v;
  v.x = df{sm.hi[row][t], kPairs ? sm.lo[row][t] : 0.0f};
  v.y = df{sm.hi[row + 1][t], kPairs ? sm.lo[row + 1][t] : 0.0f};
  v.z = df{sm.hi[row + 2][t], kPairs ? sm.lo[row + 2][t] : 0.0f};
  return v;
}
template <int kP>
__device__ __forceinline__ void st_df3(LineageSmem<kP> &sm, int row, int t, df3 v) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  sm.hi[row][t] = v.x.hi;
  sm.hi[row + 1][t] = v.y.hi;
  sm.hi[row + 2][t] = v.z.hi;
  if (kPairs) {
    sm.lo[row][t] = v.x.lo;
    sm.lo[row + 1][t] = v.y.lo;
    sm.lo[row + 2][t] = v.z.lo;
  }
}
template <int kP>
__device__ __forceinline__ float3 ld_hi3(const LineageSmem<kP> &sm, int row, int t) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  return make_float3(sm.hi[row][t], sm.hi[row + 1][t], sm.hi[row + 2][t]);
}
template <int kP>
__device__ __forceinline__ void st_f3(LineageSmem<kP> &sm, int row, int t, float3 v) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  sm.hi[row][t] = v.x;
  sm.hi[row + 1][t] = v.y;
  sm.hi[row + 2][t] = v.z;
}

// FP64 rows: the float64 value and its float32 rounding in `hi` (read by the
// float32 traversal and the segment records).
template <int kP>
__device__ __forceinline__ double3 ld_d3(const LineageSmem<kP> &sm, int row, int t) {
  return make_double3(sm.dv[row][t], sm.dv[row + 1][t], sm.dv[row + 2][t]);
}
template <int kP>
__device__ __forceinline__ void st_d3(LineageSmem<kP> &sm, int row, int t, double3 v) {
  sm.dv[row][t] = v.x;
  sm.dv[row + 1][t] = v.y;
  sm.dv[row + 2][t] = v.z;
  sm.hi[row][t] = (float)v.x;
  sm.hi[row + 1][t] = (float)v.y;
  sm.hi[row + 2][t] = (float)v.z;
}

// Start lineage `lin` (source si, beam bi) in this thread's column.
template <int kP>
__device__ __forceinline__ void init_lineage(const SceneView &a, LineageSmem<kP> &sm, int t, int64_t lin) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  const int nb = a.sc.n_bands;
  int64_t si = lin / a.n_beams, bi = lin - si * a.n_beams;
  float4 s4 = __ldg(&a.src[si]);
  float3 A = make_float3(s4.x, s4.y, s4.z);
  if (kChain64) {
    double3 d0, d1, d2;
    beam_dirs<double>(a.level, bi, d0, d1, d2);
    st_d3(sm, kRowN, t, cross_exact(d0, d1));
    st_d3(sm, kRowN + 3, t, cross_exact(d1, d2));
    st_d3(sm, kRowN + 6, t, cross_exact(d2, d0));
    st_d3(sm, kRowD, t, normalize3((d0 + d1) + d2));
    const double3 A64 = make_double3(s4.x, s4.y, s4.z);
    st_d3(sm, kRowA, t, A64);
    st_d3(sm, kRowO, t, A64);
  } else if (kPairs) {
    // table: 9 normal components then the 3 axis components, hi parts
    // first, lo parts 12 floats later
    const float *bt = a.beam_table + 24 * bi;
    for (int q = 0; q < 9; q++) {
      sm.hi[kRowN + q][t] = __ldg(bt + q);
      sm.lo[kRowN + q][t] = __ldg(bt + 12 + q);
    }
    for (int q = 0; q < 3; q++) {
      sm.hi[kRowD + q][t] = __ldg(bt + 9 + q);
      sm.lo[kRowD + q][t] = __ldg(bt + 21 + q);
      sm.lo[kRowA + q][t] = 0.0f;
      sm.lo[kRowO + q][t] = 0.0f;
    }
  } else {
    float3 d0, d1, d2;
    beam_dirs<float>(a.level, bi, d0, d1, d2);
    st_f3(sm, kRowN, t, cross_exact(d0, d1));
    st_f3(sm, kRowN + 3, t, cross_exact(d1, d2));
    st_f3(sm, kRowN + 6, t, cross_exact(d2, d0));
    st_f3(sm, kRowD, t, normalize3((d0 + d1) + d2));
  }
  st_f3(sm, kRowA, t, A);
  st_f3(sm, kRowO, t, A);
  // a directional source: its power in this beam's direction (Section 2),
  // the pattern's gain times the omnidirectional power
  float gain = 1.0f;
  if (a.dir_of) {
    const int pat = __ldg(&a.dir_of[si]);
    if (pat >= 0) gain = __ldg(&a.dir_gain[pat * a.n_beams + bi]);
  }
#pragma unroll
  for (int b = 0; b < kMaxBands; b++) sm.p[b][t] = b < nb ? gain * __ldg(&a.power[si * nb + b]) : 0.0f;
  sm.st[0][t] = 0.0f;
  sm.st[1][t] = 0.0f;
  sm.st[2][t] = 0.0f;
  sm.st[3][t] = -kInf;
}

// Per-lane scalars of a lineage besides its shared-memory column.
struct LaneState {
  int64_t lin;
  int k, start_slot;
  float dns;
  double dns64;
};

// Event counts of one launch per warp, in shared memory rather than in
// registers or per lane (4 KB less shared memory a block).  A warp handles at
// most some ten thousand segments per launch, so even its node count stays
// far below 2^32; the launch totals are formed in 64-bit.
struct TraceCounts {
  unsigned *p;  // the warp's counts
  __device__ WarpCount operator[](int i) const { return WarpCount{p + i}; }
};
__device__ __forceinline__ TraceCounts init_counts(unsigned (*wc)[kNumCounts], int t) {
  if ((t & 31) < kNumCounts) wc[t >> 5][t & 31] = 0u;
  __syncwarp();
  return TraceCounts{wc[t >> 5]};
}

// A segment is resolved: its axis ray hit triangle `slot` (or escaped, slot
// < 0).  Write the segment record and, if the beam goes on, reflect it: the
// image source (Section 2), mirrored cone and axis, energy lost at the
// reflection.  Returns true if the lineage continues.
template <int kP>
__device__ __forceinline__ bool finish_segment(const TraceArgs &a, const SceneView &v, int vi, LineageSmem<kP> &sm,
                                               int t, const Ray &r, const Best &best, int slot, LaneState &ls,
                                               const TraceCounts &cn) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  const int nb = v.sc.n_bands;
  cn[kCSeg]++;
  float4 end = make_float4(0.0f, 0.0f, 0.0f, -kInf);
  float4 v0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float4 plf = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (a.hit_log) {
    // (measurement aid: which triangle each segment's axis ray hit)
    a.hit_log[ls.lin * a.hit_log_stride + ls.k] = slot >= 0 ? __float_as_int(__ldg(&v.sc.tris[slot].v1.w)) : -1;
  }
  if (slot >= 0) {
    cn[kCHit]++;
    v0 = __ldg(&v.sc.tris[slot].v0);
    plf = __ldg(&v.sc.planes[slot]);
    // end plane on the incident side, offset relative to the apex
    float3 pn = f3(plf);
    float3 en = dot3(pn, r.d) < 0.0f ? pn : pn * -1.0f;
    float ew;
    if (kChain64) {
      double3 end = make_double3(en.x, en.y, en.z);
      ew = (float)dot3(end, make_double3(v0.x, v0.y, v0.z) - ld_d3(sm, kRowA, t));
    } else if (kPairs) {
      ew = df3_dot2(mkdf3(en), df3_sub(mkdf3(f3(v0)), ld_df3(sm, kRowA, t))).hi;
    } else {
      ew = dot3(en, f3(v0) - ld_hi3(sm, kRowA, t));
    }
    end = make_float4(en.x, en.y, en.z, ew);
  } else {
    cn[kCEsc]++;
  }
  {
    Seg s;
    for (int q = 0; q < 3; q++) {
      s.ahi[q] = sm.hi[kRowA + q][t];
      s.alo[q] = kPairs ? sm.lo[kRowA + q][t] : 0.0f;
    }
    float3 n0 = ld_hi3(sm, kRowN, t), n1 = ld_hi3(sm, kRowN + 3, t), n2 = ld_hi3(sm, kRowN + 6, t);
    s.n0 = make_float4(n0.x, n0.y, n0.z, __int_as_float(ls.start_slot));
    s.n1 = make_float4(n1.x, n1.y, n1.z, __int_as_float(slot));
    s.n2 = make_float4(n2.x, n2.y, n2.z, __int_as_float(ls.k));
    for (int q = 0; q < 9; q++) s.nlo[q] = kPairs ? sm.lo[kRowN + q][t] : 0.0f;
    s.pad[0] = s.pad[1] = s.pad[2] = 0.0f;
    if (kChain64) {
      // float64 values as float pairs, the apex with a third word so that
      // hi + lo + pad gives it back exactly
      for (int q = 0; q < 3; q++) {
        double x = sm.dv[kRowA + q][t];
        s.alo[q] = (float)(x - (double)s.ahi[q]);
        s.pad[q] = (float)((x - (double)s.ahi[q]) - (double)s.alo[q]);
      }
      for (int q = 0; q < 9; q++) s.nlo[q] = (float)(sm.dv[kRowN + q][t] - (double)sm.hi[kRowN + q][t]);
    }
    s.start = make_float4(sm.st[0][t], sm.st[1][t], sm.st[2][t], sm.st[3][t]);
    s.end = end;
    s.p03 = make_float4(sm.p[0][t], sm.p[1][t], sm.p[2][t], sm.p[3][t]);
    s.p47 = make_float4(sm.p[4][t], sm.p[5][t], sm.p[6][t], sm.p[7][t]);
    s.view = vi;
    const MicGrid &g = *v.grid;
    s.key = v.seg_key ? seg_cell_key(g, r, best.t) : 0;
    emit_segment(a, s, g.n_mics > 0 && may_reach_slab(n0, n1, n2, s.ahi[2], g), cn[kCEmit]);
  }
  if (slot < 0 || ls.k == v.max_order) return false;
  // energy lost at the reflection
  int mat = __float_as_int(v0.w);
  float wmax = 0.0f;
#pragma unroll
  for (int b = 0; b < kMaxBands; b++) {
    float p = sm.p[b][t];
    if (b < nb) p *= __ldg(&v.sc.refl[mat * nb + b]);
    sm.p[b][t] = p;
    wmax = fmaxf(wmax, p);
  }
  if (v.energy_threshold > 0.0f && wmax < v.energy_threshold) return false;
  // Image source: mirror the apex, the cone and the axis in the hit plane;
  // the reflected beam starts at the hit point on that plane.
  float3 pn = f3(plf), pv0 = f3(v0);
  float3 Dn;
  if (kChain64) {
    Plane64 pl = ldg_d4(&v.sc.planes64[slot]);
    const double3 n = make_double3(pl.x, pl.y, pl.z), v0d = make_double3(v0.x, v0.y, v0.z);
    double3 A = ld_d3(sm, kRowA, t), O = ld_d3(sm, kRowO, t), D = ld_d3(sm, kRowD, t);
    const double th = best.has64 ? best.t64 : (pl.w - dot3(n, O)) / dot3(n, D);
    const double3 H = O + D * th;
    A = A - n * (2.0 * dot3(A - v0d, n));
    st_d3(sm, kRowA, t, A);
#pragma unroll
    for (int j = 0; j < 3; j++) {
      double3 nj = ld_d3(sm, kRowN + 3 * j, t);
      st_d3(sm, kRowN + 3 * j, t, nj - n * (2.0 * dot3(nj, n)));
    }
    D = D - n * (2.0 * dot3(D, n));
    st_d3(sm, kRowO, t, H);
    st_d3(sm, kRowD, t, D);
    const double dn = dot3(n, D);
    ls.dns64 = fabs(dn);
    ls.dns = (float)ls.dns64;
    Dn = make_float3((float)D.x, (float)D.y, (float)D.z);
    const double3 sn = dn > 0.0 ? n : n * -1.0;
    const double sw = dot3(sn, v0d - A);
    sm.st[0][t] = (float)sn.x; sm.st[1][t] = (float)sn.y; sm.st[2][t] = (float)sn.z; sm.st[3][t] = (float)sw;
  } else if (kPairs) {
    // in stages, each reading its rows from shared memory and writing them
    // back before the next starts, so that few float pairs are live at once
    // (the compiler fences keep the stages apart)
    PlaneDF pd = v.sc.planes_df[slot];
    const df3 n = df3{df{pd.hi.x, pd.lo.x}, df{pd.hi.y, pd.lo.y}, df{pd.hi.z, pd.lo.z}};
    df kd = df{0.0f, 0.0f}, ka = df{0.0f, 0.0f};
    {
      // the hit point on the plane (the reflected beam's origin); n . D is
      // also the axis' own coefficient in the mirror loop below
      const df3 O = ld_df3(sm, kRowO, t), D = ld_df3(sm, kRowD, t);
      kd = df3_dot2(D, n);
      const df th = best.has64 ? d_to_df(best.t64) : df_div2(df_sub(df{pd.hi.w, pd.lo.w}, df3_dot2(n, O)), kd);
      st_df3(sm, kRowO, t, df3{df_axpy(O.x, th, D.x), df_axpy(O.y, th, D.y), df_axpy(O.z, th, D.z)});
    }
    // the cone normals, the axis and the apex (the image source) mirrored
    // by one copy of the code: v - 2 ((v - p) . n) n with p = 0 for the
    // directions and p = v0, a point of the plane, for the apex
    const df3 p0 = mkdf3(pv0);
#pragma unroll 1
    for (int j = 0; j < 5; j++) {
      asm volatile("" ::: "memory");
      const int row = j < 3 ? kRowN + 3 * j : (j == 3 ? kRowD : kRowA);
      const df3 v = ld_df3(sm, row, t);
      df k = kd;
      if (j != 3) k = df3_dot2(j == 4 ? df3_sub(v, p0) : v, n);
      if (j == 4) ka = k;
      st_df3(sm, row, t, df3_sub2kn(v, k, n));
    }
    asm volatile("" ::: "memory");
    // |n . D| is the same for the axis and its mirror image, and the image
    // source lies as far behind the plane as the apex in front of it
    ls.dns64 = fabs((double)kd.hi + (double)kd.lo);
    ls.dns = (float)ls.dns64;
    Dn = ld_hi3(sm, kRowD, t);
    const bool fwd = dot3(pn, Dn) > 0.0f;
    float3 sn = fwd ? pn : pn * -1.0f;
    float sw = fwd ? ka.hi : -ka.hi;
    sm.st[0][t] = sn.x; sm.st[1][t] = sn.y; sm.st[2][t] = sn.z; sm.st[3][t] = sw;
  } else {
    float3 A = ld_hi3(sm, kRowA, t), O = ld_hi3(sm, kRowO, t), D = ld_hi3(sm, kRowD, t);
    A = A - pn * (2.0f * dot3(A - pv0, pn));
    st_f3(sm, kRowA, t, A);
#pragma unroll
    for (int j = 0; j < 3; j++) {
      float3 nj = ld_hi3(sm, kRowN + 3 * j, t);
      st_f3(sm, kRowN + 3 * j, t, nj - pn * (2.0f * dot3(nj, pn)));
    }
    float3 H = O + D * best.t;
    Dn = D - pn * (2.0f * dot3(D, pn));
    st_f3(sm, kRowO, t, H);
    st_f3(sm, kRowD, t, Dn);
    ls.dns = fabsf(dot3(pn, Dn));
    ls.dns64 = 0.0;
    float3 sn = dot3(pn, Dn) > 0.0f ? pn : pn * -1.0f;
    float sw = dot3(sn, pv0 - A);
    sm.st[0][t] = sn.x; sm.st[1][t] = sn.y; sm.st[2][t] = sn.z; sm.st[3][t] = sw;
  }
  ls.start_slot = slot;
  ls.k++;
  return true;
}

__device__ __forceinline__ void flush_counts(const TraceArgs &a, const TraceCounts &cn, bool count_work) {
  // warp sums in 64-bit
  __syncwarp();
  unsigned long long v[kNumCounts];
  for (int q = 0; q < kNumCounts; q++) v[q] = cn.p[q];
  if (lane_id() == 0) {
    if (count_work) {
      atomicAdd(&a.ctr->nodes_visited, v[kCNodes]);
      atomicAdd(&a.ctr->tris_tested, v[kCTris]);
    }
    atomicAdd(&a.ctr->segments, v[kCSeg]);
    atomicAdd(&a.ctr->hits, v[kCHit]);
    atomicAdd(&a.ctr->escapes, v[kCEsc]);
    atomicAdd(&a.ctr->emitted, v[kCEmit]);
    if (v[kCHand]) atomicAdd(&a.ctr->handoffs, v[kCHand]);
    if (v[kCSteal]) atomicAdd(&a.ctr->steals, v[kCSteal]);
  }
}

// A warp's reservation of lineages, [next, end) relative to the launch's
// first lineage, in shared memory; `last` once the launch's counter has run
// past the end (nothing more to reserve).
struct WarpLineages {
  unsigned long long next, end;
  int last;
};

// Lineages a warp reserves at a time: what its lanes need now, or at least
// beams_per_warp, so that it draws from the launch's counter less often (at
// the price of a coarser end of the launch).
__device__ __forceinline__ unsigned long long reserve_size(const TraceArgs &a, unsigned long long need) {
  const unsigned long long b = (unsigned long long)a.beams_per_warp;
  return need > b ? need : b;
}

// Take the next lineage of the batch for every lane in `need` (warp-vote
// refill): first from the warp's reservation, then from a new one.  Returns
// the lineage index or -1 when the batch is used up.
__device__ __forceinline__ int64_t take_lineage(const TraceArgs &a, bool need, WarpLineages &wl) {
  unsigned nm = __ballot_sync(0xffffffffu, need);
  if (!nm) return -1;
  const unsigned lane = lane_id();
  if (a.beams_per_warp == 0) {
    // as many as the lanes need, straight from the launch's counter
    const int leader = __ffs(nm) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(a.lineage_next, (unsigned long long)__popc(nm));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!need) return -1;
    const int64_t mine = a.lineage_begin + (int64_t)(base + __popc(nm & ((1u << lane) - 1u)));
    return mine < a.lineage_end ? mine : -1;
  }
  const unsigned long long total = (unsigned long long)(a.lineage_end - a.lineage_begin);
  const unsigned long long n = (unsigned long long)__popc(nm);
  const unsigned long long next = wl.next, end = wl.end, have = end - next;
  const int last = wl.last;
  unsigned long long b = total, got = 0;
  if (have < n && !last && (int)lane == __ffs(nm) - 1) {
    const unsigned long long R = reserve_size(a, n - have);
    b = atomicAdd(a.lineage_next, R);
    got = b < total ? (b + R < total ? R : total - b) : 0;
    if (b + R >= total) wl.last = 1;
  }
  b = __shfl_sync(0xffffffffu, b, __ffs(nm) - 1);
  got = __shfl_sync(0xffffffffu, got, __ffs(nm) - 1);
  __syncwarp();
  if (lane == 0) {
    if (have < n && !last) {
      const unsigned long long used = n - have < got ? n - have : got;
      wl.next = b + used;
      wl.end = b + got;
    } else {
      wl.next = next + (n < have ? n : have);
    }
  }
  __syncwarp();
  if (!need) return -1;
  const unsigned long long r = (unsigned long long)__popc(nm & ((1u << lane) - 1u));
  if (r < have) return a.lineage_begin + (int64_t)(next + r);
  return r - have < got ? a.lineage_begin + (int64_t)(b + (r - have)) : -1;
}

// Persistent warps: every lane works on one lineage at a time and takes the
// next one from a global counter as soon as its lineage ends, so a warp stays
// full until the batch runs out (warp-vote refill of finished lanes).
// Index of the view whose lineage range holds global lineage `g`; `base`
// holds the views' first lineages in order (a shared-memory copy).
__device__ __forceinline__ int find_view(const int64_t *base, int n_views, int64_t g) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Lanes whose search ended (or whose lineage needs replacing) before a warp
// leaves its search phase to serve them; lanes still searching keep their
// search state and resume afterwards.  Measured on the district: 28 beat 32
// (wait for every lane) by 2.5 %; 24 and below lost, the service phase then
// running too often for too few lanes.
constexpr int kRefillLanes = 28;

// Resident blocks per SM: the traversal is latency-bound, so more warps
// help as long as the spills they force stay light.  Seven (at most 72
// registers a thread) for the single-scene MIXED kernel, whose reflection
// code is small enough (district unsplit 34.2 -> 32.8 ms against six);
// six (80 registers) for the other variants and for batches, whose lanes
// hold their scene's arrays in registers.  kBatch: the lineages of many
// scenes (views) in one launch, each lane on its own lineage's scene.
//
// Each warp alternates two phases.  In the search phase every lane with a ray
// steps through the BVH one node at a time; the phase ends once kRefillLanes
// lanes have nothing to search (their search finished, or they need a new
// lineage) or no lane is searching.  In the service phase, reconverged, the
// lanes whose search finished write their segment and reflect (or end their
// lineage), lanes without a lineage take new ones, and new searches start --
// while the lanes still searching keep their state, so a long search no longer
// holds the whole warp (dynamic ray fetch, after Aila & Laine 2009).
template <int kP, bool kCount, bool kBatch, bool kLeaves>
__global__ void __launch_bounds__(kTraceThreads, kP == kPMixed && !kBatch ? 7 : 6) k_trace(TraceArgs a) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  __shared__ LineageSmem<kP> sm;
  __shared__ int64_t view_base[kBatch ? BT_MAX_SCENES : 1];
  __shared__ WarpLineages wlin[kTraceThreads / 32];
  const int t = threadIdx.x;
  if ((t & 31) == 0) wlin[t >> 5] = WarpLineages{0ull, 0ull, 0};
  __syncwarp();
  if (kBatch) {
    for (int i = t; i < a.n_views; i += kTraceThreads) view_base[i] = a.views[i].lineage_base;
    __syncthreads();
  }
  __shared__ unsigned wcount[kTraceThreads / 32][kNumCounts];
  const TraceCounts cn = init_counts(wcount, t);
  LaneState ls = {-1, 0, -1, 0.0f, 0.0};
  int vi = 0;  // this lane's scene view
  bool done = false, searching = false, pending = false;
  HitSearch hs;
  hs.start(-1);
  int stack[kStackDepth];
  const RaySrc rs{&sm.hi[kRowO][t], kPairs ? &sm.lo[kRowO][t] : &sm.hi[kRowO][t], kTraceThreads,
                  kChain64 ? &sm.dv[kRowO][t] : nullptr, &sm.pend[0][t]};
  while (true) {
    // ---- service: finished searches write their segment and reflect
    bool fresh = false;
    if (__ballot_sync(0xffffffffu, pending) && pending) {
      const SceneView &v = kBatch ? a.views[vi] : a.v;
      const Ray r = make_ray(ld_hi3(sm, kRowO, t), ld_hi3(sm, kRowD, t), v.t_eps, ls.dns);
      if constexpr (kDefer) settle_search(v.sc, r, rs, ls.dns64, hs.best, kInf);
      if (finish_segment(a, v, vi, sm, t, r, hs.best, hs.best.slot, ls, cn)) fresh = true;
      else ls.lin = -1;
      pending = false;
    }
    // ---- service: lanes without a lineage take the next ones
    bool need = !done && ls.lin < 0;
    int64_t mine = take_lineage(a, need, wlin[t >> 5]);
    if (need) {
      if (mine >= 0) {
        if (kBatch) {
          vi = find_view(view_base, a.n_views, mine);
          mine += a.views[vi].lineage_first - view_base[vi];
        }
        ls = LaneState{mine, 0, -1, 0.0f, 0.0};
        init_lineage(kBatch ? a.views[vi] : a.v, sm, t, mine);
        fresh = true;
      } else {
        done = true;
      }
    }
    if (fresh) {
      hs.start((kBatch ? a.views[vi] : a.v).sc.root);
      if constexpr (kDefer) rs.pend[0] = 0;
      searching = true;
    }
    if (__all_sync(0xffffffffu, done)) break;
    // ---- search
    {
      const SceneView &v = kBatch ? a.views[vi] : a.v;
      const Ray r = make_ray(ld_hi3(sm, kRowO, t), ld_hi3(sm, kRowD, t), v.t_eps, ls.dns);
      const int64_t n_tri = v.sc.n_tris;
      const Node4 *const nodes = v.sc.nodes;
      const Tri *const tris = v.sc.tris;
      while (true) {
        if (searching &&
            !hs.step<kP, kCount, kLeaves>(v.sc, nodes, tris, n_tri, r, rs, ls.dns64, stack, &a.ctr->error,
                                          cn[kCNodes], cn[kCTris], kInf)) {
          searching = false;
          pending = true;
        }
        const unsigned srch = __ballot_sync(0xffffffffu, searching);
        const unsigned idle = __ballot_sync(0xffffffffu, !searching && !done);
        if (!srch || __popc(idle) >= kRefillLanes) break;
      }
    }
  }
  flush_counts(a, cn, kCount);
}

// --------------------------------------------------------------- sub-domains
// Device-scope ordered accesses for the hand-off queues.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

// Record a watchdog expiry unless an error is already recorded.
__device__ __forceinline__ void watchdog_fired(const TraceArgs &a) { atomicCAS(&a.ctr->error, 0, BT_E_TIMEOUT); }

// Bounded wait until a queue slot's sequence word reaches `want`.  False if
// the watchdog ran out first (an error is then recorded).
__device__ __forceinline__ bool wait_slot(const TraceArgs &a, const TiledArgs &ta, const unsigned *seq, unsigned want) {
  if (ld_acquire_u32(seq) == want) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    __nanosleep(32);
    if (ld_acquire_u32(seq) == want) return true;
    if (global_ns() - t0 > ta.watchdog_ns) {
      watchdog_fired(a);
      return false;
    }
  }
}

// A lineage's state in a queue slot: S points at row 0, rows c words apart.
// Queue slots are written once and read once by another SM, so both sides
// go through L2 only.
template <int kP>
__device__ __forceinline__ void save_state(uint32_t *S, size_t c, const LineageSmem<kP> &sm, int t,
                                           const LaneState &ls) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  if (kChain64) {
    // rows 0..35: the float64 chain, low word then high word
    for (int q = 0; q < kRows; q++) {
      unsigned long long b = __double_as_longlong(sm.dv[q][t]);
      __stcg(S + (2 * q) * c, (uint32_t)(b & 0xffffffffu));
      __stcg(S + (2 * q + 1) * c, (uint32_t)(b >> 32));
    }
  } else {
    for (int q = 0; q < kRows; q++) __stcg(S + q * c, __float_as_uint(sm.hi[q][t]));
    if (kPairs)
      for (int q = 0; q < kRows; q++) __stcg(S + (kRows + q) * c, __float_as_uint(sm.lo[q][t]));
  }
  for (int b = 0; b < kMaxBands; b++) __stcg(S + (36 + b) * c, __float_as_uint(sm.p[b][t]));
  for (int q = 0; q < 4; q++) __stcg(S + (44 + q) * c, __float_as_uint(sm.st[q][t]));
  __stcg(S + 48 * c, (uint32_t)(ls.lin & 0xffffffffu));
  __stcg(S + 49 * c, (uint32_t)(ls.lin >> 32));
  __stcg(S + 50 * c, (uint32_t)ls.k);
  __stcg(S + 51 * c, (uint32_t)ls.start_slot);
  __stcg(S + 52 * c, __float_as_uint(ls.dns));
  unsigned long long d = __double_as_longlong(ls.dns64);
  __stcg(S + 53 * c, (uint32_t)(d & 0xffffffffu));
  __stcg(S + 54 * c, (uint32_t)(d >> 32));
}

template <int kP>
__device__ __forceinline__ void load_state(const uint32_t *S, size_t c, LineageSmem<kP> &sm, int t,
                                           LaneState &ls) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  if (kChain64) {
    for (int q = 0; q < kRows; q++) {
      unsigned long long b = (unsigned long long)__ldcg(S + (2 * q) * c) |
                             ((unsigned long long)__ldcg(S + (2 * q + 1) * c) << 32);
      double x = __longlong_as_double((long long)b);
      sm.dv[q][t] = x;
      sm.hi[q][t] = (float)x;
    }
  } else {
    for (int q = 0; q < kRows; q++) sm.hi[q][t] = __uint_as_float(__ldcg(S + q * c));
    if (kPairs)
      for (int q = 0; q < kRows; q++) sm.lo[q][t] = __uint_as_float(__ldcg(S + (kRows + q) * c));
  }
  for (int b = 0; b < kMaxBands; b++) sm.p[b][t] = __uint_as_float(__ldcg(S + (36 + b) * c));
  for (int q = 0; q < 4; q++) sm.st[q][t] = __uint_as_float(__ldcg(S + (44 + q) * c));
  ls.lin = (int64_t)__ldcg(S + 48 * c) | ((int64_t)__ldcg(S + 49 * c) << 32);
  ls.k = (int)__ldcg(S + 50 * c);
  ls.start_slot = (int)__ldcg(S + 51 * c);
  ls.dns = __uint_as_float(__ldcg(S + 52 * c));
  ls.dns64 = __longlong_as_double(
      (long long)((unsigned long long)__ldcg(S + 53 * c) | ((unsigned long long)__ldcg(S + 54 * c) << 32)));
}

// False if the ray cannot reach any triangle under a subtree root: an empty
// tile, or both child boxes of the root missed (the test a binary traversal
// would make first; the root's binary node, half the bytes of its wide one).
// A single-triangle root is always reachable.
__device__ __forceinline__ bool root_reachable(const Node *bin, int root, const Ray &r) {
  if (root == kNoChild) return false;
  if (root < 0) return true;
  const Node *nd = bin + root;
  float4 lxy = __ldg(&nd->lxy), rxy = __ldg(&nd->rxy), lrz = __ldg(&nd->lrz);
  float tl, tr;
  return slab(r, lxy.x, lxy.y, lxy.z, lxy.w, lrz.x, lrz.y, kInf, tl) ||
         slab(r, rxy.x, rxy.y, rxy.z, rxy.w, lrz.z, lrz.w, kInf, tr);
}

// Take up to `want` queued hand-offs, from the home tile if it has any, else
// from the first tile after it that has (work stealing).  Warp-collective;
// the result is warp-uniform: the tile (-1 if none was taken), the first
// position and the count.  avail[k] counts written items not yet taken; a
// take subtracts and gives back what it could not have, so it never takes
// more than were there.
__device__ __forceinline__ int take_handoffs(const TiledArgs &ta, int home, int want, unsigned &base, int &got) {
  const unsigned lane = lane_id();
  const int T = ta.n_tiles;
  int *head = ta.ctl, *avail = ta.ctl + 2 * T;
  got = 0;
  base = 0;
  int tile = -1;
  for (int off = 0; off < T && tile < 0; off += 32) {
    int q = off + (int)lane;
    int k = home + q;
    if (k >= T) k -= T;
    bool ne = q < T && *(volatile int *)&avail[k] > 0;
    unsigned b = __ballot_sync(0xffffffffu, ne);
    if (b) {
      tile = home + off + __ffs(b) - 1;
      if (tile >= T) tile -= T;
    }
  }
  if (tile < 0) return -1;
  if (lane == 0) {
    int old = atomicSub(&avail[tile], want);
    int g = old < 0 ? 0 : (old < want ? old : want);
    if (g < want) atomicAdd(&avail[tile], want - g);
    if (g > 0) base = (unsigned)atomicAdd(&head[tile], g);
    got = g;
  }
  got = __shfl_sync(0xffffffffu, got, 0);
  base = __shfl_sync(0xffffffffu, base, 0);
  return got > 0 ? tile : -1;
}

// Take up to `want` fresh lineages of the batch without exceeding qcap
// lineages in flight.  A lineage in flight holds one of qcap credits; a warp
// draws credits from the global count in chunks, keeps those of lineages
// that end on it for its next fresh lineages, and gives back any above one
// per lane.  Warp-collective, warp-uniform result: the first lineage offset
// and the count; *exhausted is set once the batch is used up.
__device__ __forceinline__ int take_fresh(const TraceArgs &a, const TiledArgs &ta, int want, int &credits,
                                          int64_t &base, bool &exhausted, WarpLineages &wl) {
  int *used = ta.ctl + 3 * ta.n_tiles;
  int got = 0;
  unsigned long long b = 0;
  int ex = 0, c = credits;
  if (lane_id() == 0) {
    const unsigned long long n = (unsigned long long)(a.lineage_end - a.lineage_begin);
    // with beams_per_warp the warp reserves lineages ahead, and a reserved
    // lineage holds its credit from the moment it is reserved, so that
    // reservations never exceed the cap on lineages in flight
    const int bpw = a.beams_per_warp;
    const bool refill = bpw > 0 && wl.next == wl.end && !wl.last;
    const int target = bpw > 32 ? bpw : 32;
    if (c < want || (refill && c < target)) {
      int req = target - c;
      int old = atomicAdd(used, req);
      int g = (int)ta.qcap - old;
      g = g < 0 ? 0 : (g < req ? g : req);
      if (g < req) atomicSub(used, req - g);
      c += g;
    }
    if (bpw == 0) {
      int k = c < want ? c : want;
      if (k > 0) {
        b = atomicAdd(a.lineage_next, (unsigned long long)k);
        unsigned long long left = b < n ? n - b : 0;
        if (left <= (unsigned long long)k) ex = 1;
        got = left < (unsigned long long)k ? (int)left : k;
        c -= got;
      }
    } else {
      if (refill && c > 0) {
        const unsigned long long R = (unsigned long long)(c < bpw ? c : bpw);
        const unsigned long long r0 = atomicAdd(a.lineage_next, R);
        wl.next = r0 < n ? r0 : n;
        wl.end = r0 + R < n ? r0 + R : n;
        if (r0 + R >= n) wl.last = 1;
        c -= (int)(wl.end - wl.next);
      }
      const unsigned long long have = wl.end - wl.next;
      got = have < (unsigned long long)want ? (int)have : want;
      b = wl.next;
      wl.next += got;
      if (wl.last && wl.next == wl.end) ex = 1;
    }
    if (ex && c > 0) {  // no fresh lineages left for this warp: its spare credits go back
      atomicSub(used, c);
      c = 0;
    }
  }
  got = __shfl_sync(0xffffffffu, got, 0);
  b = __shfl_sync(0xffffffffu, b, 0);
  credits = __shfl_sync(0xffffffffu, c, 0);
  if (__shfl_sync(0xffffffffu, ex, 0)) exhausted = true;
  base = (int64_t)b;
  return got;
}

// Lanes that must need service before a warp of the split trace leaves its
// search phase: all of them.  A service phase of the split trace polls the
// hand-off queues, so fewer, fuller ones measured faster (60.6 ms against
// 65.0 ms at 28 on the district with 4x4 sub-domains).
constexpr int kRefillTiled = 32;

// Distance along r to its exit from tile (ix, iy) of the grid, in the xy plane.
__device__ __forceinline__ float tile_exit(const TileGrid &tg, int ix, int iy, const Ray &r) {
  float tex = kInf, tey = kInf;
  if (r.d.x > 0.0f) tex = (tg.gx0 + (ix + 1) * tg.wx - r.o.x) / r.d.x;
  else if (r.d.x < 0.0f) tex = (tg.gx0 + ix * tg.wx - r.o.x) / r.d.x;
  if (r.d.y > 0.0f) tey = (tg.gy0 + (iy + 1) * tg.wy - r.o.y) / r.d.y;
  else if (r.d.y < 0.0f) tey = (tg.gy0 + iy * tg.wy - r.o.y) / r.d.y;
  return fminf(tex, tey);
}

// The sub-domain trace (Section 3: the geometry is split into tiles; a beam
// whose ray leaves a tile is sent to the tile it enters; exchanged beams are
// served before new ones; idle workers take work from busy tiles), as one
// persistent launch per batch.  Every warp has a home tile.  Lanes without
// work take, in this order, hand-offs from the home tile's queue, hand-offs
// from the other tiles' queues (a steal), and fresh lineages of the batch.  A
// lineage keeps going while it stays in its tile -- a reflection starts in
// the tile of its hit point -- and is pushed to the queue of the next tile
// when its ray leaves the tile without a hit there.  The launch ends when the
// batch has no fresh lineages left and no lineage is in flight (traced or
// queued).  A warp with nothing to do waits at most watchdog_ns for work;
// waits on a queue slot are bounded the same way.
//
// As in k_trace, each warp alternates a search phase (every lane with a ray
// steps through its tile's hierarchy one node at a time, until kRefillTiled
// lanes need service or none is searching) and a service phase (finished
// searches write their segment and reflect, escape, or are handed to the
// next tile; lanes without a lineage take hand-offs or fresh lineages; new
// searches start), so a long search does not hold the whole warp.
// Resident blocks per SM as for k_trace: seven for the float32 variant,
// whose smaller state fits them (40.7 -> 38.3 ms on the district split 4x4),
// and for MIXED (39.8 against 40.7 ms at six); six for the float64-chain
// variants.
template <int kP, bool kCount, bool kLeaves>
__global__ void __launch_bounds__(kTraceThreads, kP == kPF32 || kP == kPMixed ? 7 : 6) k_trace_tiled(TraceArgs a, const __grid_constant__ TiledArgs ta) {
  [[maybe_unused]] constexpr bool kPairs = Prec<kP>::pairs, kChain64 = Prec<kP>::chain64, kDefer = Prec<kP>::defer;
  __shared__ LineageSmem<kP> sm;
  const int t = threadIdx.x;
  const unsigned lane = lane_id();
  const unsigned below = (1u << lane) - 1u;
  const SceneView &v = a.v;
  const TileGrid &tg = ta.tg;  // read from parameter space, not held in registers
  __shared__ unsigned wcount[kTraceThreads / 32][kNumCounts];
  const TraceCounts cn = init_counts(wcount, t);
  const size_t qc = ta.qcap;
  const unsigned qmask = ta.qcap - 1u;
  int *const used = ta.ctl + 3 * ta.n_tiles;
  int *const finished = used + 1;
  const int n_batch = (int)(a.lineage_end - a.lineage_begin);
  int credits = 0;  // warp-uniform
  __shared__ WarpLineages wlin[kTraceThreads / 32];
  if (lane == 0) wlin[threadIdx.x >> 5] = WarpLineages{0ull, 0ull, 0};
  __syncwarp();
  LaneState ls = {-1, 0, -1, 0.0f, 0.0};
  bool active = false;      // the lane holds a lineage
  bool searching = false;   // its search in the current tile is under way
  bool pending = false;     // its search is over and awaits service
  int tile = -1;
  float tlim = kInf;        // hits are accepted up to this distance
  bool exhausted = false;   // warp-uniform: the batch has no fresh lineages left
  const int home = (int)((blockIdx.x * (kTraceThreads / 32) + (threadIdx.x >> 5)) % (unsigned)ta.n_tiles);
  unsigned long long idle_since = 0, last_prog = 0;
  HitSearch hs;
  hs.start(-1);
  int stack[kStackDepth];
  const RaySrc rs{&sm.hi[kRowO][t], kPairs ? &sm.lo[kRowO][t] : &sm.hi[kRowO][t], kTraceThreads,
                  kChain64 ? &sm.dv[kRowO][t] : nullptr, &sm.pend[0][t]};
  while (true) {
    // ---- service: finished searches write their segment and reflect, end,
    // or go on to the next tile
    bool start = false, ended = false;
    int next = -1;
    if (__ballot_sync(0xffffffffu, pending) && pending) {
      pending = false;
      const Ray r = make_ray(ld_hi3(sm, kRowO, t), ld_hi3(sm, kRowD, t), v.t_eps, ls.dns);
      if constexpr (kDefer) settle_search<true>(v.sc, r, rs, ls.dns64, hs.best, tlim);
      // the hit lies in this tile (a reflected beam starts here as well); a
      // ray without one either leaves the grid, and with it every triangle
      // (it escapes), or goes on to the next tile
      int fslot = hs.best.slot;
      bool fin = fslot >= 0;
      if (!fin) {
        // step to the next tile along the ray whose geometry the ray can
        // reach -- tiles whose root boxes it misses could give no hit, so the
        // lane walks past them itself
        int ix = tile % tg.tx, iy = tile / tg.tx;
        bool leaves = false;
        while (true) {
          float tex = kInf, tey = kInf;
          // (by the ray's inverse direction: which tile comes next needs no
          // correctly rounded quotient, the tiles' triangle lists overlap by
          // 5 cm)
          if (r.d.x > 0.0f) tex = (tg.gx0 + (ix + 1) * tg.wx - r.o.x) * r.inv.x;
          else if (r.d.x < 0.0f) tex = (tg.gx0 + ix * tg.wx - r.o.x) * r.inv.x;
          if (r.d.y > 0.0f) tey = (tg.gy0 + (iy + 1) * tg.wy - r.o.y) * r.inv.y;
          else if (r.d.y < 0.0f) tey = (tg.gy0 + iy * tg.wy - r.o.y) * r.inv.y;
          leaves = tex == kInf && tey == kInf;
          if (!leaves) {
            if (tex <= tey) ix += r.d.x > 0.0f ? 1 : -1;
            if (tey <= tex) iy += r.d.y > 0.0f ? 1 : -1;
            leaves = ix < 0 || ix >= tg.tx || iy < 0 || iy >= tg.ty;
          }
          if (leaves || root_reachable(ta.bin, __ldg(&ta.roots[iy * tg.tx + ix]), r)) break;
        }
        if (leaves) fin = true;
        else next = iy * tg.tx + ix;
      }
      // one call site, so that lanes with a hit and lanes that escape run the
      // segment and reflection code together
      if (fin) {
        if (finish_segment(a, v, 0, sm, t, r, hs.best, fslot, ls, cn)) start = true;
        else ended = true;
      }
      if (ended) active = false;
    }
    unsigned em = __ballot_sync(0xffffffffu, ended);
    if (em) {
      credits += __popc(em);
      int give = credits > 32 ? credits - 32 : 0;
      credits -= give;
      if ((int)lane == __ffs(em) - 1) {
        if (give) atomicSub(used, give);
        atomicAdd(finished, __popc(em));
      }
    }
    // ---- hand-offs: one reservation per target tile, consecutive slots
    bool push = next >= 0;
    unsigned pm = __ballot_sync(0xffffffffu, push);
    if (pm && push) {
      unsigned grp = __match_any_sync(pm, next);
      int gl = __ffs(grp) - 1;
      int n = __popc(grp);
      unsigned base = 0;
      if ((int)lane == gl) base = (unsigned)atomicAdd(&ta.ctl[ta.n_tiles + next], n);
      base = __shfl_sync(grp, base, gl);
      unsigned pos = base + (unsigned)__popc(grp & below), gen = pos & ~qmask, slot = pos & qmask;
      unsigned *sq = ta.seq + (size_t)next * qc + slot;
      // with at most qcap lineages in flight the slot's previous item has
      // been taken; its consumer may still be reading it
      if (wait_slot(a, ta, sq, gen)) {
        save_state(ta.ring + (size_t)next * kStateRows * qc + slot, qc, sm, t, ls);
        // (test hook: the launch's first hand-off is never published, so its
        // consumer's bounded wait runs out)
        if (!ta.withhold || atomicAdd(ta.ctl + 3 * ta.n_tiles + 2, 1) != 0) st_release_u32(sq, gen + 1u);
      }
      __syncwarp(grp);
      if ((int)lane == gl) atomicAdd(&ta.ctl[2 * ta.n_tiles + next], n);
      cn[kCHand]++;
      active = false;
    }
    // ---- refill: hand-offs first (home tile, then steals), then fresh lineages
    unsigned nm = __ballot_sync(0xffffffffu, !active);
    if (nm) {
      unsigned base;
      int got;
      int qt = take_handoffs(ta, home, __popc(nm), base, got);
      if (qt >= 0 && !active) {
        int rank = __popc(nm & below);
        if (rank < got) {
          unsigned pos = base + (unsigned)rank, gen = pos & ~qmask, slot = pos & qmask;
          unsigned *sq = ta.seq + (size_t)qt * qc + slot;
          // the item is counted in avail only after it is written, but the
          // position handed out may belong to a producer still writing
          if (wait_slot(a, ta, sq, gen + 1u)) {
            load_state(ta.ring + (size_t)qt * kStateRows * qc + slot, qc, sm, t, ls);
            st_release_u32(sq, gen + ta.qcap);
            tile = qt;
            active = true;
            start = true;
            if (qt != home) cn[kCSteal]++;
          }
        }
      }
      nm = __ballot_sync(0xffffffffu, !active);
      if (nm && !exhausted) {
        int64_t fb;
        int got_f = take_fresh(a, ta, __popc(nm), credits, fb, exhausted, wlin[threadIdx.x >> 5]);
        int rank = __popc(nm & below);
        if (!active && rank < got_f) {
          int64_t mine = a.lineage_begin + fb + rank;
          ls = LaneState{mine, 0, -1, 0.0f, 0.0};
          init_lineage(v, sm, t, mine);
          active = true;
          start = true;
          float3 o = ld_hi3(sm, kRowO, t);
          tile = clampi((int)floorf((o.y - tg.gy0) / tg.wy), 0, tg.ty - 1) * tg.tx +
                 clampi((int)floorf((o.x - tg.gx0) / tg.wx), 0, tg.tx - 1);
        }
      }
    }
    if (start) {
      // Hits are searched up to 1 cm past the ray's exit from the tile (the
      // tile lists hold every triangle within 5 cm of the tile): a hit there
      // is the ray's first, and a ray with none goes on to the next tile.
      const Ray r = make_ray(ld_hi3(sm, kRowO, t), ld_hi3(sm, kRowD, t), v.t_eps, ls.dns);
      tlim = tile_exit(tg, tile % tg.tx, tile / tg.tx, r) + kTileEps;
      hs.start(__ldg(&ta.roots[tile]));
      if constexpr (kDefer) rs.pend[0] = 0;
      searching = true;
    }
    if (!__any_sync(0xffffffffu, active)) {
      // nothing to trace: done once every lineage of the batch has finished
      const int fin = *(volatile int *)finished;
      if (fin == n_batch) break;
      if (*(volatile int *)&a.ctr->error) break;
      // the watchdog runs while the launch as a whole makes no progress: no
      // fresh lineage taken and none finished (both counts only grow)
      const unsigned long long now = global_ns();
      const unsigned long long prog = *(volatile unsigned long long *)a.lineage_next + (unsigned)fin;
      if (idle_since == 0 || prog != last_prog) {
        idle_since = now;
        last_prog = prog;
      } else if (now - idle_since > ta.watchdog_ns) {
        if (lane == 0) watchdog_fired(a);
        break;
      }
      __nanosleep(128);
      continue;
    }
    idle_since = 0;
    // ---- search: until kRefillTiled lanes need service (a finished search,
    // or no lineage while fresh ones remain) or no lane is searching
    {
      const Ray r = make_ray(ld_hi3(sm, kRowO, t), ld_hi3(sm, kRowD, t), v.t_eps, ls.dns);
      const int64_t n_tri = v.sc.n_tris;
      const Node4 *const nodes = v.sc.nodes;
      const Tri *const tris = v.sc.tris;
      while (true) {
        if (searching && !hs.step<kP, kCount, kLeaves>(v.sc, nodes, tris, n_tri, r, rs, ls.dns64, stack,
                                                       &a.ctr->error, cn[kCNodes], cn[kCTris], tlim)) {
          searching = false;
          pending = true;
        }
        const unsigned srch = __ballot_sync(0xffffffffu, searching);
        const unsigned idle = __ballot_sync(0xffffffffu, pending || (!active && !exhausted));
        if (!srch || __popc(idle) >= kRefillTiled) break;
      }
    }
  }
  flush_counts(a, cn, kCount);
}

template <int kP, bool kCount, bool kLeaves>
static cudaError_t launch_tiled_t(cudaStream_t st, const TraceArgs &a, const TiledArgs &ta, int n_sm) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_tiled<kP, kCount, kLeaves>,
                                                                kTraceThreads, 0);
  if (e != cudaSuccess) return e;
  if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)n_sm * per_sm;
  k_trace_tiled<kP, kCount, kLeaves><<<(int)blocks, kTraceThreads, 0, st>>>(a, ta);
  return cudaGetLastError();
}

template <int kP>
static cudaError_t launch_tiled_p(cudaStream_t st, const TraceArgs &a, const TiledArgs &ta, int n_sm) {
  if (a.leaf_size > 1)
    return a.count_work ? launch_tiled_t<kP, true, true>(st, a, ta, n_sm) : launch_tiled_t<kP, false, true>(st, a, ta, n_sm);
  return a.count_work ? launch_tiled_t<kP, true, false>(st, a, ta, n_sm) : launch_tiled_t<kP, false, false>(st, a, ta, n_sm);
}

cudaError_t launch_trace_tiled(cudaStream_t st, const TraceArgs &a, const TiledArgs &ta, int n_sm) {
  cudaError_t e;
  if (a.prec == kPMixed) e = launch_tiled_p<kPMixed>(st, a, ta, n_sm);
  else if (a.prec == kPF64) e = launch_tiled_p<kPF64>(st, a, ta, n_sm);
  else if (a.prec == kPMixed64) e = launch_tiled_p<kPMixed64>(st, a, ta, n_sm);
  else e = launch_tiled_p<kPF32>(st, a, ta, n_sm);
  note_launches(1);
  return e;
}

int tiled_resident_lanes(int n_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_tiled<kPMixed, false, false>, kTraceThreads, 0) !=
      cudaSuccess)
    per_sm = 8;
  if (per_sm < 1) per_sm = 1;
  return n_sm * per_sm * kTraceThreads;
}

// Closest hit of arbitrary float32 rays (the axis-ray query of the trace
// kernel on its own), decided as in MIXED mode with the float32 origin and
// the float64-normalised direction as float pairs.  ns: optional start-plane
// normals.
__global__ void __launch_bounds__(128) k_cast(DevScene sc, const float *o, const float *d, const float *ns,
                                              int64_t n, float t_eps, float *t_out, int *tri_out, int *err) {
  __shared__ float rh[6][128], rl[6][128];
  __shared__ int pend[kPend + 1][128];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = threadIdx.x;
  float3 O = make_float3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
  double3 Dd = normalize3(make_double3(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
  df3 D = df3{d_to_df(Dd.x), d_to_df(Dd.y), d_to_df(Dd.z)};
  double dns = 0.0;
  if (ns) dns = fabs(dot3(Dd, make_double3(ns[3 * i], ns[3 * i + 1], ns[3 * i + 2])));
  rh[0][t] = O.x; rh[1][t] = O.y; rh[2][t] = O.z;
  rl[0][t] = 0.0f; rl[1][t] = 0.0f; rl[2][t] = 0.0f;
  rh[3][t] = D.x.hi; rh[4][t] = D.y.hi; rh[5][t] = D.z.hi;
  rl[3][t] = D.x.lo; rl[4][t] = D.y.lo; rl[5][t] = D.z.lo;
  Ray r = make_ray(O, df3_hi(D), t_eps, (float)dns);
  Best best;
  const WarpCount a{nullptr}, b{nullptr};
  const RaySrc rs{&rh[0][t], &rl[0][t], 128, nullptr, &pend[0][t]};
  int slot = closest_hit<kPMixed, false>(sc, r, rs, dns, best, err, a, b, sc.root);
  // the reported distance is the float64 one to the hit triangle's plane
  // along the float-pair ray (the search itself decides in float32)
  double t64 = best.t64;
  if (slot >= 0 && !best.has64) {
    double3 o64, d64;
    rs.get(o64, d64);
    t64 = plane_t64(sc, slot, o64, d64);
  }
  t_out[i] = slot >= 0 ? (float)t64 : kInf;
  tri_out[i] = slot >= 0 ? best.id : -1;
}

cudaError_t launch_cast(cudaStream_t st, const DevScene &sc, const float *o, const float *d, const float *ns,
                        int64_t n, float t_eps, float *t_out, int *tri_out, int *err) {
  if (n <= 0) return cudaSuccess;
  k_cast<<<(int)((n + 127) / 128), 128, 0, st>>>(sc, o, d, ns, n, t_eps, t_out, tri_out, err);
  note_launches(1);
  return cudaGetLastError();
}

// One persistent grid: enough blocks to fill every SM at the kernel's
// occupancy, each block looping until the batch's lineages are taken.
template <int kP, bool kCount, bool kBatch, bool kLeaves>
static cudaError_t launch_trace_t(cudaStream_t st, const TraceArgs &a, int n_sm) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<kP, kCount, kBatch, kLeaves>,
                                                                kTraceThreads, 0);
  if (e != cudaSuccess) return e;
  if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
  if (per_sm < 1) per_sm = 1;
  int64_t n = a.lineage_end - a.lineage_begin;
  int64_t blocks = (int64_t)n_sm * per_sm;
  int64_t need = (n + kTraceThreads - 1) / kTraceThreads;
  if (blocks > need) blocks = need;
  k_trace<kP, kCount, kBatch, kLeaves><<<(int)blocks, kTraceThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <int kP, bool kBatch>
static cudaError_t launch_trace_p(cudaStream_t st, const TraceArgs &a, int n_sm) {
  if (a.leaf_size > 1)
    return a.count_work ? launch_trace_t<kP, true, kBatch, true>(st, a, n_sm)
                        : launch_trace_t<kP, false, kBatch, true>(st, a, n_sm);
  return a.count_work ? launch_trace_t<kP, true, kBatch, false>(st, a, n_sm)
                      : launch_trace_t<kP, false, kBatch, false>(st, a, n_sm);
}

template <bool kBatch>
static cudaError_t launch_trace_b(cudaStream_t st, const TraceArgs &a, int n_sm) {
  if (a.prec == kPMixed) return launch_trace_p<kPMixed, kBatch>(st, a, n_sm);
  if (a.prec == kPF64) return launch_trace_p<kPF64, kBatch>(st, a, n_sm);
  if (a.prec == kPMixed64) return launch_trace_p<kPMixed64, kBatch>(st, a, n_sm);
  return launch_trace_p<kPF32, kBatch>(st, a, n_sm);
}

cudaError_t launch_trace(cudaStream_t st, const TraceArgs &a, int n_sm) {
  cudaError_t e = a.views ? launch_trace_b<true>(st, a, n_sm) : launch_trace_b<false>(st, a, n_sm);
  note_launches(1);
  return e;
}

}  // namespace bt
