// scatter.cu -- the microphone half of the hot path (Section 2 of the
// paper): a microphone measures a beam when it lies inside the beam's cone,
// past its start plane and before its end plane, and receives the beam's
// per-band intensity W_b prod(r_b) 10^(-alpha_b d / 10) / (4 pi d^2); the
// level readout turns the accumulated intensity into 10 log10(I / 1e-12) dB.
//
//   k_scatter each lane of a warp builds the footprint of one segment record
//             written by the trace kernels; the warp then flattens the
//             (segment, cell row) pairs and the microphone runs of those
//             rows, tests every candidate microphone and adds the beam's
//             intensity with float64 atomics.
//   k_levels  intensity -> level, back to the caller's microphone order.
//
// Precision.  Microphone tests are float32 relative to the apex and are
// re-tested with float pairs when a microphone lies within the rounding band
// of a cone or start/end plane (BT_PREC_MIXED and FP32), or run in float64
// throughout (BT_PREC_FP64); intensity accumulates in float64.
#include "bt_internal.cuh"

namespace bt {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// ------------------------------------------------------- footprint polygon
// Conservative xy footprint of a segment on the microphone slab: each 3D
// half-space a.m >= b becomes, over z in [zlo, zhi], the weaker half-plane
// ax x + ay y >= b - max(az zlo, az zhi), grown by a 1 cm slack; the grid
// rectangle is clipped by those half-planes (Sutherland-Hodgman).
constexpr int kPolyMax = 12;

// A polygon's vertices in one lane's column of a [vertex][32] shared-memory
// array: vertex i at x[32 i], y[32 i].
struct PolyCol {
  float *x, *y;
};

// q = p (n vertices) clipped by ax x + ay y >= b; returns q's vertex count.
// Every vertex's plane value is evaluated once; an edge that crosses the
// line contributes its crossing.
__device__ __forceinline__ int poly_clip(PolyCol p, int n, PolyCol q, float ax, float ay, float b) {
  int m = 0;
  const float f0 = ax * p.x[0] + ay * p.y[0] - b;
  float fi = f0, xi = p.x[0], yi = p.y[0];
  for (int i = 0; i < n; i++) {
    const bool last = i + 1 == n;
    const float xj = last ? p.x[0] : p.x[32 * (i + 1)], yj = last ? p.y[0] : p.y[32 * (i + 1)];
    const float fj = last ? f0 : ax * xj + ay * yj - b;
    if (fi >= 0.0f && m < kPolyMax) { q.x[32 * m] = xi; q.y[32 * m] = yi; m++; }
    if ((fi >= 0.0f) != (fj >= 0.0f) && m < kPolyMax) {
      // fi and fj have opposite signs, so |fi - fj| >= |fi| > 0
      const float t = __fdividef(fi, fi - fj);
      q.x[32 * m] = xi + t * (xj - xi);
      q.y[32 * m] = yi + t * (yj - yi);
      m++;
    }
    fi = fj; xi = xj; yi = yj;
  }
  return m;
}

// Clip polygon P (n vertices) by the relaxation of a.m >= b into Q and swap
// the two; returns false when the footprint is empty.
__device__ __forceinline__ bool poly_halfspace(PolyCol &P, PolyCol &Q, int &n, float3 a, float b, float zl, float zh) {
  if (!(b > -kInf)) return true;  // missing plane
  float bz = fmaxf(a.z * zl, a.z * zh);
  float axy = fabsf(a.x) + fabsf(a.y);
  float bb = b - bz - 0.01f * axy - 1e-6f * fabsf(b);
  if (axy == 0.0f) return bb <= 0.0f;
  n = poly_clip(P, n, Q, a.x, a.y, bb);
  PolyCol t = P;
  P = Q;
  Q = t;
  return n >= 3;
}

// Footprint of segment s over layer `layer` of the grid (the whole height
// slab when the grid has one layer), built in the columns A and B; returns
// its vertex count (0 if it is empty) with the polygon left in A.  Planes
// are relative to the apex: n . (m - A) >= w  <=>  n . m >= w + n . A.
// Reads only the apex, the cone normals and the start and end planes of s.
__device__ __forceinline__ int seg_footprint(const Seg &s, const MicGrid &g, int layer, PolyCol A, PolyCol B) {
  float zl = g.zlo, zh = g.zhi;
  if (g.nz > 1) {
    zl = fmaxf(g.zlo, g.z0 + layer * g.dz) - 1e-3f;
    zh = fminf(g.zhi, g.z0 + (layer + 1) * g.dz) + 1e-3f;
  }
  float m = 0.01f;
  float X0 = g.x0 - m, X1 = g.x0 + g.cw * g.nx + m, Y0 = g.y0 - m, Y1 = g.y0 + g.ch * g.ny + m;
  PolyCol P = A, Q = B;
  int n = 4;
  P.x[0] = X0; P.y[0] = Y0;
  P.x[32] = X1; P.y[32] = Y0;
  P.x[64] = X1; P.y[64] = Y1;
  P.x[96] = X0; P.y[96] = Y1;
  float3 ap = make_float3(s.ahi[0], s.ahi[1], s.ahi[2]);
  float3 n0 = f3(s.n0), n1 = f3(s.n1), n2 = f3(s.n2);
  float3 ns = f3(s.start), ne = f3(s.end);
  if (!poly_halfspace(P, Q, n, n0, dot3(n0, ap), zl, zh)) return 0;
  if (!poly_halfspace(P, Q, n, n1, dot3(n1, ap), zl, zh)) return 0;
  if (!poly_halfspace(P, Q, n, n2, dot3(n2, ap), zl, zh)) return 0;
  if (!poly_halfspace(P, Q, n, ns, s.start.w + dot3(ns, ap), zl, zh)) return 0;
  if (!poly_halfspace(P, Q, n, ne, s.end.w + dot3(ne, ap), zl, zh)) return 0;
  if (P.x != A.x) {
    for (int i = 0; i < n; i++) { A.x[32 * i] = P.x[32 * i]; A.y[32 * i] = P.y[32 * i]; }
  }
  return n;
}

// ------------------------------------------------------------------ scatter
// Per-warp shared state of the scatter: 32 segments, one per lane, stored as
// [field][lane] so that lanes reading different segments hit different banks.
// The rows hold what every candidate reads; what only the rare float-pair
// re-tests (and every FP64 test) need -- the cone normals' low parts, the
// apex's third word, the start and end planes' triangle slots -- is read
// from the segment record (F_SI) when needed.
constexpr int kScatterWarps = 4;
enum : int {
  F_AX = 0, F_RX = 3, F_N0 = 6, F_NS = 15, F_NE = 19, F_P = 23, F_SI = 31, F_CY0 = 32, F_PN = 33,
  F_VI = 34, F_LAYER = 35, F_PX = 36, F_PY = F_PX + kPolyMax,
  // batches only: the view's microphone array, accumulators and band count
  // (plus an air-damping flag), read for every candidate
  F_MP = F_PY + kPolyMax, F_EP = F_MP + 2, F_CP = F_EP + 2, F_FL = F_CP + 2, F_COUNT = F_FL + 1
};
// While a lane clips its footprint, its columns of the rows below F_PX
// (written only afterwards) hold the clip's second vertex buffer.
constexpr int F_QX = 0, F_QY = kPolyMax;
static_assert(F_QY + kPolyMax <= F_PX, "clip scratch overlaps the polygon rows");
// Rows a variant needs: 60 for one scene, 67 for a batch, either way six
// 128-thread blocks per SM.
template <bool kBatch>
constexpr int scatter_rows() {
  return kBatch ? F_COUNT : F_MP;
}
template <bool kBatch>
struct ScatterSmem {
  float f[kScatterWarps][scatter_rows<kBatch>()][32];
};

// A pointer kept as two float rows (bit patterns).
__device__ __forceinline__ void put_ptr(float (*F)[32], int row, unsigned lane, const void *p) {
  const unsigned long long u = (unsigned long long)p;
  F[row][lane] = __uint_as_float((unsigned)u);
  F[row + 1][lane] = __uint_as_float((unsigned)(u >> 32));
}
template <typename T>
__device__ __forceinline__ T *get_ptr(const float (*F)[32], int row, int s) {
  return (T *)((unsigned long long)__float_as_uint(F[row][s]) |
               ((unsigned long long)__float_as_uint(F[row + 1][s]) << 32));
}

__device__ __forceinline__ int warp_incl_scan(int v, unsigned lane) {
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane >= o) v += y;
  }
  return v;
}

// Largest lane whose exclusive prefix is <= i (the owner of item i).
__device__ __forceinline__ int warp_owner(int excl, int i) {
  int owner = 0;
  for (int step = 16; step >= 1; step >>= 1) {
    int ex = __shfl_sync(0xffffffffu, excl, owner + step);
    if (ex <= i) owner += step;
  }
  return owner;
}

// m - apex as float pairs (apex hi in F[F_AX..], lo parts in F[F_RX..])
__device__ __forceinline__ df3 rel_df(const float (*F)[32], int s, float4 m) {
  return df3_sub(mkdf3(make_float3(m.x, m.y, m.z)),
                 df3{df{F[F_AX][s], F[F_RX][s]}, df{F[F_AX + 1][s], F[F_RX + 1][s]}, df{F[F_AX + 2][s], F[F_RX + 2][s]}});
}

// Signed distance of m from the plane of leaf slot `slot` as a float pair,
// oriented like the float32 normal `nf` of the segment record.
__device__ __forceinline__ float plane_side_df(const SceneView &a, int slot, float3 nf, float4 m) {
  PlaneDF pd = a.sc.planes_df[slot];
  float4 v0 = __ldg(&a.sc.tris[slot].v0);
  df3 n = df3{df{pd.hi.x, pd.lo.x}, df{pd.hi.y, pd.lo.y}, df{pd.hi.z, pd.lo.z}};
  df3 rel = df3_sub(mkdf3(make_float3(m.x, m.y, m.z)), mkdf3(f3(v0)));
  df e = df3_dot(n, rel);
  float sg = pd.hi.x * nf.x + pd.hi.y * nf.y + pd.hi.z * nf.z < 0.0f ? -1.0f : 1.0f;
  return sg * (e.hi + e.lo);
}

// Signed distance of m from the float64 plane of leaf slot `slot`, oriented
// like the float32 normal `nf` of the segment record (FP64 mode).
__device__ __forceinline__ double plane_side64(const SceneView &a, int slot, float3 nf, float4 m) {
  Plane64 pl = ldg_d4(&a.sc.planes64[slot]);
  double e = pl.x * (double)m.x + pl.y * (double)m.y + pl.z * (double)m.z - pl.w;
  return pl.x * nf.x + pl.y * nf.y + pl.z * nf.z < 0.0 ? -e : e;
}

// One warp takes 32 segments at a time.  Each lane loads one segment and
// builds its footprint; the warp then walks the (segment, cell row) pairs of
// all 32 footprints 32 at a time, turns each into its run of microphones, and
// walks the runs 32 candidates at a time, so every lane has work whatever
// the footprint sizes.
template <bool kF64, bool kBatch>
__global__ void __launch_bounds__(32 * kScatterWarps) k_scatter(ScatterArgs a) {
  __shared__ ScatterSmem<kBatch> sm;
  const unsigned lane = lane_id();
  const int w = threadIdx.x >> 5;
  float(*F)[32] = sm.f[w];
  const long long n_seg = (long long)min(*a.seg_count, a.seg_capacity);
  // work items: (segment, microphone layer) pairs; one per segment when the
  // microphones lie in one layer
  const int n_layers = a.max_nz > 1 ? a.max_nz : 1;
  const long long n_items = n_seg * n_layers;
  unsigned long long n_cand = 0, n_contrib = 0;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp0 * 32; base < n_items; base += n_warps * 32) {
    // ---- 1. one item per lane: segment parameters and the layer's footprint
    const long long it = base + lane;
    const long long ii = it / n_layers;
    const int layer = (int)(it - ii * n_layers);
    // the segment record: in order of place when the scene orders its scatter
    const long long si = a.order && it < n_items ? (long long)__ldg(&a.order[ii]) : ii;
    int nrows = 0;
    if (it < n_items) {
      // the footprint needs the apex, the cone normals and the start and end
      // planes (the record's first 112 bytes); the rest is read only for a
      // non-empty footprint
      Seg sl;
      const float4 *src4 = reinterpret_cast<const float4 *>(a.segs + si);
      float4 *dst4 = reinterpret_cast<float4 *>(&sl);
#pragma unroll
      for (int q = 0; q < 7; q++) dst4[q] = __ldg(src4 + q);
      const int vi = kBatch ? sl.view : 0;
      const MicGrid &g = *(kBatch ? a.views[vi] : a.v).grid;
      // the footprint is clipped in the lane's own columns: the polygon rows
      // and, as scratch, the rows of the segment fields written below
      const int pn = layer < g.nz ? seg_footprint(sl, g, layer, PolyCol{&F[F_PX][lane], &F[F_PY][lane]},
                                                  PolyCol{&F[F_QX][lane], &F[F_QY][lane]})
                                  : 0;
      int cy0 = 0, cy1 = -1;
      if (pn > 0) {
        float ymin = kInf, ymax = -kInf;
        for (int i = 0; i < pn; i++) { ymin = fminf(ymin, F[F_PY + i][lane]); ymax = fmaxf(ymax, F[F_PY + i][lane]); }
        if (ymin <= ymax) {
          cy0 = clampi((int)floorf((ymin - g.y0) * g.inv_ch), 0, g.ny - 1);
          cy1 = clampi((int)floorf((ymax - g.y0) * g.inv_ch), 0, g.ny - 1);
        }
      }
      nrows = cy1 >= cy0 ? cy1 - cy0 + 1 : 0;
      if (nrows > 0) {
        // band powers (p03, p47); the normals' low parts stay in the record
        dst4[7] = __ldg(src4 + 7);
        dst4[8] = __ldg(src4 + 8);
        F[F_VI][lane] = __int_as_float(vi);
        F[F_SI][lane] = __int_as_float((int)si);
        if (kBatch) {
          const SceneView &V = a.views[vi];
          put_ptr(F, F_MP, lane, V.mics);
          put_ptr(F, F_EP, lane, V.energy);
          put_ptr(F, F_CP, lane, V.count);
          F[F_FL][lane] = __int_as_float(V.sc.n_bands | (V.has_alpha ? 0x100 : 0));
        }
        F[F_LAYER][lane] = __int_as_float(layer);
        for (int q = 0; q < 3; q++) {
          F[F_AX + q][lane] = sl.ahi[q];
          F[F_RX + q][lane] = sl.alo[q];
        }
        F[F_N0][lane] = sl.n0.x; F[F_N0 + 1][lane] = sl.n0.y; F[F_N0 + 2][lane] = sl.n0.z;
        F[F_N0 + 3][lane] = sl.n1.x; F[F_N0 + 4][lane] = sl.n1.y; F[F_N0 + 5][lane] = sl.n1.z;
        F[F_N0 + 6][lane] = sl.n2.x; F[F_N0 + 7][lane] = sl.n2.y; F[F_N0 + 8][lane] = sl.n2.z;
        F[F_NS][lane] = sl.start.x; F[F_NS + 1][lane] = sl.start.y; F[F_NS + 2][lane] = sl.start.z;
        F[F_NS + 3][lane] = sl.start.w;
        F[F_NE][lane] = sl.end.x; F[F_NE + 1][lane] = sl.end.y; F[F_NE + 2][lane] = sl.end.z;
        F[F_NE + 3][lane] = sl.end.w;
        F[F_P][lane] = sl.p03.x; F[F_P + 1][lane] = sl.p03.y; F[F_P + 2][lane] = sl.p03.z;
        F[F_P + 3][lane] = sl.p03.w; F[F_P + 4][lane] = sl.p47.x; F[F_P + 5][lane] = sl.p47.y;
        F[F_P + 6][lane] = sl.p47.z; F[F_P + 7][lane] = sl.p47.w;
        F[F_CY0][lane] = __int_as_float(cy0);
        F[F_PN][lane] = __int_as_float(pn);
      }
    }
    __syncwarp();
    // ---- 2. (segment, row) pairs of the 32 footprints, 32 at a time
    const int rincl = warp_incl_scan(nrows, lane);
    const int total_rows = __shfl_sync(0xffffffffu, rincl, 31);
    const int rexcl = rincl - nrows;
    for (int rb = 0; rb < total_rows; rb += 32) {
      int r = rb + (int)lane;
      int so = warp_owner(rexcl, r);  // segment lane owning pair r
      int so_excl = __shfl_sync(0xffffffffu, rexcl, so);
      int first = 0, cnt = 0;
      if (r < total_rows) {
        const SceneView &V = kBatch ? a.views[__float_as_int(F[F_VI][so])] : a.v;
        const MicGrid &g = *V.grid;
        int row = __float_as_int(F[F_CY0][so]) + (r - so_excl);
        float ya = g.y0 + row * g.ch, yb = ya + g.ch;
        float my = 1e-3f * g.ch;
        // x extent of the owner's footprint within the row's strip
        int pn = __float_as_int(F[F_PN][so]);
        float xmin = kInf, xmax = -kInf;
        float y0s = ya - my, y1s = yb + my;
        for (int i = 0; i < pn; i++) {
          int j = i + 1 == pn ? 0 : i + 1;
          float xi = F[F_PX + i][so], yi = F[F_PY + i][so], xj = F[F_PX + j][so], yj = F[F_PY + j][so];
          if (yi >= y0s && yi <= y1s) { xmin = fminf(xmin, xi); xmax = fmaxf(xmax, xi); }
          // crossings of the strip's edges; yi != yj whenever an edge
          // crosses, and the quotient lies in [0, 1]
          if ((yi < y0s) != (yj < y0s)) {
            float x = xi + __fdividef(y0s - yi, yj - yi) * (xj - xi);
            xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
          }
          if ((yi < y1s) != (yj < y1s)) {
            float x = xi + __fdividef(y1s - yi, yj - yi) * (xj - xi);
            xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
          }
        }
        if (xmin <= xmax) {
          int cx0 = clampi((int)floorf((xmin - g.x0) * g.inv_cw), 0, g.nx - 1);
          int cx1 = clampi((int)floorf((xmax - g.x0) * g.inv_cw), 0, g.nx - 1);
          const int cell0 = (__float_as_int(F[F_LAYER][so]) * g.ny + row) * g.nx;
          first = __ldg(&V.cell_start[cell0 + cx0]);
          cnt = __ldg(&V.cell_start[cell0 + cx1 + 1]) - first;
        }
      }
      // ---- 3. candidates of those runs, 32 at a time
      const int cincl = warp_incl_scan(cnt, lane);
      const int total_c = __shfl_sync(0xffffffffu, cincl, 31);
      const int cexcl = cincl - cnt;
      for (int cb = 0; cb < total_c; cb += 32) {
        int c = cb + (int)lane;
        int ro = warp_owner(cexcl, c);
        int ofirst = __shfl_sync(0xffffffffu, first, ro);
        int oexcl = __shfl_sync(0xffffffffu, cexcl, ro);
        int s = __shfl_sync(0xffffffffu, so, ro);
        if (c < total_c) {
          int mi = ofirst + (c - oexcl);
          // where the contribution goes: the scene's accumulators, band
          // count and air damping (kernel parameters for one scene, the
          // segment's rows in a batch)
          const float4 *mics;
          double *energy;
          int *count;
          int nb;
          bool has_alpha;
          if (kBatch) {
            mics = get_ptr<const float4>(F, F_MP, s);
            energy = get_ptr<double>(F, F_EP, s);
            count = get_ptr<int>(F, F_CP, s);
            const int fl = __float_as_int(F[F_FL][s]);
            nb = fl & 0xff;
            has_alpha = (fl & 0x100) != 0;
          } else {
            mics = a.v.mics;
            energy = a.v.energy;
            count = a.v.count;
            nb = a.v.sc.n_bands;
            has_alpha = a.v.has_alpha != 0;
          }
          const Seg *rec = a.segs + __float_as_int(F[F_SI][s]);
          float4 m = __ldg(&mics[mi]);
          if (kF64) {
            // FP64: every test and the contribution in float64 (apex exact
            // from its three words, cone normals from their float pairs,
            // start/end planes from the triangles' float64 planes)
            n_cand++;
            const double3 A = make_double3(((double)F[F_AX][s] + F[F_RX][s]) + __ldg(&rec->pad[0]),
                                           ((double)F[F_AX + 1][s] + F[F_RX + 1][s]) + __ldg(&rec->pad[1]),
                                           ((double)F[F_AX + 2][s] + F[F_RX + 2][s]) + __ldg(&rec->pad[2]));
            const double3 vd = make_double3((double)m.x - A.x, (double)m.y - A.y, (double)m.z - A.z);
            bool in = true;
#pragma unroll
            for (int j = 0; j < 3; j++) {
              double3 nd = make_double3((double)F[F_N0 + 3 * j][s] + __ldg(&rec->nlo[3 * j]),
                                        (double)F[F_N0 + 3 * j + 1][s] + __ldg(&rec->nlo[3 * j + 1]),
                                        (double)F[F_N0 + 3 * j + 2][s] + __ldg(&rec->nlo[3 * j + 2]));
              in = in && dot3(nd, vd) >= 0.0;
            }
            if (in) {
              const SceneView &V = kBatch ? a.views[__float_as_int(F[F_VI][s])] : a.v;
              int s_slot = __float_as_int(__ldg(&rec->n0.w)), e_slot = __float_as_int(__ldg(&rec->n1.w));
              float3 ns = make_float3(F[F_NS][s], F[F_NS + 1][s], F[F_NS + 2][s]);
              float3 ne = make_float3(F[F_NE][s], F[F_NE + 1][s], F[F_NE + 2][s]);
              double fs = s_slot >= 0 ? plane_side64(V, s_slot, ns, m) : 1.0;
              double fe = e_slot >= 0 ? plane_side64(V, e_slot, ne, m) : 1.0;
              in = fs > 0.0 && fe >= 0.0;
            }
            const double d2 = dot3(vd, vd);
            if (in && d2 > 1e-18) {
              const double gf = 1.0 / (4.0 * 3.141592653589793 * d2);
              const double dist = has_alpha ? sqrt(d2) : 0.0;
              const float *alpha = (kBatch ? a.views[__float_as_int(F[F_VI][s])] : a.v).alpha_log2;
              double *e = energy + (size_t)mi * kMaxBands;
#pragma unroll
              for (int b = 0; b < kMaxBands; b++) {
                if (b < nb) {
                  double cval = (double)F[F_P + b][s] * gf;
                  if (has_alpha) cval *= exp2((double)alpha[b] * dist);
                  atomicAdd(e + b, cval);
                }
              }
              atomicAdd(count + mi, 1);
              n_contrib++;
            }
            continue;
          }
          // m - apex with the apex as hi + lo: one extra rounding at most
          float3 v = make_float3((m.x - F[F_AX][s]) - F[F_RX][s], (m.y - F[F_AX + 1][s]) - F[F_RX + 1][s],
                                 (m.z - F[F_AX + 2][s]) - F[F_RX + 2][s]);
          n_cand++;
          // cone planes: float32; within the rounding band of a plane the
          // test is redone with float pairs
          const float band_v = 2e-6f * (fabsf(v.x) + fabsf(v.y) + fabsf(v.z));
          bool in = true;
#pragma unroll
          for (int j = 0; j < 3; j++) {
            float3 nj = make_float3(F[F_N0 + 3 * j][s], F[F_N0 + 3 * j + 1][s], F[F_N0 + 3 * j + 2][s]);
            float e = dot3(nj, v);
            if (fabsf(e) <= band_v * (fabsf(nj.x) + fabsf(nj.y) + fabsf(nj.z))) {
              df3 nd = df3{df{nj.x, __ldg(&rec->nlo[3 * j])}, df{nj.y, __ldg(&rec->nlo[3 * j + 1])},
                           df{nj.z, __ldg(&rec->nlo[3 * j + 2])}};
              df ed = df3_dot(nd, rel_df(F, s, m));
              e = ed.hi + ed.lo;
            }
            in = in && e >= 0.0f;
          }
          if (in) {
            // start/end planes: float32 relative to the apex; within the
            // rounding band the test is redone with float pairs against the
            // triangle's own plane, the form the definition uses
            float3 ns = make_float3(F[F_NS][s], F[F_NS + 1][s], F[F_NS + 2][s]);
            float3 ne = make_float3(F[F_NE][s], F[F_NE + 1][s], F[F_NE + 2][s]);
            float band = 1e-4f + 1e-6f * (fabsf(v.x) + fabsf(v.y) + fabsf(v.z));
            float fs = dot3(ns, v) - F[F_NS + 3][s], fe = dot3(ne, v) - F[F_NE + 3][s];
            if (fabsf(fs) <= band || fabsf(fe) <= band) {
              const SceneView &V = kBatch ? a.views[__float_as_int(F[F_VI][s])] : a.v;
              int s_slot = __float_as_int(__ldg(&rec->n0.w)), e_slot = __float_as_int(__ldg(&rec->n1.w));
              if (fabsf(fs) <= band && s_slot >= 0) fs = plane_side_df(V, s_slot, ns, m);
              if (fabsf(fe) <= band && e_slot >= 0) fe = plane_side_df(V, e_slot, ne, m);
            }
            in = fs > 0.0f && fe >= 0.0f;
          }
          float d2 = dot3(v, v);
          if (in && d2 > 1e-18f) {
            float gf = 1.0f / (4.0f * 3.14159265358979f * d2);
            float dist = has_alpha ? sqrtf(d2) : 0.0f;
            double *e = energy + (size_t)mi * kMaxBands;
            if (has_alpha) {
              const float *alpha = (kBatch ? a.views[__float_as_int(F[F_VI][s])] : a.v).alpha_log2;
#pragma unroll
              for (int b = 0; b < kMaxBands; b++)
                if (b < nb) atomicAdd(e + b, (double)(F[F_P + b][s] * gf * exp2f(alpha[b] * dist)));
            } else {
#pragma unroll
              for (int b = 0; b < kMaxBands; b++)
                if (b < nb) atomicAdd(e + b, (double)(F[F_P + b][s] * gf));
            }
            atomicAdd(&count[mi], 1);
            n_contrib++;
          }
        }
      }
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) {
    n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
    n_contrib += __shfl_xor_sync(0xffffffffu, n_contrib, o);
  }
  if (lane == 0) {
    atomicAdd(&a.ctr->candidates, n_cand);
    atomicAdd(&a.ctr->contributions, n_contrib);
  }
}

// ------------------------------------------------------ order of place
// With microphones through a whole volume, the accumulators and positions
// are many times the L2; segments taken in the order they were traced reach
// microphones all over the city, so nearly every atomic update and position
// load goes to HBM.  Taken in order of the cell under each segment (bins of
// 2^kOrderBits x 2^kOrderBits cells along a Morton curve), the warps
// resident at any time work in one neighbourhood and its accumulators stay
// in L2.  A counting sort: bin histogram, exclusive scan, placement; the
// order within a bin is immaterial (every contribution is added, whatever
// the order).
__device__ __forceinline__ int order_bin(const MicGrid &g, int key) {
  const unsigned x = ((unsigned)(key & 0xffff) << kOrderBits) / (unsigned)max(g.nx, 1);
  const unsigned y = ((unsigned)key >> 16 << kOrderBits) / (unsigned)max(g.ny, 1);
  unsigned m = 0;
#pragma unroll
  for (int b = 0; b < kOrderBits; b++) m |= ((x >> b) & 1u) << (2 * b) | ((y >> b) & 1u) << (2 * b + 1);
  return (int)(m & (kOrderBins - 1));
}

__global__ void __launch_bounds__(256) k_order_hist(const Seg *segs, const unsigned long long *seg_count,
                                                    unsigned long long cap, const MicGrid *grid, uint32_t *hist) {
  __shared__ uint32_t h[kOrderBins];
  for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const MicGrid g = *grid;
  const long long n = (long long)min(*seg_count, cap);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    atomicAdd(&h[order_bin(g, __ldg(&segs[i].key))], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Exclusive scan of the kOrderBins counts in place, one block.
__global__ void __launch_bounds__(1024) k_order_scan(uint32_t *hist) {
  constexpr int kPer = kOrderBins / 1024;
  __shared__ uint32_t part[1024];
  uint32_t v[kPer], sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; q++) {
    v[q] = hist[threadIdx.x * kPer + q];
    sum += v[q];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t y = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += y;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
#pragma unroll
  for (int q = 0; q < kPer; q++) {
    hist[threadIdx.x * kPer + q] = run;
    run += v[q];
  }
}

// Each record index to its bin's next place; lanes of a warp with the same
// bin take their places with one atomic.
__global__ void __launch_bounds__(256) k_order_place(const Seg *segs, const unsigned long long *seg_count,
                                                     unsigned long long cap, const MicGrid *grid, uint32_t *offs,
                                                     uint32_t *order) {
  const MicGrid g = *grid;
  const long long n = (long long)min(*seg_count, cap);
  const unsigned lane = lane_id();
  for (long long b0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) & ~31ll; b0 < n;
       b0 += (long long)gridDim.x * blockDim.x) {
    const long long i = b0 + lane;
    const bool ok = i < n;
    const int bin = ok ? order_bin(g, __ldg(&segs[i].key)) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (ok && (int)lane == leader) base = atomicAdd(&offs[bin], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (ok) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

cudaError_t launch_seg_order(cudaStream_t st, const Seg *segs, const unsigned long long *seg_count,
                             unsigned long long cap, const MicGrid *grid, uint32_t *hist, uint32_t *order, int n_sm) {
  static_assert(kOrderBins % 1024 == 0, "scan layout");
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kOrderBins, st);
  if (e != cudaSuccess) return e;
  const int blocks = n_sm * 4;
  k_order_hist<<<blocks, 256, 0, st>>>(segs, seg_count, cap, grid, hist);
  k_order_scan<<<1, 1024, 0, st>>>(hist);
  k_order_place<<<blocks, 256, 0, st>>>(segs, seg_count, cap, grid, hist, order);
  note_launches(3);
  return cudaGetLastError();
}

template <bool kF64, bool kBatch>
static cudaError_t launch_scatter_t(cudaStream_t st, const ScatterArgs &a, int n_sm) {
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<kF64, kBatch>, 32 * kScatterWarps, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k_scatter<kF64, kBatch><<<n_sm * per_sm, 32 * kScatterWarps, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scatter(cudaStream_t st, const ScatterArgs &a, int n_sm) {
  cudaError_t e;
  if (a.views) e = a.fp64 ? launch_scatter_t<true, true>(st, a, n_sm) : launch_scatter_t<false, true>(st, a, n_sm);
  else e = a.fp64 ? launch_scatter_t<true, false>(st, a, n_sm) : launch_scatter_t<false, false>(st, a, n_sm);
  note_launches(1);
  return e;
}

// ------------------------------------------------------------------ levels
// L = 10 log10(I / 1e-12) dB; -inf where no beam reached the microphone.
__global__ void k_levels(const double *energy, const int *count, const float4 *mics, int64_t n_m,
                         int n_bands, double *level_db, double *intensity, int *path_count) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_m) return;
  int64_t orig = __float_as_int(mics[p].w);
  for (int b = 0; b < n_bands; b++) {
    double I = energy[p * kMaxBands + b];
    level_db[orig * n_bands + b] = I > 0.0 ? 10.0 * log10(I) + 120.0 : -__builtin_huge_val();
    intensity[orig * n_bands + b] = I;
  }
  path_count[orig] = count[p];
}

cudaError_t launch_levels(cudaStream_t st, const double *energy, const int *count, const float4 *mics,
                          int64_t n_m, int n_bands, double *level_db, double *intensity, int *path_count) {
  if (n_m == 0) return cudaSuccess;
  int threads = 256;
  k_levels<<<(int)((n_m + threads - 1) / threads), threads, 0, st>>>(energy, count, mics, n_m, n_bands,
                                                                     level_db, intensity, path_count);
  note_launches(1);
  return cudaGetLastError();
}

// Install a result given in input microphone order (partial results of
// source shards, summed by the caller) into a scene's accumulators, which are
// kept in binned order.
__global__ void k_set_result(const double *intensity, const int *count_in, const float4 *mics, int64_t n_m,
                             int n_bands, double *energy, int *count) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_m) return;
  int64_t orig = __float_as_int(mics[p].w);
  for (int b = 0; b < kMaxBands; b++) energy[p * kMaxBands + b] = b < n_bands ? intensity[orig * n_bands + b] : 0.0;
  count[p] = count_in ? count_in[orig] : 0;
}

cudaError_t launch_set_result(cudaStream_t st, const double *intensity, const int *count_in, const float4 *mics,
                              int64_t n_m, int n_bands, double *energy, int *count) {
  if (n_m == 0) return cudaSuccess;
  int threads = 256;
  k_set_result<<<(int)((n_m + threads - 1) / threads), threads, 0, st>>>(intensity, count_in, mics, n_m,
                                                                         n_bands, energy, count);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bt
