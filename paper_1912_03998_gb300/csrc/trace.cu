// trace.cu -- the hot path of the hybrid beam/ray tracer (Section 2 of the
// paper): beam generation, axis-ray traversal, image-source reflection,
// microphone-in-beam test and per-band energy scatter, and level readout.
//
// Two kernels per batch of beam lineages:
//   k_trace   one thread per lineage (source, icosahedron face): for orders
//             0..K it casts the beam's axis ray through the BVH, writes the
//             segment (apex, cone planes, start/end planes, band power) if its
//             footprint overlaps the microphone grid, and reflects the beam
//             about the hit triangle's plane (image source).
//   k_scatter one warp per segment: the warp walks the cell rows under the
//             segment's footprint 32 rows at a time, flattens the microphone
//             runs of those rows with a warp scan, tests every candidate
//             microphone and adds the beam's intensity with float64 atomics.
#include <stdio.h>

#include "bt_internal.cuh"

namespace bt {

// Regular icosahedron: unit vertices (the cyclic permutations of
// (0, +-1, +-phi), normalised) and its 20 faces, counter-clockwise seen
// from outside.
__constant__ float c_ico_v[12][3] = {
    {0.000000000f, -0.525731112f, 0.850650808f},  {0.000000000f, 0.525731112f, 0.850650808f},
    {0.850650808f, 0.000000000f, 0.525731112f},   {-0.850650808f, 0.000000000f, 0.525731112f},
    {-0.525731112f, -0.850650808f, 0.000000000f}, {0.525731112f, -0.850650808f, 0.000000000f},
    {0.525731112f, 0.850650808f, 0.000000000f},   {-0.525731112f, 0.850650808f, 0.000000000f},
    {0.850650808f, 0.000000000f, -0.525731112f},  {-0.850650808f, 0.000000000f, -0.525731112f},
    {0.000000000f, -0.525731112f, -0.850650808f}, {0.000000000f, 0.525731112f, -0.850650808f},
};
__constant__ int c_ico_f[20][3] = {
    {0, 2, 1},  {0, 1, 3},  {0, 5, 2},  {0, 3, 4},  {1, 2, 6},   {1, 7, 3},  {0, 4, 5},
    {1, 6, 7},  {2, 5, 8},  {2, 8, 6},  {3, 9, 4},  {3, 7, 9},   {4, 10, 5}, {6, 11, 7},
    {4, 9, 10}, {5, 10, 8}, {6, 8, 11}, {7, 11, 9}, {8, 10, 11}, {9, 11, 10},
};

// Edge directions of face `i` of the level-L geodesic icosahedron.  The base
// face is i >> 2L; each further pair of bits picks one of the four children
// (a,ab,ca), (ab,b,bc), (ca,bc,c), (ab,bc,ca), ab = midpoint pushed to the
// sphere.  A vertex shared by two faces is computed from the same operands in
// both, so both faces get the bit-identical direction.
__device__ __forceinline__ void beam_dirs(int level, int64_t i, float3 &a, float3 &b, float3 &c) {
  int f = (int)(i >> (2 * level));
  a = make_float3(c_ico_v[c_ico_f[f][0]][0], c_ico_v[c_ico_f[f][0]][1], c_ico_v[c_ico_f[f][0]][2]);
  b = make_float3(c_ico_v[c_ico_f[f][1]][0], c_ico_v[c_ico_f[f][1]][1], c_ico_v[c_ico_f[f][1]][2]);
  c = make_float3(c_ico_v[c_ico_f[f][2]][0], c_ico_v[c_ico_f[f][2]][1], c_ico_v[c_ico_f[f][2]][2]);
  for (int l = level - 1; l >= 0; --l) {
    int ch = (int)((i >> (2 * l)) & 3);
    float3 ab = normalize3(a + b), bc = normalize3(b + c), ca = normalize3(c + a);
    if (ch == 0) { b = ab; c = ca; }
    else if (ch == 1) { a = ab; c = bc; }
    else if (ch == 2) { a = ca; b = bc; }
    else { a = ab; b = bc; c = ca; }
  }
}

// Closest accepted hit of the ray in the BVH; ties in distance go to the
// lowest original triangle id.  Returns the leaf slot or -1.
template <bool kCount>
__device__ __forceinline__ int closest_hit(const DevScene &sc, const Ray &r, float &best_t, int *err,
                                           unsigned long long &n_nodes, unsigned long long &n_tris) {
  best_t = kInf;
  int best_slot = -1, best_id = 0x7fffffff;
  if (sc.root == -1) return -1;
  int stack[kStackDepth];
  int sp = 0;
  int node = sc.root;
  // a well-formed BVH is visited at most once per node; the bound only
  // guarantees termination should the structure ever be malformed
  int64_t visits = 0;
  if (node < 0) {  // a single triangle
    int slot = ~node;
    if (kCount) n_tris++;
    float t = hit_watertight(r, __ldg(&sc.tris[slot].v0), __ldg(&sc.tris[slot].v1), __ldg(&sc.tris[slot].v2));
    if (t < kInf && accept_hit(r, t)) { best_t = t; best_slot = slot; }
    return best_slot;
  }
  while (true) {
    if (++visits > sc.n_tris + 64) {
      atomicExch(err, BT_E_TIMEOUT);
      break;
    }
    const Node *nd = sc.nodes + node;
    if (kCount) n_nodes++;
    float4 lxy = __ldg(&nd->lxy), rxy = __ldg(&nd->rxy), lrz = __ldg(&nd->lrz);
    int2 ch = __ldg((const int2 *)&nd->child);
    float tl, tr;
    bool hl = slab(r, lxy.x, lxy.y, lxy.z, lxy.w, lrz.x, lrz.y, best_t, tl);
    bool hr = slab(r, rxy.x, rxy.y, rxy.z, rxy.w, lrz.z, lrz.w, best_t, tr);
#pragma unroll
    for (int side = 0; side < 2; side++) {
      int c = side ? ch.y : ch.x;
      bool h = side ? hr : hl;
      if (h && c < 0) {
        int slot = ~c;
        if (kCount) n_tris++;
        const Tri *tp = sc.tris + slot;
        float4 v0 = __ldg(&tp->v0), v1 = __ldg(&tp->v1), v2 = __ldg(&tp->v2);
        float t = hit_watertight(r, v0, v1, v2);
        if (t < kInf && accept_hit(r, t)) {
          int id = __float_as_int(v1.w);
          if (t < best_t || (t == best_t && id < best_id)) { best_t = t; best_slot = slot; best_id = id; }
        }
        if (side) hr = false; else hl = false;
      }
    }
    if (hl && hr) {
      bool lf = tl <= tr;
      if (sp < kStackDepth) stack[sp++] = lf ? ch.y : ch.x;
      else atomicExch(err, BT_E_QUEUE_FULL);
      node = lf ? ch.x : ch.y;
    } else if (hl) {
      node = ch.x;
    } else if (hr) {
      node = ch.y;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return best_slot;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Row range of the segment's footprint, or false if it misses the grid.
__device__ __forceinline__ bool seg_rows(const Seg &s, const MicGrid &g, int &cy0, int &cy1) {
  Poly p;
  if (!seg_footprint(s, g, p)) return false;
  float ymin = kInf, ymax = -kInf;
  for (int i = 0; i < p.n; i++) { ymin = fminf(ymin, p.y[i]); ymax = fmaxf(ymax, p.y[i]); }
  if (!(ymin <= ymax)) return false;
  cy0 = clampi((int)floorf((ymin - g.y0) * g.inv_ch), 0, g.ny - 1);
  cy1 = clampi((int)floorf((ymax - g.y0) * g.inv_ch), 0, g.ny - 1);
  return true;
}

template <bool kCount>
__global__ void __launch_bounds__(128) k_trace(TraceArgs a) {
  const MicGrid g = *a.grid;
  const int nb = a.sc.n_bands;
  unsigned long long n_seg = 0, n_hit = 0, n_esc = 0, n_emit = 0, n_nodes = 0, n_tris = 0;
  for (int64_t lin = a.lineage_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       lin < a.lineage_end; lin += (int64_t)gridDim.x * blockDim.x) {
    int64_t si = lin / a.n_beams, bi = lin - si * a.n_beams;
    float3 d0, d1, d2;
    beam_dirs(a.level, bi, d0, d1, d2);
    float3 n0 = cross_exact(d0, d1), n1 = cross_exact(d1, d2), n2 = cross_exact(d2, d0);
    float3 A = f3(__ldg(&a.src[si]));
    float3 O = A;
    float3 D = normalize3(d0 + d1 + d2);
    float P[kMaxBands];
#pragma unroll
    for (int b = 0; b < kMaxBands; b++) P[b] = b < nb ? __ldg(&a.power[si * nb + b]) : 0.0f;
    float4 start = make_float4(0.0f, 0.0f, 0.0f, -kInf);
    float dns = 0.0f;
    for (int k = 0; k <= a.max_order; k++) {
      Ray r = make_ray(O, D, a.t_eps, dns);
      float th;
      int slot = closest_hit<kCount>(a.sc, r, th, &a.ctr->error, n_nodes, n_tris);
      n_seg++;
      float4 end = make_float4(0.0f, 0.0f, 0.0f, -kInf);
      float4 pl = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (slot >= 0) {
        n_hit++;
        pl = __ldg(&a.sc.planes[slot]);
        bool facing = pl.x * D.x + pl.y * D.y + pl.z * D.z < 0.0f;
        end = facing ? pl : make_float4(-pl.x, -pl.y, -pl.z, -pl.w);
      } else {
        n_esc++;
      }
      Seg s;
      s.apex = make_float4(A.x, A.y, A.z, 0.0f);
      s.n0 = make_float4(n0.x, n0.y, n0.z, 0.0f);
      s.n1 = make_float4(n1.x, n1.y, n1.z, __int_as_float((int)si));
      s.n2 = make_float4(n2.x, n2.y, n2.z, __int_as_float(k));
      s.start = start;
      s.end = end;
      s.p03 = make_float4(P[0], P[1], P[2], P[3]);
      s.p47 = make_float4(P[4], P[5], P[6], P[7]);
      int cy0 = 0, cy1 = -1;
      bool emit = g.n_mics > 0 && seg_rows(s, g, cy0, cy1);
      s.apex.w = __int_as_float(cy0);
      s.n0.w = __int_as_float(cy1);
      unsigned mask = __activemask();
      unsigned bal = __ballot_sync(mask, emit);
      if (bal) {
        int leader = __ffs(bal) - 1;
        unsigned long long base = 0;
        if ((int)lane_id() == leader) base = atomicAdd(a.seg_count, (unsigned long long)__popc(bal));
        base = __shfl_sync(mask, base, leader);
        if (emit) {
          unsigned long long idx = base + __popc(bal & ((1u << lane_id()) - 1u));
          if (idx < a.seg_capacity) a.segs[idx] = s;
          else atomicExch(&a.ctr->error, BT_E_QUEUE_FULL);
          n_emit++;
        }
      }
      if (slot < 0 || k == a.max_order) break;
      // Image source: mirror the apex, the cone and the axis in the hit
      // plane; the reflected beam starts on that plane and loses energy.
      float4 v0 = __ldg(&a.sc.tris[slot].v0);
      int mat = __float_as_int(v0.w);
      float wmax = 0.0f;
#pragma unroll
      for (int b = 0; b < kMaxBands; b++) {
        if (b < nb) P[b] *= __ldg(&a.sc.refl[mat * nb + b]);
        wmax = fmaxf(wmax, P[b]);
      }
      if (a.energy_threshold > 0.0f && wmax < a.energy_threshold) break;
      float3 pn = make_float3(pl.x, pl.y, pl.z);
      float3 H = O + D * th;
      float da = dot3(A - f3(v0), pn);
      A = A - pn * (2.0f * da);
      n0 = n0 - pn * (2.0f * dot3(n0, pn));
      n1 = n1 - pn * (2.0f * dot3(n1, pn));
      n2 = n2 - pn * (2.0f * dot3(n2, pn));
      D = D - pn * (2.0f * dot3(D, pn));
      O = H;
      bool toward = dot3(pn, D) > 0.0f;
      start = toward ? pl : make_float4(-pl.x, -pl.y, -pl.z, -pl.w);
      dns = fabsf(dot3(pn, D));
    }
  }
  // warp-aggregated counters
  for (int o = 16; o > 0; o >>= 1) {
    n_seg += __shfl_xor_sync(0xffffffffu, n_seg, o);
    n_hit += __shfl_xor_sync(0xffffffffu, n_hit, o);
    n_esc += __shfl_xor_sync(0xffffffffu, n_esc, o);
    n_emit += __shfl_xor_sync(0xffffffffu, n_emit, o);
    if (kCount) {
      n_nodes += __shfl_xor_sync(0xffffffffu, n_nodes, o);
      n_tris += __shfl_xor_sync(0xffffffffu, n_tris, o);
    }
  }
  if (lane_id() == 0) {
    if (kCount) {
      atomicAdd(&a.ctr->nodes_visited, n_nodes);
      atomicAdd(&a.ctr->tris_tested, n_tris);
    }
    atomicAdd(&a.ctr->segments, n_seg);
    atomicAdd(&a.ctr->hits, n_hit);
    atomicAdd(&a.ctr->escapes, n_esc);
    atomicAdd(&a.ctr->emitted, n_emit);
  }
}

cudaError_t launch_trace(cudaStream_t st, const TraceArgs &a, int n_sm) {
  int64_t n = a.lineage_end - a.lineage_begin;
  if (n <= 0) return cudaSuccess;
  int threads = 128;
  int64_t blocks = (n + threads - 1) / threads;
  int64_t cap = (int64_t)n_sm * 64;
  if (blocks > cap) blocks = cap;
  if (a.count_work) k_trace<true><<<(int)blocks, threads, 0, st>>>(a);
  else k_trace<false><<<(int)blocks, threads, 0, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ scatter
__global__ void __launch_bounds__(256) k_scatter(ScatterArgs a) {
  const MicGrid g = *a.grid;
  const unsigned lane = lane_id();
  const unsigned long long n_seg = min(*a.seg_count, a.seg_capacity);
  const int nb = a.n_bands;
  unsigned long long n_cand = 0, n_contrib = 0;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long si = warp0; si < (long long)n_seg; si += n_warps) {
    const Seg *sp = a.segs + si;
    Seg s;
    s.apex = __ldg(&sp->apex); s.n0 = __ldg(&sp->n0); s.n1 = __ldg(&sp->n1); s.n2 = __ldg(&sp->n2);
    s.start = __ldg(&sp->start); s.end = __ldg(&sp->end); s.p03 = __ldg(&sp->p03); s.p47 = __ldg(&sp->p47);
    Poly p;
    if (!seg_footprint(s, g, p)) continue;
    const int cy0 = __float_as_int(s.apex.w), cy1 = __float_as_int(s.n0.w);
    const float3 A = f3(s.apex), n0 = f3(s.n0), n1 = f3(s.n1), n2 = f3(s.n2);
    const float3 ns = f3(s.start), ne = f3(s.end);
    const float ws = s.start.w, we = s.end.w;
    const float P[kMaxBands] = {s.p03.x, s.p03.y, s.p03.z, s.p03.w, s.p47.x, s.p47.y, s.p47.z, s.p47.w};
    for (int rb = cy0; rb <= cy1; rb += 32) {
      int row = rb + (int)lane;
      int first = 0, cnt = 0;
      if (row <= cy1) {
        float ya = g.y0 + row * g.ch, yb = ya + g.ch;
        float my = 1e-3f * g.ch;
        float xmin, xmax;
        poly_strip_x(p, ya - my, yb + my, xmin, xmax);
        if (xmin <= xmax) {
          int cx0 = clampi((int)floorf((xmin - g.x0) * g.inv_cw), 0, g.nx - 1);
          int cx1 = clampi((int)floorf((xmax - g.x0) * g.inv_cw), 0, g.nx - 1);
          first = __ldg(&a.cell_start[row * g.nx + cx0]);
          cnt = __ldg(&a.cell_start[row * g.nx + cx1 + 1]) - first;
        }
      }
      int incl = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const int excl = incl - cnt;
      for (int base = 0; base < total; base += 32) {
        int i = base + (int)lane;
        int owner = 0;
        for (int step = 16; step >= 1; step >>= 1) {
          int ex = __shfl_sync(0xffffffffu, excl, owner + step);
          if (ex <= i) owner += step;
        }
        int ofirst = __shfl_sync(0xffffffffu, first, owner);
        int oexcl = __shfl_sync(0xffffffffu, excl, owner);
        if (i < total) {
          int mi = ofirst + (i - oexcl);
          float4 m = __ldg(&a.mics[mi]);
          float3 mv = f3(m);
          float3 v = mv - A;
          n_cand++;
          bool in = dot3(n0, v) >= 0.0f && dot3(n1, v) >= 0.0f && dot3(n2, v) >= 0.0f &&
                    dot3(ns, mv) - ws > 0.0f && dot3(ne, mv) - we >= 0.0f;
          float d2 = dot3(v, v);
          if (in && d2 > 1e-18f) {
            float gf = 1.0f / (4.0f * 3.14159265358979f * d2);
            float dist = a.has_alpha ? sqrtf(d2) : 0.0f;
            double *e = a.energy + (size_t)mi * kMaxBands;
#pragma unroll
            for (int b = 0; b < kMaxBands; b++) {
              if (b < nb) {
                float c = P[b] * gf;
                if (a.has_alpha) c *= exp2f(a.alpha_log2[b] * dist);
                atomicAdd(e + b, (double)c);
              }
            }
            atomicAdd(&a.count[mi], 1);
            n_contrib++;
          }
        }
      }
    }
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

cudaError_t launch_scatter(cudaStream_t st, const ScatterArgs &a, int n_sm) {
  k_scatter<<<n_sm * 8, 256, 0, st>>>(a);
  note_launches(1);
  return cudaGetLastError();
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

}  // namespace bt
