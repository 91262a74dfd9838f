// build.cu -- device-side construction of the scene's acceleration structure
// and of the microphone bins.
//
// Scene (the paper's Section 2 relies on "efficient ray shooting" over a
// hierarchical partitioning of the model): a linear BVH in the manner of
// Karras (HPG 2012) -- 30-bit Morton codes of triangle centroids, a stable
// LSD radix sort, one thread per internal node to find its key range and
// split, and a bottom-up pass that fills both child boxes of every node.
//
// Microphones (Section 3 partitions microphones together with the geometry):
// keyed by their xy cell on a uniform grid, radix-sorted, and indexed by a
// cell-start table, so a row of cells is one contiguous run of microphones.
#include <stdio.h>

#include "bt_internal.cuh"

namespace bt {

// ------------------------------------------------------------ small helpers
__device__ __forceinline__ void atomic_min_f(float *a, float v) {
  if (v >= 0.0f) atomicMin((int *)a, __float_as_int(v));
  else atomicMax((unsigned *)a, __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float *a, float v) {
  if (v >= 0.0f) atomicMax((int *)a, __float_as_int(v));
  else atomicMin((unsigned *)a, __float_as_uint(v));
}

__global__ void k_box_init(float *box) {
  if (threadIdx.x < 3) box[threadIdx.x] = kInf;
  else if (threadIdx.x < 6) box[threadIdx.x] = -kInf;
}

__device__ __forceinline__ void warp_box_reduce(float *lo, float *hi, float *box) {
  for (int k = 0; k < 3; k++) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; k++) {
      if (lo[k] <= hi[k]) {
        atomic_min_f(&box[k], lo[k]);
        atomic_max_f(&box[3 + k], hi[k]);
      }
    }
  }
}

// ------------------------------------------------------- triangle validation
// Checks indices, materials and coordinates; accumulates the scene box over
// valid triangles.  A bad triangle sets the error flag and is never read.
__global__ void k_tri_validate(const float *verts, int64_t n_verts, const int32_t *tris,
                               int64_t n_tris, const uint8_t *mat, int n_mat, float *box, int *error) {
  float lo[3] = {kInf, kInf, kInf}, hi[3] = {-kInf, -kInf, -kInf};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tris;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
    bool ok = i0 >= 0 && i0 < n_verts && i1 >= 0 && i1 < n_verts && i2 >= 0 && i2 < n_verts &&
              (int)mat[t] < n_mat;
    if (!ok) { atomicExch(error, BT_E_INVALID); continue; }
    const int32_t idx[3] = {i0, i1, i2};
    for (int v = 0; v < 3; v++) {
      for (int k = 0; k < 3; k++) {
        float c = verts[3 * (int64_t)idx[v] + k];
        if (!isfinite(c)) { atomicExch(error, BT_E_INVALID); c = 0.0f; }
        lo[k] = fminf(lo[k], c);
        hi[k] = fmaxf(hi[k], c);
      }
    }
  }
  warp_box_reduce(lo, hi, box);
}

// Spread the low 10 bits of v to every third bit.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < 10; i++) r |= ((v >> i) & 1u) << (3 * i);
  return r;
}

// Key: 30-bit Morton code of the centroid, plus bit 30 for a triangle whose
// xy extent exceeds 1/16 of the scene's (a ground sheet, a long roof).  The
// flag makes the root split those few triangles into their own subtree, so
// their scene-sized boxes do not enlarge the boxes above ordinary triangles.
// One scale for all axes (the largest extent): a flat city then splits on x
// and y far more often than on z.
__device__ __forceinline__ uint32_t tri_key(float3 a, float3 b, float3 d, const float *box) {
  float c[3] = {(a.x + b.x + d.x) * (1.0f / 3.0f), (a.y + b.y + d.y) * (1.0f / 3.0f),
                (a.z + b.z + d.z) * (1.0f / 3.0f)};
  float dx = fmaxf(fmaxf(a.x, b.x), d.x) - fminf(fminf(a.x, b.x), d.x);
  float dy = fmaxf(fmaxf(a.y, b.y), d.y) - fminf(fminf(a.y, b.y), d.y);
  float scene_xy = fmaxf(box[3] - box[0], box[4] - box[1]);
  bool large = fmaxf(dx, dy) > scene_xy * (1.0f / 16.0f);
  float ext = fmaxf(scene_xy, box[5] - box[2]);
  uint32_t q[3];
  for (int k = 0; k < 3; k++) {
    float u = ext > 0.0f ? (c[k] - box[k]) / ext : 0.5f;
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    q[k] = (uint32_t)fminf(u * 1024.0f, 1023.0f);
  }
  return (large ? (1u << 30) : 0u) | (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
}

__global__ void k_morton(const float *verts, const int32_t *tris, int64_t n_tris, const float *box,
                         uint32_t *keys, uint32_t *vals) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_tris) return;
  float3 v[3];
  for (int k = 0; k < 3; k++) {
    const float *p = verts + 3 * (int64_t)tris[3 * t + k];
    v[k] = make_float3(p[0], p[1], p[2]);
  }
  keys[t] = tri_key(v[0], v[1], v[2], box);
  vals[t] = (uint32_t)t;
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort of (key, value) pairs, 8-bit digits.  A tile of 2048
// items per 256-thread block; each warp ranks 8 rounds of 32 consecutive items
// with __match_any_sync, so ranks follow the input order.
constexpr int RS_THREADS = 256, RS_WARPS = 8, RS_ROUNDS = 8, RS_TILE = 2048;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *keys, int n, int shift,
                                                       uint32_t *hist, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    int g = base + i;
    if (g < n) atomicAdd(&h[(keys[g] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan with one block of 1024 threads (sizes up to ~1e6).
__global__ void __launch_bounds__(1024) k_scan_excl(uint32_t *a, int n) {
  __shared__ uint32_t ws[32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (int base = 0; base < n; base += 1024) {
    int i = base + threadIdx.x;
    uint32_t v = i < n ? a[i] : 0u, x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t s = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    uint32_t incl = x + (warp > 0 ? ws[warp - 1] : 0u);
    if (i < n) a[i] = carry + incl - v;
    uint32_t total = ws[31];
    __syncthreads();
    carry += total;
  }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *kin, const uint32_t *vin,
                                                          uint32_t *kout, uint32_t *vout, int n,
                                                          int shift, const uint32_t *offs, int nblk) {
  __shared__ uint32_t wh[RS_WARPS][256];
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wh[0][0])[i] = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned lt = (1u << lane) - 1u;
  int base = blockIdx.x * RS_TILE + warp * (RS_ROUNDS * 32);
  uint32_t key[RS_ROUNDS], val[RS_ROUNDS], rank[RS_ROUNDS];
  int dig[RS_ROUNDS];
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; r++) {
    int g = base + r * 32 + lane;
    bool valid = g < n;
    key[r] = valid ? kin[g] : 0u;
    val[r] = valid ? vin[g] : 0u;
    int d = valid ? (int)((key[r] >> shift) & 255u) : 256;
    dig[r] = d;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = valid ? wh[warp][d] : 0u;
    __syncwarp();
    rank[r] = before + __popc(peers & lt);
    if (valid && (peers >> lane) == 1u) wh[warp][d] = before + __popc(peers);  // highest lane of the group
    __syncwarp();
  }
  __syncthreads();
  {
    int d = threadIdx.x;  // 256 threads, one digit each
    uint32_t run = 0;
    for (int w = 0; w < RS_WARPS; w++) {
      uint32_t c = wh[w][d];
      wh[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; r++) {
    if (dig[r] < 256) {
      uint32_t pos = offs[dig[r] * nblk + blockIdx.x] + wh[warp][dig[r]] + rank[r];
      kout[pos] = key[r];
      vout[pos] = val[r];
    }
  }
}

static size_t rs_hist_entries(int n) { return (size_t)256 * ((n + RS_TILE - 1) / RS_TILE); }

// Sorts (keys, vals) in place over `bits` low key bits, using alternate
// buffers of the same size and a histogram buffer.
static cudaError_t radix_sort(cudaStream_t st, uint32_t *keys, uint32_t *vals, uint32_t *kalt,
                              uint32_t *valt, uint32_t *hist, int n, int bits) {
  if (n <= 1) return cudaSuccess;
  int nblk = (n + RS_TILE - 1) / RS_TILE;
  int passes = (bits + 7) / 8;
  uint32_t *ka = keys, *va = vals, *kb = kalt, *vb = valt;
  for (int p = 0; p < passes; p++) {
    int shift = 8 * p;
    k_rs_hist<<<nblk, RS_THREADS, 0, st>>>(ka, n, shift, hist, nblk);
    k_scan_excl<<<1, 1024, 0, st>>>(hist, 256 * nblk);
    k_rs_scatter<<<nblk, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, hist, nblk);
    note_launches(3);
    uint32_t *t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------- LBVH
__device__ __forceinline__ int lcp(const uint32_t *keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint32_t a = keys[i], b = keys[j];
  if (a == b) return 32 + __clz((unsigned)(i ^ j));
  return __clz(a ^ b);
}
__device__ __forceinline__ int lcp(const unsigned long long *keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  unsigned long long a = keys[i], b = keys[j];
  if (a == b) return 64 + __clz((unsigned)(i ^ j));
  return __clzll(a ^ b);
}

// One thread per internal node: direction, range end and split (Karras 2012).
// child.w keeps the far end j of the node's key range [min(i,j), max(i,j)].
template <typename K>
__global__ void k_lbvh_topology(const K *keys, int n, Node *nodes, int *leaf_parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (lcp(keys, n, i, i + 1) - lcp(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = lcp(keys, n, i, i - d);
  int lmax = 2;
  while (lcp(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (lcp(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = lcp(keys, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (lcp(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int gamma = i + s * d + (d < 0 ? -1 : 0);
  int lo = i < j ? i : j, hi = i < j ? j : i;
  int left = (lo == gamma) ? ~gamma : gamma;
  int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  nodes[i].child.x = left;
  nodes[i].child.y = right;
  nodes[i].child.w = j;
  if (left < 0) leaf_parent[gamma] = i; else nodes[left].child.z = i;
  if (right < 0) leaf_parent[gamma + 1] = i; else nodes[right].child.z = i;
  if (i == 0) nodes[0].child.z = -1;
}

// Triangles in leaf order with their planes; the normal is formed in double.
__global__ void k_pack_tris(const float *verts, const int32_t *tris, const uint8_t *mat,
                            const uint32_t *order, int64_t n, Tri *out, Plane *planes, Plane64 *planes64,
                            PlaneDF *planes_df) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int64_t t = order[s];
  float3 v[3];
  for (int k = 0; k < 3; k++) {
    const float *p = verts + 3 * (int64_t)tris[3 * t + k];
    v[k] = make_float3(p[0], p[1], p[2]);
  }
  out[s].v0 = make_float4(v[0].x, v[0].y, v[0].z, __int_as_float((int)mat[t]));
  out[s].v1 = make_float4(v[1].x, v[1].y, v[1].z, __int_as_float((int)t));
  out[s].v2 = make_float4(v[2].x, v[2].y, v[2].z, 0.0f);
  double e1x = (double)v[1].x - v[0].x, e1y = (double)v[1].y - v[0].y, e1z = (double)v[1].z - v[0].z;
  double e2x = (double)v[2].x - v[0].x, e2y = (double)v[2].y - v[0].y, e2z = (double)v[2].z - v[0].z;
  double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  double l = sqrt(nx * nx + ny * ny + nz * nz);
  if (l > 0.0) { nx /= l; ny /= l; nz /= l; } else { nx = ny = nz = 0.0; }
  double w = nx * v[0].x + ny * v[0].y + nz * v[0].z;
  planes[s] = make_float4((float)nx, (float)ny, (float)nz, (float)w);
  planes64[s].x = nx;
  planes64[s].y = ny;
  planes64[s].z = nz;
  planes64[s].w = w;
  float hx = (float)nx, hy = (float)ny, hz = (float)nz, hw = (float)w;
  planes_df[s].hi = make_float4(hx, hy, hz, hw);
  planes_df[s].lo = make_float4((float)(nx - hx), (float)(ny - hy), (float)(nz - hz), (float)(w - hw));
}

__device__ __forceinline__ void tri_box(const Tri &t, float lo[3], float hi[3]) {
  lo[0] = fminf(fminf(t.v0.x, t.v1.x), t.v2.x); hi[0] = fmaxf(fmaxf(t.v0.x, t.v1.x), t.v2.x);
  lo[1] = fminf(fminf(t.v0.y, t.v1.y), t.v2.y); hi[1] = fmaxf(fmaxf(t.v0.y, t.v1.y), t.v2.y);
  lo[2] = fminf(fminf(t.v0.z, t.v1.z), t.v2.z); hi[2] = fmaxf(fmaxf(t.v0.z, t.v1.z), t.v2.z);
}

__device__ __forceinline__ void child_box(int c, const Tri *tris, const float *aux, float lo[3], float hi[3]) {
  if (c < 0) {
    Tri t = tris[~c];
    tri_box(t, lo, hi);
  } else {
    for (int k = 0; k < 3; k++) {
      lo[k] = __ldcg(&aux[6 * c + k]);
      hi[k] = __ldcg(&aux[6 * c + 3 + k]);
    }
  }
}

// Bottom-up boxes: the second thread to reach a node fills it and goes on.
__global__ void k_lbvh_boxes(const Tri *tris, int n, Node *nodes, const int *leaf_parent, float *aux,
                             unsigned *flags, int *error) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p = leaf_parent[i];
  // the climb is at most the tree depth; the bound only guarantees termination
  for (int steps = 0; p >= 0; steps++) {
    if (steps > 128 || p >= n - 1) { atomicExch(error, BT_E_CUDA); return; }
    __threadfence();
    unsigned arrived = atomicAdd(&flags[p], 1u);
    if (arrived == 0u) return;
    if (arrived > 1u) { atomicExch(error, BT_E_CUDA); return; }
    __threadfence();
    int l = __ldcg(&nodes[p].child.x), r = __ldcg(&nodes[p].child.y);
    float llo[3], lhi[3], rlo[3], rhi[3];
    child_box(l, tris, aux, llo, lhi);
    child_box(r, tris, aux, rlo, rhi);
    // child boxes grown by 1e-6 relative + 0.1 mm: a float32 ray rounded from
    // a float64 one must not miss a box the float64 ray enters
    float glo[3], ghi[3], hlo[3], hhi[3];
    for (int k = 0; k < 3; k++) {
      glo[k] = llo[k] - (fabsf(llo[k]) * 1e-6f + 1e-4f);
      ghi[k] = lhi[k] + (fabsf(lhi[k]) * 1e-6f + 1e-4f);
      hlo[k] = rlo[k] - (fabsf(rlo[k]) * 1e-6f + 1e-4f);
      hhi[k] = rhi[k] + (fabsf(rhi[k]) * 1e-6f + 1e-4f);
    }
    nodes[p].lxy = make_float4(glo[0], ghi[0], glo[1], ghi[1]);
    nodes[p].rxy = make_float4(hlo[0], hhi[0], hlo[1], hhi[1]);
    nodes[p].lrz = make_float4(glo[2], ghi[2], hlo[2], hhi[2]);
    for (int k = 0; k < 3; k++) {
      aux[6 * p + k] = fminf(llo[k], rlo[k]);
      aux[6 * p + 3 + k] = fmaxf(lhi[k], rhi[k]);
    }
    p = __ldcg(&nodes[p].child.z);
  }
}

// Leaf size of the traversal: one thread per internal node rewrites its two
// child links.  A link first goes back to the node the LBVH built (a left
// child covers the key range ending at its own index, a right child the range
// starting at it, so a collapsed leaf (first, count) names its node); then a
// child node whose range holds at most leaf_size leaves becomes one leaf of
// those leaves, which are consecutive slots.  Ranges (child.w) are never
// written, so the threads do not race.
__global__ void k_collapse_leaves(Node *nodes, int n_internal, int leaf_size) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_internal) return;
  int2 ch = make_int2(nodes[p].child.x, nodes[p].child.y);
  int out[2];
  for (int side = 0; side < 2; side++) {
    int c = side == 0 ? ch.x : ch.y;
    if (c < 0 && leaf_count(~c) > 1) {
      const int v = ~c;
      c = side == 0 ? leaf_slot(v) + leaf_count(v) - 1 : leaf_slot(v);
    }
    if (c >= 0) {
      const int j = nodes[c].child.w;
      const int lo = c < j ? c : j, cnt = (c < j ? j - c : c - j) + 1;
      if (cnt <= leaf_size) c = ~(lo | ((cnt - 1) << kLeafShift));
    }
    out[side] = c;
  }
  nodes[p].child.x = out[0];
  nodes[p].child.y = out[1];
}

// The 4-wide form the traversal reads, one thread per binary node: wide node
// p lists binary node p's grandchildren -- a child that is a leaf stands for
// itself -- with the boxes the binary nodes hold for them (already grown, see
// k_lbvh_boxes), so a search from any binary node tests the same boxes as a
// binary search would, two levels per node fetch.  Child order: left
// subtree first.
__global__ void k_widen(const Node *nodes, int n_internal, Node4 *wide) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_internal) return;
  const Node b = nodes[p];
  float bx[4][6];  // lo.x, hi.x, lo.y, hi.y, lo.z, hi.z per child
  int code[4];
  int m = 0;
  auto put = [&](float4 xy, float z0, float z1, int c) {
    bx[m][0] = xy.x; bx[m][1] = xy.y; bx[m][2] = xy.z; bx[m][3] = xy.w; bx[m][4] = z0; bx[m][5] = z1;
    code[m++] = c;
  };
#pragma unroll
  for (int side = 0; side < 2; side++) {
    const int c = side == 0 ? b.child.x : b.child.y;
    if (c < 0) {
      if (side == 0) put(b.lxy, b.lrz.x, b.lrz.y, c);
      else put(b.rxy, b.lrz.z, b.lrz.w, c);
    } else {
      const Node g = nodes[c];
      put(g.lxy, g.lrz.x, g.lrz.y, g.child.x);
      put(g.rxy, g.lrz.z, g.lrz.w, g.child.y);
    }
  }
  for (int q = m; q < 4; q++) {
    for (int k = 0; k < 6; k++) bx[q][k] = 0.0f;
    code[q] = kNoChild;
  }
  Node4 w;
  w.lox = make_float4(bx[0][0], bx[1][0], bx[2][0], bx[3][0]);
  w.hix = make_float4(bx[0][1], bx[1][1], bx[2][1], bx[3][1]);
  w.loy = make_float4(bx[0][2], bx[1][2], bx[2][2], bx[3][2]);
  w.hiy = make_float4(bx[0][3], bx[1][3], bx[2][3], bx[3][3]);
  w.loz = make_float4(bx[0][4], bx[1][4], bx[2][4], bx[3][4]);
  w.hiz = make_float4(bx[0][5], bx[1][5], bx[2][5], bx[3][5]);
  w.child = make_int4(code[0], code[1], code[2], code[3]);
  w.unused = make_int4(0, 0, 0, 0);
  wide[p] = w;
}

cudaError_t widen(cudaStream_t st, void *hier, int64_t n_leaves) {
  if (n_leaves < 2) return cudaSuccess;
  const int n = (int)(n_leaves - 1);
  k_widen<<<(n + 255) / 256, 256, 0, st>>>((const Node *)hier, n, hier_wide(hier, n_leaves));
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t collapse_leaves(cudaStream_t st, void *hier, int64_t n_leaves, int leaf_size) {
  if (n_leaves < 2) return cudaSuccess;
  const int n = (int)(n_leaves - 1);
  k_collapse_leaves<<<(n + 255) / 256, 256, 0, st>>>((Node *)hier, n, leaf_size);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return widen(st, hier, n_leaves);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t build_scene_scratch_bytes(int64_t n) {
  size_t m = (size_t)(n > 0 ? n : 1);
  return 4 * align256(4 * m) + align256(4 * rs_hist_entries((int)m)) + align256(4 * m) +
         align256(24 * m) + align256(4 * m);
}

cudaError_t validate_scene(cudaStream_t st, const float *d_verts, int64_t n_verts,
                           const int32_t *d_tris, int64_t n_tris, const uint8_t *d_mat, int n_mat,
                           float *d_box, int *d_error) {
  k_box_init<<<1, 32, 0, st>>>(d_box);
  note_launches(1);
  if (n_tris == 0) return cudaGetLastError();
  int threads = 256;
  int64_t blocks = (n_tris + threads - 1) / threads;
  k_tri_validate<<<(int)(blocks < 4096 ? blocks : 4096), threads, 0, st>>>(d_verts, n_verts, d_tris,
                                                                          n_tris, d_mat, n_mat, d_box,
                                                                          d_error);
  note_launches(1);
  return cudaGetLastError();
}

// Scene build, run only after validate_scene() reported no error: every
// index and material is then in range and every coordinate finite.
cudaError_t build_scene(cudaStream_t st, const float *d_verts, const int32_t *d_tris, int64_t n_tris,
                        const uint8_t *d_mat, void *d_hier, Tri *d_tris_out, Plane *d_planes,
                        Plane64 *d_planes64, PlaneDF *d_planes_df, void *d_scratch, size_t scratch_bytes,
                        const float *d_box, int *d_error) {
  if (n_tris == 0) return cudaSuccess;
  Node *const d_nodes = (Node *)d_hier;
  if (scratch_bytes < build_scene_scratch_bytes(n_tris)) return cudaErrorInvalidValue;
  int n = (int)n_tris;
  char *s = (char *)d_scratch;
  size_t m = (size_t)n;
  uint32_t *keys = (uint32_t *)s; s += align256(4 * m);
  uint32_t *vals = (uint32_t *)s; s += align256(4 * m);
  uint32_t *kalt = (uint32_t *)s; s += align256(4 * m);
  uint32_t *valt = (uint32_t *)s; s += align256(4 * m);
  uint32_t *hist = (uint32_t *)s; s += align256(4 * rs_hist_entries(n));
  int *leaf_parent = (int *)s; s += align256(4 * m);
  float *aux = (float *)s; s += align256(24 * m);
  unsigned *flags = (unsigned *)s; s += align256(4 * m);
  int threads = 256;
  int blocks = (n + threads - 1) / threads;
  k_morton<<<blocks, threads, 0, st>>>(d_verts, d_tris, n_tris, d_box, keys, vals);
  note_launches(1);
  cudaError_t e = radix_sort(st, keys, vals, kalt, valt, hist, n, 31);
  if (e != cudaSuccess) return e;
  k_pack_tris<<<blocks, threads, 0, st>>>(d_verts, d_tris, d_mat, vals, n_tris, d_tris_out, d_planes,
                                         d_planes64, d_planes_df);
  note_launches(1);
  if (n >= 2) {
    k_lbvh_topology<uint32_t><<<(n - 1 + threads - 1) / threads, threads, 0, st>>>(keys, n, d_nodes, leaf_parent);
    cudaMemsetAsync(flags, 0, sizeof(unsigned) * m, st);
    k_lbvh_boxes<<<blocks, threads, 0, st>>>(d_tris_out, n, d_nodes, leaf_parent, aux, flags, d_error);
    note_launches(2);
    cudaError_t e2 = widen(st, d_hier, n_tris);
    if (e2 != cudaSuccess) return e2;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ sub-domains
// Tiled hierarchy (Section 3: geometry split into sub-domains).  Every
// (tile, triangle) pair whose xy boxes touch becomes a leaf; the leaves are
// sorted by (tile, large flag, Morton code), so the leaves of one tile are
// contiguous and form one subtree of the LBVH, whose root k_tile_roots finds.
// Input: the scene's packed triangles (leaf order of the 1x1 hierarchy).
// A triangle is listed in every tile its xy box, grown by 5 cm, overlaps; the
// trace accepts a hit in a tile up to 1 cm past the tile's exit along the ray,
// so every triangle such a hit could lie on is in the tile's list.
__device__ __forceinline__ void tile_span(float lo, float hi, float g0, float w, int n, int &a, int &b) {
  const float mg = 5e-2f;
  a = clampi((int)floorf((lo - mg - g0) / w), 0, n - 1);
  b = clampi((int)floorf((hi + mg - g0) / w), 0, n - 1);
}

__global__ void k_tile_count(const Tri *src, int n, TileGrid tg, uint32_t *counts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) { counts[n] = 0; return; }
  Tri t = src[i];
  int x0, x1, y0, y1;
  tile_span(fminf(fminf(t.v0.x, t.v1.x), t.v2.x), fmaxf(fmaxf(t.v0.x, t.v1.x), t.v2.x), tg.gx0, tg.wx, tg.tx, x0, x1);
  tile_span(fminf(fminf(t.v0.y, t.v1.y), t.v2.y), fmaxf(fmaxf(t.v0.y, t.v1.y), t.v2.y), tg.gy0, tg.wy, tg.ty, y0, y1);
  counts[i] = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
}

__global__ void k_tile_emit(const Tri *src, int n, TileGrid tg, const float *box, const uint32_t *offs,
                            uint32_t *pk, uint32_t *pt, uint32_t *psrc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Tri t = src[i];
  int x0, x1, y0, y1;
  tile_span(fminf(fminf(t.v0.x, t.v1.x), t.v2.x), fmaxf(fmaxf(t.v0.x, t.v1.x), t.v2.x), tg.gx0, tg.wx, tg.tx, x0, x1);
  tile_span(fminf(fminf(t.v0.y, t.v1.y), t.v2.y), fmaxf(fmaxf(t.v0.y, t.v1.y), t.v2.y), tg.gy0, tg.wy, tg.ty, y0, y1);
  uint32_t key = tri_key(f3(t.v0), f3(t.v1), f3(t.v2), box);
  uint32_t p = offs[i];
  for (int y = y0; y <= y1; y++)
    for (int x = x0; x <= x1; x++, p++) {
      pk[p] = key;
      pt[p] = (uint32_t)(y * tg.tx + x);
      psrc[p] = (uint32_t)i;
    }
}

__global__ void k_iota(uint32_t *v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

__global__ void k_gather_u32(const uint32_t *in, const uint32_t *idx, uint32_t *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[idx[i]];
}

__global__ void k_tile_keys(const uint32_t *pk, const uint32_t *pt, const uint32_t *psrc, const uint32_t *perm,
                            int n, unsigned long long *key64, uint32_t *order_src) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t p = perm[i];
  key64[i] = ((unsigned long long)pt[p] << 31) | pk[p];
  order_src[i] = psrc[p];
}

__global__ void k_pack_from_src(const Tri *src, const Plane *sp, const Plane64 *sp64, const PlaneDF *spdf,
                                const uint32_t *order_src, int n, Tri *out, Plane *planes, Plane64 *planes64,
                                PlaneDF *planes_df) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t s = order_src[i];
  out[i] = src[s];
  planes[i] = sp[s];
  planes64[i] = sp64[s];
  planes_df[i] = spdf[s];
}

__global__ void k_fill_i32(int *v, int n, int value) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = value;
}

// Root of each tile's subtree: the internal node whose key range is exactly
// the tile's run of leaves, or ~leaf for a tile with one leaf.
__global__ void k_tile_roots(const unsigned long long *key64, const Node *nodes, int n, int *roots) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto tile = [&](int k) { return (int)(key64[k] >> 31); };
  int lo, hi;
  if (i < n - 1) {
    int j = nodes[i].child.w;
    lo = i < j ? i : j;
    hi = i < j ? j : i;
    int tl = tile(lo);
    if (tile(hi) == tl && (lo == 0 || tile(lo - 1) != tl) && (hi == n - 1 || tile(hi + 1) != tl)) roots[tl] = i;
  }
  // single-leaf tiles
  int ti = tile(i);
  if ((i == 0 || tile(i - 1) != ti) && (i == n - 1 || tile(i + 1) != ti)) roots[ti] = ~i;
}

size_t build_tiled_scratch_bytes(int64_t n_src, int64_t n_pairs) {
  size_t a = (size_t)(n_src + 1), p = (size_t)(n_pairs > 0 ? n_pairs : 1);
  return align256(4 * a) + 7 * align256(4 * p) + align256(4 * rs_hist_entries((int)p)) + align256(8 * p) +
         align256(4 * p) + align256(24 * p) + align256(4 * p);
}

// Phase 1: pairs per source triangle and their exclusive offsets; offs[n_src]
// is the number of pairs.  `offs` is n_src + 1 entries of scratch.
cudaError_t tiled_count(cudaStream_t st, const Tri *src, int64_t n_src, const TileGrid &tg, uint32_t *offs) {
  int n = (int)n_src;
  k_tile_count<<<(n + 1 + 255) / 256, 256, 0, st>>>(src, n, tg, offs);
  k_scan_excl<<<1, 1024, 0, st>>>(offs, n + 1);
  note_launches(2);
  return cudaGetLastError();
}

// Phase 2, once the host knows n_pairs: sort the pairs, build the LBVH over
// them, pack the leaves and find the tile roots.
cudaError_t tiled_build(cudaStream_t st, const Tri *src, const Plane *sp, const Plane64 *sp64, const PlaneDF *spdf,
                        int64_t n_src, const TileGrid &tg, const float *d_box, const uint32_t *offs, int64_t n_pairs,
                        void *scratch, size_t scratch_bytes, void *hier, Tri *tris, Plane *planes,
                        Plane64 *planes64, PlaneDF *planes_df, int *roots, int *d_error) {
  if (scratch_bytes < build_tiled_scratch_bytes(n_src, n_pairs)) return cudaErrorInvalidValue;
  Node *const nodes = (Node *)hier;
  int n = (int)n_src, P = (int)n_pairs, T = tg.tx * tg.ty;
  char *s = (char *)scratch + align256(4 * (size_t)(n_src + 1));
  size_t p4 = align256(4 * (size_t)P);
  uint32_t *pk = (uint32_t *)s; s += p4;
  uint32_t *pt = (uint32_t *)s; s += p4;
  uint32_t *psrc = (uint32_t *)s; s += p4;
  uint32_t *ka = (uint32_t *)s; s += p4;
  uint32_t *va = (uint32_t *)s; s += p4;
  uint32_t *kb = (uint32_t *)s; s += p4;
  uint32_t *vb = (uint32_t *)s; s += p4;
  uint32_t *hist = (uint32_t *)s; s += align256(4 * rs_hist_entries(P));
  unsigned long long *key64 = (unsigned long long *)s; s += align256(8 * (size_t)P);
  int *leaf_parent = (int *)s; s += p4;
  float *aux = (float *)s; s += align256(24 * (size_t)P);
  unsigned *flags = (unsigned *)s;
  const int th = 256, bp = (P + th - 1) / th;
  k_fill_i32<<<(T + th - 1) / th, th, 0, st>>>(roots, T, (int)0x80000000);
  k_tile_emit<<<(n + th - 1) / th, th, 0, st>>>(src, n, tg, d_box, offs, pk, pt, psrc);
  // sort by (large flag, Morton) and then, stably, by tile
  cudaMemcpyAsync(ka, pk, sizeof(uint32_t) * P, cudaMemcpyDeviceToDevice, st);
  k_iota<<<bp, th, 0, st>>>(va, P);
  note_launches(3);
  cudaError_t e = radix_sort(st, ka, va, kb, vb, hist, P, 31);
  if (e != cudaSuccess) return e;
  k_gather_u32<<<bp, th, 0, st>>>(pt, va, ka, P);
  note_launches(1);
  int tbits = 1;
  while ((1 << tbits) < T) tbits++;
  e = radix_sort(st, ka, va, kb, vb, hist, P, tbits);
  if (e != cudaSuccess) return e;
  k_tile_keys<<<bp, th, 0, st>>>(pk, pt, psrc, va, P, key64, kb);
  k_pack_from_src<<<bp, th, 0, st>>>(src, sp, sp64, spdf, kb, P, tris, planes, planes64, planes_df);
  note_launches(2);
  if (P >= 2) {
    k_lbvh_topology<unsigned long long><<<(P - 1 + th - 1) / th, th, 0, st>>>(key64, P, nodes, leaf_parent);
    cudaMemsetAsync(flags, 0, sizeof(unsigned) * P, st);
    k_lbvh_boxes<<<bp, th, 0, st>>>(tris, P, nodes, leaf_parent, aux, flags, d_error);
    note_launches(2);
  }
  k_tile_roots<<<bp, th, 0, st>>>(key64, nodes, P, roots);
  note_launches(1);
  (void)n;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return widen(st, hier, P);
}

// ------------------------------------------------------------ microphones
__global__ void k_mic_validate(const float *pos, int64_t n, float *box, int *error) {
  float lo[3] = {kInf, kInf, kInf}, hi[3] = {-kInf, -kInf, -kInf};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; k++) {
      float c = pos[3 * i + k];
      if (!isfinite(c)) { atomicExch(error, BT_E_INVALID); continue; }
      lo[k] = fminf(lo[k], c);
      hi[k] = fmaxf(hi[k], c);
    }
  }
  warp_box_reduce(lo, hi, box);
}

__global__ void k_mic_grid(const float *box, int nx, int ny, int nz, int64_t n, MicGrid *g) {
  MicGrid r;
  float ex = box[3] - box[0], ey = box[4] - box[1], ez = box[5] - box[2];
  r.x0 = box[0];
  r.y0 = box[1];
  r.cw = fmaxf(ex / nx * 1.000001f, 1e-3f);
  r.ch = fmaxf(ey / ny * 1.000001f, 1e-3f);
  r.inv_cw = 1.0f / r.cw;
  r.inv_ch = 1.0f / r.ch;
  r.zlo = box[2];
  r.zhi = box[5];
  r.nx = nx;
  r.ny = ny;
  r.n_mics = (int)n;
  r.nz = nz;
  r.z0 = box[2];
  r.dz = fmaxf(ez / nz * 1.000001f, 1e-3f);
  r.inv_dz = 1.0f / r.dz;
  r.pad = 0.0f;
  *g = r;
}

__global__ void k_mic_keys(const float *pos, int64_t n, const MicGrid *g, uint32_t *keys, uint32_t *vals) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  MicGrid gr = *g;
  int cx = clampi((int)floorf((pos[3 * i] - gr.x0) * gr.inv_cw), 0, gr.nx - 1);
  int cy = clampi((int)floorf((pos[3 * i + 1] - gr.y0) * gr.inv_ch), 0, gr.ny - 1);
  int cz = gr.nz > 1 ? clampi((int)floorf((pos[3 * i + 2] - gr.z0) * gr.inv_dz), 0, gr.nz - 1) : 0;
  keys[i] = (uint32_t)((cz * gr.ny + cy) * gr.nx + cx);
  vals[i] = (uint32_t)i;
}

__global__ void k_mic_gather(const float *pos, int64_t n, const uint32_t *keys, const uint32_t *vals,
                             int n_cells, float4 *sorted, int *cell_start) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v = vals[i];
  sorted[i] = make_float4(pos[3 * (int64_t)v], pos[3 * (int64_t)v + 1], pos[3 * (int64_t)v + 2],
                          __int_as_float((int)v));
  int k = (int)keys[i];
  int kp = i > 0 ? (int)keys[i - 1] : -1;
  for (int c = kp + 1; c <= k; c++) cell_start[c] = (int)i;
  if (i == n - 1)
    for (int c = k + 1; c <= n_cells; c++) cell_start[c] = (int)n;
}

size_t build_mics_scratch_bytes(int64_t n_m) {
  size_t m = (size_t)(n_m > 0 ? n_m : 1);
  return 4 * align256(4 * m) + align256(4 * rs_hist_entries((int)m));
}

// The microphones' box (and a non-finite check); the host reads the box to
// choose the grid before build_mics.
cudaError_t mic_box(cudaStream_t st, const float *d_pos, int64_t n_m, float *d_box, int *d_error) {
  k_box_init<<<1, 32, 0, st>>>(d_box);
  int threads = 256;
  int64_t blocks = (n_m + threads - 1) / threads;
  if (blocks < 1) blocks = 1;
  k_mic_validate<<<(int)(blocks < 4096 ? blocks : 4096), threads, 0, st>>>(d_pos, n_m, d_box, d_error);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t build_mics(cudaStream_t st, const float *d_pos, int64_t n_m, int nx, int ny, int nz,
                       const float *d_box, MicGrid *d_grid, float4 *d_sorted, int *d_cell_start, void *d_scratch,
                       size_t scratch_bytes) {
  if (scratch_bytes < build_mics_scratch_bytes(n_m)) return cudaErrorInvalidValue;
  int n = (int)n_m;
  size_t m = (size_t)(n > 0 ? n : 1);
  char *s = (char *)d_scratch;
  uint32_t *keys = (uint32_t *)s; s += align256(4 * m);
  uint32_t *vals = (uint32_t *)s; s += align256(4 * m);
  uint32_t *kalt = (uint32_t *)s; s += align256(4 * m);
  uint32_t *valt = (uint32_t *)s; s += align256(4 * m);
  uint32_t *hist = (uint32_t *)s;
  k_mic_grid<<<1, 1, 0, st>>>(d_box, nx, ny, nz, n_m, d_grid);
  note_launches(1);
  const int n_cells = nx * ny * nz;
  if (n == 0) {
    cudaMemsetAsync(d_cell_start, 0, sizeof(int) * (n_cells + 1), st);
    return cudaGetLastError();
  }
  int threads = 256;
  int blocks = (n + threads - 1) / threads;
  k_mic_keys<<<blocks, threads, 0, st>>>(d_pos, n_m, d_grid, keys, vals);
  note_launches(1);
  int bits = 1;
  while ((1 << bits) < n_cells) bits++;
  cudaError_t e = radix_sort(st, keys, vals, kalt, valt, hist, n, bits);
  if (e != cudaSuccess) return e;
  k_mic_gather<<<blocks, threads, 0, st>>>(d_pos, n_m, keys, vals, n_cells, d_sorted, d_cell_start);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bt
