/*
 * btrace_oracle.c -- plain FP64 CPU oracle of the hybrid beam/ray tracer of
 * "Beam-tracing domain decomposition method for urban acoustic pollution"
 * (Gbikpi-Benissan & Magoules, arXiv:1912.03998).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this file.  It shares no code, header, table or
 * constant with the CUDA library; the two meet only at the seeded inputs.
 *
 * The paper gives the method in prose only (Section 2) and no formulas, so the
 * steps below follow that prose with these readings:
 *   - beams: the faces of a geodesic icosahedron subdivided L times, one
 *     triangular cone per face, power split by solid angle (Section 2: the
 *     source energy is split between beams by its power per direction); a
 *     directional source scales each beam's power by its pattern's gain for
 *     that beam (or_trace_dir);
 *   - only the guiding (axis) ray of a beam is intersected with the model and
 *     a beam is never split (Section 2, last paragraph);
 *   - a reflection creates an image source, the mirror of the apex in the hit
 *     plane, and the reflected beam is the mirrored cone (Section 2, image
 *     sources); energy is lost at each reflection by the material coefficient
 *     and optionally by air damping (Section 2, particle tracing);
 *   - a microphone inside a beam segment receives the beam's intensity, which
 *     equals the image-source intensity W*prod(r)/(4*pi*d^2) at distance d
 *     from the (virtual) apex;
 *   - sub-domains (Section 3, geometry and microphone partitioning): in tiled
 *     mode each tile searches only its own triangles and accepts a hit only if
 *     the hit point lies in the tile; a ray that leaves a tile without an
 *     accepted hit is handed to the next tile along the ray.
 *
 * Every floating-point step runs in double precision.  Pinned by the tests in
 * tests/test_oracle_*.py against closed forms (free field, ground plane, one
 * wall), a brute-force image-source enumeration (isrc_bruteforce.c), and
 * invariants (solid angles sum to 4*pi; tile split does not change the result).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_BANDS 8
#define OR_PI 3.14159265358979323846

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / len(a)); }
/* mirror of a direction in a plane with unit normal n */
static v3 mirror_dir(v3 d, v3 n) { return sub(d, scl(n, 2.0 * dot(d, n))); }
/* mirror of a point in the plane through p with unit normal n */
static v3 mirror_pt(v3 a, v3 p, v3 n) { return sub(a, scl(n, 2.0 * dot(sub(a, p), n))); }

/* ------------------------------------------------------------------ beams --
 * Geodesic icosahedron.  The 12 base vertices are the cyclic permutations of
 * (0, +-1, +-phi).  The 20 faces are the vertex triples whose three pairwise
 * distances equal the edge length 2, oriented counter-clockwise seen from
 * outside, listed in lexicographic order of (i<j<k).  Each face splits into
 * four at every level: (a,ab,ca), (ab,b,bc), (ca,bc,c), (ab,bc,ca), where ab is
 * the midpoint of a and b pushed back onto the unit sphere.
 */
static int icosa_base(v3 vert[12], int face[20][3]) {
  double phi = 0.5 * (1.0 + sqrt(5.0));
  int n = 0;
  for (int s1 = -1; s1 <= 1; s1 += 2)
    for (int s2 = -1; s2 <= 1; s2 += 2) {
      vert[n++] = mk(0.0, s1 * 1.0, s2 * phi);
      vert[n++] = mk(s1 * 1.0, s2 * phi, 0.0);
      vert[n++] = mk(s2 * phi, 0.0, s1 * 1.0);
    }
  int nf = 0;
  for (int i = 0; i < 12; i++)
    for (int j = i + 1; j < 12; j++)
      for (int k = j + 1; k < 12; k++) {
        double dij = dot(sub(vert[i], vert[j]), sub(vert[i], vert[j]));
        double djk = dot(sub(vert[j], vert[k]), sub(vert[j], vert[k]));
        double dki = dot(sub(vert[k], vert[i]), sub(vert[k], vert[i]));
        if (fabs(dij - 4.0) > 1e-9 || fabs(djk - 4.0) > 1e-9 || fabs(dki - 4.0) > 1e-9) continue;
        if (nf >= 20) return -1;
        double orient = dot(cross(sub(vert[j], vert[i]), sub(vert[k], vert[i])), vert[i]);
        face[nf][0] = i;
        face[nf][1] = orient > 0 ? j : k;
        face[nf][2] = orient > 0 ? k : j;
        nf++;
      }
  for (int i = 0; i < 12; i++) vert[i] = unit(vert[i]);
  return nf;
}

static void subdivide(v3 a, v3 b, v3 c, int level, v3 *out, int64_t *n) {
  if (level == 0) {
    out[3 * *n + 0] = a;
    out[3 * *n + 1] = b;
    out[3 * *n + 2] = c;
    (*n)++;
    return;
  }
  v3 ab = unit(add(a, b)), bc = unit(add(b, c)), ca = unit(add(c, a));
  subdivide(a, ab, ca, level - 1, out, n);
  subdivide(ab, b, bc, level - 1, out, n);
  subdivide(ca, bc, c, level - 1, out, n);
  subdivide(ab, bc, ca, level - 1, out, n);
}

/* Solid angle of the spherical triangle (a,b,c) of unit vectors,
 * Van Oosterom & Strackee (1983): tan(omega/2) = |a.(b x c)| / (1 + a.b + b.c + c.a). */
static double solid_angle(v3 a, v3 b, v3 c) {
  double num = fabs(dot(a, cross(b, c)));
  double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
  return 2.0 * atan2(num, den);
}

int64_t or_n_beams(int level) { return (int64_t)20 << (2 * level); }

/* Beam table: dirs[N][3][3] (three unit edge directions, CCW from outside),
 * omega[N] (solid angles).  Returns N, or -1 on a bad level. */
int64_t or_beam_table(int level, double *dirs, double *omega) {
  if (level < 0 || level > 10) return -1;
  v3 vert[12];
  int face[20][3];
  if (icosa_base(vert, face) != 20) return -1;
  int64_t n_b = or_n_beams(level), n = 0;
  v3 *tmp = (v3 *)malloc(sizeof(v3) * 3 * (size_t)n_b);
  if (!tmp) return -1;
  for (int f = 0; f < 20; f++)
    subdivide(vert[face[f][0]], vert[face[f][1]], vert[face[f][2]], level, tmp, &n);
  for (int64_t i = 0; i < n_b; i++) {
    for (int j = 0; j < 3; j++) {
      dirs[9 * i + 3 * j + 0] = tmp[3 * i + j].x;
      dirs[9 * i + 3 * j + 1] = tmp[3 * i + j].y;
      dirs[9 * i + 3 * j + 2] = tmp[3 * i + j].z;
    }
    if (omega) omega[i] = solid_angle(tmp[3 * i], tmp[3 * i + 1], tmp[3 * i + 2]);
  }
  free(tmp);
  return n_b;
}

/* ------------------------------------------------------------------ scene -- */
typedef struct {
  double lo[3], hi[3];
  int left, right; /* children, -1 for a leaf */
  int first, count; /* leaf range in the index array */
} bnode;

typedef struct {
  int n_nodes;
  bnode *nodes;
  int *idx; /* triangle ids in leaf order */
} bvh;

typedef struct {
  int64_t n_tris;
  v3 *a, *b, *c;    /* vertices of each triangle */
  v3 *n;            /* unit normal (b-a)x(c-a), normalised */
  int *mat;
  int n_mat, n_bands;
  double *refl; /* [n_mat][n_bands] */
  double lo[3], hi[3];
  bvh all;
  int tx, ty;             /* tile grid over the scene's xy box (tiled mode) */
  double gx0, gx1, gy0, gy1; /* tile grid box: scene xy box grown by 1 m */
  bvh *tile;              /* one bvh per tile */
} oscene;

static void tri_box(const oscene *s, int t, double lo[3], double hi[3]) {
  v3 p[3] = {s->a[t], s->b[t], s->c[t]};
  for (int k = 0; k < 3; k++) {
    double *l = lo, *h = hi;
    double v0 = k == 0 ? p[0].x : k == 1 ? p[0].y : p[0].z;
    l[k] = h[k] = v0;
    for (int q = 1; q < 3; q++) {
      double v = k == 0 ? p[q].x : k == 1 ? p[q].y : p[q].z;
      if (v < l[k]) l[k] = v;
      if (v > h[k]) h[k] = v;
    }
  }
}

static double centroid_axis(const oscene *s, int t, int axis) {
  v3 c = scl(add(add(s->a[t], s->b[t]), s->c[t]), 1.0 / 3.0);
  return axis == 0 ? c.x : axis == 1 ? c.y : c.z;
}

static int g_sort_axis;
static const oscene *g_sort_scene;
static int cmp_centroid(const void *pa, const void *pb) {
  double ca = centroid_axis(g_sort_scene, *(const int *)pa, g_sort_axis);
  double cb = centroid_axis(g_sort_scene, *(const int *)pb, g_sort_axis);
  if (ca < cb) return -1;
  if (ca > cb) return 1;
  return (*(const int *)pa) - (*(const int *)pb);
}

/* Median-split bounding volume hierarchy, leaves of <= 4 triangles.  It only
 * prunes triangles the ray cannot reach before the best hit so far; every
 * triangle that survives goes through the same exact test as brute force. */
static int bvh_build_rec(bvh *h, const oscene *s, int first, int count) {
  int id = h->n_nodes++;
  bnode *nd = &h->nodes[id];
  for (int k = 0; k < 3; k++) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
  for (int i = first; i < first + count; i++) {
    double lo[3], hi[3];
    tri_box(s, h->idx[i], lo, hi);
    for (int k = 0; k < 3; k++) {
      if (lo[k] < nd->lo[k]) nd->lo[k] = lo[k];
      if (hi[k] > nd->hi[k]) nd->hi[k] = hi[k];
    }
  }
  if (count <= 4) {
    nd->left = nd->right = -1;
    nd->first = first;
    nd->count = count;
    return id;
  }
  double ext[3];
  for (int k = 0; k < 3; k++) ext[k] = nd->hi[k] - nd->lo[k];
  int axis = ext[0] >= ext[1] && ext[0] >= ext[2] ? 0 : (ext[1] >= ext[2] ? 1 : 2);
  g_sort_axis = axis;
  g_sort_scene = s;
  qsort(h->idx + first, (size_t)count, sizeof(int), cmp_centroid);
  int half = count / 2;
  int l = bvh_build_rec(h, s, first, half);
  int r = bvh_build_rec(h, s, first + half, count - half);
  nd = &h->nodes[id];
  nd->left = l;
  nd->right = r;
  nd->first = first;
  nd->count = count;
  return id;
}

static int bvh_build(bvh *h, const oscene *s, const int *ids, int n) {
  h->n_nodes = 0;
  h->idx = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  h->nodes = (bnode *)malloc(sizeof(bnode) * (size_t)(2 * (n > 0 ? n : 1)));
  if (!h->idx || !h->nodes) return -1;
  memcpy(h->idx, ids, sizeof(int) * (size_t)n);
  if (n > 0) bvh_build_rec(h, s, 0, n);
  return 0;
}

static void bvh_free(bvh *h) {
  free(h->idx);
  free(h->nodes);
  h->idx = NULL;
  h->nodes = NULL;
}

void or_scene_free(void *p);

/* verts [n_v][3], tris [n_t][3], mat [n_t], refl [n_mat][n_bands]; all as the
 * library takes them (float32/int32/uint8), promoted exactly to double. */
void *or_scene_new(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                   const uint8_t *mat, const float *refl, int n_mat, int n_bands, int tiles_x,
                   int tiles_y) {
  if (n_bands < 1 || n_bands > OR_MAX_BANDS || tiles_x < 1 || tiles_y < 1 || tiles_x > 32 ||
      tiles_y > 32)
    return NULL;
  oscene *s = (oscene *)calloc(1, sizeof(oscene));
  if (!s) return NULL;
  s->n_tris = n_tris;
  s->n_mat = n_mat;
  s->n_bands = n_bands;
  size_t nt = (size_t)(n_tris > 0 ? n_tris : 1);
  s->a = (v3 *)malloc(sizeof(v3) * nt);
  s->b = (v3 *)malloc(sizeof(v3) * nt);
  s->c = (v3 *)malloc(sizeof(v3) * nt);
  s->n = (v3 *)malloc(sizeof(v3) * nt);
  s->mat = (int *)malloc(sizeof(int) * nt);
  s->refl = (double *)malloc(sizeof(double) * (size_t)(n_mat > 0 ? n_mat : 1) * (size_t)n_bands);
  int *ids = (int *)malloc(sizeof(int) * nt);
  if (!s->a || !s->b || !s->c || !s->n || !s->mat || !s->refl || !ids) {
    free(ids);
    or_scene_free(s);
    return NULL;
  }
  for (int k = 0; k < 3; k++) { s->lo[k] = 0.0; s->hi[k] = 0.0; }
  for (int64_t t = 0; t < n_tris; t++) {
    const float *pa = verts + 3 * (int64_t)tris[3 * t + 0];
    const float *pb = verts + 3 * (int64_t)tris[3 * t + 1];
    const float *pc = verts + 3 * (int64_t)tris[3 * t + 2];
    if (tris[3 * t] < 0 || tris[3 * t] >= n_verts || tris[3 * t + 1] < 0 ||
        tris[3 * t + 1] >= n_verts || tris[3 * t + 2] < 0 || tris[3 * t + 2] >= n_verts ||
        mat[t] >= n_mat) {
      free(ids);
      or_scene_free(s);
      return NULL;
    }
    s->a[t] = mk(pa[0], pa[1], pa[2]);
    s->b[t] = mk(pb[0], pb[1], pb[2]);
    s->c[t] = mk(pc[0], pc[1], pc[2]);
    v3 nn = cross(sub(s->b[t], s->a[t]), sub(s->c[t], s->a[t]));
    double l = len(nn);
    s->n[t] = l > 0 ? scl(nn, 1.0 / l) : mk(0, 0, 0);
    s->mat[t] = mat[t];
    ids[t] = (int)t;
    double lo[3], hi[3];
    tri_box(s, (int)t, lo, hi);
    for (int k = 0; k < 3; k++) {
      if (t == 0 || lo[k] < s->lo[k]) s->lo[k] = lo[k];
      if (t == 0 || hi[k] > s->hi[k]) s->hi[k] = hi[k];
    }
  }
  for (int i = 0; i < n_mat * n_bands; i++) s->refl[i] = refl[i];
  if (bvh_build(&s->all, s, ids, (int)n_tris)) {
    free(ids);
    or_scene_free(s);
    return NULL;
  }
  s->tx = tiles_x;
  s->ty = tiles_y;
  s->tile = (bvh *)calloc((size_t)(tiles_x * tiles_y), sizeof(bvh));
  if (!s->tile) { free(ids); or_scene_free(s); return NULL; }
  /* tile lists: every triangle whose xy box touches the tile's closed box */
  s->gx0 = s->lo[0] - 1.0;
  s->gx1 = s->hi[0] + 1.0;
  s->gy0 = s->lo[1] - 1.0;
  s->gy1 = s->hi[1] + 1.0;
  double wx = (s->gx1 - s->gx0) / tiles_x, wy = (s->gy1 - s->gy0) / tiles_y;
  for (int ty = 0; ty < tiles_y; ty++)
    for (int tx = 0; tx < tiles_x; tx++) {
      double x0 = s->gx0 + wx * tx, x1 = s->gx0 + wx * (tx + 1);
      double y0 = s->gy0 + wy * ty, y1 = s->gy0 + wy * (ty + 1);
      double mg = 1e-6 * (1.0 + fabs(x1) + fabs(y1));
      int n = 0;
      for (int64_t t = 0; t < n_tris; t++) {
        double lo[3], hi[3];
        tri_box(s, (int)t, lo, hi);
        if (hi[0] >= x0 - mg && lo[0] <= x1 + mg && hi[1] >= y0 - mg && lo[1] <= y1 + mg)
          ids[n++] = (int)t;
      }
      if (bvh_build(&s->tile[ty * tiles_x + tx], s, ids, n)) {
        free(ids);
        or_scene_free(s);
        return NULL;
      }
    }
  free(ids);
  return s;
}

void or_scene_free(void *p) {
  oscene *s = (oscene *)p;
  if (!s) return;
  free(s->a); free(s->b); free(s->c); free(s->n); free(s->mat); free(s->refl);
  bvh_free(&s->all);
  if (s->tile) {
    for (int i = 0; i < s->tx * s->ty; i++) bvh_free(&s->tile[i]);
    free(s->tile);
  }
  free(s);
}

/* ------------------------------------------------------------ hit testing --
 * Moller & Trumbore (1997) ray/triangle test, two-sided, edges inclusive. */
static int ray_tri(v3 o, v3 d, v3 a, v3 b, v3 c, double *t) {
  v3 e1 = sub(b, a), e2 = sub(c, a);
  v3 p = cross(d, e2);
  double det = dot(e1, p);
  if (det == 0.0) return 0;
  double inv = 1.0 / det;
  v3 s = sub(o, a);
  double u = dot(s, p) * inv;
  if (u < 0.0 || u > 1.0) return 0;
  v3 q = cross(s, e1);
  double v = dot(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return 0;
  *t = dot(e2, q) * inv;
  return 1;
}

typedef struct {
  v3 o, d;
  double t_eps;
  int has_start;  /* reflected ray: hits closer than t_eps to the start plane are ignored */
  v3 ns;          /* start-plane normal, oriented toward the ray (d.ns > 0) */
} ray_q;

/* Hit acceptance shared by every search mode: t beyond t_eps and, for a
 * reflected ray, the hit point more than t_eps away from the plane it left. */
static int accept_t(const ray_q *r, double t) {
  if (!(t > r->t_eps)) return 0;
  if (r->has_start && !(t * dot(r->d, r->ns) > r->t_eps)) return 0;
  return 1;
}

/* Tile of an xy point: half-open cells [x_i, x_i+1) of the tile grid, points
 * outside the grid clamped to the border tiles. */
static void tile_of(const oscene *s, double x, double y, int *ix, int *iy) {
  int i = (int)floor((x - s->gx0) / (s->gx1 - s->gx0) * s->tx);
  int j = (int)floor((y - s->gy0) / (s->gy1 - s->gy0) * s->ty);
  *ix = i < 0 ? 0 : i >= s->tx ? s->tx - 1 : i;
  *iy = j < 0 ? 0 : j >= s->ty ? s->ty - 1 : j;
}

static void consider(const oscene *s, const ray_q *r, int tri, double *best_t, int *best_id,
                     const int *tile_xy) {
  double t;
  if (!ray_tri(r->o, r->d, s->a[tri], s->b[tri], s->c[tri], &t)) return;
  if (!accept_t(r, t)) return;
  if (tile_xy) { /* tiled mode: the hit point must lie in this tile (half-open) */
    v3 h = add(r->o, scl(r->d, t));
    int ix, iy;
    tile_of(s, h.x, h.y, &ix, &iy);
    if (ix != tile_xy[0] || iy != tile_xy[1]) return;
  }
  /* Two surfaces hit at the same distance (a box floor lying on the ground,
   * the shared edge of two faces) form a tie in exact arithmetic; distances
   * within 1e-9 relative count as equal so that the lowest index, not the
   * rounding, decides. */
  double tol = 1e-9 * (1.0 + fabs(t));
  if (*best_id < 0 || t < *best_t - tol || (fabs(t - *best_t) <= tol && tri < *best_id)) {
    *best_t = t;
    *best_id = tri;
  }
}

/* closest hit by testing every triangle */
static void hit_bruteforce(const oscene *s, const ray_q *r, double *bt, int *bid) {
  for (int64_t t = 0; t < s->n_tris; t++) consider(s, r, (int)t, bt, bid, NULL);
}

/* Entry distance of the ray into a box grown by a margin, or +inf if missed. */
static double box_enter(const double lo[3], const double hi[3], v3 o, v3 d) {
  double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  double t0 = -INFINITY, t1 = INFINITY;
  for (int k = 0; k < 3; k++) {
    double mg = 1e-7 * (1.0 + fabs(lo[k]) + fabs(hi[k]));
    double l = lo[k] - mg, h = hi[k] + mg;
    if (dd[k] == 0.0) {
      if (oo[k] < l || oo[k] > h) return INFINITY;
      continue;
    }
    double ta = (l - oo[k]) / dd[k], tb = (h - oo[k]) / dd[k];
    if (ta > tb) { double x = ta; ta = tb; tb = x; }
    if (ta > t0) t0 = ta;
    if (tb < t1) t1 = tb;
  }
  if (t0 > t1 || t1 < 0.0) return INFINITY;
  return t0;
}

static void hit_bvh(const oscene *s, const bvh *h, const ray_q *r, double *bt, int *bid,
                    const int *tile_xy) {
  if (h->n_nodes == 0) return;
  int stack[128], sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const bnode *nd = &h->nodes[stack[--sp]];
    double te = box_enter(nd->lo, nd->hi, r->o, r->d);
    if (te == INFINITY || te > *bt + 1e-6 * (1.0 + fabs(*bt))) continue; /* margin covers the tie window */
    if (nd->left < 0) {
      for (int i = nd->first; i < nd->first + nd->count; i++)
        consider(s, r, h->idx[i], bt, bid, tile_xy);
    } else {
      stack[sp++] = nd->left;
      stack[sp++] = nd->right;
    }
  }
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : x > y;
}

/* Tiled search (Section 3, geometry and microphone partitioning): walk the
 * tiles the ray's xy projection crosses in order of t; in each, search only
 * that tile's triangles and accept only hits inside the tile; the first tile
 * with an accepted hit ends the walk, otherwise the ray passes to the next. */
static void hit_tiled(const oscene *s, const ray_q *r, double *bt, int *bid, int *handoffs) {
  double wx = (s->gx1 - s->gx0) / s->tx, wy = (s->gy1 - s->gy0) / s->ty;
  double tin = 0.0, tout = INFINITY;
  double oo[2] = {r->o.x, r->o.y}, dd[2] = {r->d.x, r->d.y};
  double lo[2] = {s->gx0, s->gy0}, hi[2] = {s->gx1, s->gy1};
  for (int k = 0; k < 2; k++) {
    if (dd[k] == 0.0) {
      if (oo[k] < lo[k] || oo[k] > hi[k]) return;
      continue;
    }
    double ta = (lo[k] - oo[k]) / dd[k], tb = (hi[k] - oo[k]) / dd[k];
    if (ta > tb) { double x = ta; ta = tb; tb = x; }
    if (ta > tin) tin = ta;
    if (tb < tout) tout = tb;
  }
  if (tin > tout) return;
  double ts[80];
  int n = 0;
  ts[n++] = tin;
  for (int i = 1; i < s->tx && r->d.x != 0.0; i++) {
    double t = (s->gx0 + wx * i - r->o.x) / r->d.x;
    if (t > tin && t < tout) ts[n++] = t;
  }
  for (int j = 1; j < s->ty && r->d.y != 0.0; j++) {
    double t = (s->gy0 + wy * j - r->o.y) / r->d.y;
    if (t > tin && t < tout) ts[n++] = t;
  }
  qsort(ts, (size_t)n, sizeof(double), cmp_double);
  int last = -1;
  for (int i = 0; i < n; i++) {
    double tb = i + 1 < n ? ts[i + 1] : tout;
    double tm = tb < INFINITY ? 0.5 * (ts[i] + tb) : ts[i] + 1.0;
    v3 p = add(r->o, scl(r->d, tm));
    int ix, iy;
    tile_of(s, p.x, p.y, &ix, &iy);
    int tid = iy * s->tx + ix;
    if (tid == last) continue;
    if (last >= 0 && handoffs) (*handoffs)++;
    last = tid;
    int txy[2] = {ix, iy};
    hit_bvh(s, &s->tile[tid], r, bt, bid, txy);
    if (*bid >= 0) return;
  }
}

/* mode 0: brute force, 1: bvh over all triangles, 2: tiled */
static void closest_hit(const oscene *s, const ray_q *r, int mode, double *bt, int *bid,
                        int *handoffs) {
  *bt = INFINITY;
  *bid = -1;
  if (mode == 0) hit_bruteforce(s, r, bt, bid);
  else if (mode == 1) hit_bvh(s, &s->all, r, bt, bid, NULL);
  else hit_tiled(s, r, bt, bid, handoffs);
}

/* Batch ray query for tests: o,d [n][3], start normal ns [n][3] used where
 * has_start[i] != 0.  Writes t (inf on a miss) and triangle id (-1). */
int or_cast_rays(const void *scene, int mode, int64_t n, const double *o, const double *d,
                 const int32_t *has_start, const double *ns, double t_eps, double *t_out,
                 int32_t *id_out) {
  const oscene *s = (const oscene *)scene;
  for (int64_t i = 0; i < n; i++) {
    ray_q r;
    r.o = mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
    r.d = mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]);
    r.t_eps = t_eps;
    r.has_start = has_start ? has_start[i] : 0;
    r.ns = r.has_start ? mk(ns[3 * i], ns[3 * i + 1], ns[3 * i + 2]) : mk(0, 0, 0);
    int id;
    closest_hit(s, &r, mode, &t_out[i], &id, NULL);
    id_out[i] = id;
  }
  return 0;
}

/* ------------------------------------------------------------- microphones -- */
typedef struct {
  int64_t n;
  const float *pos;     /* [n][3] */
  int nx, ny;           /* xy bin grid */
  double x0, y0, cw, ch; /* grid origin and cell size */
  double zlo, zhi;
  int64_t *cell_start;  /* [nx*ny+1] */
  int64_t *ids;         /* microphone ids grouped by cell */
} omics;

static int mics_build(omics *m, const float *pos, int64_t n) {
  memset(m, 0, sizeof(*m));
  m->n = n;
  m->pos = pos;
  if (n == 0) return 0;
  double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
  m->zlo = INFINITY;
  m->zhi = -INFINITY;
  for (int64_t i = 0; i < n; i++) {
    double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    if (x < x0) x0 = x;
    if (x > x1) x1 = x;
    if (y < y0) y0 = y;
    if (y > y1) y1 = y;
    if (z < m->zlo) m->zlo = z;
    if (z > m->zhi) m->zhi = z;
  }
  int side = (int)ceil(sqrt((double)n / 4.0));
  if (side < 1) side = 1;
  m->nx = m->ny = side;
  m->x0 = x0;
  m->y0 = y0;
  m->cw = (x1 - x0) / side + 1e-9 * (1.0 + fabs(x1));
  m->ch = (y1 - y0) / side + 1e-9 * (1.0 + fabs(y1));
  if (m->cw <= 0) m->cw = 1.0;
  if (m->ch <= 0) m->ch = 1.0;
  int64_t nc = (int64_t)side * side;
  m->cell_start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  m->ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!m->cell_start || !m->ids || !cell) { free(cell); return -1; }
  for (int64_t i = 0; i < n; i++) {
    int cx = (int)floor((pos[3 * i] - x0) / m->cw), cy = (int)floor((pos[3 * i + 1] - y0) / m->ch);
    if (cx < 0) cx = 0;
    if (cx >= side) cx = side - 1;
    if (cy < 0) cy = 0;
    if (cy >= side) cy = side - 1;
    cell[i] = (int64_t)cy * side + cx;
    m->cell_start[cell[i] + 1]++;
  }
  for (int64_t c = 0; c < nc; c++) m->cell_start[c + 1] += m->cell_start[c];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
  if (!fill) { free(cell); return -1; }
  memcpy(fill, m->cell_start, sizeof(int64_t) * (size_t)nc);
  for (int64_t i = 0; i < n; i++) m->ids[fill[cell[i]]++] = i;
  free(fill);
  free(cell);
  return 0;
}

static void mics_free(omics *m) {
  free(m->cell_start);
  free(m->ids);
}

/* One beam segment: apex, cone edge directions (CCW seen from outside), an
 * optional start plane (the reflector it left) and end plane (the surface its
 * axis hit), and the per-band power factor W_b * prod(r). */
typedef struct {
  v3 apex;
  v3 dir[3];
  v3 en[3];       /* edge-plane normals dir[j] x dir[j+1]; inside is en.(m-apex) >= 0 */
  int has_start;  /* inside requires ns.(m-ps) > 0 */
  v3 ns, ps;
  int has_end;    /* inside requires ne.(m-pe) >= 0 */
  v3 ne, pe;
  double w[OR_MAX_BANDS];
} segment;

/* Is microphone m inside the segment?  Returns 1/0; *tie is set when m lies on
 * a cone edge plane to within 1e-9 of its distance (measure-zero ties). */
static int mic_in_segment(const segment *g, v3 m, int *tie) {
  v3 rel = sub(m, g->apex);
  double dist = len(rel);
  *tie = 0;
  for (int j = 0; j < 3; j++) {
    double e = dot(g->en[j], rel);
    if (fabs(e) <= 1e-9 * dist * len(g->en[j])) *tie = 1;
    if (e < 0.0) return 0;
  }
  if (g->has_start && !(dot(g->ns, sub(m, g->ps)) > 0.0)) return 0;
  if (g->has_end && !(dot(g->ne, sub(m, g->pe)) >= 0.0)) return 0;
  return 1;
}

/* The cone's edge-plane normals from its edge directions. */
static void seg_edges(segment *g) {
  for (int j = 0; j < 3; j++) g->en[j] = cross(g->dir[j], g->dir[(j + 1) % 3]);
}

/* Image source (Section 2): mirror the apex and the cone's edge directions in
 * the reflecting plane (point p, normal n), and reverse the edge order so that
 * the mirrored cone stays counter-clockwise seen from outside. */
static void reflect_cone(segment *g, v3 p, v3 n) {
  v3 d0 = mirror_dir(g->dir[0], n), d1 = mirror_dir(g->dir[1], n), d2 = mirror_dir(g->dir[2], n);
  g->dir[0] = d0;
  g->dir[1] = d2;
  g->dir[2] = d1;
  g->apex = mirror_pt(g->apex, p, n);
}

/* Half-space list of a segment, each as n.x >= c with |n| = 1, for culling. */
static int seg_halfspaces(const segment *g, v3 hn[5], double hc[5]) {
  int k = 0;
  for (int j = 0; j < 3; j++) {
    double l = len(g->en[j]);
    hn[k] = scl(g->en[j], 1.0 / l);
    hc[k] = dot(hn[k], g->apex);
    k++;
  }
  if (g->has_start) { hn[k] = g->ns; hc[k] = dot(g->ns, g->ps); k++; }
  if (g->has_end) { hn[k] = g->ne; hc[k] = dot(g->ne, g->pe); k++; }
  return k;
}

typedef struct {
  double *I;          /* [n_mics][n_bands] */
  int32_t *cnt;       /* [n_mics] */
  int n_bands;
  const double *alpha; /* dB per metre per band */
  double contributions, ties;
  /* optional path log */
  int64_t log_cap, log_n;
  int32_t *log_mic, *log_src, *log_order;
  double *log_d, *log_apex;
  int cur_src, cur_order;
} accum;

/* Section 2: a microphone in the beam receives the beam's intensity, which is
 * the image-source intensity W_b prod(r_b) 10^(-alpha_b d / 10) / (4 pi d^2). */
static void contribute(accum *acc, const segment *g, int64_t mic, v3 m) {
  double d = len(sub(m, g->apex));
  if (d < 1e-9) return;
  for (int b = 0; b < acc->n_bands; b++) {
    double damp = acc->alpha[b] != 0.0 ? pow(10.0, -acc->alpha[b] * d / 10.0) : 1.0;
    acc->I[mic * acc->n_bands + b] += g->w[b] * damp / (4.0 * OR_PI * d * d);
  }
  acc->cnt[mic] += 1;
  acc->contributions += 1;
  if (acc->log_cap > 0 && acc->log_n < acc->log_cap) {
    int64_t k = acc->log_n++;
    acc->log_mic[k] = (int32_t)mic;
    acc->log_src[k] = acc->cur_src;
    acc->log_order[k] = acc->cur_order;
    acc->log_d[k] = d;
    acc->log_apex[3 * k] = g->apex.x;
    acc->log_apex[3 * k + 1] = g->apex.y;
    acc->log_apex[3 * k + 2] = g->apex.z;
  }
}

static void test_mic(accum *acc, const segment *g, const omics *mc, int64_t i) {
  v3 m = mk(mc->pos[3 * i], mc->pos[3 * i + 1], mc->pos[3 * i + 2]);
  int tie;
  if (mic_in_segment(g, m, &tie)) contribute(acc, g, i, m);
  if (tie) acc->ties += 1;
}

/* Recursive cell culling: a block of cells is skipped only when one of the
 * segment's half-spaces excludes all eight corners of the block's box
 * (xy block x [zlo, zhi]) by more than a 1e-6 m margin; surviving single
 * cells test each of their microphones exactly. */
static void cull_cells(accum *acc, const segment *g, const omics *mc, const v3 *hn,
                       const double *hc, int nh, int cx0, int cx1, int cy0, int cy1) {
  double bx0 = mc->x0 + mc->cw * cx0, bx1 = mc->x0 + mc->cw * (cx1 + 1);
  double by0 = mc->y0 + mc->ch * cy0, by1 = mc->y0 + mc->ch * (cy1 + 1);
  for (int k = 0; k < nh; k++) {
    double best = -INFINITY;
    for (int c = 0; c < 8; c++) {
      v3 p = mk(c & 1 ? bx1 : bx0, c & 2 ? by1 : by0, c & 4 ? mc->zhi : mc->zlo);
      double v = dot(hn[k], p) - hc[k];
      if (v > best) best = v;
    }
    if (best < -1e-6) return;
  }
  if (cx0 == cx1 && cy0 == cy1) {
    int64_t c = (int64_t)cy0 * mc->nx + cx0;
    for (int64_t q = mc->cell_start[c]; q < mc->cell_start[c + 1]; q++) test_mic(acc, g, mc, mc->ids[q]);
    return;
  }
  if (cx1 - cx0 >= cy1 - cy0) {
    int xm = (cx0 + cx1) / 2;
    cull_cells(acc, g, mc, hn, hc, nh, cx0, xm, cy0, cy1);
    cull_cells(acc, g, mc, hn, hc, nh, xm + 1, cx1, cy0, cy1);
  } else {
    int ym = (cy0 + cy1) / 2;
    cull_cells(acc, g, mc, hn, hc, nh, cx0, cx1, cy0, ym);
    cull_cells(acc, g, mc, hn, hc, nh, cx0, cx1, ym + 1, cy1);
  }
}

/* mic_mode 0: every microphone is tested; 1: culled by the cell grid. */
static void scatter_segment(accum *acc, const segment *g, const omics *mc, int mic_mode) {
  if (mc->n == 0) return;
  if (mic_mode == 0) {
    for (int64_t i = 0; i < mc->n; i++) test_mic(acc, g, mc, i);
    return;
  }
  v3 hn[5];
  double hc[5];
  int nh = seg_halfspaces(g, hn, hc);
  cull_cells(acc, g, mc, hn, hc, nh, 0, mc->nx - 1, 0, mc->ny - 1);
}

/* ------------------------------------------------------------------ trace -- */
typedef struct {
  int max_order;
  double t_eps;
  double energy_threshold;
  double alpha[OR_MAX_BANDS];
  int hit_mode;   /* 0 brute force, 1 bvh, 2 tiled */
  int mic_mode;   /* 0 brute force, 1 cell grid */
} oparams;

/* stats layout (doubles): [0] segments, [1] contributions, [2] hits,
 * [3] escapes, [4] hand-offs, [5] ties, [6..6+K] beam power (sum over bands
 * of W_b prod(r_b) omega/4pi) entering each order k = 0..K. */
#define OR_NSTAT_FIXED 6

typedef struct {
  const oscene *s;
  const omics *mc;
  const oparams *p;
  const float *src, *power;
  const float *dir_gain;  /* [n_patterns][n_beams] or NULL */
  const int32_t *dir_of;  /* [n_src]: pattern of each source, -1 = omnidirectional */
  int64_t n_src;
  int level;
  const double *dirs, *omega;
  int64_t n_beams;
  int tid, n_threads;
  accum acc;
  double *stats;
  int32_t *hit_log;  /* [n_src][n_beams][K+1] or NULL: hit triangle per segment, -1 escape */
} job;

/* Section 2 hybrid method, one beam from apex s along face i, orders 0..K. */
static void trace_beam(job *J, int64_t si, int64_t bi) {
  const oscene *s = J->s;
  const oparams *p = J->p;
  accum *acc = &J->acc;
  segment g;
  memset(&g, 0, sizeof(g));
  g.apex = mk(J->src[3 * si], J->src[3 * si + 1], J->src[3 * si + 2]);
  for (int j = 0; j < 3; j++)
    g.dir[j] = mk(J->dirs[9 * bi + 3 * j], J->dirs[9 * bi + 3 * j + 1], J->dirs[9 * bi + 3 * j + 2]);
  /* a directional source: its power in this beam's direction, the pattern's
   * gain times the omnidirectional power */
  double gain = 1.0;
  if (J->dir_of && J->dir_of[si] >= 0) gain = J->dir_gain[(int64_t)J->dir_of[si] * J->n_beams + bi];
  for (int b = 0; b < s->n_bands; b++) g.w[b] = gain * J->power[si * s->n_bands + b];
  ray_q r;
  r.o = g.apex;
  r.d = unit(add(add(g.dir[0], g.dir[1]), g.dir[2]));
  r.t_eps = p->t_eps;
  r.has_start = 0;
  r.ns = mk(0, 0, 0);
  double omega4pi = J->omega[bi] / (4.0 * OR_PI);
  for (int k = 0; k <= p->max_order; k++) {
    double pw = 0.0;
    for (int b = 0; b < s->n_bands; b++) pw += g.w[b] * omega4pi;
    J->stats[OR_NSTAT_FIXED + k] += pw;
    seg_edges(&g);
    double th;
    int hid, ho = 0;
    closest_hit(s, &r, p->hit_mode, &th, &hid, &ho);
    J->stats[4] += ho;
    J->stats[0] += 1;
    if (J->hit_log) J->hit_log[(si * J->n_beams + bi) * (p->max_order + 1) + k] = hid;
    if (hid >= 0) {
      J->stats[2] += 1;
      g.has_end = 1;
      g.pe = s->a[hid];
      g.ne = dot(s->n[hid], r.d) < 0.0 ? s->n[hid] : scl(s->n[hid], -1.0);
    } else {
      J->stats[3] += 1;
      g.has_end = 0;
    }
    acc->cur_order = k;
    scatter_segment(acc, &g, J->mc, p->mic_mode);
    if (hid < 0 || k == p->max_order) break;
    /* image source: the mirrored apex and cone; the reflection loses energy */
    v3 n = s->n[hid];
    reflect_cone(&g, s->a[hid], n);
    double wmax = 0.0;
    for (int b = 0; b < s->n_bands; b++) {
      g.w[b] *= s->refl[s->mat[hid] * s->n_bands + b];
      if (g.w[b] > wmax) wmax = g.w[b];
    }
    if (p->energy_threshold > 0.0 && wmax < p->energy_threshold) break;
    v3 hp = add(r.o, scl(r.d, th));
    v3 nd = mirror_dir(r.d, n);
    g.has_start = 1;
    g.ns = dot(n, nd) > 0.0 ? n : scl(n, -1.0);
    g.ps = s->a[hid];
    r.o = hp;
    r.d = nd;
    r.has_start = 1;
    r.ns = g.ns;
  }
}

static void *run_job(void *arg) {
  job *J = (job *)arg;
  for (int64_t si = J->tid; si < J->n_src; si += J->n_threads) {
    J->acc.cur_src = (int)si;
    for (int64_t bi = 0; bi < J->n_beams; bi++) trace_beam(J, si, bi);
  }
  return NULL;
}

/*
 * Full trace.  Inputs as the library takes them.  Outputs: I [n_mics][n_bands]
 * (W/m^2), cnt [n_mics] (paths per microphone), stats [6 + max_order + 1].
 * Threads split the sources statically (source s goes to thread s mod T) and
 * their partial sums are added in thread order.  An optional path log
 * (single thread only) records each contribution's microphone, source, order,
 * distance and apex.  An optional hit log [n_src][n_beams][max_order + 1]
 * receives the triangle each segment's axis ray hit (-1: it escaped); entries
 * of orders a beam did not reach are left as they were.  Returns 0, or a
 * negative value on bad input.
 */
int or_trace_dir(const void *scene, const float *src, const float *power, int64_t n_src, int level,
                 const float *dir_gain, int32_t n_patterns, const int32_t *dir_of,
                 const float *mics, int64_t n_mics, int max_order, const double *alpha,
                 double energy_threshold, double t_eps, int hit_mode, int mic_mode, int n_threads,
                 double *I, int32_t *cnt, double *stats, int64_t log_cap, int32_t *log_mic,
                 int32_t *log_src, int32_t *log_order, double *log_d, double *log_apex,
                 int64_t *log_n, int32_t *hit_log) {
  const oscene *s = (const oscene *)scene;
  if (!s || level < 0 || level > 8 || max_order < 0 || max_order > 32 || n_threads < 1) return -1;
  if (dir_of) {
    if (!dir_gain || n_patterns < 1) return -1;
    for (int64_t i = 0; i < n_src; i++)
      if (dir_of[i] < -1 || dir_of[i] >= n_patterns) return -1;
  }
  if (log_cap > 0 && n_threads != 1) return -2;
  oparams p;
  p.max_order = max_order;
  p.t_eps = t_eps;
  p.energy_threshold = energy_threshold;
  for (int b = 0; b < OR_MAX_BANDS; b++) p.alpha[b] = (alpha && b < s->n_bands) ? alpha[b] : 0.0;
  p.hit_mode = hit_mode;
  p.mic_mode = mic_mode;
  int64_t nb = or_n_beams(level);
  double *dirs = (double *)malloc(sizeof(double) * 9 * (size_t)nb);
  double *omega = (double *)malloc(sizeof(double) * (size_t)nb);
  omics mc;
  if (!dirs || !omega || mics_build(&mc, mics, n_mics)) { free(dirs); free(omega); return -3; }
  or_beam_table(level, dirs, omega);
  int nstat = OR_NSTAT_FIXED + max_order + 1;
  job *jobs = (job *)calloc((size_t)n_threads, sizeof(job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  int rc = 0;
  if (!jobs || !th) rc = -3;
  for (int i = 0; i < n_threads && !rc; i++) {
    job *J = &jobs[i];
    J->s = s; J->mc = &mc; J->p = &p; J->src = src; J->power = power; J->n_src = n_src;
    J->dir_gain = dir_of ? dir_gain : NULL; J->dir_of = dir_of;
    J->level = level; J->dirs = dirs; J->omega = omega; J->n_beams = nb;
    J->tid = i; J->n_threads = n_threads;
    J->hit_log = hit_log;
    J->acc.n_bands = s->n_bands;
    J->acc.alpha = p.alpha;
    J->acc.I = i == 0 ? I : (double *)calloc((size_t)(n_mics > 0 ? n_mics : 1) * s->n_bands, sizeof(double));
    J->acc.cnt = i == 0 ? cnt : (int32_t *)calloc((size_t)(n_mics > 0 ? n_mics : 1), sizeof(int32_t));
    J->stats = (double *)calloc((size_t)nstat, sizeof(double));
    if (!J->acc.I || !J->acc.cnt || !J->stats) rc = -3;
    if (i == 0) {
      memset(I, 0, sizeof(double) * (size_t)n_mics * s->n_bands);
      memset(cnt, 0, sizeof(int32_t) * (size_t)n_mics);
      J->acc.log_cap = log_cap;
      J->acc.log_mic = log_mic; J->acc.log_src = log_src; J->acc.log_order = log_order;
      J->acc.log_d = log_d; J->acc.log_apex = log_apex;
    }
  }
  if (!rc) {
    if (n_threads == 1) {
      run_job(&jobs[0]);
    } else {
      for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, run_job, &jobs[i]);
      for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    }
    for (int k = 0; k < nstat; k++) stats[k] = 0.0;
    for (int i = 0; i < n_threads; i++) {
      job *J = &jobs[i];
      if (i > 0) {
        for (int64_t q = 0; q < n_mics * s->n_bands; q++) I[q] += J->acc.I[q];
        for (int64_t q = 0; q < n_mics; q++) cnt[q] += J->acc.cnt[q];
      }
      for (int k = 0; k < nstat; k++) stats[k] += J->stats[k];
      stats[1] += J->acc.contributions;
      stats[5] += J->acc.ties;
    }
    if (log_n) *log_n = jobs[0].acc.log_n;
  }
  for (int i = 0; jobs && i < n_threads; i++) {
    if (i > 0) { free(jobs[i].acc.I); free(jobs[i].acc.cnt); }
    free(jobs[i].stats);
  }
  free(jobs); free(th); free(dirs); free(omega);
  mics_free(&mc);
  return rc;
}

/* or_trace_dir with every source omnidirectional. */
int or_trace(const void *scene, const float *src, const float *power, int64_t n_src, int level,
             const float *mics, int64_t n_mics, int max_order, const double *alpha,
             double energy_threshold, double t_eps, int hit_mode, int mic_mode, int n_threads,
             double *I, int32_t *cnt, double *stats, int64_t log_cap, int32_t *log_mic,
             int32_t *log_src, int32_t *log_order, double *log_d, double *log_apex,
             int64_t *log_n) {
  return or_trace_dir(scene, src, power, n_src, level, NULL, 0, NULL, mics, n_mics, max_order, alpha,
                      energy_threshold, t_eps, hit_mode, mic_mode, n_threads, I, cnt, stats, log_cap,
                      log_mic, log_src, log_order, log_d, log_apex, log_n, NULL);
}

/* Level readout: L = 10 log10(I / 1e-12) dB re 1e-12 W/m^2, -inf where I = 0. */
void or_levels(const double *I, int64_t n, double *L) {
  for (int64_t i = 0; i < n; i++) L[i] = I[i] > 0.0 ? 10.0 * log10(I[i] / 1e-12) : -INFINITY;
}

/* ------------------------------------------------------------ primitives --
 * The building blocks above, one call each, for hand-worked unit cases. */
static v3 ld3(const double *a) { return mk(a[0], a[1], a[2]); }
static void st3(double *o, v3 a) { o[0] = a.x; o[1] = a.y; o[2] = a.z; }

/* Ray (o, d) against triangle (a, b, c): 1 and *t on a hit (any sign of t),
 * else 0. */
int or_ray_tri(const double *o, const double *d, const double *a, const double *b, const double *c, double *t) {
  return ray_tri(ld3(o), ld3(d), ld3(a), ld3(b), ld3(c), t);
}

/* Mirror image of point a in the plane through p with unit normal n. */
void or_mirror_point(const double *a, const double *p, const double *n, double *out) {
  st3(out, mirror_pt(ld3(a), ld3(p), ld3(n)));
}

/* Mirror image of direction d in a plane with unit normal n. */
void or_mirror_dir(const double *d, const double *n, double *out) { st3(out, mirror_dir(ld3(d), ld3(n))); }

/* A beam's cone (apex [3], edge directions dirs [3][3]) reflected in the plane
 * through p with unit normal n, as the trace reflects it. */
void or_reflect_cone(const double *apex, const double *dirs, const double *p, const double *n, double *apex_out,
                     double *dirs_out) {
  segment g;
  memset(&g, 0, sizeof(g));
  g.apex = ld3(apex);
  for (int j = 0; j < 3; j++) g.dir[j] = ld3(dirs + 3 * j);
  reflect_cone(&g, ld3(p), ld3(n));
  st3(apex_out, g.apex);
  for (int j = 0; j < 3; j++) st3(dirs_out + 3 * j, g.dir[j]);
}

/* Is point m in the segment with apex [3], edge directions dirs [3][3], an
 * optional start plane start [6] = (normal, point) and end plane end [6]
 * (NULL: none)?  *tie as in the trace. */
int or_in_segment(const double *apex, const double *dirs, const double *start, const double *end, const double *m,
                  int *tie) {
  segment g;
  memset(&g, 0, sizeof(g));
  g.apex = ld3(apex);
  for (int j = 0; j < 3; j++) g.dir[j] = ld3(dirs + 3 * j);
  seg_edges(&g);
  if (start) { g.has_start = 1; g.ns = ld3(start); g.ps = ld3(start + 3); }
  if (end) { g.has_end = 1; g.ne = ld3(end); g.pe = ld3(end + 3); }
  return mic_in_segment(&g, ld3(m), tie);
}
