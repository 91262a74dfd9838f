/*
 * isrc_bruteforce.c -- brute-force image-source enumeration, the classical
 * image-source method that the paper's Section 2 names as the first
 * geometrical method (virtual sources mirrored at each reflection; a
 * microphone hears every virtual source whose unfolded path reaches it
 * unobstructed).
 *
 * TEST INFRASTRUCTURE.  It pins btrace_oracle.c from outside: the beam oracle
 * must reproduce these paths for microphones away from beam boundaries.  It
 * shares no code with btrace_oracle.c (its own vector helpers, its own
 * ray/segment test) and none with the CUDA library.
 *
 * For every sequence of triangles f_1..f_k (k <= K, consecutive triangles
 * never coplanar) the images are S_0 = source, S_j = mirror of S_{j-1} in the
 * plane of f_j.  For a microphone m the path is valid when, walking back from
 * Q = m: the line S_j -> Q crosses the plane of f_j strictly between them at a
 * point R_j inside triangle f_j, and Q <- R_j; and every leg
 * source -> R_1 -> ... -> R_k -> m is free of other triangles (hits closer
 * than t_eps to a leg's ends are ignored).  A valid path adds
 * W_b prod(r_b) 10^(-alpha_b d/10) / (4 pi d^2), d = |m - S_k|.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IS_MAX_BANDS 8
#define IS_PI 3.14159265358979323846

typedef struct { double v[3]; } vec;

static vec vsub(vec a, vec b) { vec r; for (int i = 0; i < 3; i++) r.v[i] = a.v[i] - b.v[i]; return r; }
static vec vadd(vec a, vec b) { vec r; for (int i = 0; i < 3; i++) r.v[i] = a.v[i] + b.v[i]; return r; }
static vec vmul(vec a, double s) { vec r; for (int i = 0; i < 3; i++) r.v[i] = a.v[i] * s; return r; }
static double vdot(vec a, vec b) { return a.v[0] * b.v[0] + a.v[1] * b.v[1] + a.v[2] * b.v[2]; }
static vec vcross(vec a, vec b) {
  vec r;
  r.v[0] = a.v[1] * b.v[2] - a.v[2] * b.v[1];
  r.v[1] = a.v[2] * b.v[0] - a.v[0] * b.v[2];
  r.v[2] = a.v[0] * b.v[1] - a.v[1] * b.v[0];
  return r;
}
static double vlen(vec a) { return sqrt(vdot(a, a)); }

typedef struct {
  vec p[3];
  vec n; /* unit normal (p1-p0)x(p2-p0) */
  int mat;
} tri;

typedef struct {
  int parent;  /* -1 for the source itself */
  int f;       /* triangle reflected on last */
  int depth;
  vec img;
  double w[IS_MAX_BANDS];
} inode;

/* Segment a->b against triangle t: parameter s in (0,1) of a crossing, or -1.
 * Plane crossing first, then an inclusive barycentric inside test. */
static double seg_cross(const tri *t, vec a, vec b) {
  double da = vdot(t->n, vsub(a, t->p[0])), db = vdot(t->n, vsub(b, t->p[0]));
  if (da == db) return -1.0;
  if ((da > 0 && db > 0) || (da < 0 && db < 0)) return -1.0;
  double s = da / (da - db);
  vec x = vadd(a, vmul(vsub(b, a), s));
  for (int e = 0; e < 3; e++) {
    vec u = vsub(t->p[(e + 1) % 3], t->p[e]);
    vec w = vsub(x, t->p[e]);
    if (vdot(vcross(u, w), t->n) < 0.0) return -1.0;
  }
  return s;
}

static int inside_tri(const tri *t, vec x) {
  for (int e = 0; e < 3; e++) {
    vec u = vsub(t->p[(e + 1) % 3], t->p[e]);
    vec w = vsub(x, t->p[e]);
    if (vdot(vcross(u, w), t->n) < 0.0) return 0;
  }
  return 1;
}

static int same_plane(const tri *a, const tri *b) {
  if (fabs(fabs(vdot(a->n, b->n)) - 1.0) > 1e-12) return 0;
  return fabs(vdot(a->n, vsub(b->p[0], a->p[0]))) < 1e-9;
}

/* leg a->b is blocked by some triangle crossed more than t_eps from both ends */
static int blocked(const tri *T, int n_t, vec a, vec b, double t_eps) {
  double L = vlen(vsub(b, a));
  for (int i = 0; i < n_t; i++) {
    double s = seg_cross(&T[i], a, b);
    if (s < 0.0) continue;
    if (s * L > t_eps && (1.0 - s) * L > t_eps) return 1;
  }
  return 0;
}

/*
 * Returns the number of image nodes, or a negative value on error.
 * closed_solids != 0 prunes reflections from the back of a triangle (valid
 * when every triangle belongs to a closed, outward-oriented solid or to an
 * upward ground, and source and microphones lie outside all solids).
 */
int64_t isrc_bruteforce(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                        const uint8_t *mat, const float *refl, int n_mat, int n_bands,
                        const float *src, const float *power, const float *mics, int64_t n_mics,
                        int max_order, const double *alpha, double t_eps, int closed_solids,
                        double *I, int32_t *cnt, int64_t log_cap, int32_t *log_mic,
                        int32_t *log_order, double *log_d, int64_t *log_n) {
  if (n_bands < 1 || n_bands > IS_MAX_BANDS || max_order < 0 || max_order > 32) return -1;
  tri *T = (tri *)malloc(sizeof(tri) * (size_t)(n_tris > 0 ? n_tris : 1));
  if (!T) return -2;
  for (int64_t i = 0; i < n_tris; i++) {
    for (int k = 0; k < 3; k++) {
      int32_t vi = tris[3 * i + k];
      if (vi < 0 || vi >= n_verts) { free(T); return -1; }
      for (int c = 0; c < 3; c++) T[i].p[k].v[c] = verts[3 * (int64_t)vi + c];
    }
    vec nn = vcross(vsub(T[i].p[1], T[i].p[0]), vsub(T[i].p[2], T[i].p[0]));
    T[i].n = vmul(nn, 1.0 / vlen(nn));
    T[i].mat = mat[i];
    if (T[i].mat >= n_mat) { free(T); return -1; }
  }
  /* image tree, breadth first */
  int64_t cap = 1024, n = 0;
  inode *nodes = (inode *)malloc(sizeof(inode) * (size_t)cap);
  if (!nodes) { free(T); return -2; }
  nodes[0].parent = -1;
  nodes[0].f = -1;
  nodes[0].depth = 0;
  for (int c = 0; c < 3; c++) nodes[0].img.v[c] = src[c];
  for (int b = 0; b < n_bands; b++) nodes[0].w[b] = power[b];
  n = 1;
  for (int64_t q = 0; q < n; q++) {
    if (nodes[q].depth >= max_order) continue;
    for (int64_t f = 0; f < n_tris; f++) {
      if (nodes[q].f >= 0 && same_plane(&T[nodes[q].f], &T[f])) continue;
      double side = vdot(T[f].n, vsub(nodes[q].img, T[f].p[0]));
      if (fabs(side) < 1e-12) continue;
      if (closed_solids && side <= 0.0) continue;
      if (n == cap) {
        cap *= 2;
        inode *nn = (inode *)realloc(nodes, sizeof(inode) * (size_t)cap);
        if (!nn) { free(nodes); free(T); return -2; }
        nodes = nn;
      }
      inode *c = &nodes[n];
      c->parent = (int)q;
      c->f = (int)f;
      c->depth = nodes[q].depth + 1;
      c->img = vsub(nodes[q].img, vmul(T[f].n, 2.0 * side));
      for (int b = 0; b < n_bands; b++) c->w[b] = nodes[q].w[b] * refl[T[f].mat * n_bands + b];
      n++;
    }
  }
  memset(I, 0, sizeof(double) * (size_t)(n_mics * n_bands));
  memset(cnt, 0, sizeof(int32_t) * (size_t)n_mics);
  int64_t nlog = 0;
  vec R[64];
  int F[64];
  vec s0 = nodes[0].img;
  for (int64_t mi = 0; mi < n_mics; mi++) {
    vec m;
    for (int c = 0; c < 3; c++) m.v[c] = mics[3 * mi + c];
    for (int64_t q = 0; q < n; q++) {
      /* walk back from the microphone through the reflectors */
      int ok = 1, k = nodes[q].depth;
      vec Q = m;
      int64_t cur = q;
      for (int j = k; j >= 1 && ok; j--) {
        const inode *nd = &nodes[cur];
        const tri *t = &T[nd->f];
        double dS = vdot(t->n, vsub(nd->img, t->p[0])), dQ = vdot(t->n, vsub(Q, t->p[0]));
        if (!(dS * dQ < 0.0)) { ok = 0; break; }
        vec x = vadd(nd->img, vmul(vsub(Q, nd->img), dS / (dS - dQ)));
        if (!inside_tri(t, x)) { ok = 0; break; }
        R[j] = x;
        F[j] = nd->f;
        Q = x;
        cur = nd->parent;
      }
      if (!ok) continue;
      /* legs source -> R_1 -> ... -> R_k -> m unobstructed */
      vec a = s0;
      for (int j = 1; j <= k + 1 && ok; j++) {
        vec b = j <= k ? R[j] : m;
        if (blocked(T, (int)n_tris, a, b, t_eps)) ok = 0;
        a = b;
      }
      if (!ok) continue;
      (void)F;
      double d = vlen(vsub(m, nodes[q].img));
      if (d < 1e-9) continue;
      for (int b = 0; b < n_bands; b++) {
        double damp = alpha && alpha[b] != 0.0 ? pow(10.0, -alpha[b] * d / 10.0) : 1.0;
        I[mi * n_bands + b] += nodes[q].w[b] * damp / (4.0 * IS_PI * d * d);
      }
      cnt[mi]++;
      if (nlog < log_cap) {
        log_mic[nlog] = (int32_t)mi;
        log_order[nlog] = k;
        log_d[nlog] = d;
        nlog++;
      }
    }
  }
  if (log_n) *log_n = nlog;
  free(nodes);
  free(T);
  return n;
}
