/*
 * CPU oracle for the residency-octree ray caster.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA library; the two meet only through the
 * seeded inputs of the synth package and the documented data layouts.
 *
 * What it computes, and the passage each part follows:
 *
 *  O-a  Residency and culling words of every octree node (Sec. 3 "Fully vs.
 *       partially mapped", Sec. 5.2 node contents and INVALID / UNKNOWN,
 *       Sec. 5.3 metadata for a volume region, Sec. 7 node layout): mask bit
 *       l of a node is set iff some resident brick of that level and channel
 *       overlaps the node's box with positive volume (by scanning bricks).
 *       The value range of a node: a leaf's is the range the data source
 *       gave for it; an inner node's is the hull of its children's when all
 *       of them are valid, else the range the data source gave for the node
 *       itself; without either the node is INVALID for the channel, and its
 *       word names the depth of the nearest ancestor that is valid for the
 *       channel (or UNKNOWN when none is).
 *
 *  O-b  Per-pixel ray march following Sec. 6.1 (Algorithm 1 and the
 *       multi-channel walk that keeps one channel index and stays in the node
 *       when a channel terminates), Sec. 6.2 (per-channel level range) and
 *       Sec. 7 (every visible channel evaluated at every sample), taking every
 *       decision in IEEE binary32 with the operation order of the contract
 *       (positions, level choice, skips, early ray termination), so that the
 *       decisions, requests, usage and the float image can be compared bit
 *       for bit.
 *
 *  O-c  The same march recomputed in binary64 along O-b's decisions: ray
 *       positions, trilinear values, transfer function, opacity correction
 *       with pow(), compositing.
 *
 * Readings of points the paper leaves open are those written in the design
 * notes (apron, quantisation, bucket occupancy, substitution order,
 * compositing, thresholds); each is restated below where it is used.
 * Built with -ffp-contract=off: the only fused multiply-adds are the fmaf()
 * calls written out.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_EXPORT __attribute__((visibility("default")))
#define OR_MAXC 16
#define OR_MAXL 16
#define OR_MAX_SAMPLES (1 << 24)

/* ------------------------------------------------------------------ inputs */

typedef struct {
  int32_t dims[3];          /* level-0 voxels per axis (x, y, z) */
  float spacing[3];         /* physical size of a level-0 voxel */
  int32_t m, k, B, bpv;     /* channels, levels, brick edge, bytes per voxel (1|2) */
  int32_t leaf[3];          /* leaf extent in level-0 voxels (powers of two, <= B) */
  const void *const *levels;/* m*k dense arrays, index c*k + l, [z][y][x] */
  const uint8_t *resident;  /* oracle brick layout (or_brick_index): 1 = resident */
  const int64_t *leaf_min;  /* m * n_leaves raw values, -1 = no metadata */
  const int64_t *leaf_max;
  /* voxel source used when levels is NULL (volumes too large to hold
   * densely): value of level-l voxel (x, y, z) of channel c, coordinates
   * already clamped to the level */
  uint32_t (*voxel_fn)(void *ctx, int c, int l, int64_t x, int64_t y, int64_t z);
  void *voxel_ctx;
  /* sample format of the brick cache: 0 = raw values, binary32 lerps;
   * 1 = binary16, 2 = bfloat16 (see trilinear_lp) */
  int32_t sample_format;
  /* ranges the data source gave for inner nodes: m * n_nodes raw values by
   * node index (depth-major), -1 = none; entries of leaves are not read.
   * NULL: none given. */
  const int64_t *node_min;
  const int64_t *node_max;
  /* downsampling between levels (Sec. 8: anisotropic downsampling ratios):
   * bit a of keep_axes[l] set = axis a keeps its resolution from level l to
   * level l + 1; clear = halved.  All zero: every level halves every axis. */
  int32_t keep_axes[OR_MAXL];
} or_volume;

typedef struct {
  int32_t W, H, perspective;
  float eye[3], fwd[3], right[3], up[3];
  float tan_x, tan_y, pixel;
  float dt;                 /* lattice spacing, physical units */
  float lod_t[OR_MAXL];     /* lod thresholds, index 1..k-1 */
  int32_t lmin[OR_MAXC], lmax[OR_MAXC];
  int32_t start_depth;
  int32_t skip;             /* 1: empty-space skipping on */
  float ert;                /* early ray termination threshold on T; 0 = off */
  float tf_lo[OR_MAXC], tf_scale[OR_MAXC];
  const float *lut;         /* m * 256 * 4 */
} or_params;

typedef struct {
  float *rgba32;            /* n*4 */
  double *rgba64;           /* n*4 */
  uint32_t *hash, *n_eval, *i_end, *n_bs;
  uint8_t *req;             /* oracle brick layout */
  uint8_t *used;            /* oracle brick layout */
  uint8_t *node_req;        /* n_nodes * m */
} or_outputs;

/* ---------------------------------------------------------------- geometry */

/* Level geometry per axis.  lvl_shift: log2 of the level-l voxel extent
 * along axis a in level-0 voxels (the number of halvings so far); lvl_dim:
 * voxels along axis a at level l (a halving rounds up: ceil(d / 2)). */
static int lvl_shift(const or_volume *v, int l, int a) {
  int s = 0;
  for (int i = 0; i < l; ++i) s += !((v->keep_axes[i] >> a) & 1);
  return s;
}

static int lvl_dim(const or_volume *v, int l, int a) {
  int d = v->dims[a];
  for (int i = 0; i < l; ++i)
    if (!((v->keep_axes[i] >> a) & 1)) d = (d + 1) / 2;
  return d;
}

/* Step exponent of level l (Sec. 6.1: the sampling distance may grow with
 * the level a brick comes from): the largest s with 2^s times the smallest
 * level-0 spacing at most the smallest physical extent of a level-l voxel.
 * With every axis halved per level this is l. */
static int lvl_step(const or_volume *v, int l) {
  double s0 = INFINITY, sl = INFINITY;
  for (int a = 0; a < 3; ++a) {
    s0 = fmin(s0, (double)v->spacing[a]);
    sl = fmin(sl, (double)v->spacing[a] * ldexp(1.0, lvl_shift(v, l, a)));
  }
  int s = 0;
  while (ldexp(s0, s + 1) <= sl) ++s;
  return s;
}

static int nbricks(const or_volume *v, int l, int a) {
  return (lvl_dim(v, l, a) + v->B - 1) / v->B;
}

/* Geometry tables computed once per call from the volume description:
 * per-level dims and bricks per axis, the offset of each (c, l) brick table,
 * the octree depth and the first node of each depth. */
typedef struct {
  int ld[OR_MAXL][3], nb[OR_MAXL][3];
  int64_t pt_off[OR_MAXC * OR_MAXL + 1];
  int D;
  int64_t nn[32][3], node_off[33];
} or_geom;

static int geom_depth(const or_volume *v);

static void make_geom(const or_volume *v, or_geom *g) {
  memset(g, 0, sizeof(*g));
  for (int l = 0; l < v->k; ++l)
    for (int a = 0; a < 3; ++a) {
      g->ld[l][a] = lvl_dim(v, l, a);
      g->nb[l][a] = (g->ld[l][a] + v->B - 1) / v->B;
    }
  int64_t off = 0;
  for (int c = 0; c < v->m; ++c)
    for (int l = 0; l < v->k; ++l) {
      g->pt_off[c * v->k + l] = off;
      off += (int64_t)g->nb[l][0] * g->nb[l][1] * g->nb[l][2];
    }
  g->pt_off[v->m * v->k] = off;
  g->D = geom_depth(v);
  int64_t noff = 0;
  for (int d = 0; d <= g->D; ++d) {
    g->node_off[d] = noff;
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      int64_t e = (int64_t)v->leaf[a] << (g->D - d);
      g->nn[d][a] = (v->dims[a] + e - 1) / e;
      cnt *= g->nn[d][a];
    }
    noff += cnt;
  }
  g->node_off[g->D + 1] = noff;
}

/* oracle brick layout: (c, l) tables in order c*k + l, each [bz][by][bx] */
static int64_t brick_index_g(const or_volume *v, const or_geom *g, int c, int l, int bx, int by, int bz) {
  if (c < 0 || c >= v->m || l < 0 || l >= v->k) return -1;
  if (bx < 0 || by < 0 || bz < 0 || bx >= g->nb[l][0] || by >= g->nb[l][1] || bz >= g->nb[l][2]) return -1;
  return g->pt_off[c * v->k + l] + ((int64_t)bz * g->nb[l][1] + by) * g->nb[l][0] + bx;
}

OR_EXPORT int64_t or_brick_index(const or_volume *v, int c, int l, int bx, int by, int bz) {
  or_geom g;
  make_geom(v, &g);
  return brick_index_g(v, &g, c, l, bx, by, bz);
}

OR_EXPORT int64_t or_brick_count(const or_volume *v) {
  int64_t n = 0;
  for (int c = 0; c < v->m; ++c)
    for (int l = 0; l < v->k; ++l) n += (int64_t)nbricks(v, l, 0) * nbricks(v, l, 1) * nbricks(v, l, 2);
  return n;
}

/* The 32-bit brick ID of Sec. 7: page-table id c*k + l in the top 8 bits,
 * then 8 bits each of z, y, x brick offset. */
static uint32_t brick_id(const or_volume *v, int c, int l, int bx, int by, int bz) {
  return ((uint32_t)(c * v->k + l) << 24) | ((uint32_t)bz << 16) | ((uint32_t)by << 8) | (uint32_t)bx;
}

/* Octree depth: the smallest D with 2^D leaves covering every axis. */
static int geom_depth(const or_volume *v) {
  int D = 0;
  for (int a = 0; a < 3; ++a) {
    int nl = (v->dims[a] + v->leaf[a] - 1) / v->leaf[a];
    int d = 0;
    while ((1 << d) < nl) ++d;
    if (d > D) D = d;
  }
  return D;
}

OR_EXPORT int or_depth(const or_volume *v) { return geom_depth(v); }

/* node extent at depth d, per axis, in level-0 voxels */
static int64_t node_ext(const or_volume *v, int D, int d, int a) { return (int64_t)v->leaf[a] << (D - d); }

static int64_t nodes_axis(const or_volume *v, int D, int d, int a) {
  int64_t e = node_ext(v, D, d, a);
  return (v->dims[a] + e - 1) / e;
}

/* pointerless full octree: depth-major, then z, y, x */
static int64_t node_offset(const or_volume *v, int D, int d) {
  int64_t off = 0;
  for (int dd = 0; dd < d; ++dd) off += nodes_axis(v, D, dd, 0) * nodes_axis(v, D, dd, 1) * nodes_axis(v, D, dd, 2);
  return off;
}

OR_EXPORT int64_t or_node_count(const or_volume *v) {
  int D = or_depth(v);
  return node_offset(v, D, D + 1);
}

/* --------------------------------------------------- O-a: node words */

typedef struct {
  const or_volume *v;
  int D;
  uint32_t *words;
  or_geom g;
} oa_ctx;

static void oa_node(const oa_ctx *x, int d, int64_t jx, int64_t jy, int64_t jz) {
  const or_volume *v = x->v;
  int D = x->D;
  int64_t j3[3] = {jx, jy, jz}, lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    int64_t e = node_ext(v, D, d, a);
    lo[a] = j3[a] * e;
    hi[a] = (j3[a] + 1) * e;
    if (hi[a] > v->dims[a]) hi[a] = v->dims[a];
  }
  int64_t nidx = x->g.node_off[d] + (jz * x->g.nn[d][1] + jy) * x->g.nn[d][0] + jx;
  int64_t nl[3], llo[3], lhi[3];
  for (int a = 0; a < 3; ++a) {
    nl[a] = (v->dims[a] + v->leaf[a] - 1) / v->leaf[a];
    llo[a] = j3[a] << (D - d);
    lhi[a] = (j3[a] + 1) << (D - d);
    if (lhi[a] > nl[a]) lhi[a] = nl[a];
  }
  int64_t nleaves = nl[0] * nl[1] * nl[2];
  for (int c = 0; c < v->m; ++c) {
    /* partial mapping, by definition: any resident brick of (c, l) whose box
     * [b*B*2^s, (b+1)*B*2^s) per axis (s the level's shift along the axis)
     * meets the node box with positive volume */
    uint32_t mask = 0;
    for (int l = 0; l < v->k; ++l) {
      int64_t b0[3], b1[3];
      for (int a = 0; a < 3; ++a) {
        int64_t BL = (int64_t)v->B << lvl_shift(v, l, a);
        b0[a] = lo[a] / BL;
        b1[a] = (hi[a] - 1) / BL;
      }
      int found = 0;
      for (int64_t bz = b0[2]; bz <= b1[2] && !found; ++bz)
        for (int64_t by = b0[1]; by <= b1[1] && !found; ++by)
          for (int64_t bx = b0[0]; bx <= b1[0] && !found; ++bx) {
            int64_t bi = brick_index_g(v, &x->g, c, l, (int)bx, (int)by, (int)bz);
            if (bi >= 0 && v->resident[bi]) found = 1;
          }
      if (found) mask |= 1u << l;
    }
    x->words[nidx * v->m + c] = mask;   /* the range bits are filled in by or_node_words */
  }
  (void)nleaves; (void)llo; (void)lhi;
}

typedef struct { oa_ctx *x; int64_t n; int64_t next; pthread_mutex_t mu; } oa_pool;

static int or_nthreads = 0;
OR_EXPORT void or_set_threads(int n) { or_nthreads = n; }
static int threads_to_use(void) {
  if (or_nthreads > 0) return or_nthreads;
  long v = sysconf(_SC_NPROCESSORS_ONLN);
  return v > 0 ? (int)(v > 64 ? 64 : v) : 1;
}
OR_EXPORT int or_threads_used(void) { return threads_to_use(); }

static void oa_by_index(oa_ctx *x, int64_t g) {
  const or_volume *v = x->v;
  int D = x->D;
  for (int d = 0; d <= D; ++d) {
    int64_t nx = x->g.nn[d][0], ny = x->g.nn[d][1], nz = x->g.nn[d][2];
    (void)v;
    if (g < nx * ny * nz) {
      oa_node(x, d, g % nx, (g / nx) % ny, g / (nx * ny));
      return;
    }
    g -= nx * ny * nz;
  }
}

static void *oa_worker(void *arg) {
  oa_pool *p = (oa_pool *)arg;
  for (;;) {
    pthread_mutex_lock(&p->mu);
    int64_t lo = p->next;
    p->next += 64;
    pthread_mutex_unlock(&p->mu);
    if (lo >= p->n) break;
    for (int64_t g = lo; g < lo + 64 && g < p->n; ++g) oa_by_index(p->x, g);
  }
  return NULL;
}

/* INVALID words: min8 = 255 and max8 = the depth of the nearest valid
 * ancestor, or OR_UNKNOWN when no ancestor is valid (both below 255, so
 * min8 > max8 marks INVALID). */
#define OR_UNKNOWN 254u

/* Value ranges of every node and channel from the data source's ranges
 * (leaves, and inner nodes where given), depth by depth from the leaves up:
 * a node is valid if all its children are (range = their hull) or if it was
 * given a range; then, from the root down, every INVALID node gets the depth
 * of its nearest valid ancestor. */
static int oa_ranges(const or_volume *v, const oa_ctx *x, uint32_t *words) {
  const int m = v->m, D = x->D;
  const int64_t n_nodes = x->g.node_off[D + 1];
  int64_t *mn = (int64_t *)malloc((size_t)n_nodes * m * sizeof(int64_t));
  int64_t *mx = (int64_t *)malloc((size_t)n_nodes * m * sizeof(int64_t));
  uint8_t *ptr = (uint8_t *)malloc((size_t)n_nodes * m);
  if (!mn || !mx || !ptr) { free(mn); free(mx); free(ptr); return -1; }
  /* leaves: the given ranges (mn = -1: invalid) */
  for (int c = 0; c < m; ++c)
    for (int64_t li = 0; li < n_nodes - x->g.node_off[D]; ++li) {
      int64_t a = v->leaf_min[(int64_t)c * (n_nodes - x->g.node_off[D]) + li];
      int64_t b = v->leaf_max[(int64_t)c * (n_nodes - x->g.node_off[D]) + li];
      int64_t n = x->g.node_off[D] + li;
      mn[n * m + c] = (a < 0 || b < 0) ? -1 : a;
      mx[n * m + c] = (a < 0 || b < 0) ? -1 : b;
    }
  /* inner nodes, deepest first */
  for (int d = D - 1; d >= 0; --d) {
    const int64_t *nn = x->g.nn[d], *nc = x->g.nn[d + 1];
    for (int64_t jz = 0; jz < nn[2]; ++jz)
      for (int64_t jy = 0; jy < nn[1]; ++jy)
        for (int64_t jx = 0; jx < nn[0]; ++jx) {
          int64_t n = x->g.node_off[d] + (jz * nn[1] + jy) * nn[0] + jx;
          for (int c = 0; c < m; ++c) {
            int all_valid = 1;
            int64_t lo = INT64_MAX, hi = -1;
            for (int cz = 0; cz < 2; ++cz)
              for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                  int64_t kx = 2 * jx + cx, ky = 2 * jy + cy, kz = 2 * jz + cz;
                  if (kx >= nc[0] || ky >= nc[1] || kz >= nc[2]) continue;
                  int64_t ch = x->g.node_off[d + 1] + (kz * nc[1] + ky) * nc[0] + kx;
                  if (mn[ch * m + c] < 0) { all_valid = 0; continue; }
                  if (mn[ch * m + c] < lo) lo = mn[ch * m + c];
                  if (mx[ch * m + c] > hi) hi = mx[ch * m + c];
                }
            if (!all_valid) {
              int64_t a = v->node_min ? v->node_min[(int64_t)c * n_nodes + n] : -1;
              int64_t b = v->node_max ? v->node_max[(int64_t)c * n_nodes + n] : -1;
              if (a >= 0 && b >= 0) { lo = a; hi = b; }
              else { lo = -1; hi = -1; }
            }
            mn[n * m + c] = lo;
            mx[n * m + c] = hi;
          }
        }
  }
  /* pointers of INVALID nodes, from the root down */
  for (int d = 0; d <= D; ++d) {
    const int64_t *nn = x->g.nn[d];
    for (int64_t jz = 0; jz < nn[2]; ++jz)
      for (int64_t jy = 0; jy < nn[1]; ++jy)
        for (int64_t jx = 0; jx < nn[0]; ++jx) {
          int64_t n = x->g.node_off[d] + (jz * nn[1] + jy) * nn[0] + jx;
          int64_t par = d > 0 ? x->g.node_off[d - 1] + ((jz / 2) * x->g.nn[d - 1][1] + jy / 2) * x->g.nn[d - 1][0] + jx / 2 : -1;
          for (int c = 0; c < m; ++c) {
            if (d == 0) ptr[n * m + c] = (uint8_t)OR_UNKNOWN;
            else ptr[n * m + c] = mn[par * m + c] >= 0 ? (uint8_t)(d - 1) : ptr[par * m + c];
          }
        }
  }
  for (int64_t n = 0; n < n_nodes; ++n)
    for (int c = 0; c < m; ++c) {
      uint32_t min8, max8;
      int64_t a = mn[n * m + c], b = mx[n * m + c];
      if (a < 0) {
        min8 = 255; max8 = ptr[n * m + c];
      } else if (v->bpv == 1) {
        min8 = (uint32_t)a; max8 = (uint32_t)b;
      } else {                  /* 16-bit data: 8-bit buckets of 256 raw values */
        min8 = (uint32_t)(a >> 8); max8 = (uint32_t)(b >> 8);
      }
      words[n * m + c] |= (min8 << 16) | (max8 << 24);
    }
  free(mn); free(mx); free(ptr);
  return 0;
}

/* Residency and culling word of every node and channel: words[node*m + c] =
 * mask[15:0] | min8[23:16] | max8[31:24] (Sec. 7), INVALID = min8 > max8
 * (then max8 = depth of the nearest valid ancestor, or OR_UNKNOWN). */
OR_EXPORT int or_node_words(const or_volume *v, uint32_t *words) {
  if (v->m < 1 || v->m > OR_MAXC || v->k < 1 || v->k > OR_MAXL || (v->bpv != 1 && v->bpv != 2) ||
      v->sample_format < 0 || v->sample_format > 2)
    return -1;
  oa_ctx x;
  x.v = v;
  x.D = or_depth(v);
  x.words = words;
  make_geom(v, &x.g);
  oa_pool p = {&x, or_node_count(v), 0};
  pthread_mutex_init(&p.mu, NULL);
  int nt = threads_to_use();
  pthread_t th[64];
  for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, oa_worker, &p);
  for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&p.mu);
  return oa_ranges(v, &x, words);
}

/* ----------------------------------------------------- O-b / O-c: march */

enum { ST_EMPTY = 0, ST_HOMOG = 1, ST_UNMAPPED = 2, ST_BRICK = 3, ST_INVALID = 4 };

typedef struct {
  const or_volume *v;
  const uint32_t *words;
  const or_params *p;
  int D;
  int sdepth[OR_MAXL];
  uint8_t occ[OR_MAXC][256];     /* bucket occupancy per channel */
  float dimm[3];                 /* largest float below each level-0 dim */
  int64_t nleaves;
  or_geom g;
} ob_frame;

/* Transfer-function coordinate of a raw value, binary32:
 * clamp((v - lo) * scale, 0, 255). */
static float tf_coord32(const or_params *p, int c, float val) {
  float t = val - p->tf_lo[c];
  float xq = t * p->tf_scale[c];
  return fminf(fmaxf(xq, 0.0f), 255.0f);
}

/* Bucket q of channel c is occupied iff the transfer function can give a
 * non-zero opacity to some raw value of the bucket (the TF-dependent side of
 * the TF-independent min/max test of Sec. 5.2): with X the binary32 TF
 * coordinate, any knot in [floor(min X), ceil(max X)] over the bucket's
 * end points with alpha > 0. */
static void frame_occupancy(ob_frame *f) {
  const or_volume *v = f->v;
  const or_params *p = f->p;
  for (int c = 0; c < v->m; ++c)
    for (int q = 0; q < 256; ++q) {
      float vlo, vhi;
      if (v->bpv == 1) { vlo = (float)q; vhi = (float)q; }
      else { vlo = (float)(q * 256); vhi = (float)(q * 256 + 255); }
      float xa = tf_coord32(p, c, vlo), xb = tf_coord32(p, c, vhi);
      float x0 = fminf(xa, xb), x1 = fmaxf(xa, xb);
      int j0 = (int)floorf(x0), j1 = (int)ceilf(x1);
      if (j1 > 255) j1 = 255;
      int occ = 0;
      for (int j = j0; j <= j1; ++j)
        if (p->lut[((size_t)c * 256 + j) * 4 + 3] > 0.0f) occ = 1;
      f->occ[c][q] = (uint8_t)occ;
    }
}

/* Traversal depth for a step of dt*2^l (Algorithm 1, chooseTraversalDepth):
 * the deepest depth whose nodes are, along every axis, at least one step
 * long physically, so that a skip is never shorter than a step. */
static void frame_sdepth(ob_frame *f) {
  const or_volume *v = f->v;
  for (int l = 0; l < OR_MAXL; ++l) {
    double step = (double)f->p->dt * ldexp(1.0, lvl_step(v, l));
    int best = 0;
    for (int d = 0; d <= f->D; ++d) {
      double mn = INFINITY;
      for (int a = 0; a < 3; ++a) {
        double e = (double)node_ext(v, f->D, d, a) * (double)v->spacing[a];
        if (e < mn) mn = e;
      }
      if (mn >= step) best = d;
    }
    f->sdepth[l] = best;
  }
}

typedef struct {
  float o[3], d[3];   /* voxel-space origin and direction (binary32) */
  float t0, t1;
  int hit;
} ray32;

/* Pixel-centre ray and its slab interval, binary32, in the contract's
 * operation order; t is physical distance along a unit direction. */
static ray32 make_ray32(const ob_frame *f, int px, int py) {
  const or_params *p = f->p;
  const or_volume *v = f->v;
  ray32 r;
  float o[3], d[3];
  float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  if (p->perspective) {
    float u = fx / (float)p->W, w = fy / (float)p->H;
    float a = (2.0f * u - 1.0f) * p->tan_x;
    float b = (1.0f - 2.0f * w) * p->tan_y;
    float dd[3];
    for (int k = 0; k < 3; ++k) dd[k] = fmaf(b, p->up[k], fmaf(a, p->right[k], p->fwd[k]));
    float n2 = fmaf(dd[2], dd[2], fmaf(dd[1], dd[1], dd[0] * dd[0]));
    float len = sqrtf(n2);
    for (int k = 0; k < 3; ++k) { o[k] = p->eye[k]; d[k] = dd[k] / len; }
  } else {
    float a = (fx - 0.5f * (float)p->W) * p->pixel;
    float b = (0.5f * (float)p->H - fy) * p->pixel;
    for (int k = 0; k < 3; ++k) { o[k] = fmaf(b, p->up[k], fmaf(a, p->right[k], p->eye[k])); d[k] = p->fwd[k]; }
  }
  float tmin = -INFINITY, tmax = INFINITY;
  r.hit = 1;
  for (int k = 0; k < 3; ++k) {
    r.o[k] = o[k] / v->spacing[k];
    r.d[k] = d[k] / v->spacing[k];
    if (r.d[k] != 0.0f) {
      float ta = (0.0f - r.o[k]) / r.d[k];
      float tb = ((float)v->dims[k] - r.o[k]) / r.d[k];
      tmin = fmaxf(tmin, fminf(ta, tb));
      tmax = fminf(tmax, fmaxf(ta, tb));
    } else if (r.o[k] < 0.0f || r.o[k] >= (float)v->dims[k]) {
      r.hit = 0;
    }
  }
  r.t0 = fmaxf(tmin, 0.0f);
  r.t1 = tmax;
  if (!(r.t0 < r.t1)) r.hit = 0;
  return r;
}

static float sample_t(const ray32 *r, const or_params *p, int64_t i) { return fmaf((float)i, p->dt, r->t0); }

static void sample_pos(const ob_frame *f, const ray32 *r, float t, float x[3]) {
  for (int k = 0; k < 3; ++k) x[k] = fminf(fmaxf(fmaf(t, r->d[k], r->o[k]), 0.0f), f->dimm[k]);
}

/* node coordinates at depth d of a level-0 position (exact power-of-two scaling) */
static void node_coords(const ob_frame *f, int d, const float x[3], int64_t j[3]) {
  for (int a = 0; a < 3; ++a) {
    float inv = ldexpf(1.0f, -(int)(__builtin_ctzll((unsigned long long)node_ext(f->v, f->D, d, a))));
    j[a] = (int64_t)(x[a] * inv);
  }
}

static int64_t node_index(const ob_frame *f, int d, const int64_t j[3]) {
  return f->g.node_off[d] + (j[2] * f->g.nn[d][1] + j[1]) * f->g.nn[d][0] + j[0];
}

/* owner brick of a position at level l: floor(x / (B 2^l)) per axis */
static void owner_brick(const ob_frame *f, int l, const float x[3], int b[3]) {
  for (int a = 0; a < 3; ++a) {
    int sh = __builtin_ctz((unsigned)f->v->B) + lvl_shift(f->v, l, a);
    b[a] = (int)(x[a] * ldexpf(1.0f, -sh));
  }
}

/* Per-channel state at one node (Algorithm 1 order: isEmpty, isHomogeneous,
 * isPartiallyMapped).  "Partially mapped" counts the levels the channel may
 * use at this sample: its desired level and every coarser one. */
static int classify(const ob_frame *f, int c, uint32_t w, int ld) {
  uint32_t min8 = (w >> 16) & 0xFFu, max8 = w >> 24;
  if (min8 > max8) return ST_INVALID;
  int any = 0;
  for (uint32_t q = min8; q <= max8; ++q) any |= f->occ[c][q];
  if (!any) return ST_EMPTY;
  if (f->v->bpv == 1 && min8 == max8) return ST_HOMOG;
  uint32_t usable = (w & 0xFFFFu) & ~((1u << ld) - 1u) & ((1u << f->v->k) - 1u);
  if (!usable) return ST_UNMAPPED;
  return ST_BRICK;
}

/* An INVALID word whose channel has a valid ancestor (Sec. 5.2: the pointer
 * to the node in the next lower subdivision level with valid information)
 * is read with that ancestor's range and its own residency mask; other
 * words are returned as they are (UNKNOWN stays INVALID). */
static uint32_t resolve_word(const ob_frame *f, uint32_t w, const float x[3], int c) {
  uint32_t min8 = (w >> 16) & 0xFFu, max8 = w >> 24;
  if (min8 <= max8 || max8 == OR_UNKNOWN) return w;
  int64_t j[3];
  node_coords(f, (int)max8, x, j);
  uint32_t a = f->words[node_index(f, (int)max8, j) * f->v->m + c];
  return (w & 0xFFFFu) | (a & 0xFFFF0000u);
}

static inline uint32_t fnv_word(uint32_t h, uint32_t w) {
  for (int b = 0; b < 4; ++b) { h ^= (w >> (8 * b)) & 0xFFu; h *= 16777619u; }
  return h;
}

static uint32_t voxel(const or_volume *v, int c, int l, int64_t x, int64_t y, int64_t z) {
  int nx = lvl_dim(v, l, 0), ny = lvl_dim(v, l, 1), nz = lvl_dim(v, l, 2);
  if (x > nx - 1) x = nx - 1;
  if (y > ny - 1) y = ny - 1;
  if (z > nz - 1) z = nz - 1;
  if (!v->levels) return v->voxel_fn(v->voxel_ctx, c, l, x, y, z);
  int64_t idx = (z * ny + y) * nx + x;
  const void *a = v->levels[c * v->k + l];
  return v->bpv == 1 ? ((const uint8_t *)a)[idx] : ((const uint16_t *)a)[idx];
}

/* Trilinear value at level l, binary32, lerps along x, then y, then z, each
 * fmaf(f, b - a, a), corners clamped to the level (clamp to edge). */
static float trilinear32(const or_volume *v, int c, int l, const float x[3]) {
  float u[3], fr[3];
  int64_t i0[3];
  for (int a = 0; a < 3; ++a) {
    float xl = ldexpf(x[a], -lvl_shift(v, l, a));
    float w = xl - 0.5f;
    w = fminf(fmaxf(w, 0.0f), (float)(lvl_dim(v, l, a) - 1));
    u[a] = w;
    i0[a] = (int64_t)w;
    fr[a] = w - (float)i0[a];
  }
  (void)u;
  float cv[2][2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) cv[dz][dy][dx] = (float)voxel(v, c, l, i0[0] + dx, i0[1] + dy, i0[2] + dz);
  float c00 = fmaf(fr[0], cv[0][0][1] - cv[0][0][0], cv[0][0][0]);
  float c10 = fmaf(fr[0], cv[0][1][1] - cv[0][1][0], cv[0][1][0]);
  float c01 = fmaf(fr[0], cv[1][0][1] - cv[1][0][0], cv[1][0][0]);
  float c11 = fmaf(fr[0], cv[1][1][1] - cv[1][1][0], cv[1][1][0]);
  float c0 = fmaf(fr[1], c10 - c00, c00);
  float c1 = fmaf(fr[1], c11 - c01, c01);
  return fmaf(fr[2], c1 - c0, c0);
}

/* Round-to-nearest-even of x to a binary format with p significant bits
 * whose smallest normal exponent is emin (gradual underflow below it):
 * binary16 p = 11, emin = -14; bfloat16 p = 8, emin = -126.  x is finite
 * and within the format's range here (values and weights lie in [-1, 1]).
 * The quantum is the unit in the last place of x's binade, so x / quantum
 * is exact and nearbyint rounds it to an integer, ties to even. */
static double fmt_quantum(double x, int p, int emin) {
  int e;
  frexp(x, &e);             /* |x| in [2^(e-1), 2^e) */
  int lead = e - 1;
  if (lead < emin) lead = emin;
  return ldexp(1.0, lead - (p - 1));
}

static double round_fmt(double x, int fmt) {
  const int p = fmt == 1 ? 11 : 8, emin = fmt == 1 ? -14 : -126;
  if (x == 0.0) return x;
  const double q = fmt_quantum(x, p, emin);
  return nearbyint(x / q) * q;
}

/* The format's rounding of an exact value given as hi + lo, hi = fl(hi + lo)
 * (an error-free sum).  Only when hi is exactly halfway between two format
 * values can lo change the result: the exact value then lies off the tie,
 * on lo's side.  Anywhere else hi and hi + lo round alike. */
static double round_fmt_pair(double hi, double lo, int fmt) {
  const int p = fmt == 1 ? 11 : 8, emin = fmt == 1 ? -14 : -126;
  if (hi == 0.0) return round_fmt(lo, fmt);
  const double q = fmt_quantum(hi, p, emin);
  const double r = hi / q, fl = floor(r);
  if (r - fl == 0.5 && lo != 0.0) return (lo > 0.0 ? fl + 1.0 : fl) * q;
  return nearbyint(r) * q;
}

/* a + b as an exact pair (Knuth's two-sum). */
static void two_sum(double a, double b, double *hi, double *lo) {
  const double s = a + b, bb = s - a;
  *hi = s;
  *lo = (a - (s - bb)) + (b - bb);
}

/* One lerp step in the format: d = q(b - a), then q(f * d + a) with one
 * rounding (a fused multiply-add in the format).  f * d is exact in a
 * double (two format values of at most 11 bits each). */
static double lerp_fmt(double f, double a, double b, int fmt) {
  double hi, lo;
  two_sum(b, -a, &hi, &lo);
  const double d = round_fmt_pair(hi, lo, fmt);
  two_sum(f * d, a, &hi, &lo);
  return round_fmt_pair(hi, lo, fmt);
}

OR_EXPORT double or_round_fmt(double x, int fmt) { return round_fmt(x, fmt); }
OR_EXPORT double or_lerp_fmt(double f, double a, double b, int fmt) { return lerp_fmt(f, a, b, fmt); }

/* Trilinear value at level l in a low-precision sample format (the paper
 * samples 8/16-bit textures and states no arithmetic; this is the reading
 * both sides implement: the cache holds q(v * 2^-S) with S = 8 (u8) or 16 (u16),
 * q = round to the format; the binary32 weights of trilinear32 are rounded
 * to the format; every lerp is lerp_fmt; the result times 2^S is returned
 * in binary32).  Order as in trilinear32: x, then y, then z. */
static float trilinear_lp(const or_volume *v, int c, int l, const float x[3], int fmt) {
  const int S = v->bpv == 1 ? 8 : 16;
  double fr[3];
  int64_t i0[3];
  for (int a = 0; a < 3; ++a) {
    float xl = ldexpf(x[a], -lvl_shift(v, l, a));
    float w = xl - 0.5f;
    w = fminf(fmaxf(w, 0.0f), (float)(lvl_dim(v, l, a) - 1));
    i0[a] = (int64_t)w;
    fr[a] = round_fmt((double)(w - (float)i0[a]), fmt);
  }
  double cv[2][2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        cv[dz][dy][dx] = round_fmt(ldexp((double)voxel(v, c, l, i0[0] + dx, i0[1] + dy, i0[2] + dz), -S), fmt);
  double c00 = lerp_fmt(fr[0], cv[0][0][0], cv[0][0][1], fmt);
  double c10 = lerp_fmt(fr[0], cv[0][1][0], cv[0][1][1], fmt);
  double c01 = lerp_fmt(fr[0], cv[1][0][0], cv[1][0][1], fmt);
  double c11 = lerp_fmt(fr[0], cv[1][1][0], cv[1][1][1], fmt);
  double c0 = lerp_fmt(fr[1], c00, c10, fmt);
  double c1 = lerp_fmt(fr[1], c01, c11, fmt);
  double cc = lerp_fmt(fr[2], c0, c1, fmt);
  return ldexpf((float)cc, S);
}

/* Same value in binary64 at a binary64 position. */
static double trilinear64(const or_volume *v, int c, int l, const double x[3]) {
  double fr[3];
  int64_t i0[3];
  for (int a = 0; a < 3; ++a) {
    double w = ldexp(x[a], -lvl_shift(v, l, a)) - 0.5;
    double hi = (double)(lvl_dim(v, l, a) - 1);
    w = w < 0.0 ? 0.0 : (w > hi ? hi : w);
    i0[a] = (int64_t)floor(w);
    fr[a] = w - (double)i0[a];
  }
  double cv[2][2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) cv[dz][dy][dx] = (double)voxel(v, c, l, i0[0] + dx, i0[1] + dy, i0[2] + dz);
  double c00 = cv[0][0][0] + fr[0] * (cv[0][0][1] - cv[0][0][0]);
  double c10 = cv[0][1][0] + fr[0] * (cv[0][1][1] - cv[0][1][0]);
  double c01 = cv[1][0][0] + fr[0] * (cv[1][0][1] - cv[1][0][0]);
  double c11 = cv[1][1][0] + fr[0] * (cv[1][1][1] - cv[1][1][0]);
  double c0 = c00 + fr[1] * (c10 - c00);
  double c1 = c01 + fr[1] * (c11 - c01);
  return c0 + fr[2] * (c1 - c0);
}

/* Transfer function: 256 RGBA knots, linear between knots, binary32. */
static void tf32(const or_params *p, int c, float val, float out[4]) {
  float xq = tf_coord32(p, c, val);
  int j = (int)xq;
  if (j > 254) j = 254;
  float fr = xq - (float)j;
  const float *L = p->lut + ((size_t)c * 256 + j) * 4;
  for (int k = 0; k < 4; ++k) out[k] = fmaf(fr, L[4 + k] - L[k], L[k]);
}

static void tf64(const or_params *p, int c, double val, double out[4]) {
  double xq = (val - (double)p->tf_lo[c]) * (double)p->tf_scale[c];
  xq = xq < 0.0 ? 0.0 : (xq > 255.0 ? 255.0 : xq);
  int j = (int)floor(xq);
  if (j > 254) j = 254;
  double fr = xq - j;
  const float *L = p->lut + ((size_t)c * 256 + j) * 4;
  for (int k = 0; k < 4; ++k) out[k] = (double)L[k] + fr * ((double)L[4 + k] - (double)L[k]);
}

typedef struct {
  uint8_t *req, *used, *node_req;
} flag_set;

typedef struct {
  double o[3], d[3], t0;
} ray64;

/* The same pixel ray in binary64 (used only for the binary64 image). */
static ray64 make_ray64(const ob_frame *f, int px, int py, float t0) {
  const or_params *p = f->p;
  const or_volume *v = f->v;
  ray64 r;
  double o[3], d[3];
  double fx = px + 0.5, fy = py + 0.5;
  if (p->perspective) {
    double a = (2.0 * fx / p->W - 1.0) * p->tan_x, b = (1.0 - 2.0 * fy / p->H) * p->tan_y, n = 0.0;
    for (int k = 0; k < 3; ++k) { d[k] = (double)p->fwd[k] + a * p->right[k] + b * p->up[k]; n += d[k] * d[k]; }
    n = sqrt(n);
    for (int k = 0; k < 3; ++k) { d[k] /= n; o[k] = p->eye[k]; }
  } else {
    double a = (fx - 0.5 * p->W) * p->pixel, b = (0.5 * p->H - fy) * p->pixel;
    for (int k = 0; k < 3; ++k) { o[k] = p->eye[k] + a * p->right[k] + b * p->up[k]; d[k] = p->fwd[k]; }
  }
  for (int k = 0; k < 3; ++k) { r.o[k] = o[k] / v->spacing[k]; r.d[k] = d[k] / v->spacing[k]; }
  r.t0 = (double)t0;   /* the lattice starts at the binary32 entry distance */
  return r;
}

static void march_pixel(const ob_frame *f, int px, int py, int64_t n_out, const or_outputs *out, flag_set *fl) {
  const or_volume *v = f->v;
  const or_params *p = f->p;
  const int m = v->m, k = v->k;
  uint32_t h = 2166136261u, n_eval = 0, n_bs = 0;
  float C[3] = {0, 0, 0}, T = 1.0f;
  double C64[3] = {0, 0, 0}, T64 = 1.0;
  int64_t i = 0;
  ray32 r = make_ray32(f, px, py);
  ray64 r64 = make_ray64(f, px, py, r.t0);
  if (r.hit) {
    for (;;) {
      if (i >= OR_MAX_SAMPLES) break;
      float t = sample_t(&r, p, i);
      if (!(t < r.t1)) break;
      float x[3];
      sample_pos(f, &r, t, x);

      /* desired level per channel (Sec. 6.2): lod from the distance, then the
       * channel's own [lmin, lmax] range */
      int lod = 0;
      for (int l = 1; l < k; ++l) lod += (t >= p->lod_t[l]);
      int ld[OR_MAXC], lmin_used = 99;
      for (int c = 0; c < m; ++c) {
        int l = lod < p->lmin[c] ? p->lmin[c] : lod;
        if (l > p->lmax[c]) l = p->lmax[c];
        ld[c] = l;
        if (l < lmin_used) lmin_used = l;
      }
      int st = f->sdepth[lmin_used];

      /* multi-channel walk of Sec. 6.1: one channel index; a channel that
       * would end the single-channel traversal here (empty, homogeneous, not
       * partially mapped, or at the traversal depth) advances the index and
       * the walk stays in the node; otherwise the walk descends. */
      int d = p->start_depth < st ? p->start_depth : st;
      int ch = 0;
      int64_t jn[3];
      while (ch < m) {
        node_coords(f, d, x, jn);
        uint32_t w = resolve_word(f, f->words[node_index(f, d, jn) * m + ch], x, ch);
        int s = classify(f, ch, w, ld[ch]);
        int terminal = (s == ST_EMPTY || s == ST_HOMOG || s == ST_UNMAPPED) || d == st;
        if (terminal) ++ch;
        else ++d;
      }
      node_coords(f, d, x, jn);
      int64_t node = node_index(f, d, jn);
      int state[OR_MAXC];
      int all_skip = 1;
      uint32_t rw[OR_MAXC];   /* the final node's words, INVALID ones resolved */
      for (int c = 0; c < m; ++c) {
        rw[c] = resolve_word(f, f->words[node * m + c], x, c);
        state[c] = classify(f, c, rw[c], ld[c]);
        if (state[c] != ST_EMPTY && state[c] != ST_UNMAPPED) all_skip = 0;
      }

      /* brick requests for channels with no usable level in this node; node
       * requests (reportNodeRequest) for channels whose own metadata is
       * missing here, unless the ancestor's range already shows the node
       * empty or homogeneous */
      for (int c = 0; c < m; ++c) {
        uint32_t w = f->words[node * m + c];
        int unm = state[c] == ST_UNMAPPED ||
                  (state[c] == ST_INVALID && ((w & 0xFFFFu) & ~((1u << ld[c]) - 1u) & ((1u << k) - 1u)) == 0);
        if (unm) {
          int b[3];
          owner_brick(f, ld[c], x, b);
          fl->req[brick_index_g(v, &f->g, c, ld[c], b[0], b[1], b[2])] = 1;
        }
        int missing = ((w >> 16) & 0xFFu) > (w >> 24);
        if (missing && state[c] != ST_EMPTY && state[c] != ST_HOMOG) fl->node_req[node * m + c] = 1;
      }

      if (all_skip && p->skip) {
        /* skipNode: continue at the first lattice sample outside the node */
        int64_t j = i + 1;
        for (;;) {
          if (j >= OR_MAX_SAMPLES) break;
          float tj = sample_t(&r, p, j);
          if (!(tj < r.t1)) break;
          float xj[3];
          int64_t jj[3];
          sample_pos(f, &r, tj, xj);
          node_coords(f, d, xj, jj);
          if (jj[0] != jn[0] || jj[1] != jn[1] || jj[2] != jn[2]) break;
          ++j;
        }
        h = fnv_word(h, (uint32_t)i);
        h = fnv_word(h, 0xFFFFFFFFu);
        h = fnv_word(h, (uint32_t)d);
        h = fnv_word(h, (uint32_t)j);
        i = j;
        continue;
      }

      /* an evaluated sample: pick each channel's brick (getBrick, and on a
       * miss reportBrickRequest + getAlternativeBrick at the next coarser
       * resident level), then read its value */
      float val[OR_MAXC];
      double val64[OR_MAXC];
      int has[OR_MAXC], lused[OR_MAXC];
      int s_used = 99;
      double x64[3];
      double t64 = r64.t0 + (double)i * (double)p->dt;
      for (int a = 0; a < 3; ++a) {
        double q = r64.o[a] + t64 * r64.d[a];
        double hi = nextafter((double)v->dims[a], 0.0);
        x64[a] = q < 0.0 ? 0.0 : (q > hi ? hi : q);
      }
      for (int c = 0; c < m; ++c) {
        has[c] = 0;
        lused[c] = -1;
        uint32_t w = rw[c];
        int s = state[c];
        if (s == ST_EMPTY || s == ST_UNMAPPED) continue;
        if (s == ST_HOMOG) {
          has[c] = 1;
          val[c] = (float)((w >> 16) & 0xFFu);
          val64[c] = (double)((w >> 16) & 0xFFu);
          h = fnv_word(h, (uint32_t)i); h = fnv_word(h, (uint32_t)c);
          h = fnv_word(h, 0xFFu); h = fnv_word(h, 0xFFFFFFFFu);
          continue;
        }
        /* ST_BRICK, or ST_INVALID with a usable level */
        if (((w & 0xFFFFu) & ~((1u << ld[c]) - 1u) & ((1u << k) - 1u)) == 0) continue;
        int found = -1, fb[3];
        for (int l = ld[c]; l < k; ++l) {
          int b[3];
          owner_brick(f, l, x, b);
          int64_t bi = brick_index_g(v, &f->g, c, l, b[0], b[1], b[2]);
          if (v->resident[bi]) { found = l; fb[0] = b[0]; fb[1] = b[1]; fb[2] = b[2]; break; }
          if (l == ld[c]) fl->req[bi] = 1;   /* the desired brick is missing */
        }
        if (found < 0) continue;            /* nothing resident: no contribution */
        fl->used[brick_index_g(v, &f->g, c, found, fb[0], fb[1], fb[2])] = 1;
        has[c] = 1;
        lused[c] = found;
        if (found < s_used) s_used = found;
        val[c] = v->sample_format ? trilinear_lp(v, c, found, x, v->sample_format) : trilinear32(v, c, found, x);
        val64[c] = trilinear64(v, c, found, x64);
        ++n_bs;
        h = fnv_word(h, (uint32_t)i); h = fnv_word(h, (uint32_t)c);
        h = fnv_word(h, (uint32_t)found); h = fnv_word(h, brick_id(v, c, found, fb[0], fb[1], fb[2]));
      }
      /* adaptive step 2^s: the step exponent of the finest level read */
      int s = lvl_step(v, s_used == 99 ? lmin_used : s_used);

      /* classification + compositing: per-channel TF, opacity corrected for
       * a step of 2^s lattice spacings, additive premultiplied colour,
       * opacities combined as 1 - prod(1 - a'), front to back */
      float col[3] = {0, 0, 0}, trans = 1.0f;
      double col64[3] = {0, 0, 0}, trans64 = 1.0;
      for (int c = 0; c < m; ++c) {
        if (!has[c]) continue;
        float rgba[4];
        tf32(p, c, val[c], rgba);
        float a = fminf(fmaxf(rgba[3], 0.0f), 1.0f);
        float q = 1.0f - a;
        for (int e = 0; e < s; ++e) q = q * q;
        float ap = 1.0f - q;
        for (int k3 = 0; k3 < 3; ++k3) col[k3] = fmaf(ap, rgba[k3], col[k3]);
        trans = trans * q;

        double rg[4];
        tf64(p, c, val64[c], rg);
        double a64 = rg[3] < 0.0 ? 0.0 : (rg[3] > 1.0 ? 1.0 : rg[3]);
        double q64 = pow(1.0 - a64, ldexp(1.0, s));
        for (int k3 = 0; k3 < 3; ++k3) col64[k3] += (1.0 - q64) * rg[k3];
        trans64 *= q64;
      }
      for (int k3 = 0; k3 < 3; ++k3) {
        C[k3] = fmaf(T, col[k3], C[k3]);
        C64[k3] += T64 * col64[k3];
      }
      T = T * trans;
      T64 *= trans64;
      ++n_eval;
      (void)lused;
      if (T < p->ert) break;     /* early ray termination */
      i += (int64_t)1 << s;
    }
  }
  out->rgba32[n_out * 4 + 0] = fminf(C[0], 1.0f);
  out->rgba32[n_out * 4 + 1] = fminf(C[1], 1.0f);
  out->rgba32[n_out * 4 + 2] = fminf(C[2], 1.0f);
  out->rgba32[n_out * 4 + 3] = 1.0f - T;
  for (int k3 = 0; k3 < 3; ++k3) out->rgba64[n_out * 4 + k3] = C64[k3] < 1.0 ? C64[k3] : 1.0;
  out->rgba64[n_out * 4 + 3] = 1.0 - T64;
  out->hash[n_out] = h;
  out->n_eval[n_out] = n_eval;
  out->i_end[n_out] = (uint32_t)i;
  out->n_bs[n_out] = n_bs;
}

typedef struct {
  const ob_frame *f;
  const int32_t *pixels;
  int64_t n;
  const or_outputs *out;
  int64_t next;
  pthread_mutex_t mu;
  int64_t nbricks, nnodes;
  int fail;
} ob_pool;

static void *ob_worker(void *arg) {
  ob_pool *p = (ob_pool *)arg;
  flag_set fl;
  fl.req = (uint8_t *)calloc((size_t)p->nbricks, 1);
  fl.used = (uint8_t *)calloc((size_t)p->nbricks, 1);
  fl.node_req = (uint8_t *)calloc((size_t)(p->nnodes * p->f->v->m), 1);
  if (!fl.req || !fl.used || !fl.node_req) {
    pthread_mutex_lock(&p->mu);
    p->fail = 1;
    pthread_mutex_unlock(&p->mu);
    free(fl.req); free(fl.used); free(fl.node_req);
    return NULL;
  }
  for (;;) {
    pthread_mutex_lock(&p->mu);
    int64_t lo = p->next;
    p->next += 16;
    pthread_mutex_unlock(&p->mu);
    if (lo >= p->n) break;
    for (int64_t q = lo; q < lo + 16 && q < p->n; ++q) march_pixel(p->f, p->pixels[2 * q], p->pixels[2 * q + 1], q, p->out, &fl);
  }
  pthread_mutex_lock(&p->mu);
  for (int64_t b = 0; b < p->nbricks; ++b) { p->out->req[b] |= fl.req[b]; p->out->used[b] |= fl.used[b]; }
  for (int64_t b = 0; b < p->nnodes * p->f->v->m; ++b) p->out->node_req[b] |= fl.node_req[b];
  pthread_mutex_unlock(&p->mu);
  free(fl.req); free(fl.used); free(fl.node_req);
  return NULL;
}

/* Render n_pixels pixels (pixels: n*2 ints (px, py)).  words: O-a table.
 * The flag outputs must be zeroed by the caller; they are OR-ed into. */
OR_EXPORT int or_render(const or_volume *v, const uint32_t *words, const or_params *p, const int32_t *pixels,
                        int64_t n_pixels, const or_outputs *out) {
  if (v->m < 1 || v->m > OR_MAXC || v->k < 1 || v->k > OR_MAXL || (v->bpv != 1 && v->bpv != 2) ||
      v->sample_format < 0 || v->sample_format > 2)
    return -1;
  for (int c = 0; c < v->m; ++c)
    if (p->lmin[c] < 0 || p->lmin[c] > p->lmax[c] || p->lmax[c] >= v->k) return -2;
  if (!(p->dt > 0.0f) || p->W < 1 || p->H < 1) return -3;
  ob_frame *f = (ob_frame *)calloc(1, sizeof(ob_frame));
  if (!f) return -4;
  f->v = v; f->words = words; f->p = p; f->D = or_depth(v);
  make_geom(v, &f->g);
  if (p->start_depth < 0 || p->start_depth > f->D) { free(f); return -5; }
  for (int a = 0; a < 3; ++a) f->dimm[a] = nextafterf((float)v->dims[a], 0.0f);
  frame_occupancy(f);
  frame_sdepth(f);
  ob_pool pool = {f, pixels, n_pixels, out, 0, PTHREAD_MUTEX_INITIALIZER, or_brick_count(v), or_node_count(v), 0};
  int nt = threads_to_use();
  pthread_t th[64];
  for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, ob_worker, &pool);
  for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
  free(f);
  return pool.fail ? -6 : 0;
}

/* Brick IDs (Sec. 7 format) of the set flags of an oracle-layout flag array,
 * in ascending order; returns how many were written (at most cap) and the
 * total count in *total. */
OR_EXPORT int64_t or_flags_to_ids(const or_volume *v, const uint8_t *flags, uint32_t *ids, int64_t cap,
                                  int64_t *total) {
  int64_t n = 0, off = 0;
  for (int c = 0; c < v->m; ++c)
    for (int l = 0; l < v->k; ++l) {
      int nx = nbricks(v, l, 0), ny = nbricks(v, l, 1), nz = nbricks(v, l, 2);
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x, ++off)
            if (flags[off]) {
              if (n < cap) ids[n] = brick_id(v, c, l, x, y, z);
              ++n;
            }
    }
  if (total) *total = n;
  return n < cap ? n : cap;
}

/* exported helpers for tests */
OR_EXPORT uint32_t or_brick_id(const or_volume *v, int c, int l, int bx, int by, int bz) {
  return brick_id(v, c, l, bx, by, bz);
}

OR_EXPORT int or_traversal_depth(const or_volume *v, float dt, int l) {
  or_params p;
  memset(&p, 0, sizeof(p));
  p.dt = dt;
  ob_frame f;
  memset(&f, 0, sizeof(f));
  f.v = v; f.p = &p; f.D = or_depth(v);
  frame_sdepth(&f);
  return (l >= 0 && l < OR_MAXL) ? f.sdepth[l] : -1;
}

OR_EXPORT int or_bucket_occupancy(const or_volume *v, const or_params *p, uint8_t *out /* m*256 */) {
  ob_frame f;
  memset(&f, 0, sizeof(f));
  f.v = v; f.p = p;
  frame_occupancy(&f);
  for (int c = 0; c < v->m; ++c) memcpy(out + 256 * c, f.occ[c], 256);
  return 0;
}
