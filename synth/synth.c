/*
 * Seeded synthetic volume source.
 *
 * This module plays the part of the data source of the paper's system
 * (Sec. 4: a server provides a bricked multi-resolution multi-volume
 * hierarchy, and optionally per-region min/max metadata).  It holds none of
 * the rendering method's arithmetic: it makes voxel values, the coarser
 * resolution levels of the hierarchy, bricks with a one-voxel border, and
 * per-leaf value ranges.  Both the CUDA library's callers and the CPU oracle
 * take their inputs from here.
 *
 * Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), written here from
 * its published definition.
 *
 * Array layout everywhere: x fastest, then y, then z (C order [z][y][x]).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <sched.h>
#include <unistd.h>

#define SY_EXPORT __attribute__((visibility("default")))

/* ---------------------------------------------------------------- random */

static inline uint64_t sy_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

typedef struct { uint64_t s; } sy_rng;

static inline uint64_t sy_next(sy_rng *r) {
  r->s += 0x9E3779B97F4A7C15ull;
  return sy_mix(r->s);
}

/* uniform in [0, 1) with 53 random bits */
static inline double sy_unif(sy_rng *r) { return (double)(sy_next(r) >> 11) * 0x1.0p-53; }

static double sy_normal(sy_rng *r) {
  double u1 = sy_unif(r), u2 = sy_unif(r);
  if (u1 < 1e-300) u1 = 1e-300;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* counter-based noise value in [0, nmax] for one voxel of one channel/level */
SY_EXPORT uint32_t sy_noise(uint64_t seed, uint32_t c, uint32_t l, uint32_t x, uint32_t y, uint32_t z,
                            uint32_t nmax) {
  uint64_t key = ((uint64_t)(c & 0xFF) << 56) ^ ((uint64_t)(l & 0xFF) << 48) ^ ((uint64_t)(z & 0xFFFF) << 32) ^
                 ((uint64_t)(y & 0xFFFF) << 16) ^ (uint64_t)(x & 0xFFFF);
  uint64_t h = sy_mix(sy_mix(seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull) ^ key);
  return (uint32_t)(h % (uint64_t)(nmax + 1u));
}

/* ------------------------------------------------------- parallel helper */

typedef void (*sy_body)(void *ctx, int64_t lo, int64_t hi);
typedef struct { sy_body f; void *ctx; int64_t n, chunk; int64_t next; pthread_mutex_t mu; } sy_pool;

static void *sy_worker(void *arg) {
  sy_pool *p = (sy_pool *)arg;
  for (;;) {
    pthread_mutex_lock(&p->mu);
    int64_t lo = p->next;
    p->next += p->chunk;
    pthread_mutex_unlock(&p->mu);
    if (lo >= p->n) break;
    int64_t hi = lo + p->chunk < p->n ? lo + p->chunk : p->n;
    p->f(p->ctx, lo, hi);
  }
  return NULL;
}

static int sy_threads = 0;
SY_EXPORT void sy_set_threads(int n) { sy_threads = n; }

static void sy_parallel(sy_body f, void *ctx, int64_t n, int64_t chunk) {
  int nt = sy_threads;
  if (nt <= 0) {
    long v = 8;
#ifdef _SC_NPROCESSORS_ONLN
    v = sysconf(_SC_NPROCESSORS_ONLN);
#endif
    nt = v > 0 ? (int)v : 1;
  }
  if (nt > 64) nt = 64;
  if (chunk < 1) chunk = 1;
  if (nt == 1 || n <= chunk) { f(ctx, 0, n); return; }
  sy_pool p = {f, ctx, n, chunk, 0};
  pthread_mutex_init(&p.mu, NULL);
  pthread_t th[64];
  for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, sy_worker, &p);
  for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&p.mu);
}

/* ------------------------------------------------ Gaussian blob volume (u8) */

typedef struct {
  int nx, ny, nz, nb;
  const double *bx, *by, *bz, *bs, *ba;
  uint64_t seed; uint32_t noise_max; uint8_t *out;
} sy_blob_ctx;

static void sy_blob_body(void *vctx, int64_t lo, int64_t hi) {
  sy_blob_ctx *c = (sy_blob_ctx *)vctx;
  for (int64_t z = lo; z < hi; ++z)
    for (int y = 0; y < c->ny; ++y)
      for (int x = 0; x < c->nx; ++x) {
        double px = x + 0.5, py = y + 0.5, pz = (double)z + 0.5, sum = 0.0;
        for (int b = 0; b < c->nb; ++b) {
          double dx = px - c->bx[b], dy = py - c->by[b], dz = pz - c->bz[b];
          double d2 = dx * dx + dy * dy + dz * dz, s = c->bs[b];
          sum += c->ba[b] * exp(-d2 / (2.0 * s * s));
        }
        int64_t v = (int64_t)floor(sum + 0.5) + sy_noise(c->seed, 0, 0, (uint32_t)x, (uint32_t)y, (uint32_t)z, c->noise_max);
        if (v > 255) v = 255;
        c->out[((int64_t)z * c->ny + y) * c->nx + x] = (uint8_t)v;
      }
}

/* Sum of n_blobs isotropic Gaussians (centres uniform in the box, sigma
 * uniform in [s_lo, s_hi], amplitude uniform in [a_lo, a_hi]) rounded to an
 * integer, plus counter-hash noise in [0, noise_max], clamped to 255. */
SY_EXPORT int sy_blobs_u8(uint64_t seed, int nx, int ny, int nz, int n_blobs, double s_lo, double s_hi,
                          double a_lo, double a_hi, uint32_t noise_max, uint8_t *out) {
  if (n_blobs < 0 || n_blobs > 100000 || nx <= 0 || ny <= 0 || nz <= 0) return -1;
  double *p = (double *)malloc(sizeof(double) * 5 * (size_t)(n_blobs > 0 ? n_blobs : 1));
  if (!p) return -2;
  sy_rng r = {seed};
  for (int b = 0; b < n_blobs; ++b) {
    p[b] = sy_unif(&r) * nx;
    p[n_blobs + b] = sy_unif(&r) * ny;
    p[2 * n_blobs + b] = sy_unif(&r) * nz;
    p[3 * n_blobs + b] = s_lo + (s_hi - s_lo) * sy_unif(&r);
    p[4 * n_blobs + b] = a_lo + (a_hi - a_lo) * sy_unif(&r);
  }
  sy_blob_ctx c = {nx, ny, nz, n_blobs, p, p + n_blobs, p + 2 * n_blobs, p + 3 * n_blobs, p + 4 * n_blobs,
                   seed, noise_max, out};
  sy_parallel(sy_blob_body, &c, nz, 1);
  free(p);
  return 0;
}

/* ---------------------------------------------- mean-downsampled level */

typedef struct {
  int bpv; int nx, ny, nz; int ox, oy, oz; const void *in; void *out; int fx, fy, fz;
} sy_down_ctx;

static void sy_down_body(void *vctx, int64_t lo, int64_t hi) {
  sy_down_ctx *c = (sy_down_ctx *)vctx;
  for (int64_t z = lo; z < hi; ++z)
    for (int y = 0; y < c->oy; ++y)
      for (int x = 0; x < c->ox; ++x) {
        uint64_t sum = 0, n = 0;
        for (int dz = 0; dz < c->fz; ++dz)
          for (int dy = 0; dy < c->fy; ++dy)
            for (int dx = 0; dx < c->fx; ++dx) {
              int64_t ix = (int64_t)c->fx * x + dx, iy = (int64_t)c->fy * y + dy, iz = (int64_t)c->fz * z + dz;
              if (ix >= c->nx || iy >= c->ny || iz >= c->nz) continue;
              int64_t idx = (iz * c->ny + iy) * c->nx + ix;
              sum += c->bpv == 1 ? ((const uint8_t *)c->in)[idx] : ((const uint16_t *)c->in)[idx];
              ++n;
            }
        uint64_t v = (sum + n / 2) / n;
        int64_t o = ((int64_t)z * c->oy + y) * c->ox + x;
        if (c->bpv == 1) ((uint8_t *)c->out)[o] = (uint8_t)v;
        else ((uint16_t *)c->out)[o] = (uint16_t)v;
      }
}

/* Next coarser level: each output voxel is the mean of the (up to 8) input
 * voxels it covers, rounded half up.  Bit a of keep set: axis a keeps its
 * resolution (factor 1), else it is halved (factor 2, output ceil(d/2)). */
SY_EXPORT int sy_downsample_axes(int bpv, int nx, int ny, int nz, int keep, const void *in, void *out) {
  if ((bpv != 1 && bpv != 2) || nx <= 0 || ny <= 0 || nz <= 0) return -1;
  const int fx = (keep & 1) ? 1 : 2, fy = (keep & 2) ? 1 : 2, fz = (keep & 4) ? 1 : 2;
  sy_down_ctx c = {bpv, nx, ny, nz, (nx + fx - 1) / fx, (ny + fy - 1) / fy, (nz + fz - 1) / fz, in, out, fx, fy, fz};
  sy_parallel(sy_down_body, &c, c.oz, 1);
  return 0;
}

SY_EXPORT int sy_downsample(int bpv, int nx, int ny, int nz, const void *in, void *out) {
  return sy_downsample_axes(bpv, nx, ny, nz, 0, in, out);
}

/* ---------------------------------------------- bricks with a border */

/* Copy n bricks of edge B from a dense level (dims nx,ny,nz) into (B+2)^3
 * blocks holding voxels b*B-1 .. (b+1)*B per axis, with indices clamped to
 * the level (clamp to edge).  coords: n*3 ints (bx, by, bz). */
SY_EXPORT int sy_bricks_from_dense(int bpv, int nx, int ny, int nz, const void *level, int B, int n,
                                   const int32_t *coords, void *out) {
  if (bpv != 1 && bpv != 2) return -1;
  int64_t E = B + 2, per = E * E * E;
  for (int i = 0; i < n; ++i) {
    int bx = coords[3 * i], by = coords[3 * i + 1], bz = coords[3 * i + 2];
    for (int64_t z = 0; z < E; ++z) {
      int64_t iz = (int64_t)bz * B - 1 + z;
      iz = iz < 0 ? 0 : (iz >= nz ? nz - 1 : iz);
      for (int64_t y = 0; y < E; ++y) {
        int64_t iy = (int64_t)by * B - 1 + y;
        iy = iy < 0 ? 0 : (iy >= ny ? ny - 1 : iy);
        for (int64_t x = 0; x < E; ++x) {
          int64_t ix = (int64_t)bx * B - 1 + x;
          ix = ix < 0 ? 0 : (ix >= nx ? nx - 1 : ix);
          int64_t src = (iz * ny + iy) * nx + ix, dst = i * per + (z * E + y) * E + x;
          if (bpv == 1) ((uint8_t *)out)[dst] = ((const uint8_t *)level)[src];
          else ((uint16_t *)out)[dst] = ((const uint16_t *)level)[src];
        }
      }
    }
  }
  return 0;
}

/* ---------------------------------------------- exact leaf value ranges */

typedef struct {
  int bpv, nx, ny, nz, ex, ey, ez, lx, ly, lz; const void *vol; uint32_t *mn, *mx;
} sy_leaf_ctx;

static void sy_leaf_body(void *vctx, int64_t lo, int64_t hi) {
  sy_leaf_ctx *c = (sy_leaf_ctx *)vctx;
  for (int64_t li = lo; li < hi; ++li) {
    int64_t jx = li % c->lx, jy = (li / c->lx) % c->ly, jz = li / ((int64_t)c->lx * c->ly);
    int64_t x0 = jx * c->ex - 1, x1 = (jx + 1) * c->ex, y0 = jy * c->ey - 1, y1 = (jy + 1) * c->ey;
    int64_t z0 = jz * c->ez - 1, z1 = (jz + 1) * c->ez;
    if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0; if (z0 < 0) z0 = 0;
    if (x1 > c->nx - 1) x1 = c->nx - 1; if (y1 > c->ny - 1) y1 = c->ny - 1; if (z1 > c->nz - 1) z1 = c->nz - 1;
    uint32_t mn = 0xFFFFFFFFu, mx = 0;
    for (int64_t z = z0; z <= z1; ++z)
      for (int64_t y = y0; y <= y1; ++y)
        for (int64_t x = x0; x <= x1; ++x) {
          int64_t idx = (z * c->ny + y) * c->nx + x;
          uint32_t v = c->bpv == 1 ? ((const uint8_t *)c->vol)[idx] : ((const uint16_t *)c->vol)[idx];
          if (v < mn) mn = v;
          if (v > mx) mx = v;
        }
    c->mn[li] = mn;
    c->mx[li] = mx;
  }
}

/* Per-leaf value range of a dense level-0 volume: min/max over the voxels
 * whose trilinear support can reach a sample inside the leaf, i.e. the leaf
 * box [j*e, (j+1)*e) widened by one voxel on each side and clipped.
 * Leaves are enumerated x fastest over ceil(dims/e) per axis. */
SY_EXPORT int sy_leaf_ranges(int bpv, int nx, int ny, int nz, const void *vol, int ex, int ey, int ez,
                             uint32_t *out_min, uint32_t *out_max) {
  if (bpv != 1 && bpv != 2) return -1;
  int lx = (nx + ex - 1) / ex, ly = (ny + ey - 1) / ey, lz = (nz + ez - 1) / ez;
  sy_leaf_ctx c = {bpv, nx, ny, nz, ex, ey, ez, lx, ly, lz, vol, out_min, out_max};
  sy_parallel(sy_leaf_body, &c, (int64_t)lx * ly * lz, 256);
  return 0;
}

/* ---------------------------------------------- Poisson ellipsoid cells */

typedef struct {
  int ncells, m;
  double box[3];       /* physical extent */
  double sp[3];        /* level-0 voxel spacing */
  int dims0[3];
  double *cx, *cy, *cz, *rx, *ry, *rz, *ca, *sa, *R;  /* centre, radii, rotation about z, bound radius */
  float *I;            /* ncells*m intensities, 0 = cell does not express the channel */
  double bin;          /* bin edge (physical) */
  int nbx, nby, nbz;
  int64_t *bstart;     /* nbins+1 */
  int32_t *bcell;      /* cell ids per bin */
  uint64_t seed;
  uint32_t noise_max;
} sy_cells;

SY_EXPORT void sy_cells_free(sy_cells *c) {
  if (!c) return;
  free(c->cx); free(c->I); free(c->bstart); free(c->bcell);
  free(c);
}

static inline int sy_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Cell field: ncells ellipsoids with centres uniform in the physical box,
 * radii uniform in [r_lo, r_hi] per axis, a random rotation about z; each
 * cell expresses each of the m channels with probability p_express, with a
 * log-normal intensity (median, sigma_ln).  Voxel value = sum of
 * I*(1 - r^2) over expressing cells with r < 1, rounded, plus counter-hash
 * noise in [0, noise_max], clamped to 65535. */
SY_EXPORT sy_cells *sy_cells_create(uint64_t seed, int ncells, int m, int nx, int ny, int nz, double sx,
                                    double sy_, double sz, double r_lo, double r_hi, double p_express,
                                    double median, double sigma_ln, uint32_t noise_max, double bin) {
  if (ncells < 0 || m < 1 || m > 64 || nx <= 0 || ny <= 0 || nz <= 0 || bin <= 0) return NULL;
  sy_cells *c = (sy_cells *)calloc(1, sizeof(sy_cells));
  if (!c) return NULL;
  c->ncells = ncells; c->m = m; c->seed = seed; c->noise_max = noise_max;
  c->dims0[0] = nx; c->dims0[1] = ny; c->dims0[2] = nz;
  c->sp[0] = sx; c->sp[1] = sy_; c->sp[2] = sz;
  c->box[0] = nx * sx; c->box[1] = ny * sy_; c->box[2] = nz * sz;
  size_t nc = ncells > 0 ? (size_t)ncells : 1;
  c->cx = (double *)malloc(sizeof(double) * 9 * nc);
  c->I = (float *)calloc(nc * (size_t)m, sizeof(float));
  if (!c->cx || !c->I) { sy_cells_free(c); return NULL; }
  c->cy = c->cx + nc; c->cz = c->cy + nc; c->rx = c->cz + nc; c->ry = c->rx + nc; c->rz = c->ry + nc;
  c->ca = c->rz + nc; c->sa = c->ca + nc; c->R = c->sa + nc;
  sy_rng r = {seed};
  for (int i = 0; i < ncells; ++i) {
    c->cx[i] = sy_unif(&r) * c->box[0];
    c->cy[i] = sy_unif(&r) * c->box[1];
    c->cz[i] = sy_unif(&r) * c->box[2];
    c->rx[i] = r_lo + (r_hi - r_lo) * sy_unif(&r);
    c->ry[i] = r_lo + (r_hi - r_lo) * sy_unif(&r);
    c->rz[i] = r_lo + (r_hi - r_lo) * sy_unif(&r);
    double th = 3.141592653589793 * sy_unif(&r);
    c->ca[i] = cos(th); c->sa[i] = sin(th);
    double R = c->rx[i] > c->ry[i] ? c->rx[i] : c->ry[i];
    c->R[i] = R > c->rz[i] ? R : c->rz[i];
    for (int ch = 0; ch < m; ++ch) {
      double u = sy_unif(&r);
      double g = sy_normal(&r);
      if (u < p_express) c->I[(size_t)i * m + ch] = (float)(median * exp(sigma_ln * g));
    }
  }
  /* spatial bins: each cell is listed in every bin its bounding box touches */
  c->bin = bin;
  c->nbx = (int)ceil(c->box[0] / bin); c->nby = (int)ceil(c->box[1] / bin); c->nbz = (int)ceil(c->box[2] / bin);
  if (c->nbx < 1) c->nbx = 1; if (c->nby < 1) c->nby = 1; if (c->nbz < 1) c->nbz = 1;
  int64_t nbins = (int64_t)c->nbx * c->nby * c->nbz;
  c->bstart = (int64_t *)calloc((size_t)nbins + 1, sizeof(int64_t));
  if (!c->bstart) { sy_cells_free(c); return NULL; }
  for (int pass = 0; pass < 2; ++pass) {
    int64_t *fill = NULL;
    if (pass == 1) {
      for (int64_t b = 0; b < nbins; ++b) c->bstart[b + 1] += c->bstart[b];
      c->bcell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(c->bstart[nbins] > 0 ? c->bstart[nbins] : 1));
      fill = (int64_t *)calloc((size_t)nbins, sizeof(int64_t));
      if (!c->bcell || !fill) { free(fill); sy_cells_free(c); return NULL; }
    }
    for (int i = 0; i < ncells; ++i) {
      int x0 = sy_clampi((int)floor((c->cx[i] - c->R[i]) / bin), 0, c->nbx - 1);
      int x1 = sy_clampi((int)floor((c->cx[i] + c->R[i]) / bin), 0, c->nbx - 1);
      int y0 = sy_clampi((int)floor((c->cy[i] - c->R[i]) / bin), 0, c->nby - 1);
      int y1 = sy_clampi((int)floor((c->cy[i] + c->R[i]) / bin), 0, c->nby - 1);
      int z0 = sy_clampi((int)floor((c->cz[i] - c->R[i]) / bin), 0, c->nbz - 1);
      int z1 = sy_clampi((int)floor((c->cz[i] + c->R[i]) / bin), 0, c->nbz - 1);
      for (int z = z0; z <= z1; ++z)
        for (int y = y0; y <= y1; ++y)
          for (int x = x0; x <= x1; ++x) {
            int64_t b = ((int64_t)z * c->nby + y) * c->nbx + x;
            if (pass == 0) c->bstart[b + 1]++;
            else c->bcell[c->bstart[b] + fill[b]++] = i;
          }
    }
    free(fill);
  }
  return c;
}

/* field value (before rounding and noise) of channel ch at a physical point */
static double sy_cells_field(const sy_cells *c, int ch, double px, double py, double pz) {
  int bx = sy_clampi((int)floor(px / c->bin), 0, c->nbx - 1);
  int by = sy_clampi((int)floor(py / c->bin), 0, c->nby - 1);
  int bz = sy_clampi((int)floor(pz / c->bin), 0, c->nbz - 1);
  int64_t b = ((int64_t)bz * c->nby + by) * c->nbx + bx;
  double v = 0.0;
  for (int64_t k = c->bstart[b]; k < c->bstart[b + 1]; ++k) {
    int i = c->bcell[k];
    float I = c->I[(size_t)i * c->m + ch];
    if (I <= 0.0f) continue;
    double dx = px - c->cx[i], dy = py - c->cy[i], dz = pz - c->cz[i];
    double u = (c->ca[i] * dx + c->sa[i] * dy) / c->rx[i];
    double w = (-c->sa[i] * dx + c->ca[i] * dy) / c->ry[i];
    double t = dz / c->rz[i];
    double r2 = u * u + w * w + t * t;
    if (r2 < 1.0) v += (double)I * (1.0 - r2);
  }
  return v;
}

/* value of level-l voxel (x,y,z) of channel ch: the field at that voxel's
 * centre, rounded, plus noise keyed by (ch, l, x, y, z) */
static inline uint16_t sy_cells_voxel(const sy_cells *c, int ch, int l, int x, int y, int z) {
  double f = (double)(1 << l);
  double px = (x + 0.5) * f * c->sp[0], py = (y + 0.5) * f * c->sp[1], pz = (z + 0.5) * f * c->sp[2];
  double v = floor(sy_cells_field(c, ch, px, py, pz) + 0.5) +
             sy_noise(c->seed, (uint32_t)ch, (uint32_t)l, (uint32_t)x, (uint32_t)y, (uint32_t)z, c->noise_max);
  return v > 65535.0 ? 65535 : (uint16_t)v;
}

typedef struct { const sy_cells *c; int ch; uint16_t *out; } sy_dense_ctx;

static void sy_dense_body(void *vctx, int64_t lo, int64_t hi) {
  sy_dense_ctx *d = (sy_dense_ctx *)vctx;
  int nx = d->c->dims0[0], ny = d->c->dims0[1];
  for (int64_t z = lo; z < hi; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) d->out[((int64_t)z * ny + y) * nx + x] = sy_cells_voxel(d->c, d->ch, 0, x, y, (int)z);
}

/* Dense level-0 volume of one channel (u16). */
SY_EXPORT int sy_cells_dense(const sy_cells *c, int ch, uint16_t *out) {
  if (!c || ch < 0 || ch >= c->m) return -1;
  sy_dense_ctx d = {c, ch, out};
  sy_parallel(sy_dense_body, &d, c->dims0[2], 1);
  return 0;
}

typedef struct { const sy_cells *c; int ch, l, B; const int32_t *coords; uint16_t *out; } sy_pbrick_ctx;

static void sy_pbrick_body(void *vctx, int64_t lo, int64_t hi) {
  sy_pbrick_ctx *p = (sy_pbrick_ctx *)vctx;
  const sy_cells *c = p->c;
  int nl[3];
  for (int a = 0; a < 3; ++a) {
    int d = c->dims0[a];
    for (int k = 0; k < p->l; ++k) d = (d + 1) / 2;
    nl[a] = d;
  }
  int64_t E = p->B + 2, per = E * E * E;
  for (int64_t i = lo; i < hi; ++i) {
    const int32_t *bc = p->coords + 3 * i;
    for (int64_t z = 0; z < E; ++z) {
      int iz = sy_clampi((int)((int64_t)bc[2] * p->B - 1 + z), 0, nl[2] - 1);
      for (int64_t y = 0; y < E; ++y) {
        int iy = sy_clampi((int)((int64_t)bc[1] * p->B - 1 + y), 0, nl[1] - 1);
        for (int64_t x = 0; x < E; ++x) {
          int ix = sy_clampi((int)((int64_t)bc[0] * p->B - 1 + x), 0, nl[0] - 1);
          p->out[i * per + (z * E + y) * E + x] = sy_cells_voxel(c, p->ch, p->l, ix, iy, iz);
        }
      }
    }
  }
}

/* n bricks of channel ch, level l (edge B) with a one-voxel clamped border,
 * evaluated directly from the cell field at level-l voxel centres (the
 * procedural hierarchy: every level samples the same continuous field). */
SY_EXPORT int sy_cells_bricks(const sy_cells *c, int ch, int l, int B, int n, const int32_t *coords,
                              uint16_t *out) {
  if (!c || ch < 0 || ch >= c->m || l < 0 || l > 15 || B < 1) return -1;
  sy_pbrick_ctx p = {c, ch, l, B, coords, out};
  sy_parallel(sy_pbrick_body, &p, n, 1);
  return 0;
}

/* Same as sy_cells_bricks, for a list of bricks of mixed channel/level:
 * keys n*5 ints (ch, l, bx, by, bz). */
typedef struct { const sy_cells *c; int B; const int32_t *keys; uint16_t *out; } sy_pmix_ctx;

static void sy_pmix_body(void *vctx, int64_t lo, int64_t hi) {
  sy_pmix_ctx *p = (sy_pmix_ctx *)vctx;
  int64_t E = p->B + 2, per = E * E * E;
  for (int64_t i = lo; i < hi; ++i) {
    const int32_t *k = p->keys + 5 * i;
    sy_pbrick_ctx one = {p->c, k[0], k[1], p->B, k + 2, p->out + i * per};
    sy_pbrick_body(&one, 0, 1);
  }
}

SY_EXPORT int sy_cells_bricks_mixed(const sy_cells *c, int B, int n, const int32_t *keys, uint16_t *out) {
  if (!c || B < 1) return -1;
  for (int i = 0; i < n; ++i)
    if (keys[5 * i] < 0 || keys[5 * i] >= c->m || keys[5 * i + 1] < 0 || keys[5 * i + 1] > 15) return -1;
  sy_pmix_ctx p = {c, B, keys, out};
  sy_parallel(sy_pmix_body, &p, n, 1);
  return 0;
}

typedef struct {
  const sy_cells *c; int ch, ex, ey, ez, lx, ly, lz; uint32_t *mn, *mx;
} sy_bound_ctx;

static void sy_bound_body(void *vctx, int64_t lo, int64_t hi) {
  sy_bound_ctx *b = (sy_bound_ctx *)vctx;
  const sy_cells *c = b->c;
  for (int64_t li = lo; li < hi; ++li) {
    int64_t jx = li % b->lx, jy = (li / b->lx) % b->ly, jz = li / ((int64_t)b->lx * b->ly);
    /* voxel index range of the widened leaf, then its voxel-centre box */
    double lo3[3], hi3[3];
    int64_t j3[3] = {jx, jy, jz}, e3[3] = {b->ex, b->ey, b->ez};
    for (int a = 0; a < 3; ++a) {
      int64_t v0 = j3[a] * e3[a] - 1, v1 = (j3[a] + 1) * e3[a];
      if (v0 < 0) v0 = 0;
      if (v1 > c->dims0[a] - 1) v1 = c->dims0[a] - 1;
      lo3[a] = (v0 + 0.5) * c->sp[a];
      hi3[a] = (v1 + 0.5) * c->sp[a];
    }
    double sum = 0.0;
    int x0 = sy_clampi((int)floor(lo3[0] / c->bin), 0, c->nbx - 1), x1 = sy_clampi((int)floor(hi3[0] / c->bin), 0, c->nbx - 1);
    int y0 = sy_clampi((int)floor(lo3[1] / c->bin), 0, c->nby - 1), y1 = sy_clampi((int)floor(hi3[1] / c->bin), 0, c->nby - 1);
    int z0 = sy_clampi((int)floor(lo3[2] / c->bin), 0, c->nbz - 1), z1 = sy_clampi((int)floor(hi3[2] / c->bin), 0, c->nbz - 1);
    for (int z = z0; z <= z1; ++z)
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
          int64_t bn = ((int64_t)z * c->nby + y) * c->nbx + x;
          for (int64_t k = c->bstart[bn]; k < c->bstart[bn + 1]; ++k) {
            int i = c->bcell[k];
            float I = c->I[(size_t)i * c->m + b->ch];
            if (I <= 0.0f) continue;
            /* count each cell once: only in the first bin of the scanned range that lists it */
            int fx = sy_clampi((int)floor((c->cx[i] - c->R[i]) / c->bin), 0, c->nbx - 1);
            int fy = sy_clampi((int)floor((c->cy[i] - c->R[i]) / c->bin), 0, c->nby - 1);
            int fz = sy_clampi((int)floor((c->cz[i] - c->R[i]) / c->bin), 0, c->nbz - 1);
            if ((fx > x0 ? fx : x0) != x || (fy > y0 ? fy : y0) != y || (fz > z0 ? fz : z0) != z) continue;
            if (c->cx[i] + c->R[i] < lo3[0] || c->cx[i] - c->R[i] > hi3[0]) continue;
            if (c->cy[i] + c->R[i] < lo3[1] || c->cy[i] - c->R[i] > hi3[1]) continue;
            if (c->cz[i] + c->R[i] < lo3[2] || c->cz[i] - c->R[i] > hi3[2]) continue;
            sum += (double)I;
          }
        }
    double mx = ceil(sum) + c->noise_max;
    b->mn[li] = 0;
    b->mx[li] = mx > 65535.0 ? 65535u : (uint32_t)mx;
  }
}

/* Conservative per-leaf value range of channel ch at level 0 for the cell
 * field, without evaluating voxels: [0, noise_max + sum of the intensities
 * of the expressing cells whose bounding sphere reaches the widened leaf]. */
SY_EXPORT int sy_cells_leaf_bounds(const sy_cells *c, int ch, int ex, int ey, int ez, uint32_t *out_min,
                                   uint32_t *out_max) {
  if (!c || ch < 0 || ch >= c->m) return -1;
  int lx = (c->dims0[0] + ex - 1) / ex, ly = (c->dims0[1] + ey - 1) / ey, lz = (c->dims0[2] + ez - 1) / ez;
  sy_bound_ctx b = {c, ch, ex, ey, ez, lx, ly, lz, out_min, out_max};
  sy_parallel(sy_bound_body, &b, (int64_t)lx * ly * lz, 1024);
  return 0;
}

/* number of cells and of expressing (cell, channel) pairs, for tests */
SY_EXPORT int64_t sy_cells_count(const sy_cells *c, int ch) {
  if (!c) return -1;
  if (ch < 0) return c->ncells;
  int64_t n = 0;
  for (int i = 0; i < c->ncells; ++i) n += c->I[(size_t)i * c->m + ch] > 0.0f;
  return n;
}

/* ------------------------------------- lazily generated voxel source */

/* Voxel access to the procedural cell field for consumers that read voxels
 * one at a time (the CPU oracle): level-l voxels are generated a whole brick
 * (B^3, no border) at a time on first touch and kept.  Insert-only
 * open-addressing table; lookups take no lock. */
typedef struct {
  const sy_cells *c;
  int B, blog2;
  int64_t cap;                 /* power of two */
  uint64_t *keys;              /* 0 = empty; key = packed (c, l, bz, by, bx) + 1 */
  uint16_t *volatile *vals;
  int nl[16][3];
  int64_t n_generated;
} sy_vcache;

SY_EXPORT sy_vcache *sy_vcache_create(const sy_cells *c, int B, int64_t capacity) {
  if (!c || B < 1 || (B & (B - 1))) return NULL;
  sy_vcache *v = (sy_vcache *)calloc(1, sizeof(sy_vcache));
  if (!v) return NULL;
  v->c = c; v->B = B;
  while ((1 << v->blog2) < B) ++v->blog2;
  v->cap = 1;
  while (v->cap < 2 * capacity) v->cap <<= 1;
  v->keys = (uint64_t *)calloc((size_t)v->cap, sizeof(uint64_t));
  v->vals = (uint16_t *volatile *)calloc((size_t)v->cap, sizeof(uint16_t *));
  if (!v->keys || !v->vals) { free(v->keys); free((void *)v->vals); free(v); return NULL; }
  for (int l = 0; l < 16; ++l)
    for (int a = 0; a < 3; ++a) {
      int d = c->dims0[a];
      for (int q = 0; q < l; ++q) d = (d + 1) / 2;
      v->nl[l][a] = d;
    }
  return v;
}

SY_EXPORT void sy_vcache_free(sy_vcache *v) {
  if (!v) return;
  for (int64_t i = 0; i < v->cap; ++i) free(v->vals[i]);
  free(v->keys);
  free((void *)v->vals);
  free(v);
}

SY_EXPORT int64_t sy_vcache_bricks(const sy_vcache *v) { return v ? __atomic_load_n(&v->n_generated, __ATOMIC_RELAXED) : -1; }

/* Value of level-l voxel (x, y, z) of channel ch (coordinates inside the
 * level); returns 0 and leaves the table untouched if it is full. */
SY_EXPORT uint32_t sy_vcache_voxel(void *vv, int ch, int l, int64_t x, int64_t y, int64_t z) {
  sy_vcache *v = (sy_vcache *)vv;
  const int sh = v->blog2;
  const uint64_t bx = (uint64_t)x >> sh, by = (uint64_t)y >> sh, bz = (uint64_t)z >> sh;
  const uint64_t key = (((((uint64_t)ch << 4 | (uint64_t)l) << 16 | bz) << 16 | by) << 16 | bx) + 1;
  uint64_t h = sy_mix(key) & (uint64_t)(v->cap - 1);
  const int B = v->B;
  for (int64_t probe = 0; probe < v->cap; ++probe, h = (h + 1) & (uint64_t)(v->cap - 1)) {
    uint64_t k = __atomic_load_n(&v->keys[h], __ATOMIC_ACQUIRE);
    if (k == 0) {
      uint64_t expect = 0;
      if (__atomic_compare_exchange_n(&v->keys[h], &expect, key, 0, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE)) {
        uint16_t *blk = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)B * B * B);
        if (!blk) return 0;
        for (int zz = 0; zz < B; ++zz)
          for (int yy = 0; yy < B; ++yy)
            for (int xx = 0; xx < B; ++xx) {
              int gx = (int)(bx * B) + xx, gy = (int)(by * B) + yy, gz = (int)(bz * B) + zz;
              uint16_t val = 0;
              if (gx < v->nl[l][0] && gy < v->nl[l][1] && gz < v->nl[l][2]) val = sy_cells_voxel(v->c, ch, l, gx, gy, gz);
              blk[((size_t)zz * B + yy) * B + xx] = val;
            }
        __atomic_store_n(&v->vals[h], blk, __ATOMIC_RELEASE);
        __atomic_add_fetch(&v->n_generated, 1, __ATOMIC_RELAXED);
        return blk[(((size_t)(z & (B - 1))) * B + (size_t)(y & (B - 1))) * B + (size_t)(x & (B - 1))];
      }
      k = expect;
    }
    if (k == key) {
      uint16_t *blk;
      while ((blk = __atomic_load_n(&v->vals[h], __ATOMIC_ACQUIRE)) == NULL) sched_yield();
      return blk[(((size_t)(z & (B - 1))) * B + (size_t)(y & (B - 1))) * B + (size_t)(x & (B - 1))];
    }
  }
  return 0;
}
