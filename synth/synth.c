/*
 * Seeded synthetic sparse matrices and vectors in CSR form.
 *
 * This module only draws inputs: it holds none of the SPC5 arithmetic
 * (no blocking, no masks, no products).  Both the CPU oracle and the CUDA
 * path are fed from it, so they see byte-identical matrices.
 *
 * Every random number is a pure function of (seed, stream, index) through a
 * counter-based splitmix64 mixer, so results do not depend on thread count
 * or loop order.  Normal deviates use the Box-Muller transform through libm,
 * so they are identical within one machine (the last ulp may differ between
 * libm builds; nothing stored in the repository depends on them).
 *
 * Workloads (the paper's SuiteSparse set is not available; these stand in
 * for its structural range, from high block filling to worst-case filling):
 *   - 2D 5-point and 3D 27-point stencils (natural x-fastest ordering),
 *   - FEM-like 3x3 dense node blocks on a random-geometric 3D mesh,
 *     nodes renumbered in Morton order,
 *   - power-law (Zipf) row lengths with columns clustered near the diagonal,
 *   - uniform-random columns at a fixed count per row,
 *   - dense n x n (the paper's "dense" matrix, Section 4.2),
 *   - small Bernoulli patterns for brute-force checks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t nrows, ncols, nnz;
  int32_t *rowptr; /* nrows + 1 */
  int32_t *colidx; /* nnz, strictly ascending within each row */
  double *vals;    /* nnz */
} synth_csr;

enum { SYNTH_OK = 0, SYNTH_EINVAL = 1, SYNTH_ENOMEM = 2, SYNTH_EOVERFLOW = 3 };

/* ---------------------------------------------------------------- rng --- */

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t rng_u64(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t key = mix64(seed * 0x9E3779B97F4A7C15ULL + stream * 0xD1B54A32D192ED03ULL +
                       0x632BE59BD9B4E019ULL);
  return mix64(key + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

/* uniform in [0, 1) with 53 random bits */
static inline double rng_unif(uint64_t seed, uint64_t stream, uint64_t i) {
  return (double)(rng_u64(seed, stream, i) >> 11) * 0x1.0p-53;
}

/* standard normal, Box-Muller on draws 2i and 2i+1 of the stream */
static inline double rng_normal(uint64_t seed, uint64_t stream, uint64_t i) {
  double u1 = ((double)(rng_u64(seed, stream, 2 * i) >> 11) + 1.0) * 0x1.0p-53; /* (0,1] */
  double u2 = rng_unif(seed, stream, 2 * i + 1);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* uniform integer in [0, m) */
static inline int64_t rng_below(uint64_t seed, uint64_t stream, uint64_t i, int64_t m) {
  int64_t v = (int64_t)(rng_unif(seed, stream, i) * (double)m);
  return v < m ? v : m - 1;
}

/* streams */
#define ST_VALUES 1u
#define ST_VECTOR 2u
#define ST_POINTS 10u
#define ST_ZIPF 20u
#define ST_ROWBASE 0x100000000ULL /* + row index: per-row column draws */
#define ST_PATTERN 30u

/* ------------------------------------------------------------ helpers --- */

void synth_free(synth_csr *m) {
  if (!m) return;
  free(m->rowptr);
  free(m->colidx);
  free(m->vals);
  m->rowptr = NULL;
  m->colidx = NULL;
  m->vals = NULL;
}

static int alloc_csr(synth_csr *m, int64_t nrows, int64_t ncols, int64_t nnz) {
  if (nnz > INT32_MAX || nrows > INT32_MAX - 1 || ncols > INT32_MAX) return SYNTH_EOVERFLOW;
  m->nrows = nrows;
  m->ncols = ncols;
  m->nnz = nnz;
  m->rowptr = (int32_t *)malloc((size_t)(nrows + 1) * sizeof(int32_t));
  m->colidx = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  m->vals = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  if (!m->rowptr || !m->colidx || !m->vals) {
    synth_free(m);
    return SYNTH_ENOMEM;
  }
  return SYNTH_OK;
}

/* value_mode 0: diagonal entries = diag, others = off.
 * value_mode 1: every value N(0,1) from (seed, ST_VALUES, element index). */
static void fill_values(synth_csr *m, int value_mode, double diag, double off, uint64_t seed) {
  int64_t n = m->nrows;
  if (value_mode == 1) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m->nnz; ++e) m->vals[e] = rng_normal(seed, ST_VALUES, (uint64_t)e);
  } else {
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = m->rowptr[i]; e < m->rowptr[i + 1]; ++e)
        m->vals[e] = (m->colidx[e] == i) ? diag : off;
  }
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* ----------------------------------------------------------- stencils --- */

/* 2D 5-point stencil on an nx-by-ny grid, row index i = x + nx*y. */
int synth_stencil2d_5pt(int64_t nx, int64_t ny, int value_mode, double diag, double off,
                        uint64_t seed, synth_csr *out) {
  memset(out, 0, sizeof(*out));
  if (nx < 1 || ny < 1) return SYNTH_EINVAL;
  int64_t n = nx * ny;
  int64_t nnz = 5 * n - 2 * nx - 2 * ny;
  int rc = alloc_csr(out, n, n, nnz);
  if (rc) return rc;
  int64_t e = 0;
  for (int64_t y = 0; y < ny; ++y)
    for (int64_t x = 0; x < nx; ++x) {
      int64_t i = x + nx * y;
      out->rowptr[i] = (int32_t)e;
      if (y > 0) out->colidx[e++] = (int32_t)(i - nx);
      if (x > 0) out->colidx[e++] = (int32_t)(i - 1);
      out->colidx[e++] = (int32_t)i;
      if (x < nx - 1) out->colidx[e++] = (int32_t)(i + 1);
      if (y < ny - 1) out->colidx[e++] = (int32_t)(i + nx);
    }
  out->rowptr[n] = (int32_t)e;
  if (e != nnz) return SYNTH_EINVAL;
  fill_values(out, value_mode, diag, off, seed);
  return SYNTH_OK;
}

/* 3D 27-point stencil on nx*ny*nz, row index i = x + nx*(y + ny*z). */
int synth_stencil3d_27pt(int64_t nx, int64_t ny, int64_t nz, int value_mode, double diag,
                         double off, uint64_t seed, synth_csr *out) {
  memset(out, 0, sizeof(*out));
  if (nx < 1 || ny < 1 || nz < 1) return SYNTH_EINVAL;
  int64_t n = nx * ny * nz;
  int64_t sx = 3 * nx - 2, sy = 3 * ny - 2, sz = 3 * nz - 2;
  if (nx == 1) sx = 1;
  if (ny == 1) sy = 1;
  if (nz == 1) sz = 1;
  int64_t nnz = sx * sy * sz;
  int rc = alloc_csr(out, n, n, nnz);
  if (rc) return rc;
  /* row lengths are separable: count(x)*count(y)*count(z) */
  int64_t e = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    out->rowptr[i] = (int32_t)e;
    for (int64_t dz = -1; dz <= 1; ++dz) {
      int64_t zz = z + dz;
      if (zz < 0 || zz >= nz) continue;
      for (int64_t dy = -1; dy <= 1; ++dy) {
        int64_t yy = y + dy;
        if (yy < 0 || yy >= ny) continue;
        for (int64_t dx = -1; dx <= 1; ++dx) {
          int64_t xx = x + dx;
          if (xx < 0 || xx >= nx) continue;
          out->colidx[e++] = (int32_t)(xx + nx * (yy + ny * zz));
        }
      }
    }
  }
  out->rowptr[n] = (int32_t)e;
  if (e != nnz) return SYNTH_EINVAL;
  fill_values(out, value_mode, diag, off, seed);
  return SYNTH_OK;
}

/* ------------------------------------------------------------- dense ---- */

int synth_dense(int64_t nrows, int64_t ncols, int value_mode, double diag, double off,
                uint64_t seed, synth_csr *out) {
  memset(out, 0, sizeof(*out));
  if (nrows < 1 || ncols < 1) return SYNTH_EINVAL;
  int rc = alloc_csr(out, nrows, ncols, nrows * ncols);
  if (rc) return rc;
  for (int64_t i = 0; i <= nrows; ++i) out->rowptr[i] = (int32_t)(i * ncols);
  for (int64_t i = 0; i < nrows; ++i)
    for (int64_t j = 0; j < ncols; ++j) out->colidx[i * ncols + j] = (int32_t)j;
  fill_values(out, value_mode, diag, off, seed);
  return SYNTH_OK;
}

/* ---------------------------------------------------- small Bernoulli --- */

/* Each entry (i, j) is stored with probability `density`.  value_mode 2:
 * small integers in {-3..3} (zero included: explicit zeros are stored);
 * value_mode 1: N(0,1). */
int synth_bernoulli(int64_t nrows, int64_t ncols, double density, int value_mode, uint64_t seed,
                    synth_csr *out) {
  memset(out, 0, sizeof(*out));
  if (nrows < 0 || ncols < 1 || density < 0.0 || density > 1.0) return SYNTH_EINVAL;
  int64_t cnt = 0;
  for (int64_t t = 0; t < nrows * ncols; ++t)
    if (rng_unif(seed, ST_PATTERN, (uint64_t)t) < density) ++cnt;
  int rc = alloc_csr(out, nrows, ncols, cnt);
  if (rc) return rc;
  int64_t e = 0;
  for (int64_t i = 0; i < nrows; ++i) {
    out->rowptr[i] = (int32_t)e;
    for (int64_t j = 0; j < ncols; ++j)
      if (rng_unif(seed, ST_PATTERN, (uint64_t)(i * ncols + j)) < density) {
        out->colidx[e] = (int32_t)j;
        if (value_mode == 2)
          out->vals[e] = (double)(rng_below(seed, ST_VALUES, (uint64_t)e, 7) - 3);
        else
          out->vals[e] = rng_normal(seed, ST_VALUES, (uint64_t)e);
        ++e;
      }
  }
  out->rowptr[nrows] = (int32_t)e;
  return SYNTH_OK;
}

/* ------------------------------------------------------ uniform random -- */

/* `per_row` distinct uniform columns in [0, ncols) for every row, sorted. */
int synth_uniform(int64_t nrows, int64_t ncols, int64_t per_row, uint64_t seed, synth_csr *out) {
  memset(out, 0, sizeof(*out));
  if (nrows < 1 || ncols < 1 || per_row < 0 || per_row > ncols) return SYNTH_EINVAL;
  int rc = alloc_csr(out, nrows, ncols, nrows * per_row);
  if (rc) return rc;
  for (int64_t i = 0; i <= nrows; ++i) out->rowptr[i] = (int32_t)(i * per_row);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < nrows; ++i) {
    int32_t *row = out->colidx + i * per_row;
    uint64_t stream = ST_ROWBASE + (uint64_t)i, draw = 0;
    int64_t have = 0;
    while (have < per_row) {
      int32_t cand = (int32_t)rng_below(seed, stream, draw++, ncols);
      int dup = 0;
      for (int64_t t = 0; t < have; ++t)
        if (row[t] == cand) {
          dup = 1;
          break;
        }
      if (!dup) row[have++] = cand;
    }
    qsort(row, (size_t)per_row, sizeof(int32_t), cmp_i32);
  }
  fill_values(out, 1, 0.0, 0.0, seed);
  return SYNTH_OK;
}

/* ----------------------------------------------------------- power law -- */

/* Row lengths k_i ~ Zipf(s) truncated to [1, n], rescaled so that their
 * sample mean is `mean`: L_i = clamp(round(mean * k_i / mean(k)), 1, n).
 * Rows with L_i <= long_row draw columns round(i + N(0, sigma)) clipped to
 * [0, n), redrawing duplicates; longer rows take L_i distinct uniform
 * columns (selection sampling).  Columns are sorted, values N(0,1). */
int synth_powerlaw(int64_t n, double s, double mean, double sigma, int64_t long_row,
                   uint64_t seed, synth_csr *out) {
  memset(out, 0, sizeof(*out));
  if (n < 1 || s <= 0.0 || mean <= 0.0 || sigma <= 0.0) return SYNTH_EINVAL;
  /* rows of up to long_row entries draw distinct columns from N(i, sigma)
   * by rejection, which needs about 4 sigma of room for long_row columns */
  if ((double)long_row > 4.0 * sigma) return SYNTH_EINVAL;
  double *cdf = (double *)malloc((size_t)n * sizeof(double));
  int64_t *len = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!cdf || !len) {
    free(cdf);
    free(len);
    return SYNTH_ENOMEM;
  }
  double acc = 0.0;
  for (int64_t k = 1; k <= n; ++k) {
    acc += pow((double)k, -s);
    cdf[k - 1] = acc;
  }
  double ksum = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double u = rng_unif(seed, ST_ZIPF, (uint64_t)i) * acc;
    int64_t lo = 0, hi = n - 1; /* first k with cdf[k] > u */
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (cdf[mid] > u)
        hi = mid;
      else
        lo = mid + 1;
    }
    len[i] = lo + 1;
    ksum += (double)(lo + 1);
  }
  free(cdf);
  double kmean = ksum / (double)n;
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t L = llround(mean * (double)len[i] / kmean);
    if (L < 1) L = 1;
    if (L > n) L = n;
    len[i] = L;
    nnz += L;
  }
  int rc = alloc_csr(out, n, n, nnz);
  if (rc) {
    free(len);
    return rc;
  }
  out->rowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) out->rowptr[i + 1] = (int32_t)(out->rowptr[i] + len[i]);
  free(len);

  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  size_t words = (size_t)((n + 63) / 64);
  uint64_t *bitmaps = (uint64_t *)calloc(words * (size_t)nthreads, sizeof(uint64_t));
  if (!bitmaps) {
    synth_free(out);
    return SYNTH_ENOMEM;
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    uint64_t *bm = bitmaps + words * (size_t)tid;
    int32_t *row = out->colidx + out->rowptr[i];
    int64_t L = out->rowptr[i + 1] - out->rowptr[i];
    uint64_t stream = ST_ROWBASE + (uint64_t)i, draw = 0;
    if (L > long_row) {
      /* uniform distinct columns: mark min(L, n-L) distinct uniform draws
       * in the bitmap, then emit the marked (or the unmarked) columns in
       * ascending order */
      int keep_marked = (2 * L <= n);
      int64_t m = keep_marked ? L : n - L, marked = 0;
      while (marked < m) {
        int64_t cand = rng_below(seed, stream, draw++, n);
        uint64_t bit = 1ULL << (cand & 63);
        if (bm[cand >> 6] & bit) continue;
        bm[cand >> 6] |= bit;
        ++marked;
      }
      int64_t t = 0;
      for (size_t w = 0; w < words; ++w) {
        uint64_t word = keep_marked ? bm[w] : ~bm[w];
        while (word) {
          int b = __builtin_ctzll(word);
          word &= word - 1;
          int64_t j = (int64_t)w * 64 + b;
          if (j < n) row[t++] = (int32_t)j;
        }
        bm[w] = 0;
      }
    } else {
      int64_t have = 0;
      while (have < L) {
        double z = rng_normal(seed, stream, draw++);
        int64_t cand = llround((double)i + sigma * z);
        if (cand < 0) cand = 0;
        if (cand >= n) cand = n - 1;
        uint64_t bit = 1ULL << (cand & 63);
        if (bm[cand >> 6] & bit) continue;
        bm[cand >> 6] |= bit;
        row[have++] = (int32_t)cand;
      }
      for (int64_t t = 0; t < L; ++t) bm[row[t] >> 6] &= ~(1ULL << (row[t] & 63));
      qsort(row, (size_t)L, sizeof(int32_t), cmp_i32);
    }
  }
  free(bitmaps);
  fill_values(out, 1, 0.0, 0.0, seed);
  return SYNTH_OK;
}

/* ----------------------------------------------------------------- FEM -- */

static uint64_t spread3(uint64_t v) { /* 21 bits -> every third bit */
  v &= 0x1FFFFFULL;
  v = (v | (v << 32)) & 0x1F00000000FFFFULL;
  v = (v | (v << 16)) & 0x1F0000FF0000FFULL;
  v = (v | (v << 8)) & 0x100F00F00F00F00FULL;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

typedef struct {
  uint64_t key;
  int64_t id;
} keyed;

static int cmp_keyed(const void *a, const void *b) {
  const keyed *x = (const keyed *)a, *y = (const keyed *)b;
  if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
  return (x->id > y->id) - (x->id < y->id);
}

/* nnodes points uniform in [0,1)^3, renumbered in Morton order; node i is
 * linked to every node within radius rho = (3*mean_nbrs/(4*pi*nnodes))^(1/3)
 * (itself included); every link is a dense 3x3 block, so the matrix has
 * n = 3*nnodes rows and about 9*(mean_nbrs+1) entries per 3 rows. */
int synth_fem3d(int64_t nnodes, double mean_nbrs, uint64_t seed, synth_csr *out) {
  memset(out, 0, sizeof(*out));
  if (nnodes < 1 || mean_nbrs < 0.0) return SYNTH_EINVAL;
  double *pt = (double *)malloc((size_t)nnodes * 3 * sizeof(double));
  keyed *order = (keyed *)malloc((size_t)nnodes * sizeof(keyed));
  if (!pt || !order) {
    free(pt);
    free(order);
    return SYNTH_ENOMEM;
  }
  for (int64_t i = 0; i < nnodes; ++i) {
    double px = rng_unif(seed, ST_POINTS, (uint64_t)(3 * i));
    double py = rng_unif(seed, ST_POINTS, (uint64_t)(3 * i + 1));
    double pz = rng_unif(seed, ST_POINTS, (uint64_t)(3 * i + 2));
    uint64_t qx = (uint64_t)(px * 2097152.0), qy = (uint64_t)(py * 2097152.0),
             qz = (uint64_t)(pz * 2097152.0);
    order[i].key = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
    order[i].id = i;
  }
  qsort(order, (size_t)nnodes, sizeof(keyed), cmp_keyed);
  /* renumbered coordinates */
  for (int64_t k = 0; k < nnodes; ++k) {
    int64_t i = order[k].id;
    pt[3 * k + 0] = rng_unif(seed, ST_POINTS, (uint64_t)(3 * i));
    pt[3 * k + 1] = rng_unif(seed, ST_POINTS, (uint64_t)(3 * i + 1));
    pt[3 * k + 2] = rng_unif(seed, ST_POINTS, (uint64_t)(3 * i + 2));
  }
  free(order);
  double rho = cbrt(3.0 * mean_nbrs / (4.0 * 3.14159265358979323846 * (double)nnodes));
  int64_t g = (int64_t)floor(1.0 / rho);
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  int64_t ncell = g * g * g;
  int64_t *cstart = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *cell_of = (int64_t *)malloc((size_t)nnodes * sizeof(int64_t));
  int64_t *members = (int64_t *)malloc((size_t)nnodes * sizeof(int64_t));
  int64_t *deg = (int64_t *)malloc((size_t)(nnodes + 1) * sizeof(int64_t));
  if (!cstart || !cell_of || !members || !deg) {
    free(pt);
    free(cstart);
    free(cell_of);
    free(members);
    free(deg);
    return SYNTH_ENOMEM;
  }
  for (int64_t k = 0; k < nnodes; ++k) {
    int64_t cx = (int64_t)(pt[3 * k] * g), cy = (int64_t)(pt[3 * k + 1] * g),
            cz = (int64_t)(pt[3 * k + 2] * g);
    if (cx >= g) cx = g - 1;
    if (cy >= g) cy = g - 1;
    if (cz >= g) cz = g - 1;
    cell_of[k] = cx + g * (cy + g * cz);
    cstart[cell_of[k] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    int64_t *fillp = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    if (!fillp) return SYNTH_ENOMEM;
    memcpy(fillp, cstart, (size_t)ncell * sizeof(int64_t));
    for (int64_t k = 0; k < nnodes; ++k) members[fillp[cell_of[k]]++] = k; /* ascending k */
    free(fillp);
  }
  double r2 = rho * rho;
  /* pass 1: degrees */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t k = 0; k < nnodes; ++k) {
    int64_t c = cell_of[k], cx = c % g, cy = (c / g) % g, cz = c / (g * g);
    int64_t d = 0;
    for (int64_t dz = -1; dz <= 1; ++dz)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dx = -1; dx <= 1; ++dx) {
          int64_t ax = cx + dx, ay = cy + dy, az = cz + dz;
          if (ax < 0 || ay < 0 || az < 0 || ax >= g || ay >= g || az >= g) continue;
          int64_t cc = ax + g * (ay + g * az);
          for (int64_t t = cstart[cc]; t < cstart[cc + 1]; ++t) {
            int64_t o = members[t];
            double ddx = pt[3 * k] - pt[3 * o], ddy = pt[3 * k + 1] - pt[3 * o + 1],
                   ddz = pt[3 * k + 2] - pt[3 * o + 2];
            if (ddx * ddx + ddy * ddy + ddz * ddz <= r2) ++d;
          }
        }
    deg[k] = d;
  }
  int64_t nlinks = 0;
  for (int64_t k = 0; k < nnodes; ++k) nlinks += deg[k];
  int64_t n = 3 * nnodes;
  int rc = alloc_csr(out, n, n, 9 * nlinks);
  if (rc) {
    free(pt);
    free(cstart);
    free(cell_of);
    free(members);
    free(deg);
    return rc;
  }
  out->rowptr[0] = 0;
  for (int64_t k = 0; k < nnodes; ++k)
    for (int a = 0; a < 3; ++a)
      out->rowptr[3 * k + a + 1] = (int32_t)(out->rowptr[3 * k + a] + 3 * deg[k]);
  /* pass 2: sorted neighbour lists expanded into 3x3 blocks */
#pragma omp parallel
  {
    int32_t *nb = (int32_t *)malloc(4096 * sizeof(int32_t));
    int64_t cap = 4096;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t k = 0; k < nnodes; ++k) {
      int64_t c = cell_of[k], cx = c % g, cy = (c / g) % g, cz = c / (g * g);
      int64_t d = 0;
      for (int64_t dz = -1; dz <= 1; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
          for (int64_t dx = -1; dx <= 1; ++dx) {
            int64_t ax = cx + dx, ay = cy + dy, az = cz + dz;
            if (ax < 0 || ay < 0 || az < 0 || ax >= g || ay >= g || az >= g) continue;
            int64_t cc = ax + g * (ay + g * az);
            for (int64_t t = cstart[cc]; t < cstart[cc + 1]; ++t) {
              int64_t o = members[t];
              double ddx = pt[3 * k] - pt[3 * o], ddy = pt[3 * k + 1] - pt[3 * o + 1],
                     ddz = pt[3 * k + 2] - pt[3 * o + 2];
              if (ddx * ddx + ddy * ddy + ddz * ddz <= r2) {
                if (d == cap) {
                  cap *= 2;
                  nb = (int32_t *)realloc(nb, (size_t)cap * sizeof(int32_t));
                }
                nb[d++] = (int32_t)o;
              }
            }
          }
      qsort(nb, (size_t)d, sizeof(int32_t), cmp_i32);
      for (int a = 0; a < 3; ++a) {
        int32_t *row = out->colidx + out->rowptr[3 * k + a];
        for (int64_t t = 0; t < d; ++t)
          for (int b = 0; b < 3; ++b) row[3 * t + b] = 3 * nb[t] + b;
      }
    }
    free(nb);
  }
  free(pt);
  free(cstart);
  free(cell_of);
  free(members);
  free(deg);
  fill_values(out, 1, 0.0, 0.0, seed);
  return SYNTH_OK;
}

/* ------------------------------------------------------------ vectors --- */

/* out[i] uniform in [lo, hi) from (seed, ST_VECTOR + stream) */
void synth_vector_uniform(int64_t n, double lo, double hi, uint64_t seed, uint64_t stream,
                          double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    out[i] = lo + (hi - lo) * rng_unif(seed, ST_VECTOR + 16 * stream, (uint64_t)i);
}

void synth_vector_normal(int64_t n, uint64_t seed, uint64_t stream, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    out[i] = rng_normal(seed, ST_VECTOR + 16 * stream + 1, (uint64_t)i);
}

/* out[i] integer in [lo, hi] */
void synth_vector_int(int64_t n, int64_t lo, int64_t hi, uint64_t seed, uint64_t stream,
                      double *out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = (double)(lo + rng_below(seed, ST_VECTOR + 16 * stream + 2, (uint64_t)i, hi - lo + 1));
}
