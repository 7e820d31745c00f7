/*
 * Seeded synthetic inputs: sparse matrices in CSR form and dense vectors.
 *
 * This module only draws inputs. It holds none of the SpMV or block-format
 * arithmetic, so both the CPU oracle and the CUDA path may use it.
 *
 * Random numbers come from one counter-based generator: the output function of
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), applied to a counter. Draw i of stream s under
 * seed q is mix(key(q, s) + (i + 1) * G), with G = 0x9e3779b97f4a7c15 and
 * key(q, s) = mix(q * G + mix(s + G)). Every draw is addressed by its index, so
 * results do not depend on the number of OpenMP threads or on the machine.
 *
 * CSR conventions (the paper's Background section): rowptr has n + 1 int64
 * entries, colidx holds int32 column indices sorted ascending within each row
 * with no duplicates, values holds float64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static inline uint64_t sm_key(uint64_t seed, uint64_t stream) {
  return sm_mix(seed * GOLDEN + sm_mix(stream + GOLDEN));
}
static inline uint64_t sm_draw(uint64_t key, uint64_t i) { return sm_mix(key + (i + 1) * GOLDEN); }
/* uniform double in [0, 1) with 53 random bits */
static inline double sm_u01(uint64_t z) { return (double)(z >> 11) * 0x1.0p-53; }
/* uniform integer in [0, k) by 128-bit multiply (Lemire), k > 0 */
static inline uint64_t sm_below(uint64_t z, uint64_t k) {
  return (uint64_t)(((unsigned __int128)z * (unsigned __int128)k) >> 64);
}

/* Streams used by the matrix builders. */
enum { ST_VALUES = 1000, ST_STRUCT = 2000, ST_PERM = 3000, ST_COUNT = 4000 };

typedef struct {
  int64_t n, m, nnz;
  int64_t* rowptr;
  int32_t* colidx;
  double* values;
} gen_csr;

void gen_free(gen_csr* a) {
  if (!a) return;
  free(a->rowptr);
  free(a->colidx);
  free(a->values);
  free(a);
}

static gen_csr* csr_alloc(int64_t n, int64_t m, int64_t nnz) {
  gen_csr* a = (gen_csr*)calloc(1, sizeof(gen_csr));
  if (!a) return NULL;
  a->n = n;
  a->m = m;
  a->nnz = nnz;
  a->rowptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  a->colidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  a->values = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!a->rowptr || !a->colidx || !a->values) {
    gen_free(a);
    return NULL;
  }
  return a;
}

/* ---------------------------------------------------------------- vectors */

void gen_fill_uniform(uint64_t seed, uint64_t stream, int64_t n, double lo, double hi, double* out) {
  uint64_t key = sm_key(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * sm_u01(sm_draw(key, (uint64_t)i));
}

/* N(0,1) by the Box-Muller transform on draws 2i and 2i+1. */
static inline double normal_at(uint64_t key, uint64_t i) {
  double u1 = ((double)(sm_draw(key, 2 * i) >> 11) + 1.0) * 0x1.0p-53; /* (0, 1] */
  double u2 = sm_u01(sm_draw(key, 2 * i + 1));
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

void gen_fill_normal(uint64_t seed, uint64_t stream, int64_t n, double* out) {
  uint64_t key = sm_key(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = normal_at(key, (uint64_t)i);
}

/* Dyadic values k / 2^bits with k uniform in [-2^bits, 2^bits]: exactly
 * representable in float32 for bits <= 23. */
void gen_fill_dyadic(uint64_t seed, uint64_t stream, int64_t n, int bits, double* out) {
  uint64_t key = sm_key(seed, stream);
  uint64_t span = (2ULL << bits) + 1ULL;
  double scale = ldexp(1.0, -bits);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t k = (int64_t)sm_below(sm_draw(key, (uint64_t)i), span) - (int64_t)(1ULL << bits);
    out[i] = (double)k * scale;
  }
}

/* Raw 64-bit draws, exposed so that tests can check the generator itself. */
void gen_fill_u64(uint64_t seed, uint64_t stream, int64_t n, uint64_t* out) {
  uint64_t key = sm_key(seed, stream);
  for (int64_t i = 0; i < n; ++i) out[i] = sm_draw(key, (uint64_t)i);
}
uint64_t gen_splitmix_mix(uint64_t z) { return sm_mix(z); }

static void fill_values_normal(gen_csr* a, uint64_t seed) {
  gen_fill_normal(seed, ST_VALUES, a->nnz, a->values);
}

/* ---------------------------------------------------------------- stencils */

/* 5-point Laplacian on an nx-by-ny grid, natural (x fastest) ordering,
 * diagonal 4, off-diagonals -1. */
gen_csr* gen_laplacian2d(int64_t nx, int64_t ny) {
  int64_t n = nx * ny;
  int64_t nnz = 5 * n - 2 * nx - 2 * ny;
  gen_csr* a = csr_alloc(n, n, nnz);
  if (!a) return NULL;
  int64_t p = 0;
  for (int64_t y = 0; y < ny; ++y)
    for (int64_t x = 0; x < nx; ++x) {
      int64_t row = y * nx + x;
      a->rowptr[row] = p;
      if (y > 0) { a->colidx[p] = (int32_t)(row - nx); a->values[p++] = -1.0; }
      if (x > 0) { a->colidx[p] = (int32_t)(row - 1); a->values[p++] = -1.0; }
      a->colidx[p] = (int32_t)row; a->values[p++] = 4.0;
      if (x + 1 < nx) { a->colidx[p] = (int32_t)(row + 1); a->values[p++] = -1.0; }
      if (y + 1 < ny) { a->colidx[p] = (int32_t)(row + nx); a->values[p++] = -1.0; }
    }
  a->rowptr[n] = p;
  a->nnz = p;
  return a;
}

/* 7-point or 27-point stencil on an nx*ny*nz grid, natural ordering.
 * value_mode 0: Poisson constants (7-point: 6 / -1; 27-point: 26 / -1).
 * value_mode 1: values N(0,1) from the values stream of `seed`. */
gen_csr* gen_stencil3d(int64_t nx, int64_t ny, int64_t nz, int points, int value_mode, uint64_t seed) {
  if (points != 7 && points != 27) return NULL;
  int64_t n = nx * ny * nz;
  /* count per row first (cheap), then fill in parallel over z-planes */
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!cnt) return NULL;
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t c = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int nd = (dx != 0) + (dy != 0) + (dz != 0);
              if (points == 7 && nd > 1) continue;
              int64_t xx = x + dx, yy = y + dy, zz = z + dz;
              if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
              ++c;
            }
        cnt[(z * ny + y) * nx + x] = c;
      }
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = cnt[i];
    cnt[i] = nnz;
    nnz += c;
  }
  cnt[n] = nnz;
  gen_csr* a = csr_alloc(n, n, nnz);
  if (!a) { free(cnt); return NULL; }
  memcpy(a->rowptr, cnt, sizeof(int64_t) * (size_t)(n + 1));
  free(cnt);
  double diag = points == 7 ? 6.0 : 26.0;
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t row = (z * ny + y) * nx + x;
        int64_t p = a->rowptr[row];
        /* dz outermost, then dy, then dx: columns come out ascending */
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int nd = (dx != 0) + (dy != 0) + (dz != 0);
              if (points == 7 && nd > 1) continue;
              int64_t xx = x + dx, yy = y + dy, zz = z + dz;
              if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
              a->colidx[p] = (int32_t)((zz * ny + yy) * nx + xx);
              a->values[p] = nd == 0 ? diag : -1.0;
              ++p;
            }
      }
  if (value_mode == 1) fill_values_normal(a, seed);
  return a;
}

/* --------------------------------------------------------------- sampling */

/* k distinct integers from [lo, lo + span) by Floyd's algorithm, written
 * sorted ascending to out; draws come from (key, base + j). */
static int sample_distinct(uint64_t key, uint64_t base, int64_t lo, int64_t span, int k, int64_t* out) {
  if (k > span) k = (int)span;
  int got = 0;
  for (int64_t j = span - k; j < span; ++j) {
    int64_t t = (int64_t)sm_below(sm_draw(key, base + (uint64_t)(j - (span - k))), (uint64_t)(j + 1));
    int seen = 0;
    for (int q = 0; q < got; ++q)
      if (out[q] == t) { seen = 1; break; }
    out[got++] = seen ? j : t;
  }
  /* insertion sort: k is small */
  for (int i = 1; i < got; ++i) {
    int64_t v = out[i];
    int q = i - 1;
    while (q >= 0 && out[q] > v) { out[q + 1] = out[q]; --q; }
    out[q + 1] = v;
  }
  for (int i = 0; i < got; ++i) out[i] += lo;
  return got;
}

/* Block-FEM-like matrix: nb block rows of bs-by-bs dense blocks. Block row I
 * has K blocks, K uniform in [bmin, bmax]; the diagonal block is always
 * present; the other K-1 block columns are distinct, uniform within
 * |J - I| <= floor(band_frac * nb). Values N(0,1). */
gen_csr* gen_block_fem(int64_t nb, int bs, int bmin, int bmax, double band_frac, uint64_t seed) {
  if (bmin < 1 || bmax < bmin || bmax > 256 || bs < 1) return NULL;
  uint64_t kcount = sm_key(seed, ST_COUNT), kstruct = sm_key(seed, ST_STRUCT);
  int64_t w = (int64_t)floor(band_frac * (double)nb);
  int64_t* kb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb + 1));
  if (!kb) return NULL;
  /* number of blocks per block row */
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < nb; ++I) {
    int64_t lo = I - w < 0 ? 0 : I - w, hi = I + w >= nb ? nb - 1 : I + w;
    int64_t k = bmin + (int64_t)sm_below(sm_draw(kcount, (uint64_t)I), (uint64_t)(bmax - bmin + 1));
    if (k > hi - lo + 1) k = hi - lo + 1;
    kb[I] = k;
  }
  int64_t tot = 0;
  for (int64_t I = 0; I < nb; ++I) {
    int64_t k = kb[I];
    kb[I] = tot;
    tot += k;
  }
  kb[nb] = tot;
  int64_t n = nb * bs;
  gen_csr* a = csr_alloc(n, n, tot * bs * bs);
  if (!a) { free(kb); return NULL; }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t I = 0; I < nb; ++I) {
    int64_t cols[257];
    int64_t lo = I - w < 0 ? 0 : I - w, hi = I + w >= nb ? nb - 1 : I + w;
    int k = (int)(kb[I + 1] - kb[I]);
    /* K-1 distinct off-diagonal block columns from the window minus I */
    int64_t span = hi - lo; /* window size minus the diagonal */
    int got = sample_distinct(kstruct, (uint64_t)I * 512, 0, span, k - 1, cols);
    for (int q = 0; q < got; ++q) {
      int64_t J = lo + cols[q];
      if (J >= I) ++J; /* skip the diagonal */
      cols[q] = J;
    }
    cols[got++] = I;
    for (int i = 1; i < got; ++i) { /* sort ascending */
      int64_t v = cols[i];
      int q = i - 1;
      while (q >= 0 && cols[q] > v) { cols[q + 1] = cols[q]; --q; }
      cols[q + 1] = v;
    }
    for (int br = 0; br < bs; ++br) {
      int64_t row = I * bs + br;
      int64_t p = kb[I] * bs * bs + (int64_t)br * got * bs;
      a->rowptr[row] = p;
      for (int q = 0; q < got; ++q)
        for (int bc = 0; bc < bs; ++bc) a->colidx[p++] = (int32_t)(cols[q] * bs + bc);
    }
  }
  a->rowptr[n] = tot * bs * bs;
  free(kb);
  fill_values_normal(a, seed);
  return a;
}

/* ------------------------------------------------------------------- sort */

/* LSD radix sort of 64-bit keys, 16-bit digits, `passes` digits. */
static int radix_sort_u64(uint64_t* key, int64_t n, int passes) {
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * 65536);
  if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
  uint64_t* src = key;
  uint64_t* dst = tmp;
  for (int p = 0; p < passes; ++p) {
    int sh = 16 * p;
    memset(cnt, 0, sizeof(int64_t) * 65536);
    for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & 0xffff]++;
    int64_t s = 0;
    for (int d = 0; d < 65536; ++d) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
    for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & 0xffff]++] = src[i];
    uint64_t* t = src; src = dst; dst = t;
  }
  if (src != key) memcpy(key, src, sizeof(uint64_t) * (size_t)n);
  free(tmp);
  free(cnt);
  return 0;
}

/* CSR from (row << 32 | col) keys: sort, drop duplicate keys, count rows. */
static gen_csr* csr_from_keys(uint64_t* keys, int64_t ne, int64_t n, int64_t m, int key_bits) {
  int passes = (key_bits + 15) / 16;
  if (radix_sort_u64(keys, ne, passes) != 0) return NULL;
  int64_t u = 0;
  for (int64_t i = 0; i < ne; ++i)
    if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
  gen_csr* a = csr_alloc(n, m, u);
  if (!a) return NULL;
  memset(a->rowptr, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < u; ++i) a->rowptr[(keys[i] >> 32) + 1]++;
  for (int64_t i = 0; i < n; ++i) a->rowptr[i + 1] += a->rowptr[i];
  for (int64_t i = 0; i < u; ++i) a->colidx[i] = (int32_t)(keys[i] & 0xffffffffULL);
  return a;
}

/* R-MAT graph with 2^scale vertices and edge_factor * 2^scale edge draws.
 * Each draw descends `scale` levels, picking quadrant (0,0), (0,1), (1,0),
 * (1,1) with probabilities a, b, c, 1-a-b-c. Repeated edges are kept once;
 * self-loops are kept. With relabel != 0 the vertices are renamed by a seeded
 * Fisher-Yates permutation, as the Graph500 generator does. Values N(0,1). */
gen_csr* gen_rmat(int scale, int edge_factor, double a, double b, double c, int relabel, uint64_t seed) {
  if (scale < 1 || scale > 30) return NULL;
  int64_t n = (int64_t)1 << scale;
  int64_t ne = (int64_t)edge_factor * n;
  uint64_t ks = sm_key(seed, ST_STRUCT);
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(ne > 0 ? ne : 1));
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!keys || !perm) { free(keys); free(perm); return NULL; }
  double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ne; ++e) {
    uint64_t row = 0, col = 0;
    for (int L = 0; L < scale; ++L) {
      double u = sm_u01(sm_draw(ks, (uint64_t)e * (uint64_t)scale + (uint64_t)L));
      int rb = u >= ab;                      /* lower half: quadrants c, d */
      int cb = (u >= a && u < ab) || u >= abc; /* right half: quadrants b, d */
      row = (row << 1) | (uint64_t)rb;
      col = (col << 1) | (uint64_t)cb;
    }
    keys[e] = (row << 32) | col;
  }
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  if (relabel) {
    uint64_t kp = sm_key(seed, ST_PERM);
    for (int64_t i = n - 1; i > 0; --i) {
      int64_t j = (int64_t)sm_below(sm_draw(kp, (uint64_t)i), (uint64_t)(i + 1));
      int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
      uint64_t row = keys[e] >> 32, col = keys[e] & 0xffffffffULL;
      keys[e] = ((uint64_t)perm[row] << 32) | (uint64_t)perm[col];
    }
  }
  free(perm);
  gen_csr* A = csr_from_keys(keys, ne, n, n, 32 + scale);
  free(keys);
  if (A) fill_values_normal(A, seed);
  return A;
}

/* n rows, exactly per_row distinct columns per row uniform in [0, m), sorted.
 * Values N(0,1). */
gen_csr* gen_uniform(int64_t n, int64_t m, int per_row, uint64_t seed) {
  if (per_row < 0 || per_row > 4096 || per_row > m) return NULL;
  gen_csr* a = csr_alloc(n, m, n * per_row);
  if (!a) return NULL;
  uint64_t ks = sm_key(seed, ST_STRUCT);
#pragma omp parallel
  {
    int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)(per_row + 1));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int got = sample_distinct(ks, (uint64_t)i * (uint64_t)per_row, 0, m, per_row, cols);
      a->rowptr[i] = i * per_row;
      for (int q = 0; q < got; ++q) a->colidx[i * per_row + q] = (int32_t)cols[q];
    }
    free(cols);
  }
  a->rowptr[n] = n * per_row;
  fill_values_normal(a, seed);
  return a;
}

/* Banded random matrix: row i keeps each column j with |i - j| <= half_bw
 * independently with probability density (the diagonal always). Values
 * N(0,1). */
gen_csr* gen_banded(int64_t n, int64_t half_bw, double density, uint64_t seed) {
  uint64_t ks = sm_key(seed, ST_STRUCT);
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!cnt) return NULL;
  int64_t width = 2 * half_bw + 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t d = -half_bw; d <= half_bw; ++d) {
      int64_t j = i + d;
      if (j < 0 || j >= n) continue;
      if (d == 0 || sm_u01(sm_draw(ks, (uint64_t)i * (uint64_t)width + (uint64_t)(d + half_bw))) < density) ++c;
    }
    cnt[i] = c;
  }
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) { int64_t c = cnt[i]; cnt[i] = nnz; nnz += c; }
  cnt[n] = nnz;
  gen_csr* a = csr_alloc(n, n, nnz);
  if (!a) { free(cnt); return NULL; }
  memcpy(a->rowptr, cnt, sizeof(int64_t) * (size_t)(n + 1));
  free(cnt);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t p = a->rowptr[i];
    for (int64_t d = -half_bw; d <= half_bw; ++d) {
      int64_t j = i + d;
      if (j < 0 || j >= n) continue;
      if (d == 0 || sm_u01(sm_draw(ks, (uint64_t)i * (uint64_t)width + (uint64_t)(d + half_bw))) < density)
        a->colidx[p++] = (int32_t)j;
    }
  }
  fill_values_normal(a, seed);
  return a;
}

/* Small random CSR for tests: each entry (i, j) present independently with
 * probability density. Values N(0,1). */
gen_csr* gen_random(int64_t n, int64_t m, double density, uint64_t seed) {
  uint64_t ks = sm_key(seed, ST_STRUCT);
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < m; ++j)
      if (sm_u01(sm_draw(ks, (uint64_t)(i * m + j))) < density) ++nnz;
  gen_csr* a = csr_alloc(n, m, nnz);
  if (!a) return NULL;
  int64_t p = 0;
  for (int64_t i = 0; i < n; ++i) {
    a->rowptr[i] = p;
    for (int64_t j = 0; j < m; ++j)
      if (sm_u01(sm_draw(ks, (uint64_t)(i * m + j))) < density) a->colidx[p++] = (int32_t)j;
  }
  a->rowptr[n] = p;
  fill_values_normal(a, seed);
  return a;
}
