/*
 * CPU oracle for the beta(r,c) sparse matrix-vector product (Bramas & Kus,
 * "Computing the sparse matrix vector product using block-based kernels
 * without zero padding on processors with AVX-512 instructions", 2018).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, obviously correct float64 code. Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark call
 * it; the CUDA library shares no code with it.
 *
 * Compile with -ffp-contract=off: the compensated dot product relies on every
 * product and sum being rounded exactly as written.
 *
 * Conventions
 *   CSR (section "Sparse Matrix Vector Product (SpMV)"): rowptr int64[n+1],
 *   colidx int32[nnz] ascending per row, values float64[nnz] row after row.
 *   beta(r,c) (section "Block-based storage without zero padding", Eq. 1):
 *   blocks are r rows high, start at a row multiple of r and at any column.
 *   I = ceil(n/r) row intervals.
 *     block_rowptr int32[I+1]  prefix of the number of blocks per interval,
 *     block_colidx int32[Nb]   column of the block's upper-left corner,
 *     block_masks  uint8[Nb*mb] one r*c-bit string per block, mb =
 *                  ceil(r*c/8) bytes; bit (i*c + k) is row i, column k of the
 *                  block; bit 0 is the least significant bit of byte 0,
 *     values       float64[nnz] in block order, row-major inside a block.
 *   The block start rule is not stated in the paper; the oracle takes greedy
 *   leftmost cover: in an interval, a block starts at the smallest column not
 *   yet covered and spans c columns. Blocks may run past column m-1; their
 *   mask bits there are zero. Rows past n in the last interval have zero bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_EUNSORTED 2
#define OR_EDUP 3
#define OR_ERANGE 4

static inline int mask_bytes(int r, int c) { return (r * c + 7) / 8; }
static inline int get_bit(const uint8_t* m, int b) { return (m[b >> 3] >> (b & 7)) & 1; }
static inline void set_bit(uint8_t* m, int b) { m[b >> 3] |= (uint8_t)(1u << (b & 7)); }

/* --------------------------------------------------------------- CSR SpMV */

/* y_i = sum over the stored entries of row i of values * x[colidx], in stored
 * order (section "Sparse Matrix Vector Product (SpMV)", CSR definition). */
void or_csr_spmv(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* val,
                 const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[colidx[p]];
    y[i] = s;
  }
}

/* The same loop with the rows shared among OpenMP threads (CPU baseline). */
void or_csr_spmv_omp(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* val,
                     const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[colidx[p]];
    y[i] = s;
  }
}

int or_omp_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Error-free transformations (Ogita, Rump & Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26(6), 2005): TwoSum (Knuth) and TwoProduct
 * through a fused multiply-add. */
static inline void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static inline void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/* Dot2 of Ogita, Rump & Oishi (Algorithm 5.3) per row: the result is as
 * accurate as if computed in twice the working precision, then rounded.
 * absy receives sum |a_ij| |x_j| (the scale of the tolerance). */
void or_csr_spmv_dot2(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* val,
                      const double* x, double* y, double* absy) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    double p = 0.0, s = 0.0, a = 0.0;
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      double h, r, t;
      two_prod(val[q], x[colidx[q]], &h, &r);
      two_sum(p, h, &p, &t);
      s += t + r;
      a += fabs(val[q]) * fabs(x[colidx[q]]);
    }
    y[i] = p + s;
    if (absy) absy[i] = a;
  }
}

/* ----------------------------------------------------------- validation */

/* Rows must list columns in ascending order (the CSR definition) without
 * repeats, inside [0, m). Returns an OR_* code and the first bad row. */
int or_csr_validate(int64_t n, int64_t m, const int64_t* rowptr, const int32_t* colidx, int64_t* bad_row) {
  if (rowptr[0] != 0) { *bad_row = 0; return OR_EINVAL; }
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) { *bad_row = i; return OR_EINVAL; }
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (colidx[p] < 0 || colidx[p] >= m) { *bad_row = i; return OR_ERANGE; }
      if (p > rowptr[i]) {
        if (colidx[p] == colidx[p - 1]) { *bad_row = i; return OR_EDUP; }
        if (colidx[p] < colidx[p - 1]) { *bad_row = i; return OR_EUNSORTED; }
      }
    }
  }
  *bad_row = -1;
  return OR_OK;
}

/* ------------------------------------------------------- CSR -> beta(r,c) */

/* Blocks of one interval under greedy leftmost cover. heads[i] walks row i. */
static int64_t interval_cover(const int64_t* rowptr, const int32_t* colidx, int64_t row0, int rows, int c,
                              int64_t* heads, int32_t* starts /* may be NULL */) {
  for (int i = 0; i < rows; ++i) heads[i] = rowptr[row0 + i];
  int64_t nb = 0;
  for (;;) {
    int64_t s = -1;
    for (int i = 0; i < rows; ++i)
      if (heads[i] < rowptr[row0 + i + 1] && (s < 0 || colidx[heads[i]] < s)) s = colidx[heads[i]];
    if (s < 0) break;
    for (int i = 0; i < rows; ++i)
      while (heads[i] < rowptr[row0 + i + 1] && colidx[heads[i]] < s + c) ++heads[i];
    if (starts) starts[nb] = (int32_t)s;
    ++nb;
  }
  return nb;
}

/* Number of blocks of every interval; returns N_blocks(r,c). */
int64_t or_beta_count(int64_t n, const int64_t* rowptr, const int32_t* colidx, int r, int c, int32_t* counts) {
  int64_t I = (n + r - 1) / r, total = 0;
  int64_t heads[64];
  for (int64_t it = 0; it < I; ++it) {
    int rows = (int)((it + 1) * r <= n ? r : n - it * r);
    int64_t nb = interval_cover(rowptr, colidx, it * r, rows, c, heads, NULL);
    if (counts) counts[it] = (int32_t)nb;
    total += nb;
  }
  return total;
}

/* Fill the four beta(r,c) arrays. The caller sizes them with or_beta_count:
 * block_rowptr[I+1], block_colidx[Nb], block_masks[Nb*mb] (zeroed here),
 * bvalues[nnz]. */
int or_beta_convert(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* val, int r, int c,
                    int32_t* block_rowptr, int32_t* block_colidx, uint8_t* block_masks, double* bvalues) {
  if (r < 1 || r > 64 || c < 1) return OR_EINVAL;
  int mb = mask_bytes(r, c);
  int64_t I = (n + r - 1) / r;
  int64_t heads[64];
  int64_t nb = 0, nv = 0;
  block_rowptr[0] = 0;
  for (int64_t it = 0; it < I; ++it) {
    int rows = (int)((it + 1) * r <= n ? r : n - it * r);
    int64_t row0 = it * r;
    for (int i = 0; i < rows; ++i) heads[i] = rowptr[row0 + i];
    for (;;) {
      int64_t s = -1;
      for (int i = 0; i < rows; ++i)
        if (heads[i] < rowptr[row0 + i + 1] && (s < 0 || colidx[heads[i]] < s)) s = colidx[heads[i]];
      if (s < 0) break;
      uint8_t* mk = block_masks + nb * mb;
      memset(mk, 0, (size_t)mb);
      /* row-major inside the block: row 0's entries, then row 1's, ... */
      for (int i = 0; i < rows; ++i)
        while (heads[i] < rowptr[row0 + i + 1] && colidx[heads[i]] < s + c) {
          set_bit(mk, i * c + (int)(colidx[heads[i]] - s));
          bvalues[nv++] = val[heads[i]];
          ++heads[i];
        }
      block_colidx[nb] = (int32_t)s;
      ++nb;
    }
    block_rowptr[it + 1] = (int32_t)nb;
  }
  return OR_OK;
}

/* beta(r,c) -> CSR. Walks the blocks of each interval in order and, for each
 * set bit (i*c + k) in bit order, emits (r*interval + i, colidx + k, next
 * value). Entries of one row come out in ascending column order because the
 * blocks of an interval do not overlap and are stored left to right. */
int or_beta_expand(int64_t n, int r, int c, const int32_t* block_rowptr, const int32_t* block_colidx,
                   const uint8_t* block_masks, const double* bvalues, int64_t* rowptr, int32_t* colidx,
                   double* val) {
  int mb = mask_bytes(r, c);
  int64_t I = (n + r - 1) / r;
  /* pass 1: row lengths from the masks */
  memset(rowptr, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t it = 0; it < I; ++it)
    for (int64_t b = block_rowptr[it]; b < block_rowptr[it + 1]; ++b)
      for (int i = 0; i < r; ++i)
        for (int k = 0; k < c; ++k)
          if (get_bit(block_masks + b * mb, i * c + k)) {
            int64_t row = it * r + i;
            if (row >= n) return OR_ERANGE;
            rowptr[row + 1]++;
          }
  for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  /* pass 2: scatter */
  int64_t* fillp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fillp) return OR_EINVAL;
  memcpy(fillp, rowptr, sizeof(int64_t) * (size_t)n);
  int64_t v = 0;
  for (int64_t it = 0; it < I; ++it)
    for (int64_t b = block_rowptr[it]; b < block_rowptr[it + 1]; ++b)
      for (int i = 0; i < r; ++i)
        for (int k = 0; k < c; ++k)
          if (get_bit(block_masks + b * mb, i * c + k)) {
            int64_t row = it * r + i;
            colidx[fillp[row]] = block_colidx[b] + k;
            val[fillp[row]] = bvalues[v++];
            fillp[row]++;
          }
  free(fillp);
  return OR_OK;
}

/* y += A x on the beta(r,c) arrays, from the storage definition (section
 * "Block-based storage without zero padding", Eq. 1): the stored values are
 * the blocks' nonzeros, block after block, and inside a block in the order of
 * the set mask bits (row-major, bit i*c + k = row i, column k). Step 1 turns
 * the arrays back into one (row, column, value) triple per stored value;
 * step 2 forms t[row] = sum of value * x[column] over the row's triples in
 * storage order, then adds t to y (the paper's kernels accumulate into y).
 * A row's triples come out left to right (an interval's blocks are disjoint
 * and stored in column order), so t[row] takes the same additions as the
 * plain CSR loop. Returns OR_ERANGE if a set bit lies past row n-1. */
int or_beta_spmv(int64_t n, int r, int c, const int32_t* block_rowptr, const int32_t* block_colidx,
                 const uint8_t* block_masks, const double* bvalues, const double* x, double* y) {
  const int mb = mask_bytes(r, c);
  const int64_t nint = (n + r - 1) / r;
  const int64_t nblocks = nint > 0 ? block_rowptr[nint] : 0;
  int64_t ntrip = 0;
  for (int64_t q = 0; q < nblocks * mb; ++q)
    for (int bit = 0; bit < 8; ++bit) ntrip += (block_masks[q] >> bit) & 1;
  int64_t* trow = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntrip > 0 ? ntrip : 1));
  int64_t* tcol = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntrip > 0 ? ntrip : 1));
  double* t = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!trow || !tcol || !t) {
    free(trow);
    free(tcol);
    free(t);
    return OR_EINVAL;
  }
  /* step 1: triples; the value of triple j is bvalues[j] */
  int64_t j = 0;
  int st = OR_OK;
  for (int64_t interval = 0; interval < nint; ++interval)
    for (int64_t blk = block_rowptr[interval]; blk < block_rowptr[interval + 1]; ++blk)
      for (int bit = 0; bit < r * c; ++bit)
        if (get_bit(block_masks + blk * mb, bit)) {
          trow[j] = interval * r + bit / c;
          tcol[j] = (int64_t)block_colidx[blk] + bit % c;
          if (trow[j] >= n) st = OR_ERANGE;
          ++j;
        }
  /* step 2: row sums in storage order, then y += t */
  if (st == OR_OK) {
    for (int64_t q = 0; q < ntrip; ++q) t[trow[q]] += bvalues[q] * x[tcol[q]];
    for (int64_t i = 0; i < n; ++i) y[i] += t[i];
  }
  free(trow);
  free(tcol);
  free(t);
  return st;
}

/* ----------------------------------------------------------- partition */

/* Static partition of the row intervals among nthreads (section
 * "Parallelization"): walking the intervals in order, the next interval joins
 * thread t's range unless that moves the range's block prefix farther from the
 * target (t+1)*Nb/T, i.e. while |target - prefix[row+1]| <= |target -
 * prefix[row]|, so each boundary lands on the prefix nearest to its target
 * (empty intervals are absorbed). The comparison in the paper's text reads
 * reversed; this is the reading that balances the blocks. The distances are
 * compared exactly, scaled by T: |(t+1)*Nb - T*prefix|. bounds receives
 * nthreads+1 interval indices. */
static int64_t or_absdiff(int64_t a, int64_t b) { return a > b ? a - b : b - a; }

void or_partition(int64_t nintervals, const int32_t* block_rowptr, int nthreads, int64_t* bounds) {
  const int64_t nb = block_rowptr[nintervals];
  int64_t row = 0;
  bounds[0] = 0;
  for (int t = 0; t < nthreads; ++t) {
    const int64_t target = (int64_t)(t + 1) * nb; /* scaled by nthreads */
    while (row < nintervals && or_absdiff(target, (int64_t)nthreads * block_rowptr[row + 1]) <=
                                   or_absdiff(target, (int64_t)nthreads * block_rowptr[row]))
      ++row;
    if (t == nthreads - 1) row = nintervals;
    bounds[t + 1] = row;
  }
}
