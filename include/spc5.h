/*
 * spc5.h - C ABI of the GB300 beta(r,c) sparse matrix-vector product library.
 *
 * The method is the mask-based block storage of Bramas & Kus (2018),
 * "Computing the sparse matrix vector product using block-based kernels
 * without zero padding": a matrix is cut into r-row intervals; each interval
 * is covered by r x c blocks that start at any column; a block stores one
 * column index, an r*c-bit mask and only its nonzero values (section "Block-
 * based storage without zero padding", Eq. 1). y = A x is computed over that
 * storage (Algorithm 1).
 *
 * General rules for every entry point:
 *   - Pointers named *_d are device pointers (cudaMalloc'd or equivalent) on
 *     the current CUDA device; pointers without the suffix are host pointers.
 *   - The caller owns every buffer it passes. A handle owns the device arrays
 *     the library allocated for it and frees them in spc5_destroy.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream). Calls return once the work is enqueued, except where a
 *     function's comment says it synchronises.
 *   - Errors are returned as spc5_status codes, never thrown or trapped on the
 *     device. Arguments are checked on the host before any launch.
 *     spc5_last_error() then gives a readable message (per host thread).
 *   - Block shapes: r in {1, 2, 4, 8}, c in {4, 8, 16}; other shapes return
 *     SPC5_EUNSUPPORTED.
 *   - Index limits: int32 column indices and block counts (the paper's
 *     S_integer = 4, Eq. 4), so m, nnz and N_blocks must be below 2^31; value
 *     offsets are int64.
 *   - Value types: SPC5_F64 stores float64 values and takes float64 x and y,
 *     accumulating in float64. SPC5_F32 and SPC5_BF16 store float32 or
 *     bfloat16 values and take float32 x and y, accumulating in float32.
 */
#ifndef SPC5_H
#define SPC5_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* spc5_stream_t; /* identical to cudaStream_t */
typedef struct spc5_matrix* spc5_handle;   /* opaque converted matrix */

typedef enum { SPC5_F64 = 0, SPC5_F32 = 1, SPC5_BF16 = 2 } spc5_dtype;

typedef enum {
  SPC5_OK = 0,
  SPC5_EINVAL = 1,       /* bad argument (null pointer, negative size, ...) */
  SPC5_EUNSORTED = 2,    /* a CSR row lists its columns out of order */
  SPC5_EDUP = 3,         /* a CSR row repeats a column */
  SPC5_ERANGE = 4,       /* a column index outside [0, m), or a size too big */
  SPC5_EUNSUPPORTED = 5, /* block shape or value type not built */
  SPC5_ENOMEM = 6,       /* device allocation failed */
  SPC5_ECUDA = 7,        /* a CUDA call failed; see spc5_last_error() */
  SPC5_ETIMEOUT = 8      /* a bounded device wait gave up */
} spc5_status;

/* Options of spc5_convert (pass NULL for the defaults). */
typedef struct {
  /* An interval with more than long_blocks blocks is processed by whole warps
   * in segments of seg_blocks blocks instead of one lane per row. 0 selects
   * the defaults: long_blocks = max(64, 4 x mean blocks per interval),
   * seg_blocks = 384. */
  int32_t long_blocks;
  int32_t seg_blocks;
  /* SpMV kernel variant for short intervals (one lane per row):
   *   0 or 5  natural interval order, next 2 nonzeros decoded per loop trip;
   *   3       natural order, 4 nonzeros per trip;
   *   1       natural order, one nonzero per trip (plain form);
   *   9 / 10  intervals taken in a work order sorted by row length inside
   *           windows of order_window rows (2 / 4 nonzeros per trip); the order is
   *           built at conversion.
   *   12 / 14 natural order, block masks read as 8-byte windows of 8/mb
   *           blocks (no memory round trip per block; for low fill),
   *           4 / 2 nonzeros per trip;
   *   13 / 15 sorted work order with mask windows, 4 / 2 nonzeros per trip;
   *   16 / 17 natural / sorted order, the c bit positions of a block row
   *           unrolled (fewest instructions for well-filled blocks; the
   *           float32 / bfloat16 choice);
   *   18 / 19 as 16 / 17 with two blocks per loop trip (c <= 8).
   *   22      r = 1 only (SPC5_EUNSUPPORTED otherwise): two lanes per row,
   *           lane g taking the row's stored values of rank g, g+2, ...
   *           (adjacent values read together, half the row's multiply-adds
   *           per lane); the two halves are added at the end, so its sums
   *           differ from the other variants' by rounding only.
   *   23      22 in the sorted work order (rows of similar length share a
   *           warp, so fewer lanes idle in each multiply-add); r = 1 only.
   *   24-27   G = 4 / 8 / 16 / 32 lanes per interval, one lane per block:
   *           the group reads G consecutive masks and column indices, a scan
   *           of their popcounts places each block's values, a shuffle tree
   *           adds the row sums (sums differ from 0-19 by rounding only);
   *   28 / 29 24 / 25 in the sorted work order.
   *   30 / 31 r = 1 only: Algorithm 2's single-value test, made once per
   *           row (a class bit built when the variant is selected): a row
   *           whose blocks all hold one value is read like CSR (no mask
   *           decode), other rows with the mask windows; sorted / natural
   *           order. Same sums as 0-19.
   *   32      r = 1 only: the warp streams the blocks of its 32 rows, two
   *           adjacent blocks per lane whatever row they belong to; a scan of
   *           the popcounts places the values, a segmented scan over the
   *           lanes adds each row's blocks, a row running past a trip carries
   *           its partial sum. Mask, column and value reads are consecutive
   *           over the warp and no lane idles on a shorter row; warps that
   *           hold a long interval take one lane per row instead. Sums differ
   *           from 0-19 by rounding only. A float32 / bfloat16 form (its
   *           float64 cost is set by the busiest lane's block).
   *   33      r = 1 only: 22 with Algorithm 2's single-value test (class bits
   *           built when the variant is selected): a row whose blocks all
   *           hold one value is read like a two-lane CSR row (no mask read);
   *           the same sums as 22, bit for bit.
   * spc5_cg uses the decode of 16 or 18 when its handle has that variant,
   * the flattened one otherwise.
   * Variants 0-19, 30 and 31 compute the same sums in the same order per
   * row, and so do 22 and 33; every variant repeats its own results bit for
   * bit. */
  int32_t variant;
  /* Rows per sorting window of the work order of the sorted variants:
   * 0 selects 1024; a negative value sorts all intervals together. */
  int32_t order_window;
  /* An interval holding more than long_values stored values is long too.
   * 0 selects max(8 x mean values per interval, 2048 r). Shards of one
   * matrix (spc5_convert_rows) given the same long_blocks and long_values
   * classify their intervals as the whole matrix would. */
  int32_t long_values;
  int32_t reserved[3];
} spc5_opts;

/* Read-only device views of a handle's arrays (layout of Eq. 1 plus derived
 * arrays), for tests and for users who keep the converted form. */
typedef struct {
  int64_t n, m, nnz, nblocks, nintervals;
  int32_t r, c, mask_bytes;
  spc5_dtype dtype;
  const int32_t* block_rowptr_d; /* int32[nintervals+1], prefix of blocks per interval */
  const int32_t* block_colidx_d; /* int32[nblocks], column of each block's upper-left corner */
  const uint8_t* block_masks_d;  /* uint8[nblocks*mask_bytes], bit i*c+k = (row i, col k), LSB first */
  const void* values_d;          /* dtype[nnz], block order, row-major inside a block */
  const int64_t* valptr_d;       /* int64[nintervals+1], first value of each interval (derived) */
  int64_t nsegments;             /* long-interval segments of the execution plan */
} spc5_arrays;

/*
 * spc5_convert - CSR -> beta(r,c) (section "Block-based storage without zero
 * padding"; conversion cost discussed in section "Test matrices").
 *   n, m, nnz   rows, columns and stored entries of the CSR matrix.
 *   rowptr_d    int64[n+1] device array, rowptr_d[0] = 0, rowptr_d[n] = nnz.
 *   colidx_d    int32[nnz] device array, ascending and unique within a row.
 *   values_d    dtype[nnz] device array (vt gives the type).
 *   r, c        block shape.
 *   opt         NULL or tuning options.
 *   out         receives the new handle (NULL on failure).
 * Block starts follow greedy leftmost cover: within an interval a block starts
 * at the smallest column not yet covered and spans c columns (it may run past
 * column m-1; those mask bits are zero). Explicit zeros are kept.
 * Errors: SPC5_EUNSORTED / SPC5_EDUP / SPC5_ERANGE for malformed CSR (checked
 * on the device, reported through a status word), SPC5_ENOMEM, SPC5_ECUDA.
 * Synchronises `stream` (the array sizes depend on the block count).
 */
spc5_status spc5_convert(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                         const void* values_d, spc5_dtype vt, int r, int c, const spc5_opts* opt,
                         spc5_stream_t stream, spc5_handle* out);

/*
 * spc5_convert_rows - CSR rows [row_begin, row_end) -> a beta(r,c) handle of
 * their own: one shard of the row-interval partition of section
 * "Parallelization" (each worker owns consecutive row intervals, balanced by
 * block count, see spc5_partition, and writes disjoint rows of y). The shard
 * keeps the full column space (x has m entries); its rows are numbered from
 * 0, so spc5_spmv(shard, x, y_d + row_begin) writes rows row_begin..row_end-1
 * of A x. row_begin must be a multiple of r (shards start at interval
 * boundaries), so a shard's intervals and blocks are those of the whole
 * matrix; with the same opt->long_blocks its products equal the rows of the
 * whole matrix's product bit for bit. Other arguments and errors as
 * spc5_convert (plus SPC5_EINVAL for bad bounds). Synchronises `stream`.
 */
spc5_status spc5_convert_rows(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              const void* values_d, spc5_dtype vt, int r, int c, int64_t row_begin, int64_t row_end,
                              const spc5_opts* opt, spc5_stream_t stream, spc5_handle* out);

/*
 * spc5_assemble - a handle from beta(r,c) arrays the caller built directly,
 * without a CSR (section "Block-based storage without zero padding": the
 * format is four arrays, Eq. 1, and the conclusion asks for producing it
 * natively). Device arrays, copied into the handle (the caller keeps its own):
 *   block_rowptr_d  int32[ceil(n/r)+1], rising from 0 to nblocks;
 *   block_colidx_d  int32[nblocks], first column of each block;
 *   block_masks_d   uint8[nblocks * ceil(r*c/8)], bit i*c+k = (row i, column
 *                   colidx+k), least significant bit first;
 *   values_d        nnz values of type vt in block order, row-major in a block.
 * Checked on the device: block_rowptr (SPC5_EINVAL); every block's column in
 * [0, m) and no set bit past column m-1 or row n-1 (SPC5_ERANGE); inside an
 * interval each block starts at or after the previous block's column + c
 * (SPC5_EUNSORTED); the masks hold exactly nnz bits (SPC5_EINVAL). The
 * message names the first bad block or interval. Sizes must fit int32
 * (SPC5_ERANGE). Options and variants as spc5_convert. Synchronises `stream`.
 */
spc5_status spc5_assemble(int64_t n, int64_t m, int64_t nnz, int64_t nblocks, const int32_t* block_rowptr_d,
                          const int32_t* block_colidx_d, const uint8_t* block_masks_d, const void* values_d,
                          spc5_dtype vt, int r, int c, const spc5_opts* opt, spc5_stream_t stream, spc5_handle* out);

/*
 * spc5_spmv - y = A x over the beta(r,c) storage (Algorithm 1; Code 1 shows
 * the paper's beta(1,8) kernel). x_d has m entries, y_d has n entries, both of
 * the handle's vector type; y is overwritten. x and y must not overlap.
 */
spc5_status spc5_spmv(spc5_handle h, const void* x_d, void* y_d, spc5_stream_t stream);

/*
 * spc5_spmv_acc - y += A x, the paper's accumulate form (Algorithm 1 adds the
 * row sums to y; Code 1 adds to y[row] too). Same arguments as spc5_spmv.
 */
spc5_status spc5_spmv_acc(spc5_handle h, const void* x_d, void* y_d, spc5_stream_t stream);

/*
 * spc5_set_variant - switch the short-interval kernel variant of a handle
 * (values as in spc5_opts.variant). Selecting 9, 10, 13, 15, 17, 19, 23, 28, 29 or 30
 * builds the sorted work order, and 30, 31 or 33 the single-value class bits, if
 * the handle has none yet (synchronises `stream`); the other values take
 * effect with no device work. SPC5_EINVAL for an unknown variant,
 * SPC5_EUNSUPPORTED for 22, 23 or 30 to 33 on a handle with r > 1.
 */
spc5_status spc5_set_variant(spc5_handle h, int variant, spc5_stream_t stream);

/*
 * spc5_autotune - time the short-interval kernel variants on this handle and
 * this GPU (median of `reps` SpMVs each, x_d / y_d as in spc5_spmv, y_d
 * overwritten) and keep the fastest; the GPU form of the paper's choice of
 * the best kernel for a matrix (section "Performance prediction and optimal
 * kernel selection"). Candidates: variants 5, 10, 13, 15, plus 16 and 18 for
 * float32 / bfloat16 values and 22, 23, 30, 33 for r = 1, and 32 for r = 1
 * with float32 / bfloat16 values (the ones that win on some matrix). Writes the
 * chosen variant and its median milliseconds (either pointer may be NULL).
 * Synchronises `stream`. On error the handle keeps its previous variant.
 */
spc5_status spc5_autotune(spc5_handle h, const void* x_d, void* y_d, int reps, int* variant_out, float* ms_out,
                          spc5_stream_t stream);

/*
 * spc5_spmv_noalloc - y = A x like spc5_spmv, for callers that cannot have a
 * library allocate device memory (their memory is owned by another
 * component's pool, or every allocation is budgeted up front). The paper has
 * no counterpart; this is an interface convenience.
 *   - Allocates nothing: the long-interval scratch lives in one fixed 4 MiB
 *     array inside the library's device image, resident on every GPU that
 *     loads the library until the process exits.
 *   - A handle needing more than 4 MiB of segment scratch (n_segments * r
 *     accumulators of 8 bytes for float64, 4 otherwise; see
 *     spc5_arrays.nsegments) is rejected with SPC5_ERANGE before any launch.
 *   - All calls on a device share that array: calls whose kernels may
 *     overlap on the GPU (unordered streams) race. Nothing needs clearing
 *     between calls.
 *   - The first call on each device looks up the array's address with that
 *     device current; make it before any stream capture begins.
 * Arguments, vector types and errors otherwise as spc5_spmv.
 */
spc5_status spc5_spmv_noalloc(spc5_handle h, const void* x_d, void* y_d, spc5_stream_t stream);

/* spc5_export - fill *view with the handle's device arrays (valid until
 * spc5_destroy). No device work. */
spc5_status spc5_export(spc5_handle h, spc5_arrays* view);

/* spc5_launch_count - number of kernels one spc5_spmv (or spc5_spmv_acc) on
 * this handle launches with its current variant: the short-interval grid
 * (shared with the long-interval segments unless variant 1 runs), a separate
 * segment kernel otherwise, and the segment fix-up. No device work. */
spc5_status spc5_launch_count(spc5_handle h, int* kernels_out);

/* spc5_device_peaks - properties of the current device for roofline
 * reports: the nominal DRAM bandwidth in GB/s (2 transfers per memory clock x
 * bus width, from the driver's attributes), the SM count and the maximum SM
 * clock in MHz. Any output pointer may be NULL (not all). No device work. */
spc5_status spc5_device_peaks(double* hbm_gbs_out, int* sm_count_out, int* sm_clock_mhz_out);

/* spc5_destroy - free the handle and its device arrays (synchronises the
 * device first so that no queued kernel still reads them). NULL is allowed.
 * The arrays of converted handles go back to a memory pool of the library's
 * own (one per device), which keeps them for the next conversion instead of
 * returning them to the driver; see spc5_pool_trim. */
spc5_status spc5_destroy(spc5_handle h);

/* spc5_pool_trim - return the memory the library's handle pools keep for
 * reuse to the driver (the arrays of live handles stay). No device work. */
spc5_status spc5_pool_trim(void);

/* spc5_last_error - message of the last failed call on this host thread. */
const char* spc5_last_error(void);

/*
 * spc5_count_blocks - N_blocks(r,c) of a CSR matrix without converting it
 * (section "Performance polynomial interpolation": the average number of
 * values per block, Avg(r,c) = nnz / N_blocks(r,c), is obtained without
 * conversion). Counts all twelve built shapes in one call: nblocks_out[12]
 * receives N_blocks for (r,c) in the order r in {1,2,4,8} outer, c in
 * {4,8,16} inner. Host output; synchronises `stream`. The CSR must be valid
 * (see spc5_convert); it is not re-checked.
 */
spc5_status spc5_count_blocks(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              int64_t* nblocks_out, spc5_stream_t stream);

/*
 * spc5_csr_spmv - y = A x directly on CSR (the comparison format of the paper,
 * section "Sparse Matrix Vector Product (SpMV)"). Same types and vector rules
 * as spc5_spmv for value type vt. rowptr_d/colidx_d/values_d as in
 * spc5_convert; the CSR is not re-checked. group = lanes per row (1, 2, 4, 8,
 * 16 or 32), or 0 to pick it from the mean row length.
 */
spc5_status spc5_csr_spmv(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                          const void* values_d, spc5_dtype vt, const void* x_d, void* y_d, int group,
                          spc5_stream_t stream);

/* CSR with long rows split (the comparator with the β path's load balancing) */
typedef struct spc5_csr_plan_s* spc5_csr_plan;

/*
 * spc5_csr_plan_create - an execution plan for y = A x on plain CSR that
 * balances power-law rows the way the β path does: rows of more than
 * long_len entries are cut into segments of seg_len entries, one warp per
 * segment (partial sums, then a fix-up adds a row's segments in order), and
 * the other rows take `group` lanes each, all in one grid. rowptr_d (int64,
 * n + 1) is the caller's and must stay valid and unchanged while the plan
 * lives. group as spc5_csr_spmv (0 = from the mean row length); long_len 0 =
 * max(1024, 16 x mean row length); seg_len 0 = 1024. Synchronises `stream`.
 */
spc5_status spc5_csr_plan_create(int64_t n, int64_t nnz, const int64_t* rowptr_d, spc5_dtype vt, int group,
                                 int64_t long_len, int64_t seg_len, spc5_stream_t stream, spc5_csr_plan* out);

/* spc5_csr_spmv_plan - y = A x with a plan (colidx_d, values_d of the
 * plan's CSR; types and vectors as spc5_csr_spmv). Runs repeat bit for bit. */
spc5_status spc5_csr_spmv_plan(spc5_csr_plan p, const int32_t* colidx_d, const void* values_d, const void* x_d,
                               void* y_d, spc5_stream_t stream);

/* spc5_csr_plan_info - the plan's lanes per short row, long-row threshold and
 * segment count (any output may be NULL). */
spc5_status spc5_csr_plan_info(spc5_csr_plan p, int* group_out, int64_t* long_len_out, int64_t* nseg_out);

/* spc5_csr_plan_destroy - free the plan (synchronises the device). NULL is allowed. */
spc5_status spc5_csr_plan_destroy(spc5_csr_plan p);

/*
 * spc5_partition - the static partition of the row intervals among `nparts`
 * workers (section "Parallelization"): walking the intervals in order, the
 * next interval joins part t while that does not move the part's block prefix
 * farther from its target (t+1) * N_b / nparts, so every boundary lands on the
 * block prefix nearest to its target and empty intervals are absorbed; the
 * last part ends at the last interval. The distances are compared exactly (in
 * integers scaled by nparts). Host function, no device work.
 *   block_rowptr  HOST int32[nintervals+1], a block prefix (rising from 0),
 *                 e.g. a host copy of spc5_arrays.block_rowptr_d.
 *   bounds_out    HOST int64[nparts+1]: part t owns intervals
 *                 [bounds_out[t], bounds_out[t+1]).
 * SPC5_EINVAL for NULL pointers, nintervals < 0 or nparts < 1.
 */
spc5_status spc5_partition(const int32_t* block_rowptr, int64_t nintervals, int nparts, int64_t* bounds_out);

/*
 * spc5_copy - dst = src for `bytes` bytes (a multiple of 16, both pointers
 * 16-byte aligned): the streaming-copy kernel that measures the achievable
 * HBM bandwidth next to the SpMV kernels.
 */
spc5_status spc5_copy(const void* src_d, void* dst_d, int64_t bytes, spc5_stream_t stream);

/*
 * spc5_spmm - Y = A X for k right-hand sides (the paper cites multiplying by
 * several vectors as a way to reuse the matrix stream, section "Sparse Matrix
 * Vector Product (SpMV)").
 *   X_d   m-by-k, row-major, leading dimension ldx >= k (row j at X_d + j*ldx).
 *   Y_d   n-by-k, row-major, leading dimension ldy >= k; overwritten.
 *   Element type of X and Y: float64 for SPC5_F64 handles, float32 otherwise.
 *   k     1..1024; ktile = column tile: 1, 4, -8, -16 or -32 (one lane per
 *         row holding 1 to 32 columns; X rows read as 16-byte vectors when
 *         X_d is 16-byte aligned and ldx a multiple of 16 bytes), 8, 16 or 32
 *         (ktile / 4 lanes per row interval, 4 columns each: per stored value
 *         the group reads one coalesced ktile-wide slice of its X row); 0 =
 *         choose from k. The grid covers ceil(k / |ktile|)
 *         tiles. k = 1 with ldx = ldy = 1 and ktile 0 or 1 is the SpMV
 *         (spc5_spmv, the handle's variant).
 * Long intervals of beta(1,c) with k >= 4: a warp per segment, groups of 1, 2,
 * 4 or 8 lanes taking its blocks in turn, 4 columns per lane (one coalesced
 * X row slice per stored value and group). A handle with long intervals keeps
 * n_segments * r * k partial sums; the first call with a larger k grows that
 * buffer (cudaMalloc, device synchronisation).
 */
spc5_status spc5_spmm(spc5_handle h, int k, const void* X_d, int64_t ldx, void* Y_d, int64_t ldy, int ktile,
                      spc5_stream_t stream);

/* ------------------------------------------------------- SM-limited streams */
/*
 * spc5_sm_stream_create - a stream whose kernels run on about `sms` SMs of the
 * current device only: the SM-count axis that stands in, on one GPU, for the
 * thread count of the paper's parallel predictor (section "Performance
 * prediction and optimal kernel selection"). Built on a green context (a
 * process-local SM partition; no device setting changes): the count is
 * rounded up to the driver's partition granularity (a multiple of 8 SMs on
 * this architecture) and written to *sms_out (nullable); sms at or above the
 * SM count gives the whole GPU. Any library call may be given the stream.
 * SPC5_EUNSUPPORTED when the driver offers no green contexts.
 */
spc5_status spc5_sm_stream_create(int sms, spc5_stream_t* stream_out, int* sms_out);

/* spc5_sm_stream_destroy - synchronise and free a stream of
 * spc5_sm_stream_create (and its green context). NULL is allowed. */
spc5_status spc5_sm_stream_destroy(spc5_stream_t stream);

/* ------------------------------------------------------------------ tuner */
#define SPC5_TUNE_NO_CACHE 1 /* spc5_tune flag: time again even when the signature is known */

typedef struct {
  int32_t r, c;       /* SpMV: fastest block shape */
  int32_t variant;    /* SpMV: fastest kernel variant on that shape (spc5_opts.variant) */
  float spmv_ms;      /* SpMV: its median milliseconds */
  int32_t spmm_r, spmm_c, ktile; /* SpMM (k_spmm > 0): fastest shape and column tile */
  float spmm_ms;      /* SpMM: its median milliseconds (-1 when k_spmm == 0) */
  int32_t from_cache; /* 1 when the result came from the signature cache */
  int32_t spmm_variant; /* SpMM: the fastest SpMV variant on the SpMM shape (k = 1 runs the SpMV) */
  uint64_t signature; /* the matrix signature the cache is keyed on */
} spc5_tune_result;

/*
 * spc5_tune - the library's autotuner: times every block shape (twelve) x the
 * kernel variants that win on some matrix (float64: 5, 10, 13, 15, 24;
 * float32 / bfloat16 also 16, 18; r = 1 also 22, 23, 30, 31, 33, and 32
 * for float32 / bfloat16) and, when
 * k_spmm > 0, every shape x SpMM column tile for k_spmm right-hand sides, on
 * this GPU (median of `reps` products after one untimed product, no cache
 * flush between them), and returns the fastest choices - the GPU form of the
 * paper's choice of the best kernel per matrix (section "Performance
 * prediction and optimal kernel selection"). The result is remembered per
 * matrix signature (n, m, nnz, value type, k_spmm, SM count, the twelve
 * N_blocks(r,c), the longest row): a later call with an equal signature
 * returns it without timing (from_cache = 1) unless flags has
 * SPC5_TUNE_NO_CACHE. The cache lives until spc5_tune_cache_clear or the end
 * of the process and is shared by all host threads.
 *   CSR arguments as spc5_convert (checked there: SPC5_EUNSORTED, ...);
 *   reps >= 1; 0 <= k_spmm <= 1024.
 * Allocates its work vectors from the stream-ordered pool; synchronises
 * `stream`.
 */
spc5_status spc5_tune(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                      const void* values_d, spc5_dtype vt, int k_spmm, int reps, int flags, spc5_tune_result* out,
                      spc5_stream_t stream);

/* spc5_tune_cache_clear - forget every remembered tuning result. */
spc5_status spc5_tune_cache_clear(void);

/* ----------------------------------------------------------------- batches */
typedef struct spc5_batch_s* spc5_batch; /* opaque batched product */

/*
 * spc5_batch_create - prepare y_j = A_j x_j for `count` handles of one value
 * type (each with its own block shape and variant) as one graph launch: the
 * short intervals of all matrices are cut into work items of 32/r intervals,
 * grouped by (block shape, row decode of the matrix's variant), one kernel per
 * group compiled for it (one warp per item); the long intervals become warp
 * segments that persistent warps take from a shared counter, then a fix-up.
 * The groups run on side streams beside the segments. The row decode: mask
 * windows (variants 12-15), Algorithm 2's test (30, 31, 33), unrolled bit
 * positions (16-19), flattened (0-10); the many-lane variants (22-29, 32) take
 * the unrolled decode for float32 / bfloat16 and the mask windows for float64.
 * A matrix whose decode sums in storage order gives the bits of its single
 * product. x_d[j] / y_d[j]: device vectors of matrix j (fixed for the batch's
 * lifetime; refill them in place between products). Everything is captured
 * into a CUDA graph here. The handles must outlive the batch. Synchronises
 * the device.
 */
spc5_status spc5_batch_create(const spc5_handle* mats, const void* const* x_d, void* const* y_d, int count,
                              spc5_batch* out);

/* spc5_batch_spmv - all products of the batch: one graph launch on `stream`. */
spc5_status spc5_batch_spmv(spc5_batch b, spc5_stream_t stream);

/* spc5_batch_spmv_direct - the same products launched without the graph. */
spc5_status spc5_batch_spmv_direct(spc5_batch b, spc5_stream_t stream);

/* spc5_batch_destroy - free the batch (not its handles); NULL is allowed. */
spc5_status spc5_batch_destroy(spc5_batch b);

/* Options of spc5_cg (zero fields select the defaults in brackets). */
typedef struct {
  double tol;              /* stop when ||b - A x||_2 <= tol ||b||_2              [1e-10] */
  int32_t max_iters;       /* CG iterations in total (inner ones when mixed)      [100000] */
  int32_t max_outer;       /* refinement steps of the mixed solver                [30] */
  double inner_tol;        /* tightest relative reduction asked of an inner solve;
                              each inner solve stops at max(inner_tol,
                              0.5 tol ||b|| / ||r||) (no further than the final
                              tolerance needs)                                  [1e-6] */
  int32_t inner_max_iters; /* iterations of one inner solve                       [2000] */
  int32_t check_every;     /* iterations before the first host read of the residual
                              norm; later reads are placed where the observed
                              convergence rate predicts the stop (between
                              check_every/4 and 8 x check_every apart); 1 reads
                              after every iteration (exact stopping point)       [8] */
  int32_t use_graph;       /* replay the iteration from a captured CUDA graph     [0: off] */
  int32_t reliable;        /* with A_inner: 1 = one float32 CG recurrence with
                              reliable updates (the float64 residual replaces
                              the recurred one whenever its norm fell 10x; no
                              restarts) instead of refinement   [0: refinement] */
  int32_t reserved[4];
} spc5_cg_opts;

typedef struct {
  int32_t iterations;  /* CG iterations run (float64 CG) or inner iterations in total (mixed) */
  int32_t outer;       /* refinement steps (mixed), 0 for float64 CG */
  int32_t inner_total; /* inner iterations in total (mixed) */
  int32_t converged;   /* 1 when rel_residual <= tol */
  double rel_residual; /* ||b - A x||_2 / ||b||_2 of the returned x, recomputed in float64 */
} spc5_cg_info;

/*
 * spc5_cg - solve A x = b for symmetric positive definite A by conjugate
 * gradients (Hestenes & Stiefel), the kind of iterative solver whose many
 * SpMVs with one matrix the paper targets (Introduction).
 *   A        SPC5_F64 handle, n == m.
 *   A_inner  NULL: plain float64 CG on A. Otherwise an SPC5_F32 or SPC5_BF16
 *            handle of the same matrix: mixed-precision iterative refinement
 *            - the residual r = b - A x, the update x += d and all norms in
 *            float64 with A; each correction d solved by CG in float32 with
 *            A_inner on r / ||r|| to a relative reduction inner_tol. With
 *            opt->reliable, one float32 CG recurrence on A_inner instead,
 *            its residual replaced by the float64 b - A x (and its iterate
 *            folded into x) whenever the recurred norm fell by 10x
 *            (info->outer counts these updates).
 *   b_d, x_d float64 device vectors of n entries; x is overwritten (the
 *            iteration starts from x = 0).
 *   info     receives iteration counts and the true relative residual.
 * Dot products reduce in a fixed order (run-to-run reproducible). Allocates
 * its workspace (a few vectors); synchronises `stream`. Returns SPC5_OK also
 * when the tolerance was not reached (see info->converged).
 */
spc5_status spc5_cg(spc5_handle A, spc5_handle A_inner, const double* b_d, double* x_d, const spc5_cg_opts* opt,
                    spc5_cg_info* info, spc5_stream_t stream);

/* ------------------------------------------------------------- selection */
#define SPC5_NFEATURES 16
#define SPC5_NFORMATS 12 /* r in {1,2,4,8} outer, c in {4,8,16} inner */

/*
 * spc5_features - the selection features of a CSR matrix, without converting
 * it (the paper's predictor uses Avg(r,c) = N_nnz / N_blocks(r,c), which is
 * cheap to obtain, section "Performance polynomial interpolation"; its
 * conclusion asks for more inputs): features_out[0..11] = Avg(r,c) for the
 * twelve shapes; [12], [13], [14] = mean, standard deviation and maximum of
 * the row lengths; [15] = log10(n). Host output (16 doubles); synchronises
 * `stream`. The CSR must be valid (not re-checked).
 */
spc5_status spc5_features(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                          double* features_out, spc5_stream_t stream);

/*
 * spc5_time_formats - the timing recorder: converts the CSR to each of the
 * twelve shapes and times `reps` SpMVs of each (after one untimed product),
 * writing the median milliseconds to ms_out[12] (host); for r = 1 the
 * shape's time is the faster of its default kernel and variant 22 (two
 * lanes per row). x_d / y_d: work vectors of the vector type (m and n
 * entries). Synchronises `stream`.
 */
spc5_status spc5_time_formats(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              const void* values_d, spc5_dtype vt, const void* x_d, void* y_d, int reps,
                              float* ms_out, spc5_stream_t stream);

/*
 * Format-scoring MLP: 16 -> 64 -> 64 -> 12, ReLU, float32, parameters flat in
 * the order W1[64][16], b1[64], W2[64][64], b2[64], W3[12][64], b3[12]
 * (spc5_mlp_nparams() floats, device memory). Inputs: x_q = (log1p(f_q) -
 * mean_q) / scale_q of the features f. Output: a score per format (the
 * trainer fits centred log times: lower is faster).
 */
int spc5_mlp_nparams(void);

/*
 * spc5_mlp_train - minibatch Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the
 * masked mean squared error sum(M (out - Y)^2) / sum(M). X_d: N x 16 inputs,
 * Y_d / M_d: N x 12 targets and 0/1 mask (device, row-major). batch 1..32;
 * samples are shuffled per epoch with `seed`. One fused kernel per step.
 * loss_history (host, `epochs` floats, nullable) receives the mean loss of
 * each epoch. Synchronises `stream`.
 */
spc5_status spc5_mlp_train(float* params_d, const float* X_d, const float* Y_d, const float* M_d, int N, int epochs,
                           int batch, float lr, uint64_t seed, float* loss_history, spc5_stream_t stream);

/*
 * spc5_mlp_grad - loss (host) and gradient (device, spc5_mlp_nparams()
 * floats) of the first B (1..32) samples, parameters unchanged.
 */
spc5_status spc5_mlp_grad(const float* params_d, const float* X_d, const float* Y_d, const float* M_d, int B,
                          float* loss_out, float* grad_d, spc5_stream_t stream);

/* spc5_mlp_infer - scores (N x 12, device) of N input rows (N x 16, device). */
spc5_status spc5_mlp_infer(const float* params_d, const float* X_d, int N, float* out_d, spc5_stream_t stream);

/*
 * Richer selection inputs (the paper's conclusion asks for statistics beyond
 * Avg(r,c) and hardware properties; its interpolation section names the
 * block distribution's effect on the x accesses as what Avg cannot tell).
 * spc5_features_ext fills 20 host doubles: [0..15] as spc5_features, [16] the
 * mean distance |col - row| of the entries from the diagonal divided by n,
 * [17] log10(1 + that mean distance), [18] the fraction of rows with at most
 * two entries, [19] sm_frac (the fraction of the SMs the products will use,
 * in (0, 1]: the hardware input). Synchronises `stream`.
 */
spc5_status spc5_features_ext(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              double sm_frac, double* features_out, spc5_stream_t stream);

/* The MLP with nfeat = 16 or 20 inputs (W1 is 64 x nfeat, the rest as above):
 * parameter count (-1 for another nfeat), training, gradient and inference as
 * spc5_mlp_train / spc5_mlp_grad / spc5_mlp_infer. */
int spc5_mlp_nparams_n(int nfeat);
spc5_status spc5_mlp_train_n(float* params_d, const float* X_d, const float* Y_d, const float* M_d, int N, int nfeat,
                             int epochs, int batch, float lr, uint64_t seed, float* loss_history,
                             spc5_stream_t stream);
spc5_status spc5_mlp_grad_n(const float* params_d, const float* X_d, const float* Y_d, const float* M_d, int B,
                            int nfeat, float* loss_out, float* grad_d, spc5_stream_t stream);
spc5_status spc5_mlp_infer_n(const float* params_d, const float* X_d, int N, int nfeat, float* out_d,
                             spc5_stream_t stream);

/*
 * spc5_poly_fit - the paper's per-kernel polynomial interpolation: for each
 * format f, least-squares coefficients c_0..c_d of perf[:, f] ~ sum_j c_j
 * avg[:, f]^j (Householder QR). avg, perf: N x 12 host arrays; coef_out:
 * 12 x (degree + 1) host array. 0 <= degree <= 6, N > degree.
 */
spc5_status spc5_poly_fit(const double* avg, const double* perf, int N, int degree, double* coef_out);

/*
 * spc5_poly2_fit - the paper's parallel predictor (section "Performance
 * prediction and optimal kernel selection", parallel part: a regression of
 * each kernel's performance on two parameters, the number of threads and
 * Avg(r,c)). Here the second parameter is the fraction s of the SMs a product
 * may use (see spc5_sm_stream_create). For each format f, least-squares
 * coefficients of perf[:, f] ~ sum of c_q Avg^a s^b over a + b <= degree,
 * the terms ordered by total degree t = a + b, then by b (so q = 0 is 1,
 * q = 1 Avg, q = 2 s, q = 3 Avg^2, ...). avg, perf: N x 12 host arrays;
 * sm_frac: N host values; coef_out: 12 x (degree+1)(degree+2)/2. 0 <=
 * degree <= 4, N >= the number of terms. Host function.
 */
spc5_status spc5_poly2_fit(const double* avg, const double* sm_frac, const double* perf, int N, int degree,
                           double* coef_out);

/* spc5_poly2_select - the format with the highest spc5_poly2_fit estimate at
 * the matrix's features (spc5_features, host, 16 values) and SM fraction
 * sm_frac; est_out (nullable, 12) receives the estimates. Host function. */
spc5_status spc5_poly2_select(const double* coef, int degree, const double* features, double sm_frac, int* r_out,
                              int* c_out, double* est_out);

typedef enum { SPC5_SELECT_EXHAUSTIVE = 0, SPC5_SELECT_POLY = 1, SPC5_SELECT_MLP = 2 } spc5_select_method;

typedef struct {
  int32_t poly_degree;      /* POLY: degree of the fitted polynomials */
  const double* poly_coef;  /* POLY: host, 12 x (degree + 1), from spc5_poly_fit on GFLOP/s */
  const float* mlp_params_d;/* MLP: device parameters */
  float feat_mean[SPC5_NFEATURES];  /* MLP input standardisation (see above) */
  float feat_scale[SPC5_NFEATURES];
} spc5_selector;

/*
 * spc5_select - pick a block shape for a CSR matrix before converting it
 * (section "Performance prediction and optimal kernel selection").
 *   EXHAUSTIVE  time every shape (spc5_time_formats) and take the fastest;
 *               needs values_d and vt; model unused.
 *   POLY        highest polynomial estimate of GFLOP/s at the matrix's Avg(r,c).
 *   MLP         lowest MLP score.
 * r_out, c_out: the choice; score_out (host, 12 floats, nullable): the
 * per-format times (EXHAUSTIVE, ms), estimates (POLY) or scores (MLP).
 * Synchronises `stream`.
 */
spc5_status spc5_select(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                        const void* values_d, spc5_dtype vt, int method, const spc5_selector* model, int* r_out,
                        int* c_out, float* score_out, spc5_stream_t stream);

/*
 * spc5_fma_rate - launch an arithmetic-rate probe: 8 CTAs of 256 threads per
 * SM, each thread running 8 independent fused multiply-add chains for `iters`
 * trips in float64 (vt = SPC5_F64) or float32 (SPC5_F32). *fmas_out receives
 * the number of multiply-adds the launch performs; timing it with events on
 * `stream` gives the measured peak of the ALU roofline. sink_d: device buffer
 * of at least 256 elements of the type (written only in an impossible case).
 */
spc5_status spc5_fma_rate(spc5_dtype vt, int64_t iters, void* sink_d, int64_t* fmas_out, spc5_stream_t stream);

/*
 * spc5_fma_rate_lanes - the same probe with only lanes 0..lanes-1 of every
 * warp doing arithmetic (1 <= lanes <= 32; the others skip the loop while
 * their warp issues it). *fmas_out counts the active lanes' multiply-adds
 * only, so the rate shows what a partly filled warp instruction costs.
 * SPC5_EINVAL for lanes outside [1, 32] or the errors of spc5_fma_rate.
 */
spc5_status spc5_fma_rate_lanes(spc5_dtype vt, int64_t iters, int lanes, void* sink_d, int64_t* fmas_out,
                                spc5_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPC5_H */
