// Internal declarations shared by the translation units of libspc5.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/spc5.h"

namespace spc5 {

// Defaults of the execution plan: an interval with more than
// max(kLongBlocks, 4 x mean blocks per interval) blocks is split into
// segments of kSegBlocks blocks, each handled by a warp.
constexpr int kLongBlocks = 64;
constexpr int kSegBlocks = 384;  // measured best of 256 / 384 / 512 on R-MAT scale 22
constexpr int kWarp = 32;
// Threads per block of the SpMV grids (short intervals, segments, CSR
// comparator). Two warps per block: a block's slot on the SM frees as soon as
// its two warps finish, so warps with short rows do not wait on a longer
// neighbour before new work enters. Measured against 256 on GB300: R-MAT
// scale 22 float64 0.4625 -> 0.4308 ms, FEM float64 0.5045 -> 0.4942 ms,
// uniform 0.0518 -> 0.0498 ms, stencil 0.1256 -> 0.1235 ms.
constexpr int kSpmvThreads = 64;

constexpr int kOrderWindow = 1024;  // rows per sorting window of the work order (best of 1024 / 2048 / 4096)

// short-interval kernel variants (spc5_opts.variant)
inline bool valid_variant(int v) {
  return v == 0 || v == 1 || v == 3 || v == 5 || v == 9 || v == 10 || (v >= 12 && v <= 19) || v == 22 || v == 23 ||
         (v >= 24 && v <= 33);
}
// variants that need r = 1 (two lanes per row, Algorithm 2's test, block streaming)
inline bool r1_variant(int v) { return v == 22 || v == 23 || v == 30 || v == 31 || v == 32 || v == 33; }
// variants that take intervals in the sorted work order
inline bool ordered_variant(int v) {
  return v == 9 || v == 10 || v == 13 || v == 15 || v == 17 || v == 19 || v == 23 || v == 28 || v == 29 || v == 30;
}
// variants with G lanes per interval, one lane per block (spmv_group.cuh)
inline bool group_variant(int v) { return v >= 24 && v <= 29; }
// variants that read the single-value class bits (Algorithm 2's test)
inline bool single_variant(int v) { return v == 30 || v == 31; }
// variants that need the single-value class bits (30, 31 and the two-lane 33)
inline bool uses_single_bits(int v) { return single_variant(v) || v == 33; }
// the warp streams the blocks of its 32 rows, lane = block (spmv_stream.cuh)
inline bool stream_variant(int v) { return v == 32; }

struct Segment {  // one warp task of a long interval
  int32_t interval;
  int32_t b_begin;
  int32_t b_end;
  int32_t count;    // segments of the interval, in its first segment; 0 in the others
  int64_t v_begin;  // value offset of block b_begin
};
static_assert(sizeof(Segment) == 24, "segment layout");

}  // namespace spc5

struct spc5_matrix {
  int64_t n = 0, m = 0, nnz = 0;
  int32_t r = 0, c = 0, mb = 0;
  spc5_dtype vt = SPC5_F64;
  int64_t I = 0;        // number of row intervals, ceil(n / r)
  int64_t nb = 0;       // N_blocks(r,c)
  int32_t* block_rowptr = nullptr;  // [I+1]
  int32_t* block_colidx = nullptr;  // [nb] (+ padding)
  uint8_t* block_masks = nullptr;   // [nb*mb] (+ padding)
  void* values = nullptr;           // [nnz] (+ padding)
  int64_t* valptr = nullptr;        // [I+1]
  // execution plan
  int32_t long_blocks = spc5::kLongBlocks;
  int64_t long_values = INT64_MAX;  // an interval with more values is long too
  int32_t seg_blocks = spc5::kSegBlocks;
  int32_t variant = 0;
  int64_t nseg = 0;
  spc5::Segment* segs = nullptr;    // [nseg]
  int64_t nlong = 0;                // long intervals
  int32_t* seg_first = nullptr;     // [nlong] first segment of each long interval
  void* partials = nullptr;         // [nseg * r] accumulation-type scratch
  // SpMM segment partials, grown on demand
  void* spmm_scratch = nullptr;
  size_t spmm_scratch_bytes = 0;
  // when not NULL, one allocation holding block_colidx, block_masks, values,
  // valptr, segs and partials (freed as a whole)
  void* arena = nullptr;
  cudaStream_t arena_stream = nullptr;  // stream of the arena's pool allocation
  // work order of the lane-per-row kernel (short intervals only)
  int64_t norder = 0;
  int32_t* order = nullptr;            // [norder] interval indices
  int32_t order_window = spc5::kOrderWindow;  // rows per sorting window; <= 0: all intervals
  // Algorithm 2's test, per interval (r = 1): bit it of single_bits is set when
  // every block of short interval it holds one value (mask 1); built on demand
  uint32_t* single_bits = nullptr;     // [(I + 31) / 32]
  int64_t nsingle = 0;                 // intervals with the bit set
};

namespace spc5 {

// thread-local last-error message
void set_error(const std::string& msg);
spc5_status fail(spc5_status st, const std::string& msg);
spc5_status cuda_fail(cudaError_t e, const char* what);

inline bool shape_supported(int r, int c) {
  return (r == 1 || r == 2 || r == 4 || r == 8) && (c == 4 || c == 8 || c == 16);
}
inline int mask_bytes(int r, int c) { return (r * c + 7) / 8; }
inline size_t value_size(spc5_dtype t) { return t == SPC5_F64 ? 8 : (t == SPC5_F32 ? 4 : 2); }

// conversion (convert.cu)
spc5_status convert_impl(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                         const void* values, spc5_dtype vt, int r, int c, const spc5_opts* opt, cudaStream_t s,
                         spc5_matrix** out);
spc5_status assemble_impl(int64_t n, int64_t m, int64_t nnz, int64_t nb, int r, int c, spc5_dtype vt,
                          const int32_t* brp, const int32_t* bcol, const uint8_t* bmask, const void* vals,
                          const spc5_opts* opt, cudaStream_t s, spc5_matrix** out);
spc5_status build_order(spc5_matrix* h, cudaStream_t s);
spc5_status build_single_bits(spc5_matrix* h, cudaStream_t s);
// block counts of the twelve shapes without conversion (counts.cu)
cudaError_t launch_block_counts(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                unsigned long long* acc, cudaStream_t s);
spc5_status count_blocks_impl(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                              int64_t* nblocks_out, cudaStream_t s);

// SpMV launchers, one per value type (spmv_f64.cu, spmv_f32.cu, spmv_bf16.cu)
cudaError_t launch_spmv_f64(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s,
                            void* partials = nullptr);
cudaError_t launch_spmv_f32(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s,
                            void* partials = nullptr);
cudaError_t launch_spmv_bf16(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s,
                            void* partials = nullptr);
// the group variants 24-29 (spmv_group_f64.cu, spmv_group_f32.cu, spmv_group_bf16.cu)
cudaError_t launch_group_f64(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s, void* partials);
cudaError_t launch_group_f32(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s, void* partials);
cudaError_t launch_group_bf16(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s, void* partials);

// CSR comparator and copy (csr.cu)
cudaError_t launch_csr_spmv(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                            const void* values, spc5_dtype vt, const void* x, void* y, cudaStream_t s);
cudaError_t launch_csr_spmv_group(int group, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                  const void* values, spc5_dtype vt, const void* x, void* y, cudaStream_t s);
int csr_auto_group(int64_t n, int64_t nnz, spc5_dtype vt);
void destroy_matrix(spc5_matrix* h);
cudaError_t trim_pools();
// exclusive scan of int32 counts into out[0..L] (out[L] = total, returned to
// the host; synchronises s) and an allocation from the library's pool
spc5_status exclusive_scan_i32(const int32_t* in, int64_t L, int32_t* out, int64_t* total_host, cudaStream_t s);
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t launch_copy(const void* src, void* dst, int64_t bytes, cudaStream_t s);
cudaError_t launch_fma_rate(spc5_dtype vt, int64_t iters, int lanes, void* sink, int64_t* fmas, cudaStream_t s);

// multi-RHS SpMM (spmm.cu)
spc5_status spmm_impl(spc5_matrix* h, int k, const void* X, int64_t ldx, void* Y, int64_t ldy, int ktile,
                      cudaStream_t s);
int spmm_auto_tile(int k);

// selection (select.cu)
spc5_status features_impl(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx, double* f,
                          cudaStream_t s);
spc5_status mlp_train_impl(float* P, const float* X, const float* Y, const float* M, int N, int epochs, int batch,
                           float lr, uint64_t seed, float* loss_hist, cudaStream_t s, int nfeat = 16);
spc5_status mlp_grad_impl(const float* P, const float* X, const float* Y, const float* M, int B, float* loss,
                          float* grad, cudaStream_t s, int nfeat = 16);
spc5_status mlp_infer_impl(const float* P, const float* X, int N, float* out, cudaStream_t s, int nfeat = 16);
// extended selection features (16 + x-access locality, short rows, SM fraction)
spc5_status features_ext_impl(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                              double sm_frac, double* f, cudaStream_t s);
spc5_status poly_fit_impl(const double* avg, const double* perf, int N, int degree, double* coef);
int poly_select_impl(const double* coef, int degree, const double* feat, double* est);
int poly2_terms(int degree);
spc5_status poly2_fit_impl(const double* avg, const double* sfrac, const double* perf, int N, int degree,
                           double* coef);
int poly2_select_impl(const double* coef, int degree, const double* feat, double sfrac, double* est);
int mlp_param_count(int nfeat = 16);

// conjugate gradients (cg.cu)
spc5_status cg_impl(const spc5_matrix* A, const spc5_matrix* L, const double* b, double* x, const spc5_cg_opts* o,
                    spc5_cg_info* info, cudaStream_t s);

int sm_count();

// The segments and the short intervals share one grid unless the plain
// variant 1 runs or the matrix has only one kind of work.
inline bool fused_launch(const spc5_matrix* h) { return h->I > 0 && h->nseg > 0 && h->variant != 1; }

// kernels one spc5_spmv launches on this handle (see launch_beta)
inline int spmv_launches(const spc5_matrix* h) {
  int k = h->I > 0 ? 1 : 0;
  if (h->nseg > 0) k += (fused_launch(h) ? 0 : 1) + 1;  // separate segment kernel, then the fix-up
  return k;
}

}  // namespace spc5
