// C ABI of libspc5 (declared in include/spc5.h): argument checks on the host,
// error reporting, and dispatch to the kernels of the other translation units.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "internal.cuh"

namespace spc5 {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

spc5_status fail(spc5_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

spc5_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return e == cudaErrorMemoryAllocation ? SPC5_ENOMEM : SPC5_ECUDA;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1;
  return sms;
}

namespace {

spc5_status check_csr_args(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                           const void* values) {
  if (n < 0 || m < 0 || nnz < 0) return fail(SPC5_EINVAL, "negative size");
  if (m > INT_MAX || nnz > INT_MAX) return fail(SPC5_ERANGE, "m and nnz must be below 2^31 (int32 indices)");
  if (n > 0 && !rowptr) return fail(SPC5_EINVAL, "rowptr is NULL");
  if (nnz > 0 && (!colidx || !values)) return fail(SPC5_EINVAL, "colidx or values is NULL");
  return SPC5_OK;
}

spc5_status spmv_common(spc5_handle h, const void* x, void* y, bool acc, cudaStream_t s) {
  if (!h) return fail(SPC5_EINVAL, "spmv: NULL handle");
  if ((h->m > 0 && !x) || (h->n > 0 && !y)) return fail(SPC5_EINVAL, "spmv: NULL vector");
  cudaError_t e;
  switch (h->vt) {
    case SPC5_F64: e = launch_spmv_f64(h, x, y, acc, s); break;
    case SPC5_F32: e = launch_spmv_f32(h, x, y, acc, s); break;
    case SPC5_BF16: e = launch_spmv_bf16(h, x, y, acc, s); break;
    default: return fail(SPC5_EUNSUPPORTED, "spmv: value type");
  }
  if (e != cudaSuccess) return cuda_fail(e, "spmv launch");
  return SPC5_OK;
}

__global__ void k_rebase_rows(int64_t rows, int64_t row_begin, const int64_t* __restrict__ rowptr,
                              int64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= rows) out[i] = rowptr[row_begin + i] - rowptr[row_begin];
}

}  // namespace
}  // namespace spc5

using namespace spc5;

extern "C" {

spc5_status spc5_convert_rows(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              const void* values_d, spc5_dtype vt, int r, int c, int64_t row_begin, int64_t row_end,
                              const spc5_opts* opt, spc5_stream_t stream, spc5_handle* out) {
  if (!out) return fail(SPC5_EINVAL, "convert_rows: out is NULL");
  *out = nullptr;
  spc5_status st = check_csr_args(n, m, nnz, rowptr_d, colidx_d, values_d);
  if (st != SPC5_OK) return st;
  if (!shape_supported(r, c)) return fail(SPC5_EUNSUPPORTED, "convert_rows: block shape must be r in {1,2,4,8}, c in {4,8,16}");
  if (vt != SPC5_F64 && vt != SPC5_F32 && vt != SPC5_BF16) return fail(SPC5_EUNSUPPORTED, "convert_rows: value type");
  if (row_begin < 0 || row_end < row_begin || row_end > n)
    return fail(SPC5_EINVAL, "convert_rows: rows must satisfy 0 <= row_begin <= row_end <= n");
  if (row_begin % r != 0) return fail(SPC5_EINVAL, "convert_rows: row_begin must be a multiple of r");
  if (opt && (opt->long_blocks < 0 || opt->seg_blocks < 0 || opt->long_values < 0)) return fail(SPC5_EINVAL, "convert_rows: negative option");
  if (opt && !valid_variant(opt->variant)) return fail(SPC5_EINVAL, "convert_rows: unknown variant");
  if (opt && r1_variant(opt->variant) && r != 1) return fail(SPC5_EUNSUPPORTED, "convert_rows: variant needs r = 1");
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t rows = row_end - row_begin;
  int64_t ends[2] = {0, 0};
  if (rows > 0) {
    cudaError_t e = cudaMemcpyAsync(&ends[0], rowptr_d + row_begin, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], rowptr_d + row_end, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "convert_rows: row bounds");
    if (ends[0] < 0 || ends[1] < ends[0] || ends[1] > nnz) return fail(SPC5_EINVAL, "convert_rows: bad row pointer");
  }
  // the rows' own CSR: a rebased row pointer, the column and value arrays
  // from the shard's first entry; the column space stays [0, m)
  int64_t* rp = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&rp, sizeof(int64_t) * (size_t)(rows + 1), s);
  if (e != cudaSuccess) return cuda_fail(e, "convert_rows: row pointer");
  if (rows > 0)
    k_rebase_rows<<<(unsigned)((rows + 1 + 255) / 256), 256, 0, s>>>(rows, row_begin, rowptr_d, rp);
  else
    e = cudaMemsetAsync(rp, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFreeAsync(rp, s);
    return cuda_fail(e, "convert_rows: row pointer");
  }
  const int64_t snnz = ends[1] - ends[0];
  const int32_t* col = snnz > 0 ? colidx_d + ends[0] : nullptr;
  const void* val = snnz > 0 ? static_cast<const char*>(values_d) + (size_t)ends[0] * value_size(vt) : nullptr;
  spc5_matrix* h = nullptr;
  st = convert_impl(rows, m, snnz, rp, col, val, vt, r, c, opt, s, &h);
  cudaFreeAsync(rp, s);
  if (st != SPC5_OK) return st;
  *out = h;
  return SPC5_OK;
}

spc5_status spc5_convert(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                         const void* values_d, spc5_dtype vt, int r, int c, const spc5_opts* opt,
                         spc5_stream_t stream, spc5_handle* out) {
  if (!out) return fail(SPC5_EINVAL, "convert: out is NULL");
  *out = nullptr;
  spc5_status st = check_csr_args(n, m, nnz, rowptr_d, colidx_d, values_d);
  if (st != SPC5_OK) return st;
  if (!shape_supported(r, c)) return fail(SPC5_EUNSUPPORTED, "convert: block shape must be r in {1,2,4,8}, c in {4,8,16}");
  if (vt != SPC5_F64 && vt != SPC5_F32 && vt != SPC5_BF16) return fail(SPC5_EUNSUPPORTED, "convert: value type");
  if (opt && (opt->long_blocks < 0 || opt->seg_blocks < 0 || opt->long_values < 0)) return fail(SPC5_EINVAL, "convert: negative option");
  if (opt && !valid_variant(opt->variant))
    return fail(SPC5_EINVAL, "convert: variant must be 0, 1, 3, 5, 9, 10, 12..19 or 22..33");
  if (opt && r1_variant(opt->variant) && r != 1)
    return fail(SPC5_EUNSUPPORTED, "convert: variants 22, 23 and 30 to 33 need r = 1");
  spc5_matrix* h = nullptr;
  st = convert_impl(n, m, nnz, rowptr_d, colidx_d, values_d, vt, r, c, opt, (cudaStream_t)stream, &h);
  if (st != SPC5_OK) return st;
  *out = h;
  return SPC5_OK;
}

spc5_status spc5_assemble(int64_t n, int64_t m, int64_t nnz, int64_t nblocks, const int32_t* block_rowptr_d,
                          const int32_t* block_colidx_d, const uint8_t* block_masks_d, const void* values_d,
                          spc5_dtype vt, int r, int c, const spc5_opts* opt, spc5_stream_t stream, spc5_handle* out) {
  if (!out) return fail(SPC5_EINVAL, "assemble: out is NULL");
  *out = nullptr;
  if (n < 0 || m < 0 || nnz < 0 || nblocks < 0) return fail(SPC5_EINVAL, "assemble: negative size");
  if (n > INT32_MAX || m > INT32_MAX || nnz > INT32_MAX || nblocks > INT32_MAX)
    return fail(SPC5_ERANGE, "assemble: sizes must fit int32 (int32 column indices and block pointers)");
  if (!shape_supported(r, c)) return fail(SPC5_EUNSUPPORTED, "assemble: block shape must be r in {1,2,4,8}, c in {4,8,16}");
  if (vt != SPC5_F64 && vt != SPC5_F32 && vt != SPC5_BF16) return fail(SPC5_EUNSUPPORTED, "assemble: value type");
  if (!block_rowptr_d || (nblocks > 0 && (!block_colidx_d || !block_masks_d)) || (nnz > 0 && !values_d))
    return fail(SPC5_EINVAL, "assemble: NULL array");
  if (opt && (opt->long_blocks < 0 || opt->seg_blocks < 0 || opt->long_values < 0)) return fail(SPC5_EINVAL, "assemble: negative option");
  if (opt && !valid_variant(opt->variant))
    return fail(SPC5_EINVAL, "assemble: variant must be 0, 1, 3, 5, 9, 10, 12..19 or 22..33");
  if (opt && r1_variant(opt->variant) && r != 1)
    return fail(SPC5_EUNSUPPORTED, "assemble: variants 22, 23 and 30 to 33 need r = 1");
  spc5_matrix* h = nullptr;
  spc5_status st = assemble_impl(n, m, nnz, nblocks, r, c, vt, block_rowptr_d, block_colidx_d, block_masks_d, values_d,
                                 opt, (cudaStream_t)stream, &h);
  if (st != SPC5_OK) return st;
  *out = h;
  return SPC5_OK;
}

spc5_status spc5_spmv(spc5_handle h, const void* x_d, void* y_d, spc5_stream_t stream) {
  return spmv_common(h, x_d, y_d, false, (cudaStream_t)stream);
}

spc5_status spc5_spmv_acc(spc5_handle h, const void* x_d, void* y_d, spc5_stream_t stream) {
  return spmv_common(h, x_d, y_d, true, (cudaStream_t)stream);
}

spc5_status spc5_set_variant(spc5_handle h, int variant, spc5_stream_t stream) {
  if (!h) return fail(SPC5_EINVAL, "set_variant: NULL handle");
  if (!valid_variant(variant))
    return fail(SPC5_EINVAL, "set_variant: variant must be 0, 1, 3, 5, 9, 10, 12..19 or 22..33");
  if (r1_variant(variant) && h->r != 1) return fail(SPC5_EUNSUPPORTED, "set_variant: variants 22, 23 and 30 to 33 need r = 1");
  if (ordered_variant(variant)) {
    spc5_status st = build_order(h, (cudaStream_t)stream);
    if (st != SPC5_OK) return st;
  }
  if (uses_single_bits(variant)) {
    spc5_status st = build_single_bits(h, (cudaStream_t)stream);
    if (st != SPC5_OK) return st;
  }
  h->variant = variant;
  return SPC5_OK;
}

spc5_status spc5_export(spc5_handle h, spc5_arrays* v) {
  if (!h || !v) return fail(SPC5_EINVAL, "export: NULL argument");
  v->n = h->n;
  v->m = h->m;
  v->nnz = h->nnz;
  v->nblocks = h->nb;
  v->nintervals = h->I;
  v->r = h->r;
  v->c = h->c;
  v->mask_bytes = h->mb;
  v->dtype = h->vt;
  v->block_rowptr_d = h->block_rowptr;
  v->block_colidx_d = h->block_colidx;
  v->block_masks_d = h->block_masks;
  v->values_d = h->values;
  v->valptr_d = h->valptr;
  v->nsegments = h->nseg;
  return SPC5_OK;
}

spc5_status spc5_poly2_fit(const double* avg, const double* sm_frac, const double* perf, int N, int degree,
                           double* coef_out) {
  if (!avg || !sm_frac || !perf || !coef_out) return fail(SPC5_EINVAL, "poly2_fit: NULL array");
  return poly2_fit_impl(avg, sm_frac, perf, N, degree, coef_out);
}

spc5_status spc5_poly2_select(const double* coef, int degree, const double* features, double sm_frac, int* r_out,
                              int* c_out, double* est_out) {
  if (!coef || !features || !r_out || !c_out) return fail(SPC5_EINVAL, "poly2_select: NULL argument");
  if (degree < 0 || degree > 4) return fail(SPC5_EINVAL, "poly2_select: need 0 <= degree <= 4");
  double est[SPC5_NFORMATS];
  const int q = poly2_select_impl(coef, degree, features, sm_frac, est);
  const int rs[4] = {1, 2, 4, 8}, cs[3] = {4, 8, 16};
  *r_out = rs[q / 3];
  *c_out = cs[q % 3];
  if (est_out)
    for (int f = 0; f < SPC5_NFORMATS; ++f) est_out[f] = est[f];
  return SPC5_OK;
}

spc5_status spc5_pool_trim(void) {
  cudaError_t e = trim_pools();
  if (e != cudaSuccess) return cuda_fail(e, "pool_trim");
  return SPC5_OK;
}

spc5_status spc5_launch_count(spc5_handle h, int* kernels_out) {
  if (!h || !kernels_out) return fail(SPC5_EINVAL, "launch_count: NULL argument");
  *kernels_out = spmv_launches(h);
  return SPC5_OK;
}

spc5_status spc5_device_peaks(double* hbm_gbs_out, int* sm_count_out, int* sm_clock_mhz_out) {
  if (!hbm_gbs_out && !sm_count_out && !sm_clock_mhz_out) return fail(SPC5_EINVAL, "device_peaks: no output");
  int dev = 0, mem_khz = 0, bus_bits = 0, sms = 0, sm_khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mem_khz, cudaDevAttrMemoryClockRate, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bus_bits, cudaDevAttrGlobalMemoryBusWidth, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_khz, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device_peaks");
  // double data rate: two transfers of bus_bits per memory clock
  if (hbm_gbs_out) *hbm_gbs_out = 2.0 * (double)mem_khz * 1e3 * (double)bus_bits / 8.0 / 1e9;
  if (sm_count_out) *sm_count_out = sms;
  if (sm_clock_mhz_out) *sm_clock_mhz_out = sm_khz / 1000;
  return SPC5_OK;
}

spc5_status spc5_destroy(spc5_handle h) {
  if (!h) return SPC5_OK;
  cudaError_t e = cudaDeviceSynchronize();
  destroy_matrix(h);
  if (e != cudaSuccess) return cuda_fail(e, "destroy: device synchronisation");
  return SPC5_OK;
}

const char* spc5_last_error(void) { return g_last_error.c_str(); }

spc5_status spc5_count_blocks(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              int64_t* nblocks_out, spc5_stream_t stream) {
  if (!nblocks_out) return fail(SPC5_EINVAL, "count_blocks: NULL output");
  spc5_status st = check_csr_args(n, m, nnz, rowptr_d, colidx_d, (const void*)colidx_d);
  if (st != SPC5_OK) return st;
  return count_blocks_impl(n, nnz, rowptr_d, colidx_d, nblocks_out, (cudaStream_t)stream);
}

spc5_status spc5_csr_spmv(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                          const void* values_d, spc5_dtype vt, const void* x_d, void* y_d, int group,
                          spc5_stream_t stream) {
  spc5_status st = check_csr_args(n, m, nnz, rowptr_d, colidx_d, values_d);
  if (st != SPC5_OK) return st;
  if (vt != SPC5_F64 && vt != SPC5_F32 && vt != SPC5_BF16) return fail(SPC5_EUNSUPPORTED, "csr_spmv: value type");
  if (!(group == 0 || group == 1 || group == 2 || group == 4 || group == 8 || group == 16 || group == 32))
    return fail(SPC5_EINVAL, "csr_spmv: group must be 0 or a power of two up to 32");
  if ((m > 0 && !x_d) || (n > 0 && !y_d)) return fail(SPC5_EINVAL, "csr_spmv: NULL vector");
  cudaError_t e = launch_csr_spmv_group(group, n, nnz, rowptr_d, colidx_d, values_d, vt, x_d, y_d, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "csr_spmv launch");
  return SPC5_OK;
}

spc5_status spc5_partition(const int32_t* block_rowptr, int64_t nintervals, int nparts, int64_t* bounds_out) {
  if (!block_rowptr || !bounds_out) return fail(SPC5_EINVAL, "partition: NULL array");
  if (nintervals < 0 || nparts < 1) return fail(SPC5_EINVAL, "partition: nintervals < 0 or nparts < 1");
  // distance of a block prefix p to part t's target, scaled by nparts:
  // |(t + 1) * N_b - nparts * p| (exact in 64 bits: both terms are below 2^62)
  const int64_t total = block_rowptr[nintervals];
  auto dist = [&](int64_t scaled_target, int64_t i) {
    const int64_t d = scaled_target - (int64_t)nparts * block_rowptr[i];
    return d < 0 ? -d : d;
  };
  int64_t at = 0;
  bounds_out[0] = 0;
  for (int t = 0; t < nparts; ++t) {
    const int64_t tgt = (int64_t)(t + 1) * total;
    if (t + 1 == nparts) {
      at = nintervals;
    } else {
      while (at < nintervals && dist(tgt, at + 1) <= dist(tgt, at)) ++at;
    }
    bounds_out[t + 1] = at;
  }
  return SPC5_OK;
}

spc5_status spc5_copy(const void* src_d, void* dst_d, int64_t bytes, spc5_stream_t stream) {
  if (bytes < 0 || (bytes % 16) != 0) return fail(SPC5_EINVAL, "copy: bytes must be a non-negative multiple of 16");
  if (bytes > 0 && (!src_d || !dst_d)) return fail(SPC5_EINVAL, "copy: NULL pointer");
  if (((uintptr_t)src_d | (uintptr_t)dst_d) & 15u) return fail(SPC5_EINVAL, "copy: pointers must be 16-byte aligned");
  cudaError_t e = launch_copy(src_d, dst_d, bytes, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy launch");
  return SPC5_OK;
}

spc5_status spc5_spmm(spc5_handle h, int k, const void* X_d, int64_t ldx, void* Y_d, int64_t ldy, int ktile,
                      spc5_stream_t stream) {
  if (!h) return fail(SPC5_EINVAL, "spmm: NULL handle");
  if (k < 1 || k > 1024) return fail(SPC5_EINVAL, "spmm: k must be in [1, 1024]");
  if (ldx < k || ldy < k) return fail(SPC5_EINVAL, "spmm: leading dimensions must be >= k");
  if (!(ktile == 0 || ktile == 1 || ktile == 4 || ktile == -8 || ktile == -16 || ktile == -32 || ktile == 8 ||
        ktile == 16 || ktile == 32))
    return fail(SPC5_EINVAL, "spmm: ktile must be 0, 1, 4, -8, -16, -32, 8, 16 or 32");
  if ((h->m > 0 && !X_d) || (h->n > 0 && !Y_d)) return fail(SPC5_EINVAL, "spmm: NULL matrix");
  // one right-hand side stored as a vector: the SpMV with the handle's variant
  if (k == 1 && ldx == 1 && ldy == 1 && (ktile == 0 || ktile == 1))
    return spmv_common(h, X_d, Y_d, false, (cudaStream_t)stream);
  return spmm_impl(h, k, X_d, ldx, Y_d, ldy, ktile, (cudaStream_t)stream);
}

spc5_status spc5_cg(spc5_handle A, spc5_handle A_inner, const double* b_d, double* x_d, const spc5_cg_opts* opt,
                    spc5_cg_info* info, spc5_stream_t stream) {
  if (!A || !info) return fail(SPC5_EINVAL, "cg: NULL handle or info");
  if (A->vt != SPC5_F64) return fail(SPC5_EINVAL, "cg: A must be a float64 handle");
  if (A->n != A->m) return fail(SPC5_EINVAL, "cg: A must be square");
  if (A_inner) {
    if (A_inner->vt != SPC5_F32 && A_inner->vt != SPC5_BF16)
      return fail(SPC5_EINVAL, "cg: A_inner must be a float32 or bfloat16 handle");
    if (A_inner->n != A->n || A_inner->m != A->m) return fail(SPC5_EINVAL, "cg: A_inner has another shape");
  }
  if (A->n > 0 && (!b_d || !x_d)) return fail(SPC5_EINVAL, "cg: NULL vector");
  spc5_cg_opts o{};
  if (opt) o = *opt;
  if (o.tol < 0 || o.inner_tol < 0 || o.max_iters < 0 || o.max_outer < 0 || o.inner_max_iters < 0 ||
      o.check_every < 0)
    return fail(SPC5_EINVAL, "cg: negative option");
  return cg_impl(A, A_inner, b_d, x_d, &o, info, (cudaStream_t)stream);
}

spc5_status spc5_features(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                          double* features_out, spc5_stream_t stream) {
  if (!features_out) return fail(SPC5_EINVAL, "features: NULL output");
  spc5_status st = check_csr_args(n, m, nnz, rowptr_d, colidx_d, (const void*)colidx_d);
  if (st != SPC5_OK) return st;
  return features_impl(n, nnz, rowptr_d, colidx_d, features_out, (cudaStream_t)stream);
}

spc5_status spc5_time_formats(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              const void* values_d, spc5_dtype vt, const void* x_d, void* y_d, int reps,
                              float* ms_out, spc5_stream_t stream) {
  if (!ms_out || reps < 1) return fail(SPC5_EINVAL, "time_formats: NULL output or reps < 1");
  if ((m > 0 && !x_d) || (n > 0 && !y_d)) return fail(SPC5_EINVAL, "time_formats: NULL vector");
  const cudaStream_t s = (cudaStream_t)stream;
  const int rs[4] = {1, 2, 4, 8}, cs[3] = {4, 8, 16};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "time_formats: events");
  spc5_status st = SPC5_OK;
  for (int q = 0; q < 12 && st == SPC5_OK; ++q) {
    spc5_handle h = nullptr;
    st = spc5_convert(n, m, nnz, rowptr_d, colidx_d, values_d, vt, rs[q / 3], cs[q % 3], nullptr, stream, &h);
    if (st != SPC5_OK) break;
    // the shape's time is that of its faster kernel form: the default one,
    // and for r = 1 also two lanes per row (variant 22)
    const int nforms = rs[q / 3] == 1 ? 2 : 1;
    for (int f = 0; f < nforms && st == SPC5_OK; ++f) {
      if (f == 1) st = spc5_set_variant(h, 22, stream);
      std::vector<float> t((size_t)reps);
      if (st == SPC5_OK) st = spc5_spmv(h, x_d, y_d, stream);  // untimed
      for (int k = 0; k < reps && st == SPC5_OK; ++k) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) st = spc5_spmv(h, x_d, y_d, stream);
        if (e == cudaSuccess && st == SPC5_OK) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess && st == SPC5_OK) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess && st == SPC5_OK) e = cudaEventElapsedTime(&t[(size_t)k], e0, e1);
        if (e != cudaSuccess) st = cuda_fail(e, "time_formats: timing");
      }
      if (st == SPC5_OK) {
        std::sort(t.begin(), t.end());
        const float med = t[(size_t)reps / 2];
        ms_out[q] = f == 0 ? med : std::min(ms_out[q], med);
      }
    }
    spc5_destroy(h);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

spc5_status spc5_autotune(spc5_handle h, const void* x_d, void* y_d, int reps, int* variant_out, float* ms_out,
                          spc5_stream_t stream) {
  if (!h) return fail(SPC5_EINVAL, "autotune: NULL handle");
  if (reps < 1) return fail(SPC5_EINVAL, "autotune: reps < 1");
  if ((h->m > 0 && !x_d) || (h->n > 0 && !y_d)) return fail(SPC5_EINVAL, "autotune: NULL vector");
  // the decodes that win somewhere: flattened (natural, sorted), mask windows
  // (sorted); for float32 / bfloat16 also the unrolled bit positions
  // (and for r = 1 two lanes per row, Algorithm 2's test, and for the narrow
  // types the block-streaming warp)
  std::vector<int> cand = h->vt == SPC5_F64 ? std::vector<int>{5, 10, 13, 15} : std::vector<int>{5, 10, 13, 15, 16, 18};
  if (h->r == 1) {
    cand.push_back(22);
    cand.push_back(23);
    cand.push_back(30);
    cand.push_back(33);
    if (h->vt != SPC5_F64) cand.push_back(32);
  }
  const int ncand = (int)cand.size();
  const cudaStream_t s = (cudaStream_t)stream;
  const int keep = h->variant;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune: events");
  spc5_status st = SPC5_OK;
  int best = keep;
  float best_ms = -1.0f;
  for (int q = 0; q < ncand && st == SPC5_OK; ++q) {
    st = spc5_set_variant(h, cand[q], stream);
    if (st == SPC5_OK) st = spc5_spmv(h, x_d, y_d, stream);  // untimed
    std::vector<float> t((size_t)reps);
    for (int k = 0; k < reps && st == SPC5_OK; ++k) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) st = spc5_spmv(h, x_d, y_d, stream);
      if (e == cudaSuccess && st == SPC5_OK) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess && st == SPC5_OK) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess && st == SPC5_OK) e = cudaEventElapsedTime(&t[(size_t)k], e0, e1);
      if (e != cudaSuccess) st = cuda_fail(e, "autotune: timing");
    }
    if (st == SPC5_OK) {
      std::sort(t.begin(), t.end());
      const float med = t[(size_t)reps / 2];
      if (best_ms < 0.0f || med < best_ms) {
        best_ms = med;
        best = cand[q];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const spc5_status st2 = spc5_set_variant(h, st == SPC5_OK ? best : keep, stream);
  if (st != SPC5_OK) return st;
  if (st2 != SPC5_OK) return st2;
  if (variant_out) *variant_out = best;
  if (ms_out) *ms_out = best_ms;
  return SPC5_OK;
}

int spc5_mlp_nparams(void) { return mlp_param_count(); }

int spc5_mlp_nparams_n(int nfeat) { return nfeat == 16 || nfeat == 20 ? mlp_param_count(nfeat) : -1; }

spc5_status spc5_features_ext(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                              double sm_frac, double* features_out, spc5_stream_t stream) {
  if (!features_out) return fail(SPC5_EINVAL, "features_ext: NULL output");
  if (!(sm_frac > 0.0 && sm_frac <= 1.0)) return fail(SPC5_EINVAL, "features_ext: sm_frac must be in (0, 1]");
  spc5_status st = check_csr_args(n, m, nnz, rowptr_d, colidx_d, (const void*)colidx_d);
  if (st != SPC5_OK) return st;
  return features_ext_impl(n, nnz, rowptr_d, colidx_d, sm_frac, features_out, (cudaStream_t)stream);
}

spc5_status spc5_mlp_train_n(float* params_d, const float* X_d, const float* Y_d, const float* M_d, int N, int nfeat,
                             int epochs, int batch, float lr, uint64_t seed, float* loss_history,
                             spc5_stream_t stream) {
  if (!params_d || N < 1 || epochs < 0 || !X_d || !Y_d || !M_d || !(lr >= 0.f))
    return fail(SPC5_EINVAL, "mlp_train: bad argument");
  return mlp_train_impl(params_d, X_d, Y_d, M_d, N, epochs, batch, lr, seed, loss_history, (cudaStream_t)stream,
                        nfeat);
}

spc5_status spc5_mlp_grad_n(const float* params_d, const float* X_d, const float* Y_d, const float* M_d, int B,
                            int nfeat, float* loss_out, float* grad_d, spc5_stream_t stream) {
  if (!params_d || !X_d || !Y_d || !M_d || !loss_out || !grad_d) return fail(SPC5_EINVAL, "mlp_grad: NULL argument");
  return mlp_grad_impl(params_d, X_d, Y_d, M_d, B, loss_out, grad_d, (cudaStream_t)stream, nfeat);
}

spc5_status spc5_mlp_infer_n(const float* params_d, const float* X_d, int N, int nfeat, float* out_d,
                             spc5_stream_t stream) {
  if (!params_d || N < 0 || (N > 0 && (!X_d || !out_d))) return fail(SPC5_EINVAL, "mlp_infer: bad argument");
  return mlp_infer_impl(params_d, X_d, N, out_d, (cudaStream_t)stream, nfeat);
}

spc5_status spc5_mlp_train(float* params_d, const float* X_d, const float* Y_d, const float* M_d, int N, int epochs,
                           int batch, float lr, uint64_t seed, float* loss_history, spc5_stream_t stream) {
  if (!params_d || N < 1 || epochs < 0 || !X_d || !Y_d || !M_d || !(lr >= 0.f))
    return fail(SPC5_EINVAL, "mlp_train: bad argument");
  return mlp_train_impl(params_d, X_d, Y_d, M_d, N, epochs, batch, lr, seed, loss_history, (cudaStream_t)stream);
}

spc5_status spc5_mlp_grad(const float* params_d, const float* X_d, const float* Y_d, const float* M_d, int B,
                          float* loss_out, float* grad_d, spc5_stream_t stream) {
  if (!params_d || !X_d || !Y_d || !M_d || !loss_out || !grad_d) return fail(SPC5_EINVAL, "mlp_grad: NULL argument");
  return mlp_grad_impl(params_d, X_d, Y_d, M_d, B, loss_out, grad_d, (cudaStream_t)stream);
}

spc5_status spc5_mlp_infer(const float* params_d, const float* X_d, int N, float* out_d, spc5_stream_t stream) {
  if (!params_d || N < 0 || (N > 0 && (!X_d || !out_d))) return fail(SPC5_EINVAL, "mlp_infer: bad argument");
  return mlp_infer_impl(params_d, X_d, N, out_d, (cudaStream_t)stream);
}

spc5_status spc5_poly_fit(const double* avg, const double* perf, int N, int degree, double* coef_out) {
  if (!avg || !perf || !coef_out) return fail(SPC5_EINVAL, "poly_fit: NULL argument");
  return poly_fit_impl(avg, perf, N, degree, coef_out);
}

spc5_status spc5_select(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                        const void* values_d, spc5_dtype vt, int method, const spc5_selector* model, int* r_out,
                        int* c_out, float* score_out, spc5_stream_t stream) {
  if (!r_out || !c_out) return fail(SPC5_EINVAL, "select: NULL output");
  const int rs[4] = {1, 2, 4, 8}, cs[3] = {4, 8, 16};
  const cudaStream_t s = (cudaStream_t)stream;
  float score[12] = {0};
  int best = 0;
  if (method == SPC5_SELECT_EXHAUSTIVE) {
    spc5_status st = check_csr_args(n, m, nnz, rowptr_d, colidx_d, values_d);
    if (st != SPC5_OK) return st;
    const size_t xs = vt == SPC5_F64 ? 8 : 4;
    void *x = nullptr, *y = nullptr;
    cudaError_t e = cudaMalloc(&x, xs * (size_t)(m > 0 ? m : 1));
    if (e == cudaSuccess) e = cudaMalloc(&y, xs * (size_t)(n > 0 ? n : 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, xs * (size_t)(m > 0 ? m : 1), s);
    if (e != cudaSuccess) {
      cudaFree(x);
      cudaFree(y);
      return cuda_fail(e, "select: work vectors");
    }
    st = spc5_time_formats(n, m, nnz, rowptr_d, colidx_d, values_d, vt, x, y, 5, score, stream);
    cudaFree(x);
    cudaFree(y);
    if (st != SPC5_OK) return st;
    for (int q = 1; q < 12; ++q)
      if (score[q] < score[best]) best = q;
  } else if (method == SPC5_SELECT_POLY || method == SPC5_SELECT_MLP) {
    if (!model) return fail(SPC5_EINVAL, "select: NULL model");
    double f[16];
    spc5_status st = spc5_features(n, m, nnz, rowptr_d, colidx_d, f, stream);
    if (st != SPC5_OK) return st;
    if (method == SPC5_SELECT_POLY) {
      if (!model->poly_coef || model->poly_degree < 0 || model->poly_degree > 6)
        return fail(SPC5_EINVAL, "select: no polynomial model");
      double est[12];
      best = poly_select_impl(model->poly_coef, model->poly_degree, f, est);
      for (int q = 0; q < 12; ++q) score[q] = (float)est[q];
    } else {
      if (!model->mlp_params_d) return fail(SPC5_EINVAL, "select: no MLP parameters");
      float xin[16];
      for (int q = 0; q < 16; ++q)
        xin[q] = (float)((std::log1p(f[q]) - (double)model->feat_mean[q]) /
                         (double)(model->feat_scale[q] != 0.f ? model->feat_scale[q] : 1.f));
      void* buf = nullptr;
      cudaError_t e = cudaMalloc(&buf, sizeof(float) * 28);
      if (e == cudaSuccess) e = cudaMemcpyAsync(buf, xin, sizeof(xin), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "select: MLP input");
      }
      st = mlp_infer_impl(model->mlp_params_d, (const float*)buf, 1, (float*)buf + 16, s);
      if (st == SPC5_OK) {
        e = cudaMemcpyAsync(score, (float*)buf + 16, sizeof(float) * 12, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "select: MLP output");
      }
      cudaFree(buf);
      if (st != SPC5_OK) return st;
      for (int q = 1; q < 12; ++q)
        if (score[q] < score[best]) best = q;
    }
  } else {
    return fail(SPC5_EINVAL, "select: unknown method");
  }
  *r_out = rs[best / 3];
  *c_out = cs[best % 3];
  if (score_out)
    for (int q = 0; q < 12; ++q) score_out[q] = score[q];
  return SPC5_OK;
}

spc5_status spc5_fma_rate(spc5_dtype vt, int64_t iters, void* sink_d, int64_t* fmas_out, spc5_stream_t stream) {
  return spc5_fma_rate_lanes(vt, iters, 32, sink_d, fmas_out, stream);
}

spc5_status spc5_fma_rate_lanes(spc5_dtype vt, int64_t iters, int lanes, void* sink_d, int64_t* fmas_out,
                                spc5_stream_t stream) {
  if ((vt != SPC5_F64 && vt != SPC5_F32) || iters < 0 || lanes < 1 || lanes > 32 || !sink_d || !fmas_out)
    return fail(SPC5_EINVAL, "fma_rate: bad argument");
  cudaError_t e = launch_fma_rate(vt, iters, lanes, sink_d, fmas_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "fma_rate launch");
  return SPC5_OK;
}

}  // extern "C"
