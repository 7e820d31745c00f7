// spc5_tune: the library's autotuner - block shape x kernel variant for the
// SpMV and, on request, block shape x column tile for the SpMM, chosen by
// timing on this GPU and remembered per matrix signature.
//
// The paper picks, per matrix, the fastest of its kernels (section
// "Performance prediction and optimal kernel selection": the exhaustive
// choice is the reference its predictors are judged against). On the GPU the
// kernel also has a work mapping (variant) and, for several right-hand
// sides, a column tile; both are timed here for every block shape. A matrix
// seen before (same signature: sizes, value type, the twelve block counts,
// the row-length maximum, k and the SM count) returns the remembered choice
// without timing, so repeated set-ups of one structure - time steps of a
// simulation, many right-hand-side batches - pay for the search once.
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace spc5 {
namespace {

std::mutex g_tune_mu;
std::unordered_map<uint64_t, spc5_tune_result> g_tune_cache;

// FNV-1a over 64-bit words
uint64_t fnv(uint64_t h, uint64_t v) {
  for (int q = 0; q < 8; ++q) {
    h ^= (v >> (8 * q)) & 0xffu;
    h *= 0x100000001b3ull;
  }
  return h;
}

__global__ void k_row_len_max(int64_t n, const int64_t* __restrict__ rowptr, unsigned long long* __restrict__ mx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long len = i < n ? (unsigned long long)(rowptr[i + 1] - rowptr[i]) : 0ull;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, len, d);
    len = o > len ? o : len;
  }
  if ((threadIdx.x & 31) == 0 && len > 0) atomicMax(mx, len);
}

// variants worth timing for a value type and shape (each wins on some matrix)
std::vector<int> tune_candidates(spc5_dtype vt, int r) {
  std::vector<int> v = vt == SPC5_F64 ? std::vector<int>{5, 10, 13, 15} : std::vector<int>{5, 10, 13, 15, 16, 18};
  v.push_back(24);
  if (r == 1) {
    v.push_back(22);
    v.push_back(23);
    v.push_back(30);
    v.push_back(31);
    v.push_back(33);
    if (vt != SPC5_F64) v.push_back(32);  // float64: the busiest lane's block sets the cost
  }
  return v;
}

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {}
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  cudaError_t init() {
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    return e;
  }
  // median milliseconds of `reps` calls of f after one untimed call
  template <class F>
  spc5_status median(F f, int reps, float* ms) {
    spc5_status st = f();
    std::vector<float> t((size_t)reps);
    for (int k = 0; k < reps && st == SPC5_OK; ++k) {
      cudaError_t e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) st = f();
      if (st != SPC5_OK) break;
      e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t[(size_t)k], e0, e1);
      if (e != cudaSuccess) st = cuda_fail(e, "tune: timing");
    }
    if (st == SPC5_OK) {
      std::sort(t.begin(), t.end());
      *ms = t[(size_t)reps / 2];
    }
    return st;
  }
};

}  // namespace

spc5_status tune_impl(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                      const void* values, spc5_dtype vt, int k, int reps, int flags, spc5_tune_result* out,
                      cudaStream_t s) {
  // signature: sizes, type, k, SM count, the twelve block counts, longest row
  int64_t nb[12];
  spc5_status st = count_blocks_impl(n, nnz, rowptr, colidx, nb, s);
  if (st != SPC5_OK) return st;
  unsigned long long lmax = 0;
  {
    void* mx = nullptr;
    cudaError_t e = cudaMallocAsync(&mx, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess && n > 0)
      k_row_len_max<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, rowptr, (unsigned long long*)mx);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lmax, mx, sizeof(lmax), cudaMemcpyDeviceToHost, s);
    if (mx) cudaFreeAsync(mx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "tune: signature");
  }
  uint64_t sig = 0xcbf29ce484222325ull;
  for (int64_t v : {n, m, nnz, (int64_t)vt, (int64_t)k, (int64_t)sm_count(), (int64_t)lmax}) sig = fnv(sig, (uint64_t)v);
  for (int q = 0; q < 12; ++q) sig = fnv(sig, (uint64_t)nb[q]);
  if (!(flags & SPC5_TUNE_NO_CACHE)) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      *out = it->second;
      out->from_cache = 1;
      return SPC5_OK;
    }
  }

  // work vectors: x = 1 (any values do; the kernels' time does not depend on them)
  const size_t xs = vt == SPC5_F64 ? 8 : 4;
  const int kk = k > 0 ? k : 1;
  void *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMallocAsync(&x, xs * (size_t)std::max<int64_t>(m, 1) * (size_t)kk, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&y, xs * (size_t)std::max<int64_t>(n, 1) * (size_t)kk, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, xs * (size_t)std::max<int64_t>(m, 1) * (size_t)kk, s);
  if (e != cudaSuccess) {
    if (x) cudaFreeAsync(x, s);
    if (y) cudaFreeAsync(y, s);
    return cuda_fail(e, "tune: work vectors");
  }
  Timer tm(s);
  e = tm.init();
  if (e != cudaSuccess) {
    cudaFreeAsync(x, s);
    cudaFreeAsync(y, s);
    return cuda_fail(e, "tune: events");
  }
  spc5_tune_result best{};
  best.spmv_ms = -1.f;
  best.spmm_ms = -1.f;
  const int rs[4] = {1, 2, 4, 8}, cs[3] = {4, 8, 16};
  const int tiles[8] = {1, 4, -8, -16, -32, 8, 16, 32};
  for (int q = 0; q < 12 && st == SPC5_OK; ++q) {
    const int r = rs[q / 3], c = cs[q % 3];
    spc5_handle h = nullptr;
    st = spc5_convert(n, m, nnz, rowptr, colidx, values, vt, r, c, nullptr, (spc5_stream_t)s, &h);
    if (st != SPC5_OK) break;
    int shape_v = 0;  // fastest variant on this shape
    float shape_ms = -1.f;
    for (int v : tune_candidates(vt, r)) {
      st = spc5_set_variant(h, v, (spc5_stream_t)s);
      float ms = 0.f;
      if (st == SPC5_OK) st = tm.median([&] { return spc5_spmv(h, x, y, (spc5_stream_t)s); }, reps, &ms);
      if (st != SPC5_OK) break;
      if (shape_ms < 0.f || ms < shape_ms) {
        shape_ms = ms;
        shape_v = v;
      }
      if (best.spmv_ms < 0.f || ms < best.spmv_ms) {
        best.spmv_ms = ms;
        best.r = r;
        best.c = c;
        best.variant = v;
      }
    }
    // the SpMM of one vector runs the SpMV: with this shape's fastest variant
    if (st == SPC5_OK && k > 0) st = spc5_set_variant(h, shape_v, (spc5_stream_t)s);
    if (st == SPC5_OK && k > 0) {
      for (int t : tiles) {
        const int at = t < 0 ? -t : t;
        if ((k == 1) != (t == 1) || at > 2 * k) continue;  // k = 1: tile 1 only; no tile wider than 2k
        float ms = 0.f;
        st = tm.median([&] { return spc5_spmm(h, k, x, k, y, k, t, (spc5_stream_t)s); }, reps, &ms);
        if (st != SPC5_OK) break;
        if (best.spmm_ms < 0.f || ms < best.spmm_ms) {
          best.spmm_ms = ms;
          best.spmm_r = r;
          best.spmm_c = c;
          best.ktile = t;
          best.spmm_variant = shape_v;
        }
      }
    }
    spc5_destroy(h);
  }
  cudaFreeAsync(x, s);
  cudaFreeAsync(y, s);
  if (st != SPC5_OK) return st;
  best.signature = sig;
  best.from_cache = 0;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[sig] = best;
  }
  *out = best;
  return SPC5_OK;
}

void tune_cache_clear() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
}

}  // namespace spc5

using namespace spc5;

extern "C" {

spc5_status spc5_tune(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr_d, const int32_t* colidx_d,
                      const void* values_d, spc5_dtype vt, int k_spmm, int reps, int flags, spc5_tune_result* out,
                      spc5_stream_t stream) {
  if (!out) return fail(SPC5_EINVAL, "tune: NULL output");
  if (n < 0 || m < 0 || nnz < 0) return fail(SPC5_EINVAL, "tune: negative size");
  if (m > INT32_MAX || nnz > INT32_MAX) return fail(SPC5_ERANGE, "tune: m and nnz must be below 2^31");
  if ((n > 0 && !rowptr_d) || (nnz > 0 && (!colidx_d || !values_d))) return fail(SPC5_EINVAL, "tune: NULL array");
  if (vt != SPC5_F64 && vt != SPC5_F32 && vt != SPC5_BF16) return fail(SPC5_EUNSUPPORTED, "tune: value type");
  if (reps < 1 || k_spmm < 0 || k_spmm > 1024) return fail(SPC5_EINVAL, "tune: reps < 1 or k outside [0, 1024]");
  if (flags & ~SPC5_TUNE_NO_CACHE) return fail(SPC5_EINVAL, "tune: unknown flag");
  return tune_impl(n, m, nnz, rowptr_d, colidx_d, values_d, vt, k_spmm, reps, flags, out, (cudaStream_t)stream);
}

spc5_status spc5_tune_cache_clear(void) {
  tune_cache_clear();
  return SPC5_OK;
}

}  // extern "C"
