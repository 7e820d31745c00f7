// Comparison kernels: plain CSR SpMV (the paper's reference format, section
// "Sparse Matrix Vector Product (SpMV)") and a streaming copy that measures
// the achievable HBM bandwidth.
//
// CSR mapping: G lanes per row (G in {1,2,4,8,16,32}); the lanes of a group
// read consecutive entries of their row, accumulate privately and reduce with
// shuffles. G = 1 is one lane per row (no reduction); larger G coalesce the
// value/index streams at the cost of log2(G) reduction steps per row.
#include "internal.cuh"

namespace spc5 {
namespace {

__device__ __forceinline__ float to_f32(uint16_t v) { return __uint_as_float(((uint32_t)v) << 16); }

template <int G, class V, class X, class A>
__global__ void __launch_bounds__(256) k_csr(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                             const V* __restrict__ val, const X* __restrict__ x, X* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = t / G;
  const int g = (int)(t % G);
  // keep whole groups alive for the shuffles; rows past n contribute nothing
  const bool live = row < n;
  A acc = 0;
  if (live) {
    const int64_t a = __ldg(rowptr + row), b = __ldg(rowptr + row + 1);
    for (int64_t p = a + g; p < b; p += G) {
      if constexpr (sizeof(V) == sizeof(A))
        acc = fma((A)__ldg(val + p), (A)__ldg(x + __ldg(colidx + p)), acc);
      else
        acc = fma(to_f32(__ldg(val + p)), (A)__ldg(x + __ldg(colidx + p)), acc);
    }
  }
  if constexpr (G > 1) {
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) acc += __shfl_xor_sync(full, acc, d, G);
  }
  if (live && g == 0) y[row] = acc;
}

template <class V, class X, class A>
cudaError_t csr_dispatch(int G, int64_t n, const int64_t* rowptr, const int32_t* colidx, const void* values,
                         const void* xv, void* yv, cudaStream_t s) {
  const V* val = static_cast<const V*>(values);
  const X* x = static_cast<const X*>(xv);
  X* y = static_cast<X*>(yv);
  const int threads = 256;
  const unsigned grid = (unsigned)((n * G + threads - 1) / threads);
  if (n == 0) return cudaSuccess;
  switch (G) {
    case 1: k_csr<1, V, X, A><<<grid, threads, 0, s>>>(n, rowptr, colidx, val, x, y); break;
    case 2: k_csr<2, V, X, A><<<grid, threads, 0, s>>>(n, rowptr, colidx, val, x, y); break;
    case 4: k_csr<4, V, X, A><<<grid, threads, 0, s>>>(n, rowptr, colidx, val, x, y); break;
    case 8: k_csr<8, V, X, A><<<grid, threads, 0, s>>>(n, rowptr, colidx, val, x, y); break;
    case 16: k_csr<16, V, X, A><<<grid, threads, 0, s>>>(n, rowptr, colidx, val, x, y); break;
    default: k_csr<32, V, X, A><<<grid, threads, 0, s>>>(n, rowptr, colidx, val, x, y); break;
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(512) k_copy(const int4* __restrict__ src, int4* __restrict__ dst, int64_t n16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
}

// Arithmetic-rate probe: each thread runs 8 independent multiply-add chains
// for `iters` trips (a measured peak for the ALU roofline of the float64
// path). The result is stored only if it hits an impossible value, so the
// chains are not removed by the compiler.
template <class A>
__global__ void __launch_bounds__(256) k_fma_rate(int64_t iters, int lanes, A a, A b, A* sink) {
  A c0 = (A)threadIdx.x * (A)1e-3, c1 = c0 + 1, c2 = c0 + 2, c3 = c0 + 3, c4 = c0 + 4, c5 = c0 + 5, c6 = c0 + 6,
    c7 = c0 + 7;
  // lanes >= `lanes` of every warp skip the arithmetic (their warps still issue it)
  const int64_t my_iters = (int)(threadIdx.x & 31) < lanes ? iters : 0;
  for (int64_t i = 0; i < my_iters; ++i) {
    c0 = fma(c0, a, b); c1 = fma(c1, a, b); c2 = fma(c2, a, b); c3 = fma(c3, a, b);
    c4 = fma(c4, a, b); c5 = fma(c5, a, b); c6 = fma(c6, a, b); c7 = fma(c7, a, b);
  }
  const A s = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
  if (s == (A)-12345.678) sink[threadIdx.x] = s;
}

}  // namespace

cudaError_t launch_fma_rate(spc5_dtype vt, int64_t iters, int lanes, void* sink, int64_t* fmas, cudaStream_t s) {
  const unsigned grid = (unsigned)(sm_count() * 8);
  *fmas = (int64_t)grid * 8 * lanes * iters * 8;  // 8 warps per CTA, `lanes` active lanes, 8 chains
  if (vt == SPC5_F64)
    k_fma_rate<double><<<grid, 256, 0, s>>>(iters, lanes, 0.999, 1e-4, (double*)sink);
  else
    k_fma_rate<float><<<grid, 256, 0, s>>>(iters, lanes, 0.999f, 1e-4f, (float*)sink);
  return cudaGetLastError();
}

int csr_auto_group(int64_t n, int64_t nnz, spc5_dtype vt) {
  const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
  // float64: fused multiply-adds dominate, favour one lane per row; narrower
  // types are load bound, favour coalesced groups.
  const double per_lane = vt == SPC5_F64 ? 24.0 : 4.0;
  int g = 1;
  while (g < 32 && avg / g > per_lane) g *= 2;
  return g;
}

cudaError_t launch_csr_spmv_group(int group, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                  const void* values, spc5_dtype vt, const void* x, void* y, cudaStream_t s) {
  const int G = group > 0 ? group : csr_auto_group(n, nnz, vt);
  switch (vt) {
    case SPC5_F64: return csr_dispatch<double, double, double>(G, n, rowptr, colidx, values, x, y, s);
    case SPC5_F32: return csr_dispatch<float, float, float>(G, n, rowptr, colidx, values, x, y, s);
    default: return csr_dispatch<uint16_t, float, float>(G, n, rowptr, colidx, values, x, y, s);
  }
}

cudaError_t launch_csr_spmv(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx, const void* values,
                            spc5_dtype vt, const void* x, void* y, cudaStream_t s) {
  return launch_csr_spmv_group(0, n, nnz, rowptr, colidx, values, vt, x, y, s);
}

cudaError_t launch_copy(const void* src, void* dst, int64_t bytes, cudaStream_t s) {
  const int64_t n16 = bytes / 16;
  if (n16 == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(sm_count() * 4);
  k_copy<<<grid, 512, 0, s>>>(static_cast<const int4*>(src), static_cast<int4*>(dst), n16);
  return cudaGetLastError();
}

}  // namespace spc5
