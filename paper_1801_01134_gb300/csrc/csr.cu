// Comparison kernels: plain CSR SpMV (the paper's reference format, section
// "Sparse Matrix Vector Product (SpMV)") and a streaming copy that measures
// the achievable HBM bandwidth.
//
// CSR mapping: G lanes per row (G in {1,2,4,8,16,32}); the lanes of a group
// read consecutive entries of their row, accumulate privately and reduce with
// shuffles. G = 1 is one lane per row (no reduction); larger G coalesce the
// value/index streams at the cost of log2(G) reduction steps per row.
#include <climits>

#include "internal.cuh"

namespace spc5 {
namespace {

__device__ __forceinline__ float to_f32(uint16_t v) { return __uint_as_float(((uint32_t)v) << 16); }

template <int G, class V, class X, class A>
__device__ __forceinline__ void csr_rows_body(int64_t bid, int64_t n, int64_t long_len,
                                              const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                              const V* __restrict__ val, const X* __restrict__ x, X* __restrict__ y) {
  const int64_t t = bid * blockDim.x + threadIdx.x;
  const int64_t row = t / G;
  const int g = (int)(t % G);
  // keep whole groups alive for the shuffles; rows past n contribute nothing,
  // rows longer than long_len belong to the segment path
  bool live = row < n;
  int64_t a = 0, b = 0;
  if (live) {
    a = __ldg(rowptr + row);
    b = __ldg(rowptr + row + 1);
    live = b - a <= long_len;
  }
  A acc = 0;
  if (live) {
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

template <int G, class V, class X, class A>
__global__ void __launch_bounds__(256) k_csr(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                             const V* __restrict__ val, const X* __restrict__ x, X* __restrict__ y) {
  csr_rows_body<G, V, X, A>(blockIdx.x, n, INT64_MAX, rowptr, colidx, val, x, y);
}

// ------------------------------------------------------------ CSR plan
// The comparator with the β path's load balancing: rows longer than
// long_len entries are cut into segments of seg_len entries, a warp per
// segment (lanes take entries j, j + 32, ..., then a fixed shuffle tree),
// partial sums per segment; the segments and the short rows (G lanes per
// row) share one grid, segment thread blocks first; a fix-up adds each long
// row's segments in order and writes y. Same summation order run to run.
struct CsrSeg {
  int64_t begin, end;  // entries of the segment
  int32_t row;         // its row
  int32_t count;       // segments of the row, in its first segment; 0 in the others
};

template <class V, class X, class A>
__device__ __forceinline__ void csr_seg_body(int64_t bid, int64_t nseg, const CsrSeg* __restrict__ segs,
                                             const int32_t* __restrict__ colidx, const V* __restrict__ val,
                                             const X* __restrict__ x, A* __restrict__ part) {
  const int64_t q = (bid * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nseg) return;  // whole warp
  const CsrSeg sg = segs[q];
  A acc = 0;
  for (int64_t p = sg.begin + lane; p < sg.end; p += 32) {
    if constexpr (sizeof(V) == sizeof(A))
      acc = fma((A)__ldg(val + p), (A)__ldg(x + __ldg(colidx + p)), acc);
    else
      acc = fma(to_f32(__ldg(val + p)), (A)__ldg(x + __ldg(colidx + p)), acc);
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane == 0) part[q] = acc;
}

template <int G, class V, class X, class A>
__global__ void __launch_bounds__(256) k_csr_plan(int64_t seg_ctas, int64_t n, int64_t long_len,
                                                  const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ colidx, const V* __restrict__ val,
                                                  const X* __restrict__ x, X* __restrict__ y, int64_t nseg,
                                                  const CsrSeg* __restrict__ segs, A* __restrict__ part) {
  if ((int64_t)blockIdx.x < seg_ctas)
    csr_seg_body<V, X, A>(blockIdx.x, nseg, segs, colidx, val, x, part);
  else
    csr_rows_body<G, V, X, A>((int64_t)blockIdx.x - seg_ctas, n, long_len, rowptr, colidx, val, x, y);
}

template <class X, class A>
__global__ void k_csr_plan_fixup(int64_t nseg, const CsrSeg* __restrict__ segs, const A* __restrict__ part,
                                 X* __restrict__ y) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nseg) return;
  const int32_t count = segs[q].count;
  if (count == 0) return;
  A s = 0;
  for (int32_t k = 0; k < count; ++k) s += part[q + k];
  y[segs[q].row] = s;
}

// segments per row: 0 for short rows
__global__ void k_csr_seg_counts(int64_t n, int64_t long_len, int64_t seg_len, const int64_t* __restrict__ rowptr,
                                 int32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t len = rowptr[i + 1] - rowptr[i];
  cnt[i] = len > long_len ? (int32_t)((len + seg_len - 1) / seg_len) : 0;
}

__global__ void k_csr_seg_fill(int64_t n, int64_t seg_len, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ off, CsrSeg* __restrict__ segs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t k0 = off[i], k1 = off[i + 1];
  const int64_t a = rowptr[i], b = rowptr[i + 1];
  for (int32_t k = k0; k < k1; ++k) {
    CsrSeg sg;
    sg.begin = a + (int64_t)(k - k0) * seg_len;
    sg.end = sg.begin + seg_len < b ? sg.begin + seg_len : b;
    sg.row = (int32_t)i;
    sg.count = k == k0 ? k1 - k0 : 0;
    segs[k] = sg;
  }
}

template <class V, class X, class A>
cudaError_t csr_dispatch(int G, int64_t n, const int64_t* rowptr, const int32_t* colidx, const void* values,
                         const void* xv, void* yv, cudaStream_t s) {
  const V* val = static_cast<const V*>(values);
  const X* x = static_cast<const X*>(xv);
  X* y = static_cast<X*>(yv);
  const int threads = kSpmvThreads;
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

template <class V, class X, class A>
cudaError_t csr_plan_launch(int G, int64_t n, int64_t long_len, const int64_t* rowptr, const int32_t* colidx,
                            const void* values, const void* xv, void* yv, int64_t nseg, const CsrSeg* segs,
                            void* partials, cudaStream_t s) {
  const V* val = static_cast<const V*>(values);
  const X* x = static_cast<const X*>(xv);
  X* y = static_cast<X*>(yv);
  A* part = static_cast<A*>(partials);
  const int threads = kSpmvThreads;
  const int64_t seg_ctas = (nseg * 32 + threads - 1) / threads;
  const unsigned grid = (unsigned)(seg_ctas + (n * G + threads - 1) / threads);
  if (grid == 0) return cudaSuccess;
  switch (G) {
    case 1: k_csr_plan<1, V, X, A><<<grid, threads, 0, s>>>(seg_ctas, n, long_len, rowptr, colidx, val, x, y, nseg, segs, part); break;
    case 2: k_csr_plan<2, V, X, A><<<grid, threads, 0, s>>>(seg_ctas, n, long_len, rowptr, colidx, val, x, y, nseg, segs, part); break;
    case 4: k_csr_plan<4, V, X, A><<<grid, threads, 0, s>>>(seg_ctas, n, long_len, rowptr, colidx, val, x, y, nseg, segs, part); break;
    case 8: k_csr_plan<8, V, X, A><<<grid, threads, 0, s>>>(seg_ctas, n, long_len, rowptr, colidx, val, x, y, nseg, segs, part); break;
    case 16: k_csr_plan<16, V, X, A><<<grid, threads, 0, s>>>(seg_ctas, n, long_len, rowptr, colidx, val, x, y, nseg, segs, part); break;
    default: k_csr_plan<32, V, X, A><<<grid, threads, 0, s>>>(seg_ctas, n, long_len, rowptr, colidx, val, x, y, nseg, segs, part); break;
  }
  if (nseg > 0)
    k_csr_plan_fixup<X, A><<<(unsigned)((nseg + 255) / 256), 256, 0, s>>>(nseg, segs, part, y);
  return cudaGetLastError();
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

struct spc5_csr_plan_s {
  int64_t n = 0, nnz = 0, long_len = 0, seg_len = 0, nseg = 0;
  int group = 1;
  spc5_dtype vt = SPC5_F64;
  const int64_t* rowptr = nullptr;  // the caller's
  spc5::CsrSeg* segs = nullptr;
  void* partials = nullptr;
  cudaStream_t s = nullptr;
};

using namespace spc5;

extern "C" {

spc5_status spc5_csr_plan_create(int64_t n, int64_t nnz, const int64_t* rowptr_d, spc5_dtype vt, int group,
                                 int64_t long_len, int64_t seg_len, spc5_stream_t stream, spc5_csr_plan* out) {
  if (!out) return fail(SPC5_EINVAL, "csr_plan_create: NULL output");
  *out = nullptr;
  if (n < 0 || nnz < 0 || long_len < 0 || seg_len < 0) return fail(SPC5_EINVAL, "csr_plan_create: negative size");
  if (n > INT32_MAX || nnz > INT32_MAX) return fail(SPC5_ERANGE, "csr_plan_create: n and nnz must be below 2^31");
  if (n > 0 && !rowptr_d) return fail(SPC5_EINVAL, "csr_plan_create: rowptr is NULL");
  if (vt != SPC5_F64 && vt != SPC5_F32 && vt != SPC5_BF16) return fail(SPC5_EUNSUPPORTED, "csr_plan_create: value type");
  if (!(group == 0 || group == 1 || group == 2 || group == 4 || group == 8 || group == 16 || group == 32))
    return fail(SPC5_EINVAL, "csr_plan_create: group must be 0 or a power of two up to 32");
  const cudaStream_t s = (cudaStream_t)stream;
  spc5_csr_plan_s* p = new spc5_csr_plan_s();
  p->n = n;
  p->nnz = nnz;
  p->vt = vt;
  p->rowptr = rowptr_d;
  p->s = s;
  p->group = group > 0 ? group : csr_auto_group(n, nnz, vt);
  const double mean = n > 0 ? (double)nnz / (double)n : 0.0;
  p->long_len = long_len > 0 ? long_len : (int64_t)(16.0 * mean > 1024.0 ? 16.0 * mean : 1024.0);
  p->seg_len = seg_len > 0 ? seg_len : 1024;
  auto bail = [&](spc5_status st) {
    if (p->segs) cudaFreeAsync(p->segs, s);
    if (p->partials) cudaFreeAsync(p->partials, s);
    delete p;
    return st;
  };
  if (n > 0) {
    int32_t *cnt = nullptr, *off = nullptr;
    cudaError_t e = pool_alloc((void**)&cnt, sizeof(int32_t) * (size_t)(n + 1), s);
    if (e == cudaSuccess) e = pool_alloc((void**)&off, sizeof(int32_t) * (size_t)(n + 1), s);
    if (e == cudaSuccess) {
      k_csr_seg_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, p->long_len, p->seg_len, rowptr_d, cnt);
      e = cudaGetLastError();
    }
    spc5_status st = e == cudaSuccess ? exclusive_scan_i32(cnt, n, off, &p->nseg, s) : cuda_fail(e, "csr_plan_create");
    if (st == SPC5_OK && p->nseg > 0) {
      e = pool_alloc((void**)&p->segs, sizeof(CsrSeg) * (size_t)p->nseg, s);
      if (e == cudaSuccess) e = pool_alloc(&p->partials, (vt == SPC5_F64 ? 8 : 4) * (size_t)p->nseg, s);
      if (e == cudaSuccess) {
        k_csr_seg_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, p->seg_len, rowptr_d, off, p->segs);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) st = cuda_fail(e, "csr_plan_create: segments");
    }
    if (cnt) cudaFreeAsync(cnt, s);
    if (off) cudaFreeAsync(off, s);
    if (st == SPC5_OK) {
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "csr_plan_create");
    }
    if (st != SPC5_OK) return bail(st);
  }
  *out = p;
  return SPC5_OK;
}

spc5_status spc5_csr_spmv_plan(spc5_csr_plan p, const int32_t* colidx_d, const void* values_d, const void* x_d,
                               void* y_d, spc5_stream_t stream) {
  if (!p) return fail(SPC5_EINVAL, "csr_spmv_plan: NULL plan");
  if (p->nnz > 0 && (!colidx_d || !values_d)) return fail(SPC5_EINVAL, "csr_spmv_plan: NULL array");
  if (p->n > 0 && (!x_d || !y_d)) return fail(SPC5_EINVAL, "csr_spmv_plan: NULL vector");
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  switch (p->vt) {
    case SPC5_F64:
      e = csr_plan_launch<double, double, double>(p->group, p->n, p->long_len, p->rowptr, colidx_d, values_d, x_d, y_d,
                                                  p->nseg, p->segs, p->partials, s);
      break;
    case SPC5_F32:
      e = csr_plan_launch<float, float, float>(p->group, p->n, p->long_len, p->rowptr, colidx_d, values_d, x_d, y_d,
                                               p->nseg, p->segs, p->partials, s);
      break;
    default:
      e = csr_plan_launch<uint16_t, float, float>(p->group, p->n, p->long_len, p->rowptr, colidx_d, values_d, x_d,
                                                  y_d, p->nseg, p->segs, p->partials, s);
      break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "csr_spmv_plan launch");
  return SPC5_OK;
}

spc5_status spc5_csr_plan_destroy(spc5_csr_plan p) {
  if (!p) return SPC5_OK;
  const cudaError_t e = cudaDeviceSynchronize();
  if (p->segs) cudaFreeAsync(p->segs, nullptr);
  if (p->partials) cudaFreeAsync(p->partials, nullptr);
  delete p;
  if (e != cudaSuccess) return cuda_fail(e, "csr_plan_destroy: device synchronisation");
  return SPC5_OK;
}

spc5_status spc5_csr_plan_info(spc5_csr_plan p, int* group_out, int64_t* long_len_out, int64_t* nseg_out) {
  if (!p) return fail(SPC5_EINVAL, "csr_plan_info: NULL plan");
  if (group_out) *group_out = p->group;
  if (long_len_out) *long_len_out = p->long_len;
  if (nseg_out) *nseg_out = p->nseg;
  return SPC5_OK;
}

}  // extern "C"
