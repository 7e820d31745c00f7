// N_blocks(r,c) of all twelve shapes from a CSR, without conversion (section
// "Performance polynomial interpolation": the selection inputs Avg(r,c) =
// nnz / N_blocks(r,c) are cheap to compute) plus the row-length statistics of
// the selection features.
//
//   * r = 1: the greedy cover of a row splits at every gap of at least c
//     between neighbouring columns (the block holding the left column ends
//     before the right one), so the runs between gaps are covered
//     independently: k_count_r1 spreads the entries over threads (8 each),
//     and a thread counts the blocks of the runs that start in its range,
//     for c = 4, 8 and 16 at once.
//   * r > 1: one thread per interval walks the merged columns of its r rows
//     (heads kept in registers, one load per step) and counts the greedy
//     blocks for c = 4, 8 and 16 in the same walk.
// All counts are integers summed with atomics, so the order of the sums does
// not matter.
#include <climits>

#include "internal.cuh"

namespace spc5 {
namespace {

constexpr int kPerThread = 8;

__device__ __forceinline__ int64_t row_holding(const int64_t* __restrict__ rowptr, int64_t n, int64_t j) {
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (rowptr[mid] <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// warp sum then one atomic per warp
__device__ __forceinline__ void warp_add(unsigned long long* dst, unsigned long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

__global__ void __launch_bounds__(256) k_count_r1(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ colidx,
                                                  unsigned long long* __restrict__ acc) {
  const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kPerThread;
  unsigned long long cnt[3] = {0ull, 0ull, 0ull};
  if (j0 < nnz) {
    const int64_t j1 = j0 + kPerThread < nnz ? j0 + kPerThread : nnz;
    int64_t row = row_holding(rowptr, n, j0);
    int64_t rs = rowptr[row], re = rowptr[row + 1];
    int32_t prev = j0 > rs ? colidx[j0 - 1] : 0;
    for (int64_t j = j0; j < j1; ++j) {
      while (j >= re) {
        ++row;
        rs = rowptr[row];
        re = rowptr[row + 1];
      }
      const int32_t col = colidx[j];
      const int32_t gap = col - prev;
      prev = col;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int c = 4 << q;
        if (j != rs && gap < c) continue;  // inside a run that starts earlier
        int32_t s0 = col, last = col;
        ++cnt[q];
        for (int64_t k = j + 1; k < re; ++k) {
          const int32_t ck = colidx[k];
          if (ck - last >= c) break;
          if (ck - s0 >= c) {
            s0 = ck;
            ++cnt[q];
          }
          last = ck;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) warp_add(&acc[q], cnt[q]);
}

template <int R>
__global__ void __launch_bounds__(256) k_count_rk(int64_t n, int64_t I, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ colidx,
                                                  unsigned long long* __restrict__ acc) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt[3] = {0ull, 0ull, 0ull};
  if (it < I) {
    const int64_t row0 = it * R;
    int64_t h[R], e[R];
    int32_t cur[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if (row0 + i < n) {
        h[i] = rowptr[row0 + i];
        e[i] = rowptr[row0 + i + 1];
      } else {
        h[i] = e[i] = 0;
      }
      cur[i] = h[i] < e[i] ? colidx[h[i]] : INT_MAX;
    }
    int64_t end[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (;;) {
      int32_t s = INT_MAX;
#pragma unroll
      for (int i = 0; i < R; ++i) s = cur[i] < s ? cur[i] : s;
      if (s == INT_MAX) break;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if ((int64_t)s >= end[q]) {
          ++cnt[q];
          end[q] = (int64_t)s + (4 << q);
        }
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        if (cur[i] == s) {
          ++h[i];
          cur[i] = h[i] < e[i] ? colidx[h[i]] : INT_MAX;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) warp_add(&acc[q], cnt[q]);
}

// acc[0] += row lengths, acc[1] += squares, acc[2] = max
__global__ void __launch_bounds__(256) k_row_stats(int64_t n, const int64_t* __restrict__ rowptr,
                                                   unsigned long long* __restrict__ acc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long len = i < n ? (unsigned long long)(rowptr[i + 1] - rowptr[i]) : 0ull;
  unsigned long long s1 = len, s2 = len * len, mx = len;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, d);
    s2 += __shfl_xor_sync(0xffffffffu, s2, d);
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, d);
    mx = o > mx ? o : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], s1);
    atomicAdd(&acc[1], s2);
    atomicMax(&acc[2], mx);
  }
}

}  // namespace

// acc (device, 15 entries, zeroed here): [0..11] N_blocks in the order r in
// {1,2,4,8} outer, c in {4,8,16} inner; [12..14] sum, sum of squares and max of
// the row lengths.
cudaError_t launch_block_counts(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                unsigned long long* acc, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 15, s);
  if (e != cudaSuccess) return e;
  const int64_t th = (nnz + kPerThread - 1) / kPerThread;
  if (th > 0) k_count_r1<<<(unsigned)((th + 255) / 256), 256, 0, s>>>(n, nnz, rowptr, colidx, acc);
  const int64_t I2 = (n + 1) / 2, I4 = (n + 3) / 4, I8 = (n + 7) / 8;
  if (I2 > 0) k_count_rk<2><<<(unsigned)((I2 + 255) / 256), 256, 0, s>>>(n, I2, rowptr, colidx, acc + 3);
  if (I4 > 0) k_count_rk<4><<<(unsigned)((I4 + 255) / 256), 256, 0, s>>>(n, I4, rowptr, colidx, acc + 6);
  if (I8 > 0) k_count_rk<8><<<(unsigned)((I8 + 255) / 256), 256, 0, s>>>(n, I8, rowptr, colidx, acc + 9);
  if (n > 0) k_row_stats<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, rowptr, acc + 12);
  return cudaGetLastError();
}

spc5_status count_blocks_impl(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                              int64_t* nblocks_out, cudaStream_t s) {
  unsigned long long* acc = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&acc, sizeof(unsigned long long) * 16, s);
  if (e != cudaSuccess) return cuda_fail(e, "count_blocks: scratch");
  unsigned long long h[15];
  e = launch_block_counts(n, nnz, rowptr, colidx, acc, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(acc, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "count_blocks");
  for (int q = 0; q < 12; ++q) nblocks_out[q] = (int64_t)h[q];
  return SPC5_OK;
}

}  // namespace spc5
