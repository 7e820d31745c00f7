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
//     blocks for c = 4, 8 and 16 in the same walk; intervals with more than
//     kLongEntries entries (power-law hubs) are cut into chunks along their
//     longest row at columns that start a block in every cover (no merged
//     column in the 16 before them), one thread per chunk.
// All counts are integers summed with atomics, so the order of the sums does
// not matter.
#include <climits>
#include <vector>

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

// Greedy block counts (c = 4, 8, 16) of the merged columns of rows
// row0 .. row0 + R - 1 that lie in [lo, hi); lo must start a block for every c
// (the first column of the interval, or one with no merged column in the 16
// before it).
template <int R>
__device__ __forceinline__ void count_merged(int64_t n, int64_t row0, const int64_t* __restrict__ rowptr,
                                             const int32_t* __restrict__ colidx, int32_t lo, int32_t hi,
                                             unsigned long long (&cnt)[3]) {
  int64_t h[R], e[R];
  int32_t cur[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (row0 + i < n) {
      h[i] = rowptr[row0 + i];
      e[i] = rowptr[row0 + i + 1];
      if (lo > INT_MIN) {  // first entry >= lo
        int64_t a = h[i], b = e[i];
        while (a < b) {
          const int64_t mid = (a + b) >> 1;
          if (colidx[mid] < lo) a = mid + 1; else b = mid;
        }
        h[i] = a;
      }
    } else {
      h[i] = e[i] = 0;
    }
    cur[i] = h[i] < e[i] && colidx[h[i]] < hi ? colidx[h[i]] : INT_MAX;
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
        cur[i] = h[i] < e[i] && colidx[h[i]] < hi ? colidx[h[i]] : INT_MAX;
      }
    }
  }
}

constexpr int64_t kLongEntries = 1024;  // intervals with more entries are counted in chunks
constexpr int kChunk = 256;             // entries of the longest row per chunk

struct LongInterval {
  int64_t it;       // interval
  int64_t row;      // its longest row
  int64_t first;    // that row's first entry
  int64_t len;      // and its length
};

template <int R>
__global__ void __launch_bounds__(256) k_count_rk(int64_t n, int64_t I, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ colidx,
                                                  unsigned long long* __restrict__ acc, LongInterval* __restrict__ longs,
                                                  unsigned long long* __restrict__ nlong, int64_t cap) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt[3] = {0ull, 0ull, 0ull};
  if (it < I) {
    const int64_t row0 = it * R;
    const int64_t rend = row0 + R < n ? row0 + R : n;
    if (rowptr[rend] - rowptr[row0] > kLongEntries) {
      // counted by k_count_long in chunks along its longest row
      LongInterval li{it, row0, rowptr[row0], 0};
      for (int64_t row = row0; row < rend; ++row) {
        const int64_t len = rowptr[row + 1] - rowptr[row];
        if (len > li.len) li = LongInterval{it, row, rowptr[row], len};
      }
      const unsigned long long slot = atomicAdd(nlong, 1ull);
      if ((int64_t)slot < cap) longs[slot] = li;
    } else {
      count_merged<R>(n, row0, rowptr, colidx, INT_MIN, INT_MAX, cnt);
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) warp_add(&acc[q], cnt[q]);
}

// A long interval in chunks: chunk j looks for its start among the entries
// j*kChunk .. (j+1)*kChunk - 1 of the longest row, taking the first column
// with no merged column of the interval in the 16 before it (such a column
// starts a block in every cover with c <= 16, so the covers on either side
// are independent); it counts the blocks from there to the next chunk's start
// (the first such column from entry (j+1)*kChunk on). A chunk without such a
// column counts nothing: the chunk before it runs on through its range.
// task = (index into longs, chunk)
template <int R>
__device__ __forceinline__ bool clean_start(int64_t n, int64_t row0, const int64_t* __restrict__ rowptr,
                                            const int32_t* __restrict__ colidx, int32_t b) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (row0 + i >= n) break;
    int64_t a = rowptr[row0 + i], e = rowptr[row0 + i + 1];
    while (a < e) {  // first entry >= b
      const int64_t mid = (a + e) >> 1;
      if (colidx[mid] < b) a = mid + 1; else e = mid;
    }
    if (a > rowptr[row0 + i] && colidx[a - 1] > b - 16) return false;
  }
  return true;
}

template <int R>
__device__ __forceinline__ int32_t next_start(int64_t n, const LongInterval& li, const int64_t* __restrict__ rowptr,
                                              const int32_t* __restrict__ colidx, int64_t from, int64_t to) {
  for (int64_t p = from; p < to && p < li.len; ++p) {
    const int32_t b = colidx[li.first + p];
    if (clean_start<R>(n, li.it * R, rowptr, colidx, b)) return b;
  }
  return INT_MAX;
}

template <int R>
__global__ void __launch_bounds__(256) k_count_long(int64_t n, const int64_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ colidx,
                                                    const LongInterval* __restrict__ longs, const int2* __restrict__ tasks,
                                                    int64_t ntasks, unsigned long long* __restrict__ acc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt[3] = {0ull, 0ull, 0ull};
  if (t < ntasks) {
    const int2 tk = tasks[t];
    const LongInterval li = longs[tk.x];
    const int64_t j = tk.y;
    const int32_t lo = j == 0 ? INT_MIN : next_start<R>(n, li, rowptr, colidx, j * kChunk, (j + 1) * kChunk);
    if (lo != INT_MAX) {
      const int32_t hi = next_start<R>(n, li, rowptr, colidx, (j + 1) * kChunk, li.len);
      count_merged<R>(n, li.it * R, rowptr, colidx, lo, hi, cnt);
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
  if (n > 0) k_row_stats<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, rowptr, acc + 12);
  // r = 2, 4, 8: short intervals directly, long ones listed and then counted in chunks
  const int64_t cap = nnz / kLongEntries + 1;
  LongInterval* longs = nullptr;
  unsigned long long* nlong = nullptr;
  e = cudaMallocAsync((void**)&longs, sizeof(LongInterval) * (size_t)cap, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&nlong, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  for (int a = 1; a < 4 && e == cudaSuccess; ++a) {
    const int r = 1 << a;
    const int64_t I = (n + r - 1) / r;
    if (I == 0) continue;
    e = cudaMemsetAsync(nlong, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) break;
    const unsigned g = (unsigned)((I + 255) / 256);
    unsigned long long* dst = acc + 3 * a;
    switch (r) {
      case 2: k_count_rk<2><<<g, 256, 0, s>>>(n, I, rowptr, colidx, dst, longs, nlong, cap); break;
      case 4: k_count_rk<4><<<g, 256, 0, s>>>(n, I, rowptr, colidx, dst, longs, nlong, cap); break;
      default: k_count_rk<8><<<g, 256, 0, s>>>(n, I, rowptr, colidx, dst, longs, nlong, cap); break;
    }
    unsigned long long nl = 0;
    e = cudaMemcpyAsync(&nl, nlong, sizeof(nl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || nl == 0) continue;
    std::vector<LongInterval> hl((size_t)nl);
    e = cudaMemcpyAsync(hl.data(), longs, sizeof(LongInterval) * (size_t)nl, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    std::vector<int2> tasks;
    for (size_t q = 0; q < hl.size(); ++q)
      for (int64_t j = 0; j * kChunk < hl[q].len; ++j) tasks.push_back(make_int2((int)q, (int)j));
    int2* td = nullptr;
    e = cudaMallocAsync((void**)&td, sizeof(int2) * tasks.size(), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(td, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      const int64_t nt = (int64_t)tasks.size();
      const unsigned gt = (unsigned)((nt + 255) / 256);
      switch (r) {
        case 2: k_count_long<2><<<gt, 256, 0, s>>>(n, rowptr, colidx, longs, td, nt, dst); break;
        case 4: k_count_long<4><<<gt, 256, 0, s>>>(n, rowptr, colidx, longs, td, nt, dst); break;
        default: k_count_long<8><<<gt, 256, 0, s>>>(n, rowptr, colidx, longs, td, nt, dst); break;
      }
      e = cudaGetLastError();
      // the host task list must live until the copy ran
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (td) cudaFreeAsync(td, s);
  }
  cudaFreeAsync(longs, s);
  cudaFreeAsync(nlong, s);
  if (e != cudaSuccess) return e;
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
