// CSR -> beta(r,c) conversion on the GPU (section "Block-based storage
// without zero padding"; the paper measures conversion at about two
// sequential SpMVs, section "Test matrices").
//
// Pipeline, all on the caller's stream:
//   1. k_validate   one thread per row: columns ascending, unique, in [0, m).
//   2. k_count      one thread per interval: greedy leftmost cover of the
//                   merged columns of the interval's r rows -> blocks per
//                   interval, and the number of warp segments of long ones.
//   3. scan         exclusive prefix sums -> block_rowptr, segment pointers.
//   4. k_fill       one thread per interval: the same cover again, emitting
//                   block_colidx, the r*c-bit masks, the values in block
//                   order (row-major inside a block) and the segment table.
//   5. k_valptr     first value of each interval = rowptr[min(r*i, n)].
// Steps 2 and 4 run the same device function, so the block decisions of the
// two passes are identical by construction.
#include <algorithm>
#include <climits>
#include <vector>

#include "internal.cuh"

namespace spc5 {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ------------------------------------------------------------ validation
// status[0] receives min over bad rows of (row * 8 + code).
__global__ void k_validate(int64_t n, int64_t m, int64_t nnz, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ colidx, unsigned long long* __restrict__ status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t a = rowptr[i], b = rowptr[i + 1];
  int code = 0;
  if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == n - 1 && b != nnz)) {
    code = SPC5_EINVAL;
  } else {
    int32_t prev = -1;
    for (int64_t p = a; p < b; ++p) {
      int32_t col = colidx[p];
      if (col < 0 || col >= m) { code = SPC5_ERANGE; break; }
      if (p > a) {
        if (col == prev) { code = SPC5_EDUP; break; }
        if (col < prev) { code = SPC5_EUNSORTED; break; }
      }
      prev = col;
    }
  }
  if (code) atomicMin(status, (unsigned long long)i * 8ull + (unsigned long long)code);
}

// ------------------------------------------------------------ block cover
// Greedy leftmost cover of one interval. For every block, `emit(s, lo, hi)`
// receives the block start s and, per row i, the entry range [lo[i], hi[i])
// whose columns fall in [s, s + c). Returns the number of blocks.
template <int R, class Emit>
__device__ __forceinline__ int32_t cover_interval(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                                  int64_t row0, int rows, int c, Emit&& emit) {
  int64_t h[R], e[R];
  int64_t cur[R];  // column at the head of each row, or LLONG_MAX once exhausted
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (i < rows) {
      h[i] = rowptr[row0 + i];
      e[i] = rowptr[row0 + i + 1];
    } else {
      h[i] = e[i] = 0;
    }
    cur[i] = h[i] < e[i] ? (int64_t)colidx[h[i]] : LLONG_MAX;
  }
  int32_t nb = 0;
  for (;;) {
    int64_t s = LLONG_MAX;
#pragma unroll
    for (int i = 0; i < R; ++i) s = cur[i] < s ? cur[i] : s;
    if (s == LLONG_MAX) break;
    int64_t lo[R], hi[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      lo[i] = h[i];
      while (cur[i] < s + c) {
        ++h[i];
        cur[i] = h[i] < e[i] ? (int64_t)colidx[h[i]] : LLONG_MAX;
      }
      hi[i] = h[i];
    }
    emit(s, nb, lo, hi);
    ++nb;
  }
  return nb;
}

template <int R>
__global__ void k_count(int64_t n, int64_t I, int c, const int64_t* __restrict__ rowptr,
                        const int32_t* __restrict__ colidx, int32_t* __restrict__ counts) {
  int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  int64_t row0 = it * R;
  int rows = (int)(n - row0 < (int64_t)R ? n - row0 : (int64_t)R);
  counts[it] = cover_interval<R>(rowptr, colidx, row0, rows, c, [](int64_t, int32_t, const int64_t*, const int64_t*) {});
}

// Warp segments of each long interval (0 for short ones). An interval is long
// when it has more than long_blocks blocks or more than long_values values:
// one lane per row would then hold up its whole warp.
__global__ void k_nseg(int64_t n, int64_t I, int r, int long_blocks, int64_t long_values, int seg_blocks,
                       const int32_t* __restrict__ counts, const int64_t* __restrict__ rowptr,
                       int32_t* __restrict__ nseg) {
  int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  int32_t nb = counts[it];
  const int64_t r0 = it * r, r1 = (it + 1) * r < n ? (it + 1) * r : n;
  const int64_t nv = rowptr[r1] - rowptr[r0];
  const bool lng = nb > long_blocks || nv > long_values;
  nseg[it] = lng ? (nb + seg_blocks - 1) / seg_blocks : 0;
}

__global__ void k_long_flags(int64_t I, const int32_t* __restrict__ segptr, int32_t* __restrict__ flag) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it < I) flag[it] = segptr[it + 1] > segptr[it] ? 1 : 0;
}

__global__ void k_seg_first(int64_t I, const int32_t* __restrict__ segptr, const int32_t* __restrict__ flag,
                            const int32_t* __restrict__ pos, int32_t* __restrict__ first) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it < I && flag[it]) first[pos[it]] = segptr[it];
}

template <int R, class VT>
__global__ void k_fill(int64_t n, int64_t I, int c, int mb, int seg_blocks, const int64_t* __restrict__ rowptr,
                       const int32_t* __restrict__ colidx, const VT* __restrict__ values,
                       const int32_t* __restrict__ block_rowptr, const int32_t* __restrict__ segptr,
                       int32_t* __restrict__ bcol, uint8_t* __restrict__ bmask, VT* __restrict__ bval,
                       Segment* __restrict__ segs) {
  int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  int64_t row0 = it * R;
  int rows = (int)(n - row0 < (int64_t)R ? n - row0 : (int64_t)R);
  int32_t b0 = block_rowptr[it];
  int32_t bend = block_rowptr[it + 1];
  bool is_long = segptr != nullptr && segptr[it + 1] > segptr[it];
  int32_t seg0 = is_long ? segptr[it] : 0;
  int64_t vo = rowptr[row0];  // the interval's values start where its first row starts in CSR
  cover_interval<R>(rowptr, colidx, row0, rows, c, [&](int64_t s, int32_t j, const int64_t* lo, const int64_t* hi) {
    int32_t b = b0 + j;
    if (is_long && j % seg_blocks == 0) {
      Segment sg;
      sg.interval = (int32_t)it;
      sg.b_begin = b;
      sg.b_end = min(b + seg_blocks, bend);
      sg.count = j == 0 ? (bend - b0 + seg_blocks - 1) / seg_blocks : 0;
      sg.v_begin = vo;
      segs[seg0 + j / seg_blocks] = sg;
    }
    uint32_t mw[4] = {0u, 0u, 0u, 0u};  // up to 128 mask bits
#pragma unroll
    for (int i = 0; i < R; ++i) {
      for (int64_t p = lo[i]; p < hi[i]; ++p) {
        int bit = i * c + (int)(colidx[p] - s);
        mw[bit >> 5] |= 1u << (bit & 31);
        bval[vo++] = values[p];
      }
    }
    bcol[b] = (int32_t)s;
    uint8_t* dst = bmask + (int64_t)b * mb;
    for (int q = 0; q < mb; ++q) dst[q] = (uint8_t)(mw[q >> 2] >> (8 * (q & 3)));
  });
}

__global__ void k_valptr(int64_t n, int64_t I, int r, const int64_t* __restrict__ rowptr, int64_t* __restrict__ valptr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > I) return;
  int64_t row = i * r;
  valptr[i] = rowptr[row < n ? row : n];
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of int32 counts into int64 partial results.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t ws = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    int64_t wi = ws;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - ws;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  int64_t r = warp_sums[w] + incl - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_tiles(const int32_t* __restrict__ in, int64_t L, int64_t* __restrict__ out,
                             int64_t* __restrict__ tile_sums) {
  __shared__ int64_t tot;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < L ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int64_t pre = block_exclusive_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < L) out[base + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// one CTA: exclusive scan of the tile sums, in chunks, with a running carry
__global__ void k_scan_tile_sums(int64_t* __restrict__ tile_sums, int64_t ntiles, int64_t* __restrict__ grand_total) {
  __shared__ int64_t tot;
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < ntiles ? tile_sums[i] : 0;
    int64_t pre = block_exclusive_scan(v, &tot);
    if (i < ntiles) tile_sums[i] = carry + pre;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand_total = carry;
}

// add tile offsets; write int32 results (caller checked the total) and the total at index L
__global__ void k_scan_finish(const int64_t* __restrict__ part, const int64_t* __restrict__ tile_sums, int64_t L,
                              const int64_t* __restrict__ grand_total, int32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) out[i] = (int32_t)(part[i] + tile_sums[i / kScanTile]);
  if (i == L) out[L] = (int32_t)*grand_total;
}

struct DeviceBuf {
  void* p = nullptr;
  ~DeviceBuf() {
    if (p) cudaFree(p);
  }
};

// Exclusive scan of in[0..L) into out[0..L] (out[L] = total). Returns the
// total through *total_host (synchronises the stream).
spc5_status scan_counts(const int32_t* in, int64_t L, int32_t* out, int64_t* total_host, cudaStream_t s) {
  int64_t ntiles = (L + kScanTile - 1) / kScanTile;
  if (ntiles < 1) ntiles = 1;
  DeviceBuf part, sums;
  cudaError_t e = cudaMalloc(&part.p, sizeof(int64_t) * (size_t)(L > 0 ? L : 1));
  if (e != cudaSuccess) return cuda_fail(e, "scan scratch");
  e = cudaMalloc(&sums.p, sizeof(int64_t) * (size_t)(ntiles + 1));
  if (e != cudaSuccess) return cuda_fail(e, "scan scratch");
  int64_t* p64 = (int64_t*)part.p;
  int64_t* t64 = (int64_t*)sums.p;
  k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, L, p64, t64);
  k_scan_tile_sums<<<1, kScanThreads, 0, s>>>(t64, ntiles, t64 + ntiles);
  int64_t tot = 0;
  e = cudaMemcpyAsync(&tot, t64 + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "scan");
  *total_host = tot;
  if (tot > INT_MAX) return fail(SPC5_ERANGE, "prefix sum exceeds int32 (too many blocks)");
  k_scan_finish<<<(unsigned)((L + 1 + 255) / 256), 256, 0, s>>>(p64, t64, L, t64 + ntiles, out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // scratch is freed on return
  if (e != cudaSuccess) return cuda_fail(e, "scan");
  return SPC5_OK;
}

template <int R>
void launch_count(int64_t n, int64_t I, int c, const int64_t* rowptr, const int32_t* colidx, int32_t* counts,
                  cudaStream_t s) {
  if (I == 0) return;
  k_count<R><<<(unsigned)((I + 127) / 128), 128, 0, s>>>(n, I, c, rowptr, colidx, counts);
}

template <class VT>
void launch_fill_r(int r, int64_t n, int64_t I, int c, int mb, int sb, const int64_t* rowptr, const int32_t* colidx,
                   const void* values, const int32_t* brp, const int32_t* segptr, spc5_matrix* h, cudaStream_t s) {
  if (I == 0) return;
  unsigned grid = (unsigned)((I + 127) / 128);
  const VT* v = (const VT*)values;
  VT* bv = (VT*)h->values;
  switch (r) {
    case 1: k_fill<1, VT><<<grid, 128, 0, s>>>(n, I, c, mb, sb, rowptr, colidx, v, brp, segptr, h->block_colidx, h->block_masks, bv, h->segs); break;
    case 2: k_fill<2, VT><<<grid, 128, 0, s>>>(n, I, c, mb, sb, rowptr, colidx, v, brp, segptr, h->block_colidx, h->block_masks, bv, h->segs); break;
    case 4: k_fill<4, VT><<<grid, 128, 0, s>>>(n, I, c, mb, sb, rowptr, colidx, v, brp, segptr, h->block_colidx, h->block_masks, bv, h->segs); break;
    default: k_fill<8, VT><<<grid, 128, 0, s>>>(n, I, c, mb, sb, rowptr, colidx, v, brp, segptr, h->block_colidx, h->block_masks, bv, h->segs); break;
  }
}

void count_r(int r, int64_t n, int64_t I, int c, const int64_t* rowptr, const int32_t* colidx, int32_t* counts,
             cudaStream_t s) {
  switch (r) {
    case 1: launch_count<1>(n, I, c, rowptr, colidx, counts, s); break;
    case 2: launch_count<2>(n, I, c, rowptr, colidx, counts, s); break;
    case 4: launch_count<4>(n, I, c, rowptr, colidx, counts, s); break;
    default: launch_count<8>(n, I, c, rowptr, colidx, counts, s); break;
  }
}

void free_matrix(spc5_matrix* h) {
  if (!h) return;
  cudaFree(h->order);
  cudaFree(h->spmm_scratch);
  cudaFree(h->block_rowptr);
  cudaFree(h->block_colidx);
  cudaFree(h->block_masks);
  cudaFree(h->values);
  cudaFree(h->valptr);
  cudaFree(h->segs);
  cudaFree(h->seg_first);
  cudaFree(h->partials);
  delete h;
}

// allocation padded to a multiple of 16 bytes plus 16 (bulk copies may round up)
cudaError_t alloc_padded(void** p, size_t bytes, cudaStream_t s) {
  size_t b = ((bytes + 15) / 16) * 16 + 16;
  cudaError_t e = cudaMalloc(p, b);
  if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, b, s);
  return e;
}

// Longest row (in stored entries) of each short interval, from the masks;
// -1 for the intervals of the segment path.
template <int R, int C>
__global__ void k_order_key(int64_t I, int32_t long_blocks, int64_t long_values, const int32_t* __restrict__ brp,
                            const uint8_t* __restrict__ masks, const int64_t* __restrict__ valptr,
                            int32_t* __restrict__ key) {
  constexpr int MB = (R * C + 7) / 8;
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  const int32_t b0 = brp[it], b1 = brp[it + 1];
  if (b1 - b0 > long_blocks || valptr[it + 1] - valptr[it] > long_values) {
    key[it] = -1;
    return;
  }
  int32_t len[R];
#pragma unroll
  for (int i = 0; i < R; ++i) len[i] = 0;
  for (int32_t b = b0; b < b1; ++b) {
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (int q = 0; q < MB; ++q) w[q >> 2] |= (uint32_t)masks[(int64_t)b * MB + q] << (8 * (q & 3));
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int p = i * C;
      len[i] += __popc((w[p >> 5] >> (p & 31)) & (C == 32 ? 0xffffffffu : ((1u << C) - 1u)));
    }
  }
  int32_t mx = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) mx = len[i] > mx ? len[i] : mx;
  key[it] = mx;
}

template <int R>
void launch_order_key(int c, const spc5_matrix* h, int32_t* key, cudaStream_t s) {
  const unsigned grid = (unsigned)((h->I + 255) / 256);
  switch (c) {
    case 4: k_order_key<R, 4><<<grid, 256, 0, s>>>(h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_masks, h->valptr, key); break;
    case 8: k_order_key<R, 8><<<grid, 256, 0, s>>>(h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_masks, h->valptr, key); break;
    default: k_order_key<R, 16><<<grid, 256, 0, s>>>(h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_masks, h->valptr, key); break;
  }
}

}  // namespace

// Work order of the lane-per-row kernel (variants 9, 10, 13, 15): the short
// intervals, sorted by their longest row (descending, stable) inside windows
// of order_window rows (all intervals together when order_window <= 0), so
// that the 32/r intervals of one warp have rows of similar length and the
// warp's multiply-adds are fully packed. Small windows keep the rows that
// neighbouring warps read close together in memory (measured: one global
// sort, or handing whole thread blocks out heaviest first, is slower on
// power-law graphs than 4096-row windows). The storage is untouched; only the
// assignment of intervals to lanes changes.
spc5_status build_order(spc5_matrix* h, cudaStream_t s) {
  if (h->order || h->I == 0) return SPC5_OK;
  const int64_t I = h->I;
  DeviceBuf keyd;
  cudaError_t e = cudaMalloc(&keyd.p, sizeof(int32_t) * (size_t)I);
  if (e != cudaSuccess) return cuda_fail(e, "work order: scratch");
  switch (h->r) {
    case 1: launch_order_key<1>(h->c, h, (int32_t*)keyd.p, s); break;
    case 2: launch_order_key<2>(h->c, h, (int32_t*)keyd.p, s); break;
    case 4: launch_order_key<4>(h->c, h, (int32_t*)keyd.p, s); break;
    default: launch_order_key<8>(h->c, h, (int32_t*)keyd.p, s); break;
  }
  std::vector<int32_t> key((size_t)I);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(key.data(), keyd.p, sizeof(int32_t) * (size_t)I, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "work order: keys");
  std::vector<int32_t> order;
  order.reserve((size_t)I);
  std::vector<std::pair<int32_t, int32_t>> win;
  const int64_t wiv = h->order_window > 0 ? (h->order_window + h->r - 1) / h->r : I;
  for (int64_t w0 = 0; w0 < I; w0 += wiv) {
    const int64_t w1 = w0 + wiv < I ? w0 + wiv : I;
    win.clear();
    for (int64_t it = w0; it < w1; ++it)
      if (key[(size_t)it] >= 0) win.emplace_back(-key[(size_t)it], (int32_t)it);
    std::stable_sort(win.begin(), win.end(), [](const std::pair<int32_t, int32_t>& a,
                                                const std::pair<int32_t, int32_t>& b) { return a.first < b.first; });
    for (auto& pr : win) order.push_back(pr.second);
  }
  if (!order.empty()) {
    int32_t* d = nullptr;
    e = alloc_padded((void**)&d, sizeof(int32_t) * order.size(), s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "work order: upload");
    }
    h->order = d;
  }
  h->norder = (int64_t)order.size();
  return SPC5_OK;
}

void destroy_matrix(spc5_matrix* h) { free_matrix(h); }

spc5_status convert_impl(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                         const void* values, spc5_dtype vt, int r, int c, const spc5_opts* opt, cudaStream_t s,
                         spc5_matrix** out) {
  *out = nullptr;
  spc5_matrix* h = new spc5_matrix();
  h->n = n;
  h->m = m;
  h->nnz = nnz;
  h->r = r;
  h->c = c;
  h->mb = mask_bytes(r, c);
  h->vt = vt;
  h->I = (n + r - 1) / r;
  int32_t user_long = 0;
  if (opt) {
    user_long = opt->long_blocks;
    if (opt->seg_blocks > 0) h->seg_blocks = opt->seg_blocks;
    h->variant = opt->variant;
    if (opt->order_window != 0) h->order_window = opt->order_window;
  }
  const int64_t I = h->I;
  cudaError_t e;
  auto bail = [&](spc5_status st) {
    free_matrix(h);
    return st;
  };

  // 1. validate
  DeviceBuf status, counts, nseg;
  e = cudaMalloc(&status.p, sizeof(unsigned long long));
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: status word"));
  e = cudaMemsetAsync(status.p, 0xff, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: status word"));
  if (n > 0)
    k_validate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, m, nnz, rowptr, colidx, (unsigned long long*)status.p);
  // 2. count
  e = cudaMalloc(&counts.p, sizeof(int32_t) * (size_t)(I + 1));
  if (e == cudaSuccess) e = cudaMalloc(&nseg.p, sizeof(int32_t) * (size_t)(I + 1));
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: counts"));
  unsigned long long st_host = ~0ull;
  e = cudaMemcpyAsync(&st_host, status.p, sizeof(st_host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: validation"));
  if (st_host != ~0ull) {
    int code = (int)(st_host & 7ull);
    long long row = (long long)(st_host >> 3);
    const char* what = code == SPC5_EUNSORTED ? "columns out of order" : code == SPC5_EDUP ? "repeated column"
                       : code == SPC5_ERANGE  ? "column index out of range" : "bad row pointer";
    return bail(fail((spc5_status)code, std::string("convert: CSR row ") + std::to_string(row) + ": " + what));
  }
  count_r(r, n, I, c, rowptr, colidx, (int32_t*)counts.p, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: count kernel"));

  // 3. scans
  e = alloc_padded((void**)&h->block_rowptr, sizeof(int32_t) * (size_t)(I + 1), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: block_rowptr"));
  int64_t nb = 0, ns = 0;
  spc5_status st = scan_counts((const int32_t*)counts.p, I, h->block_rowptr, &nb, s);
  if (st != SPC5_OK) return bail(st);
  // An interval goes to the warp-segment path when it is much longer than
  // the mean (lane-per-row warps then idle behind it) or than the absolute
  // floor; the caller may fix the threshold instead.
  if (user_long > 0) {
    h->long_blocks = user_long;
  } else {
    const double mean = I > 0 ? (double)nb / (double)I : 0.0;
    const double lim = 4.0 * mean;
    h->long_blocks = lim > kLongBlocks ? (lim < (double)INT_MAX ? (int32_t)lim : INT_MAX) : kLongBlocks;
  }
  {
    // an interval is also long when it holds many more values than the mean
    const double mean_v = I > 0 ? (double)nnz / (double)I : 0.0;
    const double lv = 8.0 * mean_v;
    h->long_values = lv > 2048.0 * r ? (int64_t)lv : (int64_t)2048 * r;
  }
  if (I > 0)
    k_nseg<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(n, I, r, h->long_blocks, h->long_values, h->seg_blocks,
                                                      (const int32_t*)counts.p, rowptr, (int32_t*)nseg.p);
  DeviceBuf segptr;
  e = cudaMalloc(&segptr.p, sizeof(int32_t) * (size_t)(I + 1));
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: segment pointers"));
  st = scan_counts((const int32_t*)nseg.p, I, (int32_t*)segptr.p, &ns, s);
  if (st != SPC5_OK) return bail(st);
  h->nb = nb;
  h->nseg = ns;

  // 4. arrays + fill
  e = alloc_padded((void**)&h->block_colidx, sizeof(int32_t) * (size_t)nb, s);
  if (e == cudaSuccess) e = alloc_padded((void**)&h->block_masks, (size_t)nb * (size_t)h->mb, s);
  if (e == cudaSuccess) e = alloc_padded(&h->values, value_size(vt) * (size_t)nnz, s);
  if (e == cudaSuccess) e = alloc_padded((void**)&h->valptr, sizeof(int64_t) * (size_t)(I + 1), s);
  if (e == cudaSuccess) e = alloc_padded((void**)&h->segs, sizeof(Segment) * (size_t)ns, s);
  if (e == cudaSuccess) e = alloc_padded(&h->partials, (vt == SPC5_F64 ? 8 : 4) * (size_t)ns * (size_t)r, s);
  if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? fail(SPC5_ENOMEM, "convert: out of device memory")
                                                                    : cuda_fail(e, "convert: allocation"));
  const int32_t* sp = ns > 0 ? (const int32_t*)segptr.p : nullptr;
  switch (vt) {
    case SPC5_F64: launch_fill_r<uint64_t>(r, n, I, c, h->mb, h->seg_blocks, rowptr, colidx, values, h->block_rowptr, sp, h, s); break;
    case SPC5_F32: launch_fill_r<uint32_t>(r, n, I, c, h->mb, h->seg_blocks, rowptr, colidx, values, h->block_rowptr, sp, h, s); break;
    default: launch_fill_r<uint16_t>(r, n, I, c, h->mb, h->seg_blocks, rowptr, colidx, values, h->block_rowptr, sp, h, s); break;
  }
  if (n > 0) k_valptr<<<(unsigned)((I + 1 + 255) / 256), 256, 0, s>>>(n, I, r, rowptr, h->valptr);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: fill"));

  // 5. first segment of every long interval, in interval order (the fix-up's work list)
  if (ns > 0) {
    int32_t* flag = (int32_t*)counts.p;  // free after the fill
    int32_t* pos = (int32_t*)nseg.p;
    k_long_flags<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(I, sp, flag);
    int64_t nlong = 0;
    st = scan_counts(flag, I, pos, &nlong, s);
    if (st != SPC5_OK) return bail(st);
    e = alloc_padded((void**)&h->seg_first, sizeof(int32_t) * (size_t)nlong, s);
    if (e == cudaSuccess) {
      k_seg_first<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(I, sp, flag, pos, h->seg_first);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "convert: long-interval list"));
    h->nlong = nlong;
  }

  if (ordered_variant(h->variant)) {
    spc5_status st2 = build_order(h, s);
    if (st2 != SPC5_OK) return bail(st2);
  }
  *out = h;
  return SPC5_OK;
}

// N_blocks for the twelve shapes (r outer in {1,2,4,8}, c inner in {4,8,16}).
spc5_status count_blocks_impl(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                              int64_t* nblocks_out, cudaStream_t s) {
  (void)nnz;
  const int rs[4] = {1, 2, 4, 8};
  const int cs[3] = {4, 8, 16};
  DeviceBuf counts;
  int64_t I1 = n;  // r = 1 has the most intervals
  cudaError_t e = cudaMalloc(&counts.p, sizeof(int32_t) * (size_t)(I1 + 1));
  if (e != cudaSuccess) return cuda_fail(e, "count_blocks: scratch");
  DeviceBuf out;
  e = cudaMalloc(&out.p, sizeof(int32_t) * (size_t)(I1 + 1));
  if (e != cudaSuccess) return cuda_fail(e, "count_blocks: scratch");
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 3; ++b) {
      int64_t I = (n + rs[a] - 1) / rs[a];
      count_r(rs[a], n, I, cs[b], rowptr, colidx, (int32_t*)counts.p, s);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "count_blocks: count kernel");
      int64_t tot = 0;
      spc5_status st = scan_counts((const int32_t*)counts.p, I, (int32_t*)out.p, &tot, s);
      if (st != SPC5_OK) return st;
      nblocks_out[a * 3 + b] = tot;
    }
  return SPC5_OK;
}

}  // namespace spc5
