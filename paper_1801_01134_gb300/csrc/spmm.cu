// Y = A X for k right-hand sides over the beta(r,c) storage (multi-RHS SpMM).
//
// The paper cites multiplication by several vectors as a known way to reuse
// the matrix stream (section "Sparse Matrix Vector Product (SpMV)"): every
// decoded nonzero of A is applied to k values of X at once. X is m-by-k and
// Y n-by-k, both row-major with leading dimensions ldx, ldy >= k.
//
// Mappings for the short intervals, chosen by the column tile ktile:
//   ktile 1, 4, -8, -16, -32   one lane per row keeps 1 to 32 accumulators
//                  and, per nonzero, reads one matrix value and that wide a
//                  slice of an X row (16-byte loads when X rows are aligned);
//   ktile 8/16/32  ktile / 4 lanes per interval, 4 columns each: per stored
//                  value the group reads one coalesced ktile-wide slice of
//                  its X row (for large k, where X dominates).
// The grid's y dimension covers the column tiles. Long intervals go through
// warp segments and a fix-up, as in the SpMV, with per-row partials per
// segment and column (beta(1,c) with k >= 4: column groups, see
// k_spmm_seg_cols).
//
// The one-lane-per-row and segment kernels take the block shape at run time
// (the decode is amortised over k multiply-adds per nonzero, and it keeps the
// number of kernel instantiations small); the column-group kernel of the short
// intervals is compiled per shape.
#include "spmv_beta.cuh"

namespace spc5 {
namespace {

struct RtMask {
  uint32_t w[4];
};

__device__ __forceinline__ RtMask load_mask_rt(const uint8_t* __restrict__ masks, int64_t b, int mb) {
  RtMask m{{0u, 0u, 0u, 0u}};
  switch (mb) {
    case 1: m.w[0] = __ldg(masks + b); break;
    case 2: m.w[0] = __ldg(reinterpret_cast<const uint16_t*>(masks) + b); break;
    case 4: m.w[0] = __ldg(reinterpret_cast<const uint32_t*>(masks) + b); break;
    case 8: {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(masks) + b);
      m.w[0] = v.x;
      m.w[1] = v.y;
      break;
    }
    default: {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(masks) + b);
      m.w[0] = v.x;
      m.w[1] = v.y;
      m.w[2] = v.z;
      m.w[3] = v.w;
    }
  }
  return m;
}

__device__ __forceinline__ uint32_t row_bits_rt(const RtMask& m, int i, int c) {
  const int p = i * c;
  return (m.w[p >> 5] >> (p & 31)) & ((1u << c) - 1u);
}

__device__ __forceinline__ int popc_below_rt(const RtMask& m, int i, int c) {
  const int p = i * c;
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < (p >> 5)) cnt += __popc(m.w[q]);
  if (p & 31) cnt += __popc(m.w[p >> 5] & ((1u << (p & 31)) - 1u));
  return cnt;
}

__device__ __forceinline__ int popc_all_rt(const RtMask& m) {
  return __popc(m.w[0]) + __popc(m.w[1]) + __popc(m.w[2]) + __popc(m.w[3]);
}

template <class T, int KT>
__device__ __forceinline__ void fma_row(typename T::A (&acc)[KT], typename T::A v, const typename T::X* __restrict__ xr,
                                        int kk) {
#pragma unroll
  for (int t = 0; t < KT; ++t)
    if (t < kk) acc[t] = fma(v, (typename T::A)__ldg(xr + t), acc[t]);
}

// the same with the KT values of the X row read as 16-byte vectors (the
// caller checked the alignment and that the tile is full)
template <class T, int KT>
__device__ __forceinline__ void fma_row_vec(typename T::A (&acc)[KT], typename T::A v,
                                            const typename T::X* __restrict__ xr) {
  if constexpr (sizeof(typename T::X) == 4) {
#pragma unroll
    for (int q = 0; q < KT / 4; ++q) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(xr) + q);
      acc[4 * q + 0] = fma(v, (typename T::A)t.x, acc[4 * q + 0]);
      acc[4 * q + 1] = fma(v, (typename T::A)t.y, acc[4 * q + 1]);
      acc[4 * q + 2] = fma(v, (typename T::A)t.z, acc[4 * q + 2]);
      acc[4 * q + 3] = fma(v, (typename T::A)t.w, acc[4 * q + 3]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < KT / 2; ++q) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(xr) + q);
      acc[2 * q + 0] = fma(v, (typename T::A)t.x, acc[2 * q + 0]);
      acc[2 * q + 1] = fma(v, (typename T::A)t.y, acc[2 * q + 1]);
    }
  }
}

// short intervals: one lane per row, KT columns of X per lane
template <class T, int KT>
__global__ void __launch_bounds__(256) k_spmm_rows(int64_t n, int64_t I, int r, int c, int mb, int32_t long_blocks,
                                                   int64_t long_values, const int32_t* __restrict__ brp,
                                                   const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                   const typename T::V* __restrict__ val,
                                                   const int64_t* __restrict__ valptr,
                                                   const typename T::X* __restrict__ X, int64_t ldx,
                                                   typename T::X* __restrict__ Y, int64_t ldy, int k, bool vec) {
  using A = typename T::A;
  const int lane = threadIdx.x & 31;
  const int S = kWarp / r;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t it = warp * S + lane / r;
  const int i = lane % r;
  const int j0 = blockIdx.y * KT;
  const int kk = k - j0 < KT ? k - j0 : KT;
  const bool full_vec = vec && kk == KT;  // 16-byte X loads for this tile
  if (it >= I || lane >= S * r) return;
  int32_t b = __ldg(brp + it);
  const int32_t bend = __ldg(brp + it + 1);
  const int64_t v0 = __ldg(valptr + it);
  if (bend - b > long_blocks || __ldg(valptr + it + 1) - v0 > long_values) return;  // the segment path's
  const typename T::V* __restrict__ vrow = val + v0;
  A acc[KT];
#pragma unroll
  for (int t = 0; t < KT; ++t) acc[t] = 0;
  int32_t vbase = 0;
  for (; b < bend; ++b) {
    const RtMask mk = load_mask_rt(bmask, b, mb);
    uint32_t bits = row_bits_rt(mk, i, c);
    int32_t vo = vbase + popc_below_rt(mk, i, c);
    vbase += popc_all_rt(mk);
    if (!bits) continue;
    const int64_t col0 = __ldg(bcol + b);
    while (bits) {
      const int kb = __ffs(bits) - 1;
      bits &= bits - 1;
      if constexpr (KT >= 4) {
        if (full_vec) {
          fma_row_vec<T, KT>(acc, T::val(vrow, vo++), X + (col0 + kb) * ldx + j0);
          continue;
        }
      }
      fma_row<T, KT>(acc, T::val(vrow, vo++), X + (col0 + kb) * ldx + j0, kk);
    }
  }
  const int64_t row = it * r + i;
  if (row < n) {
#pragma unroll
    for (int t = 0; t < KT; ++t)
      if (t < kk) Y[row * ldy + j0 + t] = acc[t];
  }
}

// short intervals, G lanes per interval (ktile 8 / 16 / 32, G = ktile / 4):
// lane g of a group owns the 4 columns j = tile * ktile + 4 g .. + 3 of X and
// Y and keeps the interval's R row sums for each. The group walks the
// interval's blocks and each block row's set bits one by one: per stored
// value one value read (one address for the whole group), the 4-column slice
// of the X row of its column (one 16-byte load when X rows are aligned; the
// group's slices form one coalesced stretch of ktile values) and 4
// multiply-adds; the next block's mask and column are read one block ahead.
// No lane talks to another. Each (row, column) sum adds the row's products in
// storage order, as the SpMV does. (Measured on GB300: unrolling every bit
// position of a block and reading the X rows of its columns once for all its
// rows issued six times the instructions of the multiply-adds and ran 1.3 to
// 1.5x slower: 27-point stencil 128^3, k = 32 0.74 -> 0.56 ms.)
template <class T, int V>
struct XQuad {
  typename T::A v[V];
};

template <class T, int V>
__device__ __forceinline__ XQuad<T, V> load_xq(const typename T::X* __restrict__ p, int nv, bool vec) {
  XQuad<T, V> q;
  if constexpr (sizeof(typename T::X) == 4 && V == 4) {
    if (vec) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p));
      q.v[0] = t.x;
      q.v[1] = t.y;
      q.v[2] = t.z;
      q.v[3] = t.w;
      return q;
    }
  }
#pragma unroll
  for (int t = 0; t < V; ++t) q.v[t] = t < nv ? (typename T::A)__ldg(p + t) : typename T::A(0);
  return q;
}

template <class T, int R, int C, int G>
__global__ void __launch_bounds__(256) k_spmm_blk(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                   const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                   const uint8_t* __restrict__ bmask,
                                                   const typename T::V* __restrict__ val,
                                                   const int64_t* __restrict__ valptr,
                                                   const typename T::X* __restrict__ X, int64_t ldx,
                                                   typename T::X* __restrict__ Y, int64_t ldy, int k, bool vec) {
  using A = typename T::A;
  constexpr int MB = (R * C + 7) / 8;
  constexpr int V = 4;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t it = t / G;
  const int j = blockIdx.y * (G * V) + (int)(t % G) * V;
  if (it >= I || j >= k) return;
  const int nv = k - j < V ? k - j : V;
  const bool full = vec && nv == V;
  int32_t b = __ldg(brp + it);
  const int32_t bend = __ldg(brp + it + 1);
  const int64_t v0 = __ldg(valptr + it);
  if (bend - b > long_blocks || __ldg(valptr + it + 1) - v0 > long_values) return;  // the segment path's
  const typename T::V* __restrict__ vrow = val + v0;
  const typename T::X* __restrict__ xcol = X + j;
  A acc[R][V];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int q = 0; q < V; ++q) acc[i][q] = A(0);
  int32_t vv = 0;
  Mask<MB> m0 = b < bend ? load_mask<MB>(bmask, b) : zero_mask<MB>();
  int64_t c0 = b < bend ? __ldg(bcol + b) : 0;
  for (; b < bend; ++b) {
    const Mask<MB> mk = m0;
    const typename T::X* __restrict__ xb = xcol + c0 * ldx;
    if (b + 1 < bend) {
      m0 = load_mask<MB>(bmask, b + 1);
      c0 = __ldg(bcol + b + 1);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
      uint32_t bits = row_bits<C>(mk, i);
      while (bits) {
        const int kk = __ffs(bits) - 1;
        bits &= bits - 1;
        const A v = T::val(vrow, vv++);
        const XQuad<T, V> xq = load_xq<T, V>(xb + kk * ldx, nv, full);
#pragma unroll
        for (int q = 0; q < V; ++q) acc[i][q] = fma(v, xq.v[q], acc[i][q]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int64_t row = it * R + i;
    if (row < n)
#pragma unroll
      for (int q = 0; q < V; ++q)
        if (q < nv) Y[row * ldy + j + q] = acc[i][q];
  }
}

template <class T, int G>
void launch_spmm_blk(const spc5_matrix* h, int k, const typename T::X* Xm, int64_t ldx, typename T::X* Ym,
                     int64_t ldy, cudaStream_t s) {
  const typename T::V* val = static_cast<const typename T::V*>(h->values);
  dim3 grid((unsigned)((h->I * G + 255) / 256), (unsigned)((k + 4 * G - 1) / (4 * G)));
  // 16-byte X loads when every lane's 4 columns start on a 16-byte boundary
  const bool vec = sizeof(typename T::X) == 4 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(Xm) & 15u) == 0;
#define SPC5_BLK(RR, CC)                                                                                            \
  if (h->r == RR && h->c == CC) {                                                                                   \
    k_spmm_blk<T, RR, CC, G><<<grid, 256, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr,     \
                                                  h->block_colidx, h->block_masks, val, h->valptr, Xm, ldx, Ym, ldy, \
                                                  k, vec);                                                          \
    return;                                                                                                         \
  }
  SPC5_BLK(1, 4) SPC5_BLK(1, 8) SPC5_BLK(1, 16)
  SPC5_BLK(2, 4) SPC5_BLK(2, 8) SPC5_BLK(2, 16)
  SPC5_BLK(4, 4) SPC5_BLK(4, 8) SPC5_BLK(4, 16)
  SPC5_BLK(8, 4) SPC5_BLK(8, 8) SPC5_BLK(8, 16)
#undef SPC5_BLK
}

// long intervals: a warp per segment, lane = (block slot, row); KT partials
// per (segment, row) go to part[(seg * r + i) * k + j]
template <class T, int KT>
__global__ void __launch_bounds__(256) k_spmm_segments(int64_t nseg, int r, int c, int mb,
                                                       const Segment* __restrict__ segs,
                                                       const int32_t* __restrict__ bcol,
                                                       const uint8_t* __restrict__ bmask,
                                                       const typename T::V* __restrict__ val,
                                                       const typename T::X* __restrict__ X, int64_t ldx,
                                                       typename T::A* __restrict__ part, int k) {
  using A = typename T::A;
  const int lane = threadIdx.x & 31;
  const int64_t seg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (seg >= nseg) return;
  const int S = kWarp / r;
  const int slot = lane / r, i = lane % r;
  const bool active = lane < S * r;
  const int j0 = blockIdx.y * KT;
  const int kk = k - j0 < KT ? k - j0 : KT;
  const Segment sg = segs[seg];
  int64_t vbase = sg.v_begin;
  A acc[KT];
#pragma unroll
  for (int t = 0; t < KT; ++t) acc[t] = 0;
  for (int32_t b0 = sg.b_begin; b0 < sg.b_end; b0 += S) {
    const int32_t b = b0 + slot;
    const bool valid = active && b < sg.b_end;
    RtMask mk{{0u, 0u, 0u, 0u}};
    if (valid) mk = load_mask_rt(bmask, b, mb);
    const int cnt = popc_all_rt(mk);
    int incl = cnt;
    for (int d = r; d < kWarp; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
    int64_t vo = vbase + (incl - cnt) + (valid ? popc_below_rt(mk, i, c) : 0);
    uint32_t bits = valid ? row_bits_rt(mk, i, c) : 0u;
    const int64_t col0 = valid ? __ldg(bcol + b) : 0;
    while (bits) {
      const int kb = __ffs(bits) - 1;
      bits &= bits - 1;
      fma_row<T, KT>(acc, T::val(val, vo++), X + (col0 + kb) * ldx + j0, kk);
    }
    vbase += total;
  }
#pragma unroll
  for (int t = 0; t < KT; ++t)
    for (int d = kWarp / 2; d >= r; d >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], d);
  if (lane < r) {
#pragma unroll
    for (int t = 0; t < KT; ++t)
      if (t < kk) part[(seg * r + lane) * (int64_t)k + j0 + t] = acc[t];
  }
}

// first segment of each long interval adds its segments' partials in order
template <class T>
__global__ void k_spmm_fixup(int64_t n, int64_t nseg, int r, const Segment* __restrict__ segs,
                             const typename T::A* __restrict__ part, typename T::X* __restrict__ Y, int64_t ldy,
                             int k) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t seg = t / ((int64_t)r * k);
  const int rem = (int)(t % ((int64_t)r * k));
  const int i = rem / k, j = rem % k;
  if (seg >= nseg) return;
  const int32_t count = segs[seg].count;  // segments of the interval, in its first segment only
  if (count == 0) return;
  const int32_t it = segs[seg].interval;
  typename T::A s = 0;
  for (int32_t q = 0; q < count; ++q) s += part[((seg + q) * r + i) * (int64_t)k + j];
  const int64_t row = (int64_t)it * r + i;
  if (row < n) Y[row * ldy + j] = s;
}

// Long intervals of beta(1,c) with column groups (k >= 4): a warp per
// segment walks its blocks 32 at a time - lane t reads block t's mask and
// column (consecutive over the warp) and a shuffle scan of the popcounts
// places the blocks' values - and the warp's 32/G groups of G lanes then take
// the trip's blocks in turn (group q: blocks q, q + 32/G, ...). Lane g of a
// group owns the 4 columns j0 + 4 g .. + 3: per stored value it reads that
// stretch of the X row (one 16-byte load when aligned), so a group reads a
// whole row slice of 4 G values as one coalesced request, where one lane per
// block run would read it as 4 G scalar or 16-byte pieces of its own. All
// blocks belong to the segment's row: after the last trip an xor tree adds
// the groups' sums, and group 0 writes the segment's partials. The order of
// the sums depends only on the structure (results repeat bit for bit).
template <class T, int G>
__global__ void __launch_bounds__(256) k_spmm_seg_cols(int64_t nseg, int c, int mb, const Segment* __restrict__ segs,
                                                       const int32_t* __restrict__ bcol,
                                                       const uint8_t* __restrict__ bmask,
                                                       const typename T::V* __restrict__ val,
                                                       const typename T::X* __restrict__ X, int64_t ldx,
                                                       typename T::A* __restrict__ part, int k, bool vec) {
  using A = typename T::A;
  constexpr int V = 4;
  constexpr int NG = kWarp / G;  // groups per warp
  const int lane = threadIdx.x & 31;
  const int64_t seg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (seg >= nseg) return;  // whole warp
  const int grp = lane / G, gl = lane % G;
  const int j = blockIdx.y * (G * V) + gl * V;
  const int nv = k - j < V ? (k - j > 0 ? k - j : 0) : V;
  const bool full = vec && nv == V;
  const Segment sg = segs[seg];
  int64_t vbase = sg.v_begin;
  A acc[V];
#pragma unroll
  for (int q = 0; q < V; ++q) acc[q] = A(0);
  for (int32_t b0 = sg.b_begin; b0 < sg.b_end; b0 += kWarp) {
    const int32_t b = b0 + lane;
    const bool valid = b < sg.b_end;
    const uint32_t m = valid ? load_mask_rt(bmask, b, mb).w[0] : 0u;  // r = 1: c <= 16 bits
    const int32_t col = valid ? __ldg(bcol + b) : 0;
    const int cnt = __popc(m);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    const int excl = incl - cnt;
#pragma unroll 2
    for (int q0 = 0; q0 < kWarp; q0 += NG) {
      const int q = q0 + grp;
      uint32_t mq = __shfl_sync(0xffffffffu, m, q);
      const int64_t cq = __shfl_sync(0xffffffffu, col, q);
      int64_t vo = vbase + __shfl_sync(0xffffffffu, excl, q);
      while (mq) {
        const int kb = __ffs(mq) - 1;
        mq &= mq - 1;
        const A v = T::val(val, vo++);
        if (nv > 0) {
          const XQuad<T, V> xq = load_xq<T, V>(X + (cq + kb) * ldx + j, nv, full);
#pragma unroll
          for (int t = 0; t < V; ++t) acc[t] = fma(v, xq.v[t], acc[t]);
        }
      }
    }
    vbase += __shfl_sync(0xffffffffu, incl, kWarp - 1);
  }
#pragma unroll
  for (int t = 0; t < V; ++t)
#pragma unroll
    for (int d = G; d < kWarp; d <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], d);
  if (grp == 0) {
#pragma unroll
    for (int t = 0; t < V; ++t)
      if (t < nv) part[seg * (int64_t)k + j + t] = acc[t];
  }
}

// the long intervals' segments and fix-up; beta(1,c) with k >= 4 takes the
// column groups above (G = 1, 2, 4 or 8 lanes: 4, 8, 16 or 32 columns per
// tile), other shapes a lane per (block run, row) with KT columns
template <class T, int KT>
void spmm_long(const spc5_matrix* h, int k, const typename T::X* Xm, int64_t ldx, typename T::X* Ym, int64_t ldy,
               typename T::A* part, cudaStream_t s) {
  const typename T::V* val = static_cast<const typename T::V*>(h->values);
  if (h->r == 1 && k >= 4) {
    const bool vec = sizeof(typename T::X) == 4 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(Xm) & 15u) == 0;
    const unsigned gx = (unsigned)((h->nseg * kWarp + 255) / 256);
    if (k < 8) {
      k_spmm_seg_cols<T, 1><<<dim3(gx, (unsigned)((k + 3) / 4)), 256, 0, s>>>(
          h->nseg, h->c, h->mb, h->segs, h->block_colidx, h->block_masks, val, Xm, ldx, part, k, vec);
    } else if (k >= 32) {
      k_spmm_seg_cols<T, 8><<<dim3(gx, (unsigned)((k + 31) / 32)), 256, 0, s>>>(
          h->nseg, h->c, h->mb, h->segs, h->block_colidx, h->block_masks, val, Xm, ldx, part, k, vec);
    } else if (k >= 16) {
      k_spmm_seg_cols<T, 4><<<dim3(gx, (unsigned)((k + 15) / 16)), 256, 0, s>>>(
          h->nseg, h->c, h->mb, h->segs, h->block_colidx, h->block_masks, val, Xm, ldx, part, k, vec);
    } else {
      k_spmm_seg_cols<T, 2><<<dim3(gx, (unsigned)((k + 7) / 8)), 256, 0, s>>>(
          h->nseg, h->c, h->mb, h->segs, h->block_colidx, h->block_masks, val, Xm, ldx, part, k, vec);
    }
  } else {
    dim3 grid((unsigned)((h->nseg * kWarp + 255) / 256), (unsigned)((k + KT - 1) / KT));
    k_spmm_segments<T, KT><<<grid, 256, 0, s>>>(h->nseg, h->r, h->c, h->mb, h->segs, h->block_colidx, h->block_masks,
                                                val, Xm, ldx, part, k);
  }
  const int64_t nt = h->nseg * h->r * (int64_t)k;
  k_spmm_fixup<T><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(h->n, h->nseg, h->r, h->segs, part, Ym, ldy, k);
}

template <class T, int KT>
cudaError_t spmm_launch(const spc5_matrix* h, int k, const void* Xv, int64_t ldx, void* Yv, int64_t ldy, void* part,
                        cudaStream_t s) {
  using X = typename T::X;
  using A = typename T::A;
  const X* Xm = static_cast<const X*>(Xv);
  X* Ym = static_cast<X*>(Yv);
  const typename T::V* val = static_cast<const typename T::V*>(h->values);
  const int S = kWarp / h->r;
  const unsigned tiles = (unsigned)((k + KT - 1) / KT);
  if (h->I > 0) {
    const int64_t warps = (h->I + S - 1) / S;
    dim3 grid((unsigned)((warps * kWarp + 255) / 256), tiles);
    // 16-byte X loads when every tile start is 16-byte aligned
    constexpr int N = 16 / (int)sizeof(X);
    const bool vec = KT >= 4 && KT % N == 0 && ldx % N == 0 && (reinterpret_cast<uintptr_t>(Xm) & 15u) == 0;
    k_spmm_rows<T, KT><<<grid, 256, 0, s>>>(h->n, h->I, h->r, h->c, h->mb, h->long_blocks, h->long_values,
                                            h->block_rowptr, h->block_colidx, h->block_masks, val, h->valptr, Xm, ldx,
                                            Ym, ldy, k, vec);
  }
  if (h->nseg > 0) spmm_long<T, KT>(h, k, Xm, ldx, Ym, ldy, static_cast<A*>(part), s);
  return cudaGetLastError();
}

// ktile columns per interval for the short intervals; the long ones take
// spmm_long
template <class T, int G>
cudaError_t spmm_launch_cols(const spc5_matrix* h, int k, const void* Xv, int64_t ldx, void* Yv, int64_t ldy,
                             void* part, cudaStream_t s) {
  using X = typename T::X;
  using A = typename T::A;
  const X* Xm = static_cast<const X*>(Xv);
  X* Ym = static_cast<X*>(Yv);
  const typename T::V* val = static_cast<const typename T::V*>(h->values);
  if (h->I > 0) launch_spmm_blk<T, G / 4>(h, k, Xm, ldx, Ym, ldy, s);
  if (h->nseg > 0) spmm_long<T, 8>(h, k, Xm, ldx, Ym, ldy, static_cast<A*>(part), s);
  return cudaGetLastError();
}

// ktile 1 or 4, and -8 / -16 / -32: one lane per row holding 1, 4, 8, 16 or
// 32 columns; 8, 16, 32: ktile / 4 lanes per interval, 4 columns each
template <class T>
cudaError_t spmm_tile(int kt, const spc5_matrix* h, int k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                      void* part, cudaStream_t s) {
  switch (kt) {
    case 1: return spmm_launch<T, 1>(h, k, X, ldx, Y, ldy, part, s);
    case 4: return spmm_launch<T, 4>(h, k, X, ldx, Y, ldy, part, s);
    case -8: return spmm_launch<T, 8>(h, k, X, ldx, Y, ldy, part, s);
    case -16: return spmm_launch<T, 16>(h, k, X, ldx, Y, ldy, part, s);
    case -32: return spmm_launch<T, 32>(h, k, X, ldx, Y, ldy, part, s);
    case 8: return spmm_launch_cols<T, 8>(h, k, X, ldx, Y, ldy, part, s);
    case 16: return spmm_launch_cols<T, 16>(h, k, X, ldx, Y, ldy, part, s);
    default: return spmm_launch_cols<T, 32>(h, k, X, ldx, Y, ldy, part, s);
  }
}

}  // namespace

int spmm_auto_tile(int k) {
  if (k <= 1) return 1;
  if (k <= 4) return 4;
  if (k <= 8) return 8;
  if (k <= 16) return 16;
  return 32;
}

spc5_status spmm_impl(spc5_matrix* h, int k, const void* X, int64_t ldx, void* Y, int64_t ldy, int ktile,
                      cudaStream_t s) {
  const int kt = ktile != 0 ? ktile : spmm_auto_tile(k);
  // segment partials: n_segments * r * k accumulators, kept by the handle and
  // grown on demand (the growth synchronises the device)
  const size_t need = (size_t)h->nseg * (size_t)h->r * (size_t)k * (h->vt == SPC5_F64 ? 8 : 4);
  if (need > h->spmm_scratch_bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) return cuda_fail(e, "spmm: segment scratch");
    cudaFree(h->spmm_scratch);  // synchronises: no queued kernel still uses the old buffer
    h->spmm_scratch = p;
    h->spmm_scratch_bytes = need;
  }
  cudaError_t e;
  switch (h->vt) {
    case SPC5_F64: e = spmm_tile<F64>(kt, h, k, X, ldx, Y, ldy, h->spmm_scratch, s); break;
    case SPC5_F32: e = spmm_tile<F32>(kt, h, k, X, ldx, Y, ldy, h->spmm_scratch, s); break;
    default: e = spmm_tile<BF16>(kt, h, k, X, ldx, Y, ldy, h->spmm_scratch, s); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "spmm launch");
  return SPC5_OK;
}

}  // namespace spc5
