// y = A x over the beta(r,c) storage with G lanes per interval, one lane per
// block (variants 24-29): the warp-cooperative block-row traversal.
//
// A group of G consecutive lanes owns one short interval and walks its blocks
// G at a time: lane g reads block bb + g's mask and column index (the group's
// reads are consecutive, so they coalesce), an exclusive scan of the G
// popcounts over the group gives every block its first value (the blocks'
// values are stored one after another, Eq. 1), and each lane then multiplies
// its block's values - a contiguous stretch next to its neighbours' - by the
// x entries of its block's window, keeping one partial sum per block row.
// After the last block a shuffle tree adds the group's partial sums row by
// row. Against the lane-per-row kernels this turns the value, column and
// mask streams into coalesced group reads and issues all of a block's loads
// at once; the price is the scan and the final tree, cheap when the interval
// holds a few blocks per lane. Long intervals stay on the segment path.
//
// Summation order of a row: each lane adds its blocks' products (block by
// block, bits ascending), then the fixed xor tree over the G lanes; it
// depends only on G and the interval's block count, so results repeat bit for
// bit (they differ from the lane-per-row variants' by rounding only).
#pragma once

#include "spmv_beta.cuh"

namespace spc5 {

// variants 24 / 25 / 26 / 27: G = 4 / 8 / 16 / 32 lanes per interval in
// natural order; 28 / 29: G = 4 / 8 in the sorted work order
constexpr int group_lanes(int v) {
  return v == 24 || v == 28 ? 4 : v == 25 || v == 29 ? 8 : v == 26 ? 16 : 32;
}

// Adds the products of one block (mask mk, first column col, values from
// vblk) to the row sums acc[0..R-1]. Small blocks unroll their R*C bit
// positions (all loads of the block issued before the first multiply-add);
// larger ones loop over the set bits of each block row.
template <int R, int C, class T>
__device__ __forceinline__ void block_products(const Mask<(R * C + 7) / 8>& mk, int32_t col,
                                               const typename T::V* __restrict__ vblk,
                                               const typename T::X* __restrict__ x, typename T::A (&acc)[R]) {
  using A = typename T::A;
  const typename T::X* __restrict__ xw = x + col;
  if constexpr (R * C <= 16) {
    A v[R][C], xx[R][C];
    uint32_t rb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      rb[i] = row_bits<C>(mk, i);
      const int vo = popc_below<C>(mk, i);
#pragma unroll
      for (int k = 0; k < C; ++k) {
        const bool on = (rb[i] >> k) & 1u;
        const int rank = vo + __popc(rb[i] & ((1u << k) - 1u));
        v[i][k] = on ? T::val(vblk, rank) : A(0);
        xx[i][k] = on ? T::xv(xw, k) : A(0);
      }
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int k = 0; k < C; ++k)
        if ((rb[i] >> k) & 1u) acc[i] = fmadd<T>(v[i][k], xx[i][k], acc[i]);
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      uint32_t bits = row_bits<C>(mk, i);
      int vo = popc_below<C>(mk, i);
      while (bits) {
        const int k = __ffs(bits) - 1;
        bits &= bits - 1;
        acc[i] = fmadd<T>(T::val(vblk, vo), T::xv(xw, k), acc[i]);
        ++vo;
      }
    }
  }
}

template <int R, int C, class T, bool ACCUM, int G, bool ORDER>
__device__ __forceinline__ void rows_grp_body(int64_t bid, int64_t n, int64_t I, int32_t long_blocks,
                                              int64_t long_values, const int32_t* __restrict__ brp,
                                              const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                              const typename T::V* __restrict__ val,
                                              const int64_t* __restrict__ valptr,
                                              const typename T::X* __restrict__ x, typename T::X* __restrict__ y,
                                              const int32_t* __restrict__ order, int64_t norder) {
  static_assert(G == 4 || G == 8 || G == 16 || G == 32, "group of 4, 8, 16 or 32 lanes");
  constexpr int MB = (R * C + 7) / 8;
  using A = typename T::A;
  const int lane = threadIdx.x & 31;
  const int g = lane & (G - 1);
  // the group's lanes; every shuffle below runs on exactly these lanes, and
  // every branch before it is uniform over the group
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int64_t slots = ORDER ? norder : I;
  const int64_t pos = (bid * blockDim.x + threadIdx.x) / G;
  if (pos >= slots) return;
  const int64_t it = ORDER ? (int64_t)__ldg(order + pos) : pos;
  const int32_t b0 = __ldg(brp + it), b1 = __ldg(brp + it + 1);
  int64_t vbase = __ldg(valptr + it);
  if (b1 - b0 > long_blocks || __ldg(valptr + it + 1) - vbase > long_values) return;  // the segment path's
  A acc[R];
#pragma unroll
  for (int i = 0; i < R; ++i) acc[i] = A(0);
  // the next trip's mask and column are read one trip ahead
  Mask<MB> nmk = b0 + g < b1 ? load_mask<MB>(bmask, b0 + g) : zero_mask<MB>();
  int32_t ncol = b0 + g < b1 ? __ldg(bcol + b0 + g) : 0;
  for (int32_t bb = b0; bb < b1; bb += G) {
    const int32_t b = bb + g;
    const bool have = b < b1;
    const Mask<MB> mk = nmk;
    const int32_t col = ncol;
    if (b + G < b1) {
      nmk = load_mask<MB>(bmask, b + G);
      ncol = __ldg(bcol + b + G);
    } else {
      nmk = zero_mask<MB>();
      ncol = 0;
    }
    const int cnt = popc_all(mk);
    int incl = cnt;  // inclusive scan of the popcounts over the group
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
      const int t = __shfl_up_sync(gmask, incl, d, G);
      if (g >= d) incl += t;
    }
    const int64_t off = vbase + (incl - cnt);
    vbase += __shfl_sync(gmask, incl, G - 1, G);
    if (have) block_products<R, C, T>(mk, col, val + off, x, acc);
  }
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) acc[i] += __shfl_xor_sync(gmask, acc[i], d, G);
  // lane g writes rows g, g + G, ... of the interval (after the tree every
  // lane holds every row's sum)
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int64_t row = it * R + i;
    if (i % G == g && row < n) {
      if (ACCUM)
        y[row] = y[row] + acc[i];
      else
        y[row] = acc[i];
    }
  }
}

template <int R, int C, class T, bool ACCUM, int G, bool ORDER>
__global__ void __launch_bounds__(256) k_spmv_grp(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                  const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                  const uint8_t* __restrict__ bmask,
                                                  const typename T::V* __restrict__ val,
                                                  const int64_t* __restrict__ valptr,
                                                  const typename T::X* __restrict__ x, typename T::X* __restrict__ y,
                                                  const int32_t* __restrict__ order, int64_t norder) {
  rows_grp_body<R, C, T, ACCUM, G, ORDER>(blockIdx.x, n, I, long_blocks, long_values, brp, bcol, bmask, val, valptr,
                                          x, y, order, norder);
}

// the long intervals' segments (thread blocks [0, seg_ctas)) and the groups in
// one grid, as k_spmv_rows_segs does for the lane-per-row kernels
template <int R, int C, class T, bool ACCUM, int G, bool ORDER>
__global__ void __launch_bounds__(256) k_spmv_grp_segs(int64_t seg_ctas, int64_t n, int64_t I, int32_t long_blocks,
                                                       int64_t long_values, const int32_t* __restrict__ brp,
                                                       const int32_t* __restrict__ bcol,
                                                       const uint8_t* __restrict__ bmask,
                                                       const typename T::V* __restrict__ val,
                                                       const int64_t* __restrict__ valptr,
                                                       const typename T::X* __restrict__ x,
                                                       typename T::X* __restrict__ y,
                                                       const int32_t* __restrict__ order, int64_t norder,
                                                       int64_t nseg, const Segment* __restrict__ segs,
                                                       typename T::A* __restrict__ partials) {
  if ((int64_t)blockIdx.x < seg_ctas)
    segments_body<R, C, T, 4, 1>(blockIdx.x, nseg, segs, bcol, bmask, val, x, partials);
  else
    rows_grp_body<R, C, T, ACCUM, G, ORDER>((int64_t)blockIdx.x - seg_ctas, n, I, long_blocks, long_values, brp, bcol,
                                            bmask, val, valptr, x, y, order, norder);
}

template <int R, int C, class T, int G, bool ORDER>
cudaError_t launch_grp_g(const spc5_matrix* h, const void* xv, void* yv, bool acc, void* partials, cudaStream_t s) {
  using X = typename T::X;
  using A = typename T::A;
  const X* x = static_cast<const X*>(xv);
  X* y = static_cast<X*>(yv);
  const typename T::V* val = static_cast<const typename T::V*>(h->values);
  A* part = static_cast<A*>(partials);
  const int threads = kSpmvThreads;
  const int64_t slots = ORDER ? h->norder : h->I;
  const int64_t seg_ctas = (h->nseg * kWarp + threads - 1) / threads;
  const unsigned grid = (unsigned)((slots * G + threads - 1) / threads);
  const int32_t* order = ORDER ? h->order : nullptr;
  const int64_t norder = ORDER ? h->norder : 0;
  if (fused_launch(h)) {
    auto kern = acc ? k_spmv_grp_segs<R, C, T, true, G, ORDER> : k_spmv_grp_segs<R, C, T, false, G, ORDER>;
    kern<<<(unsigned)(seg_ctas + grid), threads, 0, s>>>(seg_ctas, h->n, h->I, h->long_blocks, h->long_values,
                                                         h->block_rowptr, h->block_colidx, h->block_masks, val,
                                                         h->valptr, x, y, order, norder, h->nseg, h->segs, part);
  } else if (grid > 0) {
    auto kern = acc ? k_spmv_grp<R, C, T, true, G, ORDER> : k_spmv_grp<R, C, T, false, G, ORDER>;
    kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                  h->block_masks, val, h->valptr, x, y, order, norder);
  }
  if (h->nseg > 0) {
    const unsigned g2 = (unsigned)((h->nlong + 255) / 256);
    if (acc)
      k_spmv_fixup<R, T, true><<<g2, 256, 0, s>>>(h->n, h->nlong, h->seg_first, h->segs, part, y);
    else
      k_spmv_fixup<R, T, false><<<g2, 256, 0, s>>>(h->n, h->nlong, h->seg_first, h->segs, part, y);
  }
  return cudaGetLastError();
}

template <int R, int C, class T>
cudaError_t launch_grp(const spc5_matrix* h, const void* x, void* y, bool acc, void* partials, cudaStream_t s) {
  const bool ordered = ordered_variant(h->variant) && h->norder > 0;
  switch (h->variant) {
    case 24: return launch_grp_g<R, C, T, 4, false>(h, x, y, acc, partials, s);
    case 25: return launch_grp_g<R, C, T, 8, false>(h, x, y, acc, partials, s);
    case 26: return launch_grp_g<R, C, T, 16, false>(h, x, y, acc, partials, s);
    case 27: return launch_grp_g<R, C, T, 32, false>(h, x, y, acc, partials, s);
    case 28:
      return ordered ? launch_grp_g<R, C, T, 4, true>(h, x, y, acc, partials, s)
                     : launch_grp_g<R, C, T, 4, false>(h, x, y, acc, partials, s);
    default:
      return ordered ? launch_grp_g<R, C, T, 8, true>(h, x, y, acc, partials, s)
                     : launch_grp_g<R, C, T, 8, false>(h, x, y, acc, partials, s);
  }
}

template <class T>
cudaError_t dispatch_grp(const spc5_matrix* h, const void* x, void* y, bool acc, void* partials, cudaStream_t s) {
#define SPC5_CASE(RR, CC) \
  if (h->r == RR && h->c == CC) return launch_grp<RR, CC, T>(h, x, y, acc, partials, s);
  SPC5_CASE(1, 4) SPC5_CASE(1, 8) SPC5_CASE(1, 16)
  SPC5_CASE(2, 4) SPC5_CASE(2, 8) SPC5_CASE(2, 16)
  SPC5_CASE(4, 4) SPC5_CASE(4, 8) SPC5_CASE(4, 16)
  SPC5_CASE(8, 4) SPC5_CASE(8, 8) SPC5_CASE(8, 16)
#undef SPC5_CASE
  return cudaErrorInvalidValue;
}

}  // namespace spc5
