// y = A x over the beta(1,c) storage with the warp streaming the blocks of
// its rows (variant 32).
//
// A warp owns 32 consecutive rows. Their blocks form one contiguous stretch
// of the block arrays, and their values one contiguous stretch of the value
// array (Eq. 1 stores a row's blocks, and the blocks' values, one after
// another). The warp walks that stretch 64 blocks per trip, two adjacent
// blocks per lane, whatever row each block belongs to: the mask, column and
// value reads of a trip are consecutive over the warp, no lane idles while a
// neighbour's row is longer, and rows of a few blocks cost no more than long
// ones. Per trip:
//   * a shuffle scan of the lanes' popcounts places every block's values (the
//     trip's values start where the previous trip's ended);
//   * each lane multiplies its blocks' values by the x entries of their
//     windows, bits ascending (the block product of Algorithm 1);
//   * the rows starting in the trip are marked in two 32-bit words (one bit
//     per block position, an OR over the warp of the row starts), and a
//     segmented shuffle scan over the lanes adds each row's run of blocks;
//   * lane q collects row q's sum when the row's last block falls in the
//     trip; a row that runs on into the next trip leaves its partial sum as a
//     carry, added before its next run.
// After the last trip lane q writes y for row q (one coalesced store).
//
// Rows longer than the long-interval threshold are taken by the segment path;
// a warp whose 32 rows include one falls back to one lane per row (the mask
// window decode) for its other rows, so no block is visited twice.
//
// Summation order of a row: each block's products bits ascending, the blocks
// of one run by the segmented scan's fixed tree, runs added in trip order.
// It depends only on the matrix structure, so results repeat bit for bit; they
// differ from the lane-per-row variants' by rounding only.
//
// Measured on GB300 (float32 / bfloat16, beta(1,4)): the fastest form on the
// FEM matrix (about 18 blocks per row of unequal length), where the per-row
// lanes of the other kernels idle; slower than one lane per row on the
// 27-point stencil and the uniform matrix, whose equal short rows keep those
// lanes busy at fewer instructions per block. With float64 values the products
// of a block are one multiply-add instruction per set bit for the whole warp,
// so the busiest lane sets the cost: not a float64 kernel. Reading x windows as
// aligned float4 pairs cut the L1 requests by a third but cost more
// instructions (the realignment) than it saved.
#pragma once

#include "spmv_group.cuh"

namespace spc5 {

// The masks and first columns of blocks b and b + 1 (b even): one 2- or
// 4-byte mask read and one 8-byte column read. The arrays are padded past
// their end, so the pair read at b = N_blocks - 1 stays inside them.
template <int MB>
__device__ __forceinline__ void load_pair(const uint8_t* __restrict__ masks, const int32_t* __restrict__ bcol,
                                          int32_t b, uint32_t& ma, uint32_t& mb, int32_t& ca, int32_t& cb) {
  static_assert(MB == 1 || MB == 2, "beta(1,c) masks of c <= 16 bits");
  if constexpr (MB == 1) {
    const uint32_t w = __ldg(reinterpret_cast<const uint16_t*>(masks) + (b >> 1));
    ma = w & 0xffu;
    mb = w >> 8;
  } else {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(masks) + (b >> 1));
    ma = w & 0xffffu;
    mb = w >> 16;
  }
  const int2 c2 = __ldg(reinterpret_cast<const int2*>(bcol) + (b >> 1));
  ca = c2.x;
  cb = c2.y;
}

// Product of one beta(1,c) block (mask mk, first column col, values from
// vblk), bits ascending.
template <int C, class T>
__device__ __forceinline__ typename T::A block_product1(uint32_t mk, int32_t col,
                                                        const typename T::V* __restrict__ vblk,
                                                        const typename T::X* __restrict__ x) {
  Mask<(C + 7) / 8> mm;
  mm.w[0] = mk;
  typename T::A acc[1] = {typename T::A(0)};
  block_products<1, C, T>(mm, col, vblk, x, acc);
  return acc[0];
}

template <int C, class T, bool ACCUM>
__device__ __forceinline__ void rows_s_body(int64_t bid, int64_t n, int64_t I, int32_t long_blocks,
                                            int64_t long_values, const int32_t* __restrict__ brp,
                                            const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                            const typename T::V* __restrict__ val,
                                            const int64_t* __restrict__ valptr, const typename T::X* __restrict__ x,
                                            typename T::X* __restrict__ y) {
  constexpr int MB = (C + 7) / 8;
  constexpr unsigned kAll = 0xffffffffu;
  constexpr int kTrip = 2 * kWarp;  // blocks per trip, two per lane
  using A = typename T::A;
  const int lane = threadIdx.x & 31;
  const int64_t r0 = ((bid * blockDim.x + threadIdx.x) >> 5) * kWarp;
  if (r0 >= I) return;  // whole warp
  const int64_t row = r0 + lane;
  const bool have = row < I;
  int32_t b0 = 0, b1 = 0;
  int64_t v0 = 0;
  bool lng = false;
  if (have) {
    b0 = __ldg(brp + row);
    b1 = __ldg(brp + row + 1);
    v0 = __ldg(valptr + row);
    lng = b1 - b0 > long_blocks || __ldg(valptr + row + 1) - v0 > long_values;
  }
  if (__any_sync(kAll, lng)) {  // a long row among the 32: one lane per row for the others
    if (have && !lng) {
      const A acc = row_sum<1, C, T, 2, 1>(0, b0, b1, val + v0, bcol, bmask, x);
      if (row < n) y[row] = ACCUM ? y[row] + acc : acc;
    }
    return;
  }
  const int last = (int)(I - 1 - r0 < 31 ? I - 1 - r0 : 31);
  const int32_t B0 = __shfl_sync(kAll, b0, 0);
  const int32_t B1 = __shfl_sync(kAll, b1, last);
  int64_t vcur = __shfl_sync(kAll, v0, 0);  // first value of the current trip
  const bool nonempty = have && b1 > b0;
  A ysum = A(0);   // row `row`'s sum (empty rows keep 0)
  A carry = A(0);  // the run-on row's sum over the trips before
  // trips start on an even block (pair reads); a block before B0 counts nothing
  const int32_t S0 = B0 & ~1;
  uint32_t nma = 0, nmb = 0;
  int32_t nca = 0, ncb = 0;
  if (S0 + 2 * lane < B1) load_pair<MB>(bmask, bcol, S0 + 2 * lane, nma, nmb, nca, ncb);
  for (int32_t t0 = S0; t0 < B1; t0 += kTrip) {
    const int32_t ba = t0 + 2 * lane;
    const bool ina = ba >= B0 && ba < B1, inb = ba + 1 < B1;
    const uint32_t ma = ina ? nma : 0u, mb = inb ? nmb : 0u;
    const int32_t ca = nca, cb = ncb;
    if (ba + kTrip < B1) {  // the next trip's masks and columns, one trip ahead
      load_pair<MB>(bmask, bcol, ba + kTrip, nma, nmb, nca, ncb);
    }
    const int cnta = __popc(ma), cnt = cnta + __popc(mb);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
      const int t = __shfl_up_sync(kAll, incl, d);
      if (lane >= d) incl += t;
    }
    const typename T::V* __restrict__ vlane = val + vcur + (incl - cnt);
    const A pa = ina ? block_product1<C, T>(ma, ca, vlane, x) : A(0);
    const A pb = inb ? block_product1<C, T>(mb, cb, vlane + cnta, x) : A(0);
    vcur += __shfl_sync(kAll, incl, kWarp - 1);
    // rows starting in this trip, one bit per block position (two words)
    const int32_t rs = b0 - t0;
    const bool starts = nonempty && rs >= 0 && rs < kTrip;
    const uint32_t hlo = __reduce_or_sync(kAll, starts && rs < kWarp ? (1u << rs) : 0u);
    const uint32_t hhi = __reduce_or_sync(kAll, starts && rs >= kWarp ? (1u << (rs - kWarp)) : 0u);
    const uint32_t hw = lane < 16 ? hlo : hhi;
    const int hs = 2 * (lane & 15);
    const bool fa = (hw >> hs) & 1u, fb = (hw >> (hs + 1)) & 1u;
    // lane flags: a row starts at one of the lane's blocks; the lane's value
    // is what it adds to the run open after its blocks
    const uint32_t flags = __ballot_sync(kAll, fa || fb);
    const uint32_t upto = flags & (kAll >> (31 - lane));
    const int first = upto ? 31 - __clz(upto) : 0;
    A s = fb ? pb : pa + pb;
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
      const A t = __shfl_up_sync(kAll, s, d);
      if (lane - d >= first) s += t;
    }
    // the run through block a: the lane before's run plus pa, or pa alone
    const A prev = __shfl_up_sync(kAll, s, 1);
    const A ea = (fa || lane == 0) ? pa : prev + pa;
    // lane q takes row q's sum when the row's last block is in this trip
    const int32_t re = b1 - 1 - t0;
    const bool ends = nonempty && re >= 0 && re < kTrip;
    const int src = ends ? (re >> 1) : 0;
    const A got_s = __shfl_sync(kAll, s, src);
    const A got_a = __shfl_sync(kAll, ea, src);
    if (ends) {
      const A got = (re & 1) ? got_s : got_a;
      ysum = b0 < t0 ? carry + got : got;
    }
    const A tail = __shfl_sync(kAll, s, kWarp - 1);
    carry = (hlo | hhi) ? tail : carry + tail;
  }
  if (have && row < n) y[row] = ACCUM ? y[row] + ysum : ysum;
}

template <int C, class T, bool ACCUM, int MINB>
__global__ void __launch_bounds__(256, MINB) k_spmv_s(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                const uint8_t* __restrict__ bmask,
                                                const typename T::V* __restrict__ val,
                                                const int64_t* __restrict__ valptr,
                                                const typename T::X* __restrict__ x, typename T::X* __restrict__ y) {
  rows_s_body<C, T, ACCUM>(blockIdx.x, n, I, long_blocks, long_values, brp, bcol, bmask, val, valptr, x, y);
}

// the long intervals' segments (thread blocks [0, seg_ctas)) and the streaming
// warps in one grid
template <int C, class T, bool ACCUM, int MINB>
__global__ void __launch_bounds__(256, MINB) k_spmv_s_segs(int64_t seg_ctas, int64_t n, int64_t I,
                                                           int32_t long_blocks,
                                                     int64_t long_values, const int32_t* __restrict__ brp,
                                                     const int32_t* __restrict__ bcol,
                                                     const uint8_t* __restrict__ bmask,
                                                     const typename T::V* __restrict__ val,
                                                     const int64_t* __restrict__ valptr,
                                                     const typename T::X* __restrict__ x, typename T::X* __restrict__ y,
                                                     int64_t nseg, const Segment* __restrict__ segs,
                                                     typename T::A* __restrict__ partials) {
  if ((int64_t)blockIdx.x < seg_ctas)
    segments_body<1, C, T, 4, 1>(blockIdx.x, nseg, segs, bcol, bmask, val, x, partials);
  else
    rows_s_body<C, T, ACCUM>((int64_t)blockIdx.x - seg_ctas, n, I, long_blocks, long_values, brp, bcol, bmask, val,
                             valptr, x, y);
}

template <int C, class T, int MINB>
cudaError_t launch_stream_c(const spc5_matrix* h, const void* xv, void* yv, bool acc, void* partials,
                            cudaStream_t s) {
  using X = typename T::X;
  using A = typename T::A;
  const X* x = static_cast<const X*>(xv);
  X* y = static_cast<X*>(yv);
  const typename T::V* val = static_cast<const typename T::V*>(h->values);
  A* part = static_cast<A*>(partials);
  const int threads = kSpmvThreads;
  const int64_t seg_ctas = (h->nseg * kWarp + threads - 1) / threads;
  const int64_t warps = (h->I + kWarp - 1) / kWarp;
  const unsigned grid = (unsigned)((warps * kWarp + threads - 1) / threads);
  if (fused_launch(h)) {
    auto kern = acc ? k_spmv_s_segs<C, T, true, MINB> : k_spmv_s_segs<C, T, false, MINB>;
    kern<<<(unsigned)(seg_ctas + grid), threads, 0, s>>>(seg_ctas, h->n, h->I, h->long_blocks, h->long_values,
                                                         h->block_rowptr, h->block_colidx, h->block_masks, val,
                                                         h->valptr, x, y, h->nseg, h->segs, part);
  } else if (grid > 0) {
    auto kern = acc ? k_spmv_s<C, T, true, MINB> : k_spmv_s<C, T, false, MINB>;
    kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                  h->block_masks, val, h->valptr, x, y);
  }
  if (h->nseg > 0) {
    const unsigned g2 = (unsigned)((h->nlong + 255) / 256);
    if (acc)
      k_spmv_fixup<1, T, true><<<g2, 256, 0, s>>>(h->n, h->nlong, h->seg_first, h->segs, part, y);
    else
      k_spmv_fixup<1, T, false><<<g2, 256, 0, s>>>(h->n, h->nlong, h->seg_first, h->segs, part, y);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t dispatch_stream(const spc5_matrix* h, const void* x, void* y, bool acc, void* partials, cudaStream_t s) {
  if (h->r != 1) return cudaErrorInvalidValue;
  // c = 4: a register cap of 40 (six blocks of 256 threads per SM) costs no
  // spills there; the larger block products keep their registers
  switch (h->c) {
    case 4: return launch_stream_c<4, T, 6>(h, x, y, acc, partials, s);
    case 8: return launch_stream_c<8, T, 1>(h, x, y, acc, partials, s);
    case 16: return launch_stream_c<16, T, 1>(h, x, y, acc, partials, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace spc5
