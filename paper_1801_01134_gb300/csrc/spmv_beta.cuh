// y = A x over the beta(r,c) storage (Algorithm 1 of Bramas & Kus 2018).
//
// The paper's AVX-512 kernel expands popcount(mask) packed values into the
// set lanes of a vector (vexpandpd, section "Vectorization"), multiplies by an
// unaligned c-wide load of x and advances its value index by the popcount
// (Code 1). On the GPU the expand becomes arithmetic: the value of bit p of a
// block sits at (block's first value) + popc(mask & ((1 << p) - 1)).
//
// Work mapping (one warp = 32 lanes):
//   * short intervals (<= long_blocks blocks): lane = one row of one
//     interval; a warp owns 32/r consecutive intervals. Each lane walks the
//     blocks of its interval and consumes only its own row's bits, so every
//     multiply-add of a warp instruction belongs to a different row and no
//     cross-lane reduction is needed. The loop is flattened over the row's
//     nonzeros (block changes happen inside), so a warp issues max(row length)
//     fused multiply-adds. On GB300 a float64 FMA costs the same warp
//     instruction slot however many lanes are active, which makes this
//     packing the bound for float64.
//   * long intervals: split into segments of seg_blocks blocks (built at
//     conversion); a warp per segment, lane = (block slot, row), 32/r blocks
//     per step; per-step value offsets come from a shuffle scan of the block
//     popcounts. Each segment leaves r partial sums; a fix-up kernel adds the
//     segments of one interval in order (deterministic) and writes y.
#pragma once

#include "internal.cuh"

namespace spc5 {

// ---------------------------------------------------------------- masks
// A block mask of MB bytes held as 32-bit words; bit (i*C + k) = row i, col k.
template <int MB>
struct Mask {
  static constexpr int W = MB <= 4 ? 1 : MB / 4;
  uint32_t w[W];
};

template <int MB>
__device__ __forceinline__ Mask<MB> load_mask(const uint8_t* __restrict__ masks, int64_t b) {
  Mask<MB> m;
  if constexpr (MB == 1) {
    m.w[0] = __ldg(masks + b);
  } else if constexpr (MB == 2) {
    m.w[0] = __ldg(reinterpret_cast<const uint16_t*>(masks) + b);
  } else if constexpr (MB == 4) {
    m.w[0] = __ldg(reinterpret_cast<const uint32_t*>(masks) + b);
  } else if constexpr (MB == 8) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(masks) + b);
    m.w[0] = v.x;
    m.w[1] = v.y;
  } else {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(masks) + b);
    m.w[0] = v.x;
    m.w[1] = v.y;
    m.w[2] = v.z;
    m.w[3] = v.w;
  }
  return m;
}

template <int MB>
__device__ __forceinline__ Mask<MB> zero_mask() {
  Mask<MB> m;
#pragma unroll
  for (int q = 0; q < Mask<MB>::W; ++q) m.w[q] = 0u;
  return m;
}

// the C bits of block row i (C divides 32, so a row never straddles words)
template <int C, int MB>
__device__ __forceinline__ uint32_t row_bits(const Mask<MB>& m, int i) {
  const int p = i * C;
  const uint32_t full = C == 32 ? 0xffffffffu : ((1u << C) - 1u);
  return (m.w[p >> 5] >> (p & 31)) & full;
}

// number of set bits below bit position p = i * C
template <int C, int MB>
__device__ __forceinline__ int popc_below(const Mask<MB>& m, int i) {
  const int p = i * C;
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < Mask<MB>::W; ++q) {
    if (q < (p >> 5)) cnt += __popc(m.w[q]);
  }
  const int sh = p & 31;
  if (sh) cnt += __popc(m.w[p >> 5] & ((1u << sh) - 1u));
  return cnt;
}

template <int MB>
__device__ __forceinline__ int popc_all(const Mask<MB>& m) {
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < Mask<MB>::W; ++q) cnt += __popc(m.w[q]);
  return cnt;
}

// ---------------------------------------------------------------- types
struct F64 {
  using V = double;
  using X = double;
  using A = double;
  static __device__ __forceinline__ A val(const V* p, int64_t i) { return __ldg(p + i); }
  static __device__ __forceinline__ A xv(const X* p, int64_t i) { return __ldg(p + i); }
};
struct F32 {
  using V = float;
  using X = float;
  using A = float;
  static __device__ __forceinline__ A val(const V* p, int64_t i) { return __ldg(p + i); }
  static __device__ __forceinline__ A xv(const X* p, int64_t i) { return __ldg(p + i); }
};
struct BF16 {
  using V = uint16_t;  // bfloat16 bit pattern
  using X = float;
  using A = float;
  static __device__ __forceinline__ A val(const V* p, int64_t i) {
    return __uint_as_float(((uint32_t)__ldg(p + i)) << 16);
  }
  static __device__ __forceinline__ A xv(const X* p, int64_t i) { return __ldg(p + i); }
};

// value read from shared memory (generic load)
template <class T>
__device__ __forceinline__ typename T::A sval(const typename T::V* p, int i) {
  if constexpr (sizeof(typename T::V) == 2)
    return __uint_as_float(((uint32_t)p[i]) << 16);
  else
    return p[i];
}

template <class T>
__device__ __forceinline__ typename T::A fmadd(typename T::A a, typename T::A b, typename T::A c) {
  return fma(a, b, c);
}

// ------------------------------------------------------- short intervals
template <int R, int C, class T, bool ACCUM>
__global__ void __launch_bounds__(256) k_spmv_rows(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                   const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                   const uint8_t* __restrict__ bmask, const typename T::V* __restrict__ val,
                                                   const int64_t* __restrict__ valptr, const typename T::X* __restrict__ x,
                                                   typename T::X* __restrict__ y) {
  constexpr int MB = (R * C + 7) / 8;
  constexpr int S = kWarp / R;  // intervals per warp
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t it = warp * S + lane / R;
  const int i = lane % R;
  if (it >= I) return;
  int32_t b = __ldg(brp + it);
  const int32_t bend = __ldg(brp + it + 1);
  int64_t vbase = __ldg(valptr + it);
  if (bend - b > long_blocks || __ldg(valptr + it + 1) - vbase > long_values) return;  // the segment path's
  typename T::A acc = 0;
  uint32_t bits = 0;
  int32_t col0 = 0;
  int64_t vo = 0;
  for (;;) {
    while (bits == 0 && b < bend) {
      const Mask<MB> mk = load_mask<MB>(bmask, b);
      col0 = __ldg(bcol + b);
      bits = row_bits<C>(mk, i);
      vo = vbase + popc_below<C>(mk, i);
      vbase += popc_all(mk);
      ++b;
    }
    if (bits == 0) break;
    const int k = __ffs(bits) - 1;
    bits &= bits - 1;
    acc = fmadd<T>(T::val(val, vo), T::xv(x, (int64_t)col0 + k), acc);
    ++vo;
  }
  const int64_t row = it * R + i;
  if (row < n) {
    if (ACCUM)
      y[row] = y[row] + acc;
    else
      y[row] = acc;
  }
}

// Sum of one row of a short interval (lane-per-row form): walks blocks
// [b, bend) of the interval whose values start at vrow, consuming the bits of
// block row i, U nonzeros decoded per trip (see k_spmv_rows_u).
template <int R, int C, class T, int U>
__device__ __forceinline__ typename T::A row_sum_u(int i, int32_t b, int32_t bend,
                                                   const typename T::V* __restrict__ vrow,
                                                   const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                   const typename T::X* __restrict__ x) {
  constexpr int MB = (R * C + 7) / 8;
  using A = typename T::A;
  int32_t vbase = 0;  // offset of block b's first value inside the interval
  uint32_t bits = 0;
  int32_t col0 = 0, vo = 0;
  Mask<MB> nmk = b < bend ? load_mask<MB>(bmask, b) : zero_mask<MB>();
  int32_t ncol = b < bend ? __ldg(bcol + b) : 0;
  A acc = 0;
  for (;;) {
    int32_t vi[U], xi[U];
    bool h[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      while (bits == 0 && b < bend) {
        const Mask<MB> mk = nmk;
        col0 = ncol;
        if (b + 1 < bend) {
          nmk = load_mask<MB>(bmask, b + 1);
          ncol = __ldg(bcol + b + 1);
        }
        bits = row_bits<C>(mk, i);
        vo = vbase + popc_below<C>(mk, i);
        vbase += popc_all(mk);
        ++b;
      }
      h[u] = bits != 0;
      const int k = __ffs(bits) - 1;
      bits &= bits - 1;
      vi[u] = vo;
      vo += h[u] ? 1 : 0;
      xi[u] = col0 + k;
    }
    if (!h[0]) break;
    A v[U], xx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v[u] = h[u] ? T::val(vrow, vi[u]) : A(0);
      xx[u] = h[u] ? T::xv(x, xi[u]) : A(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (h[u]) acc = fmadd<T>(v[u], xx[u], acc);
  }
  return acc;
}

// ------------------------------------------- short intervals, unrolled form
// Same mapping, arithmetic and summation order as k_spmv_rows; each loop trip
// decodes the lane's next U nonzeros first (the mask and column index of the
// following block are already loaded one block ahead), then issues their U
// value loads and U x loads together, then the U multiply-adds (predicated
// off past the end of the row). U independent loads per lane are in flight
// instead of one.
//
// With ORDER, lane slot q of the warp takes interval order[q] instead of q
// (the sorted work order built at conversion; long intervals are not in it).
template <int R, int C, class T, bool ACCUM, int U, bool ORDER>
__global__ void __launch_bounds__(256) k_spmv_rows_u(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                     const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                     const uint8_t* __restrict__ bmask,
                                                     const typename T::V* __restrict__ val,
                                                     const int64_t* __restrict__ valptr,
                                                     const typename T::X* __restrict__ x,
                                                     typename T::X* __restrict__ y,
                                                     const int32_t* __restrict__ order, int64_t norder) {
  constexpr int S = kWarp / R;
  using A = typename T::A;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t it = warp * S + lane / R;
  if (ORDER) {
    if (it >= norder) return;
    it = __ldg(order + it);
  }
  const int i = lane % R;
  if (it >= I) return;
  int32_t b = __ldg(brp + it);
  const int32_t bend = __ldg(brp + it + 1);
  const int64_t vbase0 = __ldg(valptr + it);
  if (bend - b > long_blocks || __ldg(valptr + it + 1) - vbase0 > long_values) return;  // the segment path's
  const typename T::A acc = row_sum_u<R, C, T, U>(i, b, bend, val + vbase0, bcol, bmask, x);
  const int64_t row = it * R + i;
  if (row < n) {
    if (ACCUM)
      y[row] = y[row] + acc;
    else
      y[row] = acc;
  }
}

// -------------------------------------------------------- long intervals
template <int R, int C, class T>
__global__ void __launch_bounds__(256) k_spmv_segments(int64_t nseg, const Segment* __restrict__ segs,
                                                       const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                       const typename T::V* __restrict__ val,
                                                       const typename T::X* __restrict__ x,
                                                       typename T::A* __restrict__ partials) {
  constexpr int MB = (R * C + 7) / 8;
  constexpr int S = kWarp / R;  // block slots per step
  const int lane = threadIdx.x & 31;
  const int64_t seg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (seg >= nseg) return;  // whole warp leaves together
  const int slot = lane / R, i = lane % R;
  const Segment sg = segs[seg];
  int64_t vbase = sg.v_begin;
  typename T::A acc = 0;
  for (int32_t b0 = sg.b_begin; b0 < sg.b_end; b0 += S) {
    const int32_t b = b0 + slot;
    const bool valid = b < sg.b_end;
    const Mask<MB> mk = valid ? load_mask<MB>(bmask, b) : zero_mask<MB>();
    const int cnt = popc_all(mk);
    // inclusive scan of the block popcounts over the slots (stride R lanes)
    int incl = cnt;
#pragma unroll
    for (int d = R; d < kWarp; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
    int64_t vo = vbase + (incl - cnt) + popc_below<C>(mk, i);
    uint32_t bits = valid ? row_bits<C>(mk, i) : 0u;
    const int32_t col0 = valid ? __ldg(bcol + b) : 0;
    while (bits) {
      const int k = __ffs(bits) - 1;
      bits &= bits - 1;
      acc = fmadd<T>(T::val(val, vo), T::xv(x, (int64_t)col0 + k), acc);
      ++vo;
    }
    vbase += total;
  }
  // sum over the slots of each row (lanes i, i + R, i + 2R, ...)
#pragma unroll
  for (int d = kWarp / 2; d >= R; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane < R) partials[seg * R + lane] = acc;
}

// first segment of each long interval adds its interval's partials in order
template <int R, class T, bool ACCUM>
__global__ void k_spmv_fixup(int64_t n, int64_t nseg, const Segment* __restrict__ segs,
                             const typename T::A* __restrict__ partials, typename T::X* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t seg = t / R;
  const int i = (int)(t % R);
  if (seg >= nseg) return;
  const int32_t it = segs[seg].interval;
  if (seg > 0 && segs[seg - 1].interval == it) return;
  typename T::A s = 0;
  for (int64_t k = seg; k < nseg && segs[k].interval == it; ++k) s += partials[k * R + i];
  const int64_t row = (int64_t)it * R + i;
  if (row < n) {
    if (ACCUM)
      y[row] = y[row] + s;
    else
      y[row] = s;
  }
}

// --------------------------------------------------------------- launch
template <int R, int C, class T>
cudaError_t launch_beta(const spc5_matrix* h, const void* xv, void* yv, bool acc, cudaStream_t s) {
  using V = typename T::V;
  using X = typename T::X;
  using A = typename T::A;
  const X* x = static_cast<const X*>(xv);
  X* y = static_cast<X*>(yv);
  const V* val = static_cast<const V*>(h->values);
  constexpr int S = kWarp / R;
  const int threads = 256;
  if (h->I > 0) {
    const int64_t warps = (h->I + S - 1) / S;
    if (h->variant == 1) {
      const unsigned grid = (unsigned)((warps * kWarp + threads - 1) / threads);
      if (acc)
        k_spmv_rows<R, C, T, true><<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr,
                                                            h->block_colidx, h->block_masks, val, h->valptr, x, y);
      else
        k_spmv_rows<R, C, T, false><<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr,
                                                             h->block_colidx, h->block_masks, val, h->valptr, x, y);
    } else if ((h->variant == 9 || h->variant == 10) && h->norder > 0) {
      // sorted work order
      const int64_t owarps = (h->norder + S - 1) / S;
      const unsigned grid = (unsigned)((owarps * kWarp + threads - 1) / threads);
      auto go = [&](auto kern) {
        kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                      h->block_masks, val, h->valptr, x, y, h->order, h->norder);
      };
      if (h->variant == 10) {
        if (acc) go(k_spmv_rows_u<R, C, T, true, 4, true>); else go(k_spmv_rows_u<R, C, T, false, 4, true>);
      } else {
        if (acc) go(k_spmv_rows_u<R, C, T, true, 2, true>); else go(k_spmv_rows_u<R, C, T, false, 2, true>);
      }
    } else {
      // natural order; variant 3 unrolls by 4, the default (0 or 5) by 2
      const unsigned grid = (unsigned)((warps * kWarp + threads - 1) / threads);
      auto go = [&](auto kern) {
        kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                      h->block_masks, val, h->valptr, x, y, nullptr, (int64_t)0);
      };
      if (h->variant == 3) {
        if (acc) go(k_spmv_rows_u<R, C, T, true, 4, false>); else go(k_spmv_rows_u<R, C, T, false, 4, false>);
      } else {
        if (acc) go(k_spmv_rows_u<R, C, T, true, 2, false>); else go(k_spmv_rows_u<R, C, T, false, 2, false>);
      }
    }
  }
  if (h->nseg > 0) {
    A* part = static_cast<A*>(h->partials);
    const unsigned grid = (unsigned)((h->nseg * kWarp + threads - 1) / threads);
    k_spmv_segments<R, C, T><<<grid, threads, 0, s>>>(h->nseg, h->segs, h->block_colidx, h->block_masks, val, x, part);
    const unsigned g2 = (unsigned)((h->nseg * R + 255) / 256);
    if (acc)
      k_spmv_fixup<R, T, true><<<g2, 256, 0, s>>>(h->n, h->nseg, h->segs, part, y);
    else
      k_spmv_fixup<R, T, false><<<g2, 256, 0, s>>>(h->n, h->nseg, h->segs, part, y);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t dispatch_beta(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s) {
#define SPC5_CASE(RR, CC) \
  if (h->r == RR && h->c == CC) return launch_beta<RR, CC, T>(h, x, y, acc, s);
  SPC5_CASE(1, 4) SPC5_CASE(1, 8) SPC5_CASE(1, 16)
  SPC5_CASE(2, 4) SPC5_CASE(2, 8) SPC5_CASE(2, 16)
  SPC5_CASE(4, 4) SPC5_CASE(4, 8) SPC5_CASE(4, 16)
  SPC5_CASE(8, 4) SPC5_CASE(8, 8) SPC5_CASE(8, 16)
#undef SPC5_CASE
  return cudaErrorInvalidValue;
}

}  // namespace spc5
