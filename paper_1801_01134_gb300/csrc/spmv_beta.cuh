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
//     conversion); a warp per segment, the segment cut into 32/r contiguous
//     runs of blocks, lane = (run, row); run value offsets come from a
//     shuffle scan of the runs' popcounts. Each segment leaves r partial
//     sums; a fix-up kernel adds the segments of one interval in a fixed
//     order (deterministic) and writes y.
//   * mask windows (variants 12-15 and the segments): the masks of 8/mb
//     consecutive blocks are read as one 8-byte word, so walking low-fill
//     blocks does not wait on memory once per block.
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

// The 8 mask bytes that start at block b: blocks b .. b + 8/MB - 1 (MB <= 8),
// bit j*8*MB + q of the result = bit q of block b + j. Reads the two aligned
// 8-byte words around them; mask arrays carry 16 bytes of padding past their
// end, so the second word is always inside the allocation.
template <int MB>
__device__ __forceinline__ uint64_t load_window(const uint8_t* __restrict__ masks, int32_t b) {
  static_assert(MB <= 8, "a window holds at most 8 mask bytes");
  const uint64_t o = (uint64_t)(uint32_t)b * MB;
  const unsigned long long* p = reinterpret_cast<const unsigned long long*>(masks) + (o >> 3);
  if constexpr (MB == 8) {
    return __ldg(p);
  } else {
    const unsigned sh = (unsigned)(o & 7) * 8;
    const uint64_t lo = __ldg(p), hi = __ldg(p + 1);
    return sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
  }
}

// mask of block w of a window
template <int MB>
__device__ __forceinline__ Mask<MB> window_mask(uint64_t win, int w) {
  Mask<MB> m;
  if constexpr (MB == 8) {
    m.w[0] = (uint32_t)win;
    m.w[1] = (uint32_t)(win >> 32);
  } else if constexpr (MB == 4) {
    m.w[0] = (uint32_t)(win >> (32 * w));
  } else {
    m.w[0] = (uint32_t)(win >> (8 * MB * w)) & ((1u << (8 * MB)) - 1u);
  }
  return m;
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

// Same sum as row_sum_u (same nonzeros, same order), decoded from mask
// windows: the masks of 8/MB consecutive blocks arrive in one 8-byte read and
// the next window is requested while the current one is consumed, so stepping
// from block to block costs no global-memory round trip. The column index of
// each decoded nonzero is loaded beside its value (one load per nonzero; the
// indices of neighbouring blocks share sectors). For low fill (about one
// nonzero per block, as in power-law graphs) a trip of U nonzeros then waits
// for two memory latencies instead of one per block.
template <int R, int C, class T, int U>
__device__ __forceinline__ typename T::A row_sum_w(int i, int32_t b, int32_t bend,
                                                   const typename T::V* __restrict__ vrow,
                                                   const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                   const typename T::X* __restrict__ x) {
  constexpr int MB = (R * C + 7) / 8;
  constexpr int K = 8 / MB;  // blocks per window
  using A = typename T::A;
  uint64_t cur = b < bend ? load_window<MB>(bmask, b) : 0ull;
  uint64_t nxt = b + K < bend ? load_window<MB>(bmask, b + K) : 0ull;
  int32_t wb = b;  // first block of the current window
  int w = 0;       // blocks of the current window entered so far
  int32_t vbase = 0, vo = 0, blk = 0;
  uint32_t bits = 0;
  A acc = 0;
  for (;;) {
    int32_t vi[U], bi[U], ki[U];
    bool h[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      while (bits == 0 && wb + w < bend) {
        if (w == K) {
          cur = nxt;
          wb += K;
          w = 0;
          nxt = wb + K < bend ? load_window<MB>(bmask, wb + K) : 0ull;
        }
        const Mask<MB> mk = window_mask<MB>(cur, w);
        bits = row_bits<C>(mk, i);
        vo = vbase + popc_below<C>(mk, i);
        vbase += popc_all(mk);
        blk = wb + w;
        ++w;
      }
      h[u] = bits != 0;
      ki[u] = __ffs(bits) - 1;
      bits &= bits - 1;
      vi[u] = vo;
      vo += h[u] ? 1 : 0;
      bi[u] = blk;
    }
    if (!h[0]) break;
    A v[U], xx[U];
    int32_t cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v[u] = h[u] ? T::val(vrow, vi[u]) : A(0);
      cc[u] = h[u] ? __ldg(bcol + bi[u]) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xx[u] = h[u] ? T::xv(x, (int64_t)cc[u] + ki[u]) : A(0);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (h[u]) acc = fmadd<T>(v[u], xx[u], acc);
  }
  return acc;
}

// Same sum again, block by block with the C bit positions of the block row
// unrolled at compile time (the column of position k is col0 + k, an
// immediate offset from the block's x window). No per-nonzero bit search or
// loop trip: fewer instructions per stored value when blocks are well filled
// and multiply-adds are cheap (float32 / bfloat16), but every position costs
// a predicated slot, so float64 - where a multiply-add occupies the float64
// pipe whatever the active lanes - usually prefers the flattened forms.
template <int R, int C, class T>
__device__ __forceinline__ typename T::A row_sum_e(int i, int32_t b, int32_t bend,
                                                   const typename T::V* __restrict__ vrow,
                                                   const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                   const typename T::X* __restrict__ x) {
  constexpr int MB = (R * C + 7) / 8;
  using A = typename T::A;
  A acc = 0;
  int32_t vbase = 0;
  Mask<MB> nmk = b < bend ? load_mask<MB>(bmask, b) : zero_mask<MB>();
  int32_t ncol = b < bend ? __ldg(bcol + b) : 0;
  for (; b < bend; ++b) {
    const Mask<MB> mk = nmk;
    const int32_t col0 = ncol;
    if (b + 1 < bend) {  // next block's mask and column one block ahead
      nmk = load_mask<MB>(bmask, b + 1);
      ncol = __ldg(bcol + b + 1);
    }
    const uint32_t rbits = row_bits<C>(mk, i);
    int32_t vo = vbase + popc_below<C>(mk, i);
    vbase += popc_all(mk);
    const typename T::X* __restrict__ xw = x + col0;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (rbits & (1u << k)) {
        acc = fmadd<T>(T::val(vrow, vo), T::xv(xw, k), acc);
        ++vo;
      }
    }
  }
  return acc;
}

// row_sum_e taking two blocks per trip (c <= 8): the value and x loads of
// both blocks are issued before the first multiply-add, halving the memory
// round trips per row; the products are still added block by block, bits
// ascending.
template <int R, int C, class T>
__device__ __forceinline__ typename T::A row_sum_e2(int i, int32_t b, int32_t bend,
                                                    const typename T::V* __restrict__ vrow,
                                                    const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                    const typename T::X* __restrict__ x) {
  constexpr int MB = (R * C + 7) / 8;
  using A = typename T::A;
  A acc = 0;
  int32_t vbase = 0;
  Mask<MB> m0 = b < bend ? load_mask<MB>(bmask, b) : zero_mask<MB>();
  Mask<MB> m1 = b + 1 < bend ? load_mask<MB>(bmask, b + 1) : zero_mask<MB>();
  int32_t c0 = b < bend ? __ldg(bcol + b) : 0;
  int32_t c1 = b + 1 < bend ? __ldg(bcol + b + 1) : 0;
  for (; b < bend; b += 2) {
    const Mask<MB> mk0 = m0, mk1 = m1;
    const int32_t col0 = c0, col1 = c1;
    const bool two = b + 1 < bend;
    if (b + 2 < bend) {  // the next pair's masks and columns one trip ahead
      m0 = load_mask<MB>(bmask, b + 2);
      c0 = __ldg(bcol + b + 2);
    }
    if (b + 3 < bend) {
      m1 = load_mask<MB>(bmask, b + 3);
      c1 = __ldg(bcol + b + 3);
    }
    const uint32_t rb0 = row_bits<C>(mk0, i);
    const uint32_t rb1 = two ? row_bits<C>(mk1, i) : 0u;
    int32_t vo0 = vbase + popc_below<C>(mk0, i);
    vbase += popc_all(mk0);
    int32_t vo1 = vbase + popc_below<C>(mk1, i);
    vbase += two ? popc_all(mk1) : 0;
    const typename T::X* __restrict__ xw0 = x + col0;
    const typename T::X* __restrict__ xw1 = x + col1;
    A v0[C], a0[C], v1[C], a1[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (rb0 & (1u << k)) {
        v0[k] = T::val(vrow, vo0);
        a0[k] = T::xv(xw0, k);
        ++vo0;
      }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (rb1 & (1u << k)) {
        v1[k] = T::val(vrow, vo1);
        a1[k] = T::xv(xw1, k);
        ++vo1;
      }
    }
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (rb0 & (1u << k)) acc = fmadd<T>(v0[k], a0[k], acc);
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (rb1 & (1u << k)) acc = fmadd<T>(v1[k], a1[k], acc);
  }
  return acc;
}

// row_sum_w where a window fits the shape's masks (up to 64 mask bits per
// block), row_sum_u otherwise
// DEC selects the decode: 0 row_sum_u, 1 row_sum_w (row_sum_u where a window
// cannot hold a block's masks, above 64 mask bits), 2 row_sum_e, 3 row_sum_e2
// (row_sum_e for c = 16).
template <int R, int C, class T, int U, int DEC>
__device__ __forceinline__ typename T::A row_sum(int i, int32_t b, int32_t bend, const typename T::V* __restrict__ vrow,
                                                 const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                 const typename T::X* __restrict__ x) {
  if constexpr (DEC == 3 && C <= 8)
    return row_sum_e2<R, C, T>(i, b, bend, vrow, bcol, bmask, x);
  else if constexpr (DEC == 2 || DEC == 3)
    return row_sum_e<R, C, T>(i, b, bend, vrow, bcol, bmask, x);
  else if constexpr (DEC == 1 && R * C <= 64)
    return row_sum_w<R, C, T, U>(i, b, bend, vrow, bcol, bmask, x);
  else
    return row_sum_u<R, C, T, U>(i, b, bend, vrow, bcol, bmask, x);
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
// DEC picks the row decode (see row_sum).
template <int R, int C, class T, bool ACCUM, int U, bool ORDER, int DEC>
__device__ __forceinline__ void rows_u_body(int64_t bid, int64_t n, int64_t I, int32_t long_blocks,
                                            int64_t long_values, const int32_t* __restrict__ brp,
                                            const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                            const typename T::V* __restrict__ val,
                                            const int64_t* __restrict__ valptr, const typename T::X* __restrict__ x,
                                            typename T::X* __restrict__ y, const int32_t* __restrict__ order,
                                            int64_t norder) {
  constexpr int S = kWarp / R;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (bid * blockDim.x + threadIdx.x) >> 5;
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
  const typename T::A acc = row_sum<R, C, T, U, DEC>(i, b, bend, val + vbase0, bcol, bmask, x);
  const int64_t row = it * R + i;
  if (row < n) {
    if (ACCUM)
      y[row] = y[row] + acc;
    else
      y[row] = acc;
  }
}

template <int R, int C, class T, bool ACCUM, int U, bool ORDER, int DEC>
__global__ void __launch_bounds__(256) k_spmv_rows_u(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                     const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                     const uint8_t* __restrict__ bmask,
                                                     const typename T::V* __restrict__ val,
                                                     const int64_t* __restrict__ valptr,
                                                     const typename T::X* __restrict__ x,
                                                     typename T::X* __restrict__ y,
                                                     const int32_t* __restrict__ order, int64_t norder) {
  rows_u_body<R, C, T, ACCUM, U, ORDER, DEC>(blockIdx.x, n, I, long_blocks, long_values, brp, bcol, bmask, val, valptr,
                                             x, y, order, norder);
}

// ---------------------------------------- two lanes per row (beta(1,c))
// Variant 22, r = 1: the two lanes of a pair share a short row and lane g
// takes the row's stored values of rank g, g + 2, ... (rank = position among
// the row's values). Its values are then every other one, so the pair reads
// them as one contiguous stretch and each lane makes half the row's
// multiply-adds (within one of its partner's), as in a two-lane CSR kernel,
// while the column indices are still read once per block. The bits of a mask
// with even (odd) rank inside the block are those where the inclusive prefix
// parity of the mask is 1 (0). (Measured on GB300: float64 FEM beta(1,8)
// 534 -> 640 GFLOP/s against the one-lane flattened decode, uniform
// 286 -> 309; four lanes per row, with a two-plane prefix count, was slower
// on every test matrix, and 1 or 4 values per trip slower than 2.)
template <int G, int NB>
__device__ __forceinline__ uint32_t rank_class_bits(uint32_t m, int cls) {
  static_assert(G == 2, "two lanes per row");
  // inclusive prefix parity of the NB-bit mask
  uint32_t p = m;
#pragma unroll
  for (int s = 1; s < NB; s <<= 1) p ^= p << s;
  // a set bit of rank j has inclusive count j + 1
  return m & (cls == 0 ? p : ~p);
}

// With ORDER, row slot q of the warp takes row order[q] (the sorted work
// order, short rows only) instead of row q. With SGL (variant 33), a row whose
// single-value class bit is set (Algorithm 2's test: every block holds one
// value, at its first column) skips the masks: value j belongs to block
// b0 + j, so lane g reads blocks g, g + 2, ... and their values like a
// two-lane CSR kernel - the same values in the same order as the parity path.
template <int C, class T, bool ACCUM, int G, int U, bool ORDER = false, bool SGL = false>
__device__ __forceinline__ void rows_g_body(int64_t bid, int64_t n, int64_t I, int32_t long_blocks,
                                            int64_t long_values, const int32_t* __restrict__ brp,
                                            const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                            const typename T::V* __restrict__ val,
                                            const int64_t* __restrict__ valptr, const typename T::X* __restrict__ x,
                                            typename T::X* __restrict__ y, const int32_t* __restrict__ order = nullptr,
                                            int64_t norder = 0, const uint32_t* __restrict__ single = nullptr) {
  constexpr int MB = (C + 7) / 8;
  constexpr int S = kWarp / G;  // rows per warp
  using A = typename T::A;
  const int lane = threadIdx.x & 31;
  const int g = lane & (G - 1);
  const int64_t warp = (bid * blockDim.x + threadIdx.x) >> 5;
  const int64_t slots = ORDER ? norder : I;
  if (warp * S >= slots) return;  // whole warp
  const int64_t pos = warp * S + lane / G;
  bool have = pos < slots;
  const int64_t it = ORDER ? (have ? (int64_t)__ldg(order + pos) : 0) : pos;
  int32_t b = 0, bend = 0;
  int64_t vp = 0;
  if (have) {
    b = __ldg(brp + it);
    bend = __ldg(brp + it + 1);
    const int64_t v0 = __ldg(valptr + it);
    if (bend - b > long_blocks || __ldg(valptr + it + 1) - v0 > long_values) have = false;  // the segment path's
    vp = v0 + g;
  }
  if (!have) bend = b;  // no work, but the group still meets at the shuffle below
  A acc = 0;
  if constexpr (SGL) {
    if (have && ((__ldg(single + (it >> 5)) >> (it & 31)) & 1u)) {
      const typename T::V* __restrict__ vrow = val + (vp - g);
      const int32_t len = bend - b;
      int32_t j = g;
      for (; j + G * (U - 1) < len; j += G * U) {
        int32_t cc[U];
        A v[U], xx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          cc[u] = __ldg(bcol + b + j + G * u);
          v[u] = T::val(vrow, j + G * u);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xx[u] = T::xv(x, cc[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc = fmadd<T>(v[u], xx[u], acc);
      }
      for (; j < len; j += G) acc = fmadd<T>(T::val(vrow, j), T::xv(x, __ldg(bcol + b + j)), acc);
      bend = b;  // the parity walk below has nothing left
    }
  }
  uint32_t sel = 0, nm = b < bend ? load_mask<MB>(bmask, b).w[0] : 0u;
  int32_t col0 = 0, ncol = b < bend ? __ldg(bcol + b) : 0;
  int before = 0;  // values of the row in the blocks already entered
  for (;;) {
    int64_t vi[U];
    int32_t xi[U];
    bool h[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      while (sel == 0 && b < bend) {
        const uint32_t m = nm;
        col0 = ncol;
        if (b + 1 < bend) {
          nm = load_mask<MB>(bmask, b + 1).w[0];
          ncol = __ldg(bcol + b + 1);
        }
        sel = rank_class_bits<G, C>(m, (g - before) & (G - 1));
        before += __popc(m);
        ++b;
      }
      h[u] = sel != 0;
      const int k = __ffs(sel) - 1;
      sel &= sel - 1;
      vi[u] = vp;
      vp += h[u] ? G : 0;
      xi[u] = col0 + k;
    }
    if (!h[0]) break;
    A v[U], xx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v[u] = h[u] ? T::val(val, vi[u]) : A(0);
      xx[u] = h[u] ? T::xv(x, xi[u]) : A(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (h[u]) acc = fmadd<T>(v[u], xx[u], acc);
  }
#pragma unroll
  for (int d = G / 2; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d, G);
  if (have && g == 0 && it < n) {
    if (ACCUM)
      y[it] = y[it] + acc;
    else
      y[it] = acc;
  }
}

template <int C, class T, bool ACCUM, int G, int U, bool ORDER>
__global__ void __launch_bounds__(256) k_spmv_rows_g(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                     const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                     const uint8_t* __restrict__ bmask,
                                                     const typename T::V* __restrict__ val,
                                                     const int64_t* __restrict__ valptr,
                                                     const typename T::X* __restrict__ x,
                                                     typename T::X* __restrict__ y, const int32_t* __restrict__ order,
                                                     int64_t norder) {
  rows_g_body<C, T, ACCUM, G, U, ORDER>(blockIdx.x, n, I, long_blocks, long_values, brp, bcol, bmask, val, valptr, x,
                                        y, order, norder);
}

// variant 33: two lanes per row with Algorithm 2's test (natural order)
template <int C, class T, bool ACCUM, int U>
__global__ void __launch_bounds__(256) k_spmv_rows_g1(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                      const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                      const uint8_t* __restrict__ bmask,
                                                      const typename T::V* __restrict__ val,
                                                      const int64_t* __restrict__ valptr,
                                                      const typename T::X* __restrict__ x,
                                                      typename T::X* __restrict__ y,
                                                      const uint32_t* __restrict__ single) {
  rows_g_body<C, T, ACCUM, 2, U, false, true>(blockIdx.x, n, I, long_blocks, long_values, brp, bcol, bmask, val, valptr,
                                              x, y, nullptr, 0, single);
}

// ------------------------------------- Algorithm 2's test (beta(1,c))
// Variants 30 (sorted work order) and 31 (natural order), r = 1: the paper
// gives blocks holding a single value (mask 1) a scalar loop of their own, so
// that very sparse rows do not pay for the expand of a whole block. Here the
// test is made once per row at set-up (single_bits): in a row whose blocks all
// hold one value, value j belongs to block b0 + j and sits at its first
// column, so the lane reads the row like CSR - U column indices and U values
// per trip, no mask read, no popcount; other rows take the mask-window decode.
// Both paths add the row's products in storage order, so the results equal
// the other one-lane variants' bit for bit.
template <int C, class T, bool ACCUM, int U, bool ORDER>
__device__ __forceinline__ void rows_t_body(int64_t bid, int64_t n, int64_t I, int32_t long_blocks,
                                            int64_t long_values, const int32_t* __restrict__ brp,
                                            const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                            const typename T::V* __restrict__ val,
                                            const int64_t* __restrict__ valptr, const typename T::X* __restrict__ x,
                                            typename T::X* __restrict__ y, const int32_t* __restrict__ order,
                                            int64_t norder, const uint32_t* __restrict__ single) {
  using A = typename T::A;
  const int64_t slot = bid * blockDim.x + threadIdx.x;  // one lane per row
  if (slot >= (ORDER ? norder : I)) return;
  const int64_t it = ORDER ? (int64_t)__ldg(order + slot) : slot;
  const int32_t b0 = __ldg(brp + it), b1 = __ldg(brp + it + 1);
  const int64_t v0 = __ldg(valptr + it);
  if (b1 - b0 > long_blocks || __ldg(valptr + it + 1) - v0 > long_values) return;  // the segment path's
  const typename T::V* __restrict__ vrow = val + v0;
  A acc = 0;
  if ((__ldg(single + (it >> 5)) >> (it & 31)) & 1u) {
    const int32_t* __restrict__ crow = bcol + b0;
    const int32_t len = b1 - b0;
    int32_t j = 0;
    for (; j + U <= len; j += U) {
      int32_t cc[U];
      A v[U], xx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cc[u] = __ldg(crow + j + u);
        v[u] = T::val(vrow, j + u);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) xx[u] = T::xv(x, cc[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) acc = fmadd<T>(v[u], xx[u], acc);
    }
    for (; j < len; ++j) acc = fmadd<T>(T::val(vrow, j), T::xv(x, __ldg(crow + j)), acc);
  } else {
    acc = row_sum<1, C, T, 2, 1>(0, b0, b1, vrow, bcol, bmask, x);
  }
  if (it < n) {
    if (ACCUM)
      y[it] = y[it] + acc;
    else
      y[it] = acc;
  }
}

template <int C, class T, bool ACCUM, int U, bool ORDER>
__global__ void __launch_bounds__(256) k_spmv_rows_t(int64_t n, int64_t I, int32_t long_blocks, int64_t long_values,
                                                     const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                                                     const uint8_t* __restrict__ bmask,
                                                     const typename T::V* __restrict__ val,
                                                     const int64_t* __restrict__ valptr,
                                                     const typename T::X* __restrict__ x,
                                                     typename T::X* __restrict__ y, const int32_t* __restrict__ order,
                                                     int64_t norder, const uint32_t* __restrict__ single) {
  rows_t_body<C, T, ACCUM, U, ORDER>(blockIdx.x, n, I, long_blocks, long_values, brp, bcol, bmask, val, valptr, x, y,
                                     order, norder, single);
}

// -------------------------------------------------------- long intervals
// A warp per segment (at most seg_blocks blocks of one long interval). The
// segment's blocks are cut into S = 32/r contiguous runs, one per group of r
// lanes (lane = run slot, row i). A first pass counts the stored values of
// each run from its masks and a shuffle scan over the slots gives every run
// its first value; each lane then sums its row over its run with the
// short-interval decode, and the run sums of a row are added over the slots
// by a fixed shuffle tree. Lanes 0..r-1 store the segment's r partial sums.
// (Measured on GB300: giving each lane a whole segment instead, like a short
// interval, is about 1.35x slower on power-law rows; the warp's lanes then
// stream 32 separate stretches of memory.)
template <int R, int C, class T, int U, int DEC>
__device__ __forceinline__ void segments_body(int64_t bid, int64_t nseg, const Segment* __restrict__ segs,
                                              const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                              const typename T::V* __restrict__ val,
                                              const typename T::X* __restrict__ x,
                                              typename T::A* __restrict__ partials) {
  constexpr int MB = (R * C + 7) / 8;
  constexpr int S = kWarp / R;  // runs per segment
  const int lane = threadIdx.x & 31;
  const int64_t seg = (bid * blockDim.x + threadIdx.x) >> 5;
  if (seg >= nseg) return;  // whole warp leaves together
  const int slot = lane / R, i = lane % R;
  const Segment sg = segs[seg];
  const int32_t per = (sg.b_end - sg.b_begin + S - 1) / S;
  const int32_t rb = min(sg.b_begin + slot * per, sg.b_end);
  const int32_t re = min(rb + per, sg.b_end);
  // stored values of the run (the r lanes of a slot share its blocks)
  int cnt = 0;
  if constexpr (MB <= 8) {
    constexpr int K = 8 / MB;
    for (int32_t bb = rb + i * K; bb < re; bb += R * K) {
      uint64_t wv = load_window<MB>(bmask, bb);
      const int nblk = re - bb;
      if (nblk < K) wv &= (1ull << (8 * MB * nblk)) - 1ull;
      cnt += __popcll(wv);
    }
  } else {
    for (int32_t bb = rb + i; bb < re; bb += R) cnt += popc_all(load_mask<MB>(bmask, bb));
  }
#pragma unroll
  for (int d = 1; d < R; d <<= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
  int incl = cnt;  // inclusive scan of the run totals over the slots
#pragma unroll
  for (int d = R; d < kWarp; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  typename T::A acc = row_sum<R, C, T, U, DEC>(i, rb, re, val + sg.v_begin + (incl - cnt), bcol, bmask, x);
#pragma unroll
  for (int d = kWarp / 2; d >= R; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane < R) partials[seg * R + lane] = acc;
}

template <int R, int C, class T, int U, int DEC>
__global__ void __launch_bounds__(256) k_spmv_segments(int64_t nseg, const Segment* __restrict__ segs,
                                                       const int32_t* __restrict__ bcol, const uint8_t* __restrict__ bmask,
                                                       const typename T::V* __restrict__ val,
                                                       const typename T::X* __restrict__ x,
                                                       typename T::A* __restrict__ partials) {
  segments_body<R, C, T, U, DEC>(blockIdx.x, nseg, segs, bcol, bmask, val, x, partials);
}

// Both kinds of work in one launch: thread blocks [0, seg_ctas) take the
// segments of the long intervals, the rest the short intervals. One grid lets
// the short-interval blocks fill the SMs that the segment blocks leave idle
// (and the reverse) instead of each launch draining before the next starts;
// the sums are those of the two separate kernels, bit for bit.
template <int R, int C, class T, bool ACCUM, int U, bool ORDER, int DEC, int G = 1>
__global__ void __launch_bounds__(256) k_spmv_rows_segs(int64_t seg_ctas, int64_t n, int64_t I, int32_t long_blocks,
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
  else if constexpr (G == 1)
    rows_u_body<R, C, T, ACCUM, U, ORDER, DEC>((int64_t)blockIdx.x - seg_ctas, n, I, long_blocks, long_values, brp,
                                               bcol, bmask, val, valptr, x, y, order, norder);
  else
    rows_g_body<C, T, ACCUM, G, U, ORDER>((int64_t)blockIdx.x - seg_ctas, n, I, long_blocks, long_values, brp, bcol,
                                          bmask, val, valptr, x, y, order, norder);
}

// segments and the two-lane single-value test kernel in one grid (variant 33)
template <int C, class T, bool ACCUM, int U>
__global__ void __launch_bounds__(256) k_spmv_g1_segs(int64_t seg_ctas, int64_t n, int64_t I, int32_t long_blocks,
                                                      int64_t long_values, const int32_t* __restrict__ brp,
                                                      const int32_t* __restrict__ bcol,
                                                      const uint8_t* __restrict__ bmask,
                                                      const typename T::V* __restrict__ val,
                                                      const int64_t* __restrict__ valptr,
                                                      const typename T::X* __restrict__ x, typename T::X* __restrict__ y,
                                                      const uint32_t* __restrict__ single, int64_t nseg,
                                                      const Segment* __restrict__ segs,
                                                      typename T::A* __restrict__ partials) {
  if ((int64_t)blockIdx.x < seg_ctas)
    segments_body<1, C, T, 4, 1>(blockIdx.x, nseg, segs, bcol, bmask, val, x, partials);
  else
    rows_g_body<C, T, ACCUM, 2, U, false, true>((int64_t)blockIdx.x - seg_ctas, n, I, long_blocks, long_values, brp,
                                                bcol, bmask, val, valptr, x, y, nullptr, 0, single);
}

// segments and the single-value test kernel in one grid (variants 30 / 31)
template <int C, class T, bool ACCUM, int U, bool ORDER>
__global__ void __launch_bounds__(256) k_spmv_t_segs(int64_t seg_ctas, int64_t n, int64_t I, int32_t long_blocks,
                                                     int64_t long_values, const int32_t* __restrict__ brp,
                                                     const int32_t* __restrict__ bcol,
                                                     const uint8_t* __restrict__ bmask,
                                                     const typename T::V* __restrict__ val,
                                                     const int64_t* __restrict__ valptr,
                                                     const typename T::X* __restrict__ x, typename T::X* __restrict__ y,
                                                     const int32_t* __restrict__ order, int64_t norder,
                                                     const uint32_t* __restrict__ single, int64_t nseg,
                                                     const Segment* __restrict__ segs,
                                                     typename T::A* __restrict__ partials) {
  if ((int64_t)blockIdx.x < seg_ctas)
    segments_body<1, C, T, 4, 1>(blockIdx.x, nseg, segs, bcol, bmask, val, x, partials);
  else
    rows_t_body<C, T, ACCUM, U, ORDER>((int64_t)blockIdx.x - seg_ctas, n, I, long_blocks, long_values, brp, bcol,
                                       bmask, val, valptr, x, y, order, norder, single);
}

// Finishes the long intervals (list of first segments built at conversion;
// the first segment holds the interval's segment count). One lane per long
// interval: with at most kFixupSerial segments it adds their partials row by
// row in segment order; longer lists are taken by the whole warp, one
// interval after another - lane j adds segments j, j + 32, ... in order and a
// fixed shuffle tree adds the lanes. Either way the summation order depends
// only on the segment count.
constexpr int kFixupSerial = 32;

template <class A, class X, bool ACCUM>
__device__ __forceinline__ void fixup_lane_interval(bool have, int64_t s0, int32_t count, int32_t it, int r, int64_t n,
                                                    const A* __restrict__ part, X* __restrict__ y) {
  if (have && count <= kFixupSerial) {
    for (int i = 0; i < r; ++i) {
      A s = 0;
      for (int q = 0; q < count; ++q) s += part[(s0 + q) * r + i];
      const int64_t row = (int64_t)it * r + i;
      if (row < n) {
        if (ACCUM)
          y[row] = y[row] + s;
        else
          y[row] = s;
      }
    }
  }
}

template <class A, class X, bool ACCUM>
__device__ __forceinline__ void fixup_warp_interval(int64_t s0, int32_t count, int32_t it, int r, int64_t n,
                                                    const A* __restrict__ part, X* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < r; ++i) {
    A s = 0;
    for (int q = lane; q < count; q += kWarp) s += part[(s0 + q) * r + i];
#pragma unroll
    for (int d = kWarp / 2; d >= 1; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    const int64_t row = (int64_t)it * r + i;
    if (lane == 0 && row < n) {
      if (ACCUM)
        y[row] = y[row] + s;
      else
        y[row] = s;
    }
  }
}

template <int R, class T, bool ACCUM>
__global__ void __launch_bounds__(256) k_spmv_fixup(int64_t n, int64_t nlong, const int32_t* __restrict__ seg_first,
                                                    const Segment* __restrict__ segs,
                                                    const typename T::A* __restrict__ partials,
                                                    typename T::X* __restrict__ y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >= nlong) return;  // whole warp
  const bool have = e < nlong;
  const int64_t s0 = have ? __ldg(seg_first + e) : 0;
  const int32_t count = have ? segs[s0].count : 0;
  const int32_t it = have ? segs[s0].interval : 0;
  fixup_lane_interval<typename T::A, typename T::X, ACCUM>(have, s0, count, it, R, n, partials, y);
  unsigned big = __ballot_sync(0xffffffffu, have && count > kFixupSerial);
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1;
    fixup_warp_interval<typename T::A, typename T::X, ACCUM>(__shfl_sync(0xffffffffu, s0, src),
                                                             __shfl_sync(0xffffffffu, count, src),
                                                             __shfl_sync(0xffffffffu, it, src), R, n, partials, y);
  }
}

// --------------------------------------------------------------- launch
// Variants of the short-interval kernel: 1 plain; 0/5 natural order U=2;
// 3 natural U=4; 9/10 sorted order U=2/U=4; 12/14 natural order, mask
// windows, U=4/U=2; 13/15 sorted order, mask windows, U=4/U=2; 16/17
// natural / sorted order, bit positions unrolled (row_sum_e); 18/19 the same
// two blocks per trip (row_sum_e2); 22 (r = 1) two lanes per row taking
// alternate stored values (rows_g_body), 23 the same in the sorted order,
// 33 the same in natural order with Algorithm 2's single-value test;
// 30 / 31 (r = 1) Algorithm 2's single-value test in sorted / natural order
// (rows_t_body). (Measured:
// 8 nonzeros per trip is slower than 2 or 4 on every test matrix.)
// `partials` is the segment scratch (n_segments * r accumulators).
template <int R, int C, class T>
cudaError_t launch_beta(const spc5_matrix* h, const void* xv, void* yv, bool acc, void* partials, cudaStream_t s) {
  using V = typename T::V;
  using X = typename T::X;
  using A = typename T::A;
  const X* x = static_cast<const X*>(xv);
  X* y = static_cast<X*>(yv);
  const V* val = static_cast<const V*>(h->values);
  constexpr int S = kWarp / R;
  const int threads = kSpmvThreads;
  const int v = h->variant;
  const bool ordered = ordered_variant(v) && h->norder > 0;
  A* part = static_cast<A*>(partials);
  // segments and short intervals in one launch (not for the plain variant 1)
  const bool fused = fused_launch(h);
  const int64_t seg_ctas = (h->nseg * kWarp + threads - 1) / threads;
  bool rows_done = false;  // the short intervals already launched (G lanes per row)
  if constexpr (R == 1) {
    if (single_variant(v) && h->I > 0 && h->single_bits) {
      constexpr int U = 4;
      const bool ord = v == 30 && ordered;
      const int64_t slots = ord ? h->norder : h->I;
      const unsigned grid = (unsigned)((slots + threads - 1) / threads);
      const int32_t* order = ord ? h->order : nullptr;
      const int64_t norder = ord ? h->norder : 0;
      auto go = [&](auto kern) {
        if (grid > 0)
          kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                        h->block_masks, val, h->valptr, x, y, order, norder, h->single_bits);
      };
      auto go_both = [&](auto kern) {
        kern<<<(unsigned)(seg_ctas + grid), threads, 0, s>>>(seg_ctas, h->n, h->I, h->long_blocks, h->long_values,
                                                             h->block_rowptr, h->block_colidx, h->block_masks, val,
                                                             h->valptr, x, y, order, norder, h->single_bits, h->nseg,
                                                             h->segs, part);
      };
      if (ord) {
        if (fused)
          acc ? go_both(k_spmv_t_segs<C, T, true, U, true>) : go_both(k_spmv_t_segs<C, T, false, U, true>);
        else
          acc ? go(k_spmv_rows_t<C, T, true, U, true>) : go(k_spmv_rows_t<C, T, false, U, true>);
      } else {
        if (fused)
          acc ? go_both(k_spmv_t_segs<C, T, true, U, false>) : go_both(k_spmv_t_segs<C, T, false, U, false>);
        else
          acc ? go(k_spmv_rows_t<C, T, true, U, false>) : go(k_spmv_rows_t<C, T, false, U, false>);
      }
      rows_done = true;
    }
    if (!rows_done && v == 33 && h->I > 0 && h->single_bits) {
      constexpr int U = 2;
      const int64_t warps = (h->I + kWarp / 2 - 1) / (kWarp / 2);
      const unsigned grid = (unsigned)((warps * kWarp + threads - 1) / threads);
      if (fused) {
        auto kern = acc ? k_spmv_g1_segs<C, T, true, U> : k_spmv_g1_segs<C, T, false, U>;
        kern<<<(unsigned)(seg_ctas + grid), threads, 0, s>>>(seg_ctas, h->n, h->I, h->long_blocks, h->long_values,
                                                             h->block_rowptr, h->block_colidx, h->block_masks, val,
                                                             h->valptr, x, y, h->single_bits, h->nseg, h->segs, part);
      } else {
        auto kern = acc ? k_spmv_rows_g1<C, T, true, U> : k_spmv_rows_g1<C, T, false, U>;
        kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                      h->block_masks, val, h->valptr, x, y, h->single_bits);
      }
      rows_done = true;
    }
    if (!rows_done && (v == 22 || v == 23 || v == 33) && h->I > 0) {
      constexpr int U = 2;
      const int64_t slots = ordered ? h->norder : h->I;
      const int64_t warps = (slots + kWarp / 2 - 1) / (kWarp / 2);
      const unsigned grid = (unsigned)((warps * kWarp + threads - 1) / threads);
      const int32_t* order = ordered ? h->order : nullptr;
      const int64_t norder = ordered ? h->norder : 0;
      auto go = [&](auto kern) {
        kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                      h->block_masks, val, h->valptr, x, y, order, norder);
      };
      auto go_both = [&](auto kern) {
        kern<<<(unsigned)(seg_ctas + grid), threads, 0, s>>>(seg_ctas, h->n, h->I, h->long_blocks, h->long_values,
                                                             h->block_rowptr, h->block_colidx, h->block_masks, val,
                                                             h->valptr, x, y, order, norder, h->nseg, h->segs, part);
      };
      if (ordered) {
        if (fused)
          acc ? go_both(k_spmv_rows_segs<1, C, T, true, U, true, 0, 2>)
              : go_both(k_spmv_rows_segs<1, C, T, false, U, true, 0, 2>);
        else
          acc ? go(k_spmv_rows_g<C, T, true, 2, U, true>) : go(k_spmv_rows_g<C, T, false, 2, U, true>);
      } else {
        if (fused)
          acc ? go_both(k_spmv_rows_segs<1, C, T, true, U, false, 0, 2>)
              : go_both(k_spmv_rows_segs<1, C, T, false, U, false, 0, 2>);
        else
          acc ? go(k_spmv_rows_g<C, T, true, 2, U, false>) : go(k_spmv_rows_g<C, T, false, 2, U, false>);
      }
      rows_done = true;
    }
  }
  if (h->I > 0 && !rows_done) {
    const int64_t warps = ordered ? (h->norder + S - 1) / S : (h->I + S - 1) / S;
    const unsigned grid = (unsigned)((warps * kWarp + threads - 1) / threads);
    const int32_t* order = ordered ? h->order : nullptr;
    const int64_t norder = ordered ? h->norder : 0;
    auto go = [&](auto kern) {
      kern<<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_colidx,
                                    h->block_masks, val, h->valptr, x, y, order, norder);
    };
    auto go_both = [&](auto kern) {
      kern<<<(unsigned)(seg_ctas + grid), threads, 0, s>>>(seg_ctas, h->n, h->I, h->long_blocks, h->long_values,
                                                           h->block_rowptr, h->block_colidx, h->block_masks, val,
                                                           h->valptr, x, y, order, norder, h->nseg, h->segs, part);
    };
#define SPC5_GO(U, ORD, DEC)                                                                                   \
  (fused ? (acc ? go_both(k_spmv_rows_segs<R, C, T, true, U, ORD, DEC>)                                         \
                : go_both(k_spmv_rows_segs<R, C, T, false, U, ORD, DEC>))                                       \
         : (acc ? go(k_spmv_rows_u<R, C, T, true, U, ORD, DEC>) : go(k_spmv_rows_u<R, C, T, false, U, ORD, DEC>)))
    if (v == 1) {
      if (acc)
        k_spmv_rows<R, C, T, true><<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr,
                                                            h->block_colidx, h->block_masks, val, h->valptr, x, y);
      else
        k_spmv_rows<R, C, T, false><<<grid, threads, 0, s>>>(h->n, h->I, h->long_blocks, h->long_values, h->block_rowptr,
                                                             h->block_colidx, h->block_masks, val, h->valptr, x, y);
    } else if (ordered) {
      if (v == 10) SPC5_GO(4, true, 0);
      else if (v == 13) SPC5_GO(4, true, 1);
      else if (v == 15) SPC5_GO(2, true, 1);
      else if (v == 17) SPC5_GO(1, true, 2);
      else if (v == 19) SPC5_GO(1, true, 3);
      else SPC5_GO(2, true, 0);
    } else {
      if (v == 3) SPC5_GO(4, false, 0);
      else if (v == 12) SPC5_GO(4, false, 1);
      else if (v == 14) SPC5_GO(2, false, 1);
      else if (v == 16) SPC5_GO(1, false, 2);
      else if (v == 18) SPC5_GO(1, false, 3);
      else SPC5_GO(2, false, 0);
    }
#undef SPC5_GO
  }
  if (h->nseg > 0) {
    if (!fused)
      k_spmv_segments<R, C, T, 4, 1><<<(unsigned)seg_ctas, threads, 0, s>>>(h->nseg, h->segs, h->block_colidx,
                                                                            h->block_masks, val, x, part);
    const unsigned g2 = (unsigned)((h->nlong + 255) / 256);
    if (acc)
      k_spmv_fixup<R, T, true><<<g2, 256, 0, s>>>(h->n, h->nlong, h->seg_first, h->segs, part, y);
    else
      k_spmv_fixup<R, T, false><<<g2, 256, 0, s>>>(h->n, h->nlong, h->seg_first, h->segs, part, y);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t dispatch_beta(const spc5_matrix* h, const void* x, void* y, bool acc, void* partials, cudaStream_t s) {
#define SPC5_CASE(RR, CC) \
  if (h->r == RR && h->c == CC) return launch_beta<RR, CC, T>(h, x, y, acc, partials, s);
  SPC5_CASE(1, 4) SPC5_CASE(1, 8) SPC5_CASE(1, 16)
  SPC5_CASE(2, 4) SPC5_CASE(2, 8) SPC5_CASE(2, 16)
  SPC5_CASE(4, 4) SPC5_CASE(4, 8) SPC5_CASE(4, 16)
  SPC5_CASE(8, 4) SPC5_CASE(8, 8) SPC5_CASE(8, 16)
#undef SPC5_CASE
  return cudaErrorInvalidValue;
}

}  // namespace spc5
