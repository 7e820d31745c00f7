// CSR -> beta(r,c) conversion on the GPU (section "Block-based storage
// without zero padding"; the paper measures conversion at about two
// sequential SpMVs, section "Test matrices").
//
// Pipeline, all on the caller's stream:
//   1. k_validate_rows / k_validate_cols: row pointers, then every entry
//                   (in range, ascending, unique within its row), the work
//                   spread over the entries; on any error the row-by-row
//                   k_validate names the first bad row.
//   2. k_count      (r > 1) one thread per interval: greedy leftmost cover of
//                   the merged columns of the interval's r rows -> blocks per
//                   interval, and the number of warp segments of long ones.
//      k_r1_flags   (r = 1) block starts marked over the entries, one bit
//                   each (see there); the block index of an entry is then
//                   the scanned popcount of the mark words before it plus
//                   the marks below it in its word.
//   3. scan         exclusive prefix sums -> block_rowptr, segment pointers.
//   4. k_fill       (r > 1) one thread per interval: the same cover again,
//                   emitting block_colidx, the r*c-bit masks, each block's
//                   value offset and the segments; k_fill_values then moves
//                   the values to block order (row-major inside a block),
//                   the work spread over the entries.
//      k_r1_fill    (r = 1) the same from the marks; values copied as-is.
//   5. k_valptr     first value of each interval = rowptr[min(r*i, n)].
// Steps 2 and 4 decide blocks with the same rule (the same device function
// for r > 1, the same marks for r = 1), so the two passes agree.
#include <algorithm>
#include <climits>
#include <mutex>
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

// Fast validation, work spread over the entries instead of the rows (one
// thread per row serialises on power-law hubs): k_validate_rows checks the
// row pointer, k_validate_cols (below) every entry's range and its order
// against the previous entry of its row. Both only detect; when either flags
// anything the caller reruns k_validate for the canonical first bad row and
// code.
__global__ void k_validate_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                                unsigned long long* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t a = rowptr[i], b = rowptr[i + 1];
  if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == n - 1 && b != nnz))
    atomicMin(status, (unsigned long long)i * 8ull + (unsigned long long)SPC5_EINVAL);
}

constexpr int kEntriesPerThread = 8;  // entries per thread of the entry-parallel passes (one row search each; 32 measured slower: the walks stop coalescing)

// the row holding entry j (0 <= j < rowptr[n]): the last row whose pointer is
// <= j, which skips empty rows; stays inside [0, n-1] whatever rowptr holds
__device__ __forceinline__ int64_t row_of_entry(const int64_t* __restrict__ rowptr, int64_t n, int64_t j) {
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (rowptr[mid] <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// Row hints: the row of the first entry of every chunk of kHintChunk entries
// (and of entry nnz), so that an entry's row is searched between the rows of
// its chunk's ends - a few steps - instead of over all rows.
constexpr int kHintShift = 8;
constexpr int64_t kHintChunk = int64_t(1) << kHintShift;

__global__ void k_row_hints(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr, int64_t* __restrict__ hints) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nch = (nnz + kHintChunk - 1) / kHintChunk;
  if (k > nch) return;
  const int64_t j = k * kHintChunk < nnz ? k * kHintChunk : (nnz > 0 ? nnz - 1 : 0);
  hints[k] = row_of_entry(rowptr, n, j);
}

// the row of entry j (same result as row_of_entry) from the hints
__device__ __forceinline__ int64_t row_of_entry_hint(const int64_t* __restrict__ rowptr, int64_t n,
                                                     const int64_t* __restrict__ hints, int64_t j) {
  int64_t lo = hints[j >> kHintShift], hi = hints[(j >> kHintShift) + 1] + 1;
  if (hi > n) hi = n;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (rowptr[mid] <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// A warp checks 2048 consecutive entries with coalesced loads: the rows that
// start inside the chunk become a bitmap (from the row pointers), then each
// entry is checked for range and, unless it starts a row, against its left
// neighbour. Detection only (status set to 0 on any error).
constexpr int kValChunk = 2048;

__global__ void __launch_bounds__(256) k_validate_cols(int64_t n, int64_t m, int64_t nnz,
                                                       const int64_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ colidx,
                                                       unsigned long long* __restrict__ status) {
  __shared__ uint32_t starts[8][kValChunk / 32];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kValChunk;
  if (base >= nnz) return;  // whole warp
  const int64_t end = base + kValChunk < nnz ? base + kValChunk : nnz;
  uint32_t* st = starts[wb];
  for (int q = lane; q < kValChunk / 32; q += 32) st[q] = 0u;
  __syncwarp();
  // first row whose pointer is >= base
  int64_t lo = 0, hi = n + 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (rowptr[mid] < base) lo = mid + 1; else hi = mid;
  }
  for (int64_t q0 = lo;; q0 += 32) {
    const int64_t q = q0 + lane;
    const int64_t v = q <= n ? rowptr[q] : LLONG_MAX;
    const bool in = v >= base && v < end;
    if (in) atomicOr(&st[(v - base) >> 5], 1u << ((v - base) & 31));
    if (!__any_sync(0xffffffffu, v < end)) break;
  }
  __syncwarp();
  bool bad = false;
#pragma unroll 4
  for (int k = 0; k < kValChunk / 32; ++k) {
    const int64_t j = base + k * 32 + lane;
    const int32_t col = j < end ? colidx[j] : 0;
    int32_t prev = __shfl_up_sync(0xffffffffu, col, 1);
    if (lane == 0) prev = j > 0 ? colidx[j - 1] : 0;
    if (j < end) {
      const int o = (int)(j - base);
      const bool row_start = (st[o >> 5] >> (o & 31)) & 1u;
      if (col < 0 || col >= m) bad = true;
      if (!row_start && j > 0 && col <= prev) bad = true;
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMin(status, 0ull);
}

// ------------------------------------------------------ one-row intervals
// For r = 1 the cover splits at every gap of at least c between neighbouring
// columns of a row: whichever block holds the left column ends before the
// right one, so the right column starts a block in any cover. The runs
// between such gaps are covered independently, so the work spreads over the
// entries (one thread per kEntriesPerThread entries, each walking the runs
// that start in its range) instead of one thread per row. Pass 1 sets one
// bit per entry that starts a block (nnz/8 bytes of marks); an exclusive scan
// of the popcounts of the 32-bit mark words numbers the blocks in storage
// order (rows in order, blocks by column), the block of a marked entry being
// the prefix of its word plus the marks below it; pass 2 writes each block's
// column, mask and, for long rows, its segment record. With one row per
// interval the values keep CSR order and are copied as they are.
__global__ void k_r1_flags(int64_t n, int64_t nnz, int c, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ colidx, const int64_t* __restrict__ hints,
                           uint32_t* __restrict__ marks) {
  static_assert(32 % kEntriesPerThread == 0, "a thread's entries share one mark word");
  const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kEntriesPerThread;
  if (j0 >= nnz) return;
  const int64_t j1 = j0 + kEntriesPerThread < nnz ? j0 + kEntriesPerThread : nnz;
  int64_t row = row_of_entry_hint(rowptr, n, hints, j0);
  int64_t rs = rowptr[row], re = rowptr[row + 1];
  int32_t prev = j0 > rs ? colidx[j0 - 1] : 0;
  uint32_t mine = 0u;  // marks of this thread's own entries (one word); others by atomicOr
  for (int64_t j = j0; j < j1; ++j) {
    while (j >= re) {
      ++row;
      rs = rowptr[row];
      re = rowptr[row + 1];
    }
    const int32_t col = colidx[j];
    const bool run_start = j == rs || col - prev >= c;
    prev = col;
    if (!run_start) continue;
    // greedy cover of the run that starts here
    int32_t s0 = col, last = col;
    mine |= 1u << (j & 31);
    for (int64_t k = j + 1; k < re; ++k) {
      const int32_t ck = colidx[k];
      if (ck - last >= c) break;  // the next run
      if (ck - s0 >= c) {
        s0 = ck;
        if (k < j1)
          mine |= 1u << (k & 31);
        else
          atomicOr(marks + (k >> 5), 1u << (k & 31));
      }
      last = ck;
    }
  }
  if (mine) atomicOr(marks + (j0 >> 5), mine);
}

// popcount of every mark word (the scan input)
__global__ void k_mark_counts(int64_t nwords, const uint32_t* __restrict__ marks, int32_t* __restrict__ counts) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w < nwords) counts[w] = __popc(marks[w]);
}

// blocks that start before entry e: marks in whole words before e's word
// (prefix) plus those below e in its word
__device__ __forceinline__ int32_t blocks_before(int64_t e, int64_t nwords, const uint32_t* __restrict__ marks,
                                                 const int32_t* __restrict__ prefix) {
  const int64_t w = e >> 5;
  if (w >= nwords) return prefix[nwords];
  return prefix[w] + __popc(marks[w] & ((1u << (e & 31)) - 1u));
}

__global__ void k_r1_rowptr(int64_t n, const int64_t* __restrict__ rowptr, int64_t nwords,
                            const uint32_t* __restrict__ marks, const int32_t* __restrict__ prefix,
                            int32_t* __restrict__ brp, int32_t* __restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int32_t b = blocks_before(rowptr[i], nwords, marks, prefix);
  brp[i] = b;
  if (i < n) counts[i] = blocks_before(rowptr[i + 1], nwords, marks, prefix) - b;
}
template <class W>
__global__ void k_r1_fill(int64_t n, int64_t nnz, int c, int mb, int seg_blocks, const int64_t* __restrict__ rowptr,
                          const int32_t* __restrict__ colidx, const int64_t* __restrict__ hints,
                          const W* __restrict__ vin, W* __restrict__ vout, int64_t nwords,
                          const uint32_t* __restrict__ marks, const int32_t* __restrict__ prefix,
                          const int32_t* __restrict__ brp,
                          const int32_t* __restrict__ segptr, int32_t* __restrict__ bcol,
                          uint8_t* __restrict__ bmask, Segment* __restrict__ segs) {
  // the values keep CSR order (one row per interval): the warp copies its
  // 32 x kEntriesPerThread entries' values with coalesced accesses
  {
    const int64_t wbase = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 * kEntriesPerThread);
    for (int64_t q = wbase + (threadIdx.x & 31); q < wbase + 32 * kEntriesPerThread && q < nnz; q += 32)
      vout[q] = vin[q];
  }
  const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kEntriesPerThread;
  if (j0 >= nnz) return;
  const int64_t j1 = j0 + kEntriesPerThread < nnz ? j0 + kEntriesPerThread : nnz;
  int64_t row = row_of_entry_hint(rowptr, n, hints, j0);
  int64_t re = rowptr[row + 1];
  for (int64_t j = j0; j < j1; ++j) {
    while (j >= re) {
      ++row;
      re = rowptr[row + 1];
    }
    const uint32_t word = marks[j >> 5];
    if (!((word >> (j & 31)) & 1u)) continue;
    const int32_t b = prefix[j >> 5] + __popc(word & ((1u << (j & 31)) - 1u));
    const int32_t s0 = colidx[j];
    uint32_t mask = 0u;
    for (int64_t k = j; k < re; ++k) {
      const int32_t d = colidx[k] - s0;
      if (d >= c) break;
      mask |= 1u << d;
    }
    bcol[b] = s0;
    bmask[(int64_t)b * mb] = (uint8_t)mask;
    if (mb > 1) bmask[(int64_t)b * mb + 1] = (uint8_t)(mask >> 8);
    if (segptr != nullptr && segptr[row + 1] > segptr[row]) {
      const int32_t jb = b - brp[row];
      if (jb % seg_blocks == 0) {
        Segment sg;
        sg.interval = (int32_t)row;
        sg.b_begin = b;
        sg.b_end = min(b + seg_blocks, brp[row + 1]);
        sg.count = jb == 0 ? segptr[row + 1] - segptr[row] : 0;
        sg.v_begin = j;
        segs[segptr[row] + jb / seg_blocks] = sg;
      }
    }
  }
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

// Structure pass for r > 1: one thread per interval walks the cover again and
// writes each block's column, mask, value offset inside the interval (bvo)
// and the segment records. The values move in k_fill_values.
template <int R>
__global__ void k_fill(int64_t n, int64_t I, int c, int mb, int seg_blocks, const int64_t* __restrict__ rowptr,
                       const int32_t* __restrict__ colidx, const int32_t* __restrict__ block_rowptr,
                       const int32_t* __restrict__ segptr, int32_t* __restrict__ bcol, uint8_t* __restrict__ bmask,
                       int32_t* __restrict__ bvo, Segment* __restrict__ segs) {
  int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  int64_t row0 = it * R;
  int rows = (int)(n - row0 < (int64_t)R ? n - row0 : (int64_t)R);
  int32_t b0 = block_rowptr[it];
  int32_t bend = block_rowptr[it + 1];
  bool is_long = segptr != nullptr && segptr[it + 1] > segptr[it];
  int32_t seg0 = is_long ? segptr[it] : 0;
  const int64_t v0 = rowptr[row0];  // the interval's values start where its first row starts in CSR
  int64_t vo = v0;
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
    bvo[b] = (int32_t)(vo - v0);
    uint32_t mw[4] = {0u, 0u, 0u, 0u};  // up to 128 mask bits
#pragma unroll
    for (int i = 0; i < R; ++i) {
      for (int64_t p = lo[i]; p < hi[i]; ++p) {
        int bit = i * c + (int)(colidx[p] - s);
        mw[bit >> 5] |= 1u << (bit & 31);
      }
      vo += hi[i] - lo[i];
    }
    bcol[b] = (int32_t)s;
    uint8_t* dst = bmask + (int64_t)b * mb;
    for (int q = 0; q < mb; ++q) dst[q] = (uint8_t)(mw[q >> 2] >> (8 * (q & 3)));
  });
}

// Value pass for r > 1, spread over the entries (kEntriesPerThread consecutive
// CSR entries per thread, walking rows): entry (row i of interval it, column
// col) lies in the interval's last block starting at or before col, and its
// place in block order is the interval's first value + the block's offset +
// the mask bits before (i, col - start). Consecutive entries of a row move
// through the interval's blocks in order, so only the first needs a search.
template <int R, class VT>
__global__ void k_fill_values(int64_t n, int64_t nnz, int c, int mb, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colidx, const int64_t* __restrict__ hints,
                              const VT* __restrict__ values,
                              const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                              const uint8_t* __restrict__ bmask, const int32_t* __restrict__ bvo,
                              VT* __restrict__ bval) {
  const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kEntriesPerThread;
  if (j0 >= nnz) return;
  const int64_t j1 = j0 + kEntriesPerThread < nnz ? j0 + kEntriesPerThread : nnz;
  int64_t row = row_of_entry_hint(rowptr, n, hints, j0);
  int64_t re = rowptr[row + 1];
  int64_t it = row / R, vstart = rowptr[it * R];
  int i = (int)(row - it * R);
  int32_t bb = brp[it], be = brp[it + 1];
  bool fresh = true;  // block of the first entry of this row still to search
  int32_t b = bb;
  for (int64_t j = j0; j < j1; ++j) {
    while (j >= re) {
      ++row;
      re = rowptr[row + 1];
      it = row / R;
      i = (int)(row - it * R);
      vstart = rowptr[it * R];
      bb = brp[it];
      be = brp[it + 1];
      fresh = true;
    }
    const int32_t col = colidx[j];
    if (fresh) {  // last block of the interval starting at or before col
      int32_t lo = bb, hi = be;
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (bcol[mid] <= col) lo = mid; else hi = mid;
      }
      b = lo;
      fresh = false;
    } else {
      while (b + 1 < be && bcol[b + 1] <= col) ++b;
    }
    const int bit = i * c + (col - bcol[b]);
    const uint8_t* mk = bmask + (int64_t)b * mb;
    int below = 0;
    for (int q = 0; q < (bit >> 3); ++q) below += __popc((uint32_t)mk[q]);
    below += __popc((uint32_t)mk[bit >> 3] & ((1u << (bit & 7)) - 1u));
    bval[vstart + bvo[b] + below] = values[j];
  }
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

// sum of each tile of kScanTile counts (coalesced loads)
__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t L, int64_t* __restrict__ tile_sums) {
  __shared__ int64_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kScanThreads + threadIdx.x;
    sum += i < L ? (int64_t)in[i] : 0;
  }
  block_exclusive_scan(sum, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// one CTA of 1024 threads: exclusive scan of the tile sums, 4096 per step
// (4 consecutive per thread), with a running carry
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) k_scan_tile_sums(int64_t* __restrict__ tile_sums, int64_t ntiles,
                                                               int64_t* __restrict__ grand_total) {
  __shared__ int64_t warp_sums[kSumThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += 4 * kSumThreads) {
    const int64_t i0 = base + 4 * (int64_t)threadIdx.x;
    int64_t v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = i0 + k < ntiles ? tile_sums[i0 + k] : 0;
      sum += v[k];
    }
    int64_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int64_t ws = warp_sums[lane];
      int64_t wi = ws;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, wi, d);
        if (lane >= d) wi += t;
      }
      warp_sums[lane] = wi - ws;  // exclusive warp offsets; lane 31's wi is the step total
    }
    __syncthreads();
    int64_t pre = carry + warp_sums[w] + (incl - sum);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i0 + k < ntiles) tile_sums[i0 + k] = pre;
      pre += v[k];
    }
    // the step total: the last thread's running prefix
    __shared__ int64_t step_end;
    if (threadIdx.x == kSumThreads - 1) step_end = pre;
    __syncthreads();
    carry = step_end;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand_total = carry;
}

// exclusive scan of each tile (coalesced loads through shared memory) plus
// the tile's offset; int32 results (the caller checked the total), the total
// at index L
__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t L, const int64_t* __restrict__ tile_sums,
                             const int64_t* __restrict__ grand_total, int32_t* __restrict__ out) {
  __shared__ int64_t tot;
  __shared__ int32_t tile[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kScanThreads + threadIdx.x;
    tile[k * kScanThreads + threadIdx.x] = i < L ? in[i] : 0;
  }
  __syncthreads();
  int32_t v[kScanItems];
  int64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = tile[threadIdx.x * kScanItems + k];
    sum += v[k];
  }
  int64_t pre = block_exclusive_scan(sum, &tot) + tile_sums[blockIdx.x];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    tile[threadIdx.x * kScanItems + k] = (int32_t)pre;
    pre += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kScanThreads + threadIdx.x;
    if (i < L) out[i] = tile[k * kScanThreads + threadIdx.x];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[L] = (int32_t)*grand_total;
}

// The handles' arenas come from a memory pool of the library's own (one per
// device) that keeps freed memory for the next handle instead of returning
// it to the driver: a fresh cudaMalloc of a 1.6 GB handle costs more than
// its conversion kernels, and conversions of one matrix to several shapes,
// or of one structure at every time step, come in series. spc5_pool_trim
// hands the kept memory back.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaError_t handle_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;  // never release on synchronisation
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    g_pools[dev] = p;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

// Scratch memory taken from the library's pool: allocation and release are
// queued on the conversion stream, so neither waits for the GPU, and the
// memory stays in the pool for the next conversion.
struct DeviceBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t alloc(size_t bytes, cudaStream_t st) {
    s = st;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = handle_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(&p, bytes > 0 ? bytes : 16, pool, st);
  }
  ~DeviceBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

// Exclusive scan of in[0..L) into out[0..L] (out[L] = total). Returns the
// total through *total_host (synchronises the stream).
spc5_status scan_counts(const int32_t* in, int64_t L, int32_t* out, int64_t* total_host, cudaStream_t s) {
  int64_t ntiles = (L + kScanTile - 1) / kScanTile;
  if (ntiles < 1) ntiles = 1;
  DeviceBuf sums;
  cudaError_t e = sums.alloc(sizeof(int64_t) * (size_t)(ntiles + 1), s);
  if (e != cudaSuccess) return cuda_fail(e, "scan scratch");
  int64_t* t64 = (int64_t*)sums.p;
  k_scan_reduce<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, L, t64);
  k_scan_tile_sums<<<1, kSumThreads, 0, s>>>(t64, ntiles, t64 + ntiles);
  int64_t tot = 0;
  e = cudaMemcpyAsync(&tot, t64 + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "scan");
  *total_host = tot;
  if (tot > INT_MAX) return fail(SPC5_ERANGE, "prefix sum exceeds int32 (too many blocks)");
  k_scan_apply<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, L, t64, t64 + ntiles, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "scan");
  return SPC5_OK;
}

template <int R>
void launch_count(int64_t n, int64_t I, int c, const int64_t* rowptr, const int32_t* colidx, int32_t* counts,
                  cudaStream_t s) {
  if (I == 0) return;
  k_count<R><<<(unsigned)((I + 127) / 128), 128, 0, s>>>(n, I, c, rowptr, colidx, counts);
}

void launch_fill_r(int r, int64_t n, int64_t I, int c, int mb, int sb, const int64_t* rowptr, const int32_t* colidx,
                   const int32_t* brp, const int32_t* segptr, int32_t* bvo, spc5_matrix* h, cudaStream_t s) {
  if (I == 0) return;
  unsigned grid = (unsigned)((I + 127) / 128);
  switch (r) {
    case 2: k_fill<2><<<grid, 128, 0, s>>>(n, I, c, mb, sb, rowptr, colidx, brp, segptr, h->block_colidx, h->block_masks, bvo, h->segs); break;
    case 4: k_fill<4><<<grid, 128, 0, s>>>(n, I, c, mb, sb, rowptr, colidx, brp, segptr, h->block_colidx, h->block_masks, bvo, h->segs); break;
    default: k_fill<8><<<grid, 128, 0, s>>>(n, I, c, mb, sb, rowptr, colidx, brp, segptr, h->block_colidx, h->block_masks, bvo, h->segs); break;
  }
}

template <class VT>
void launch_fill_values(int r, int64_t n, int64_t nnz, int c, int mb, const int64_t* rowptr, const int32_t* colidx,
                        const int64_t* hints, const void* values, const int32_t* bvo, spc5_matrix* h,
                        cudaStream_t s) {
  const int64_t th = (nnz + kEntriesPerThread - 1) / kEntriesPerThread;
  if (th == 0) return;
  const unsigned grid = (unsigned)((th + 255) / 256);
  const VT* v = (const VT*)values;
  VT* bv = (VT*)h->values;
  switch (r) {
    case 2: k_fill_values<2, VT><<<grid, 256, 0, s>>>(n, nnz, c, mb, rowptr, colidx, hints, v, h->block_rowptr, h->block_colidx, h->block_masks, bvo, bv); break;
    case 4: k_fill_values<4, VT><<<grid, 256, 0, s>>>(n, nnz, c, mb, rowptr, colidx, hints, v, h->block_rowptr, h->block_colidx, h->block_masks, bvo, bv); break;
    default: k_fill_values<8, VT><<<grid, 256, 0, s>>>(n, nnz, c, mb, rowptr, colidx, hints, v, h->block_rowptr, h->block_colidx, h->block_masks, bvo, bv); break;
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

// The handle's arrays are pool memory, freed in stream order: on the
// conversion's stream while a conversion fails, on the legacy stream after
// spc5_destroy's device synchronisation (the SpMM scratch is cudaMalloc'd).
void free_matrix(spc5_matrix* h) {
  if (!h) return;
  const cudaStream_t s = h->arena_stream;
  auto release = [s](void* p) {
    if (p) cudaFreeAsync(p, s);
  };
  release(h->order);
  release(h->single_bits);
  cudaFree(h->spmm_scratch);
  release(h->block_rowptr);
  release(h->seg_first);
  if (h->arena) {
    release(h->arena);
  } else {
    release(h->block_colidx);
    release(h->block_masks);
    release(h->values);
    release(h->valptr);
    release(h->segs);
    release(h->partials);
  }
  delete h;
}

// One allocation for the arrays whose sizes are known once the blocks are
// counted: each region starts on a 256-byte boundary and is followed by at
// least 16 bytes of padding (zeroed; the window and vector loads may read
// into it).
cudaError_t alloc_arena(spc5_matrix* h, int64_t nb, int64_t nnz, int64_t ns, cudaStream_t s) {
  const size_t vsz = value_size(h->vt), asz = h->vt == SPC5_F64 ? 8 : 4;
  const size_t bytes[6] = {sizeof(int32_t) * (size_t)nb,        (size_t)nb * (size_t)h->mb,
                           vsz * (size_t)nnz,                   sizeof(int64_t) * (size_t)(h->I + 1),
                           sizeof(Segment) * (size_t)ns,        asz * (size_t)ns * (size_t)h->r};
  size_t off[6], total = 0;
  for (int q = 0; q < 6; ++q) {
    off[q] = total;
    total += ((bytes[q] + 16 + 255) / 256) * 256;
  }
  uint8_t* base = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = handle_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&base, total, pool, s);
  if (e != cudaSuccess) return e;
  h->arena = base;
  h->arena_stream = s;
  h->block_colidx = reinterpret_cast<int32_t*>(base + off[0]);
  h->block_masks = base + off[1];
  h->values = base + off[2];
  h->valptr = reinterpret_cast<int64_t*>(base + off[3]);
  h->segs = reinterpret_cast<Segment*>(base + off[4]);
  h->partials = base + off[5];
  for (int q = 0; q < 6 && e == cudaSuccess; ++q) {
    const size_t end = q < 5 ? off[q + 1] : total;
    e = cudaMemsetAsync(base + off[q] + bytes[q], 0, end - off[q] - bytes[q], s);  // the padding
  }
  return e;
}

// allocation padded to a multiple of 16 bytes plus 16 (bulk copies may round
// up), zeroed, from the library's pool in the order of stream s
cudaError_t alloc_padded(void** p, size_t bytes, cudaStream_t s) {
  size_t b = ((bytes + 15) / 16) * 16 + 16;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = handle_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, b, pool, s);
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

// Algorithm 2's test made once per interval (r = 1): bit it is set when
// every block of short interval it holds a single value. Under greedy
// leftmost cover a single-value block of one row has mask 1 (its value sits
// at the block's first column), so such a row reads like CSR: value j of the
// row belongs to block b0 + j at column block_colidx[b0 + j]. One warp forms
// each 32-interval word with a ballot; the count of set bits goes to *nset.
template <int MB>
__global__ void k_single_bits(int64_t I, int32_t long_blocks, int64_t long_values, const int32_t* __restrict__ brp,
                              const uint8_t* __restrict__ masks, const int64_t* __restrict__ valptr,
                              uint32_t* __restrict__ bits, unsigned long long* __restrict__ nset) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool one = false;
  if (it < I) {
    const int32_t b0 = brp[it], b1 = brp[it + 1];
    const bool lng = b1 - b0 > long_blocks || valptr[it + 1] - valptr[it] > long_values;
    // a single-value row has as many values as blocks; then every mask is 1
    one = !lng && b1 > b0 && valptr[it + 1] - valptr[it] == (int64_t)(b1 - b0);
    for (int32_t b = b0; one && b < b1; ++b) {
      uint32_t w = masks[(int64_t)b * MB];
      if (MB == 2) w |= (uint32_t)masks[(int64_t)b * MB + 1] << 8;
      one = w == 1u;
    }
  }
  const unsigned word = __ballot_sync(0xffffffffu, one);
  if ((threadIdx.x & 31) == 0 && it < I) {
    bits[it >> 5] = word;
    atomicAdd(nset, (unsigned long long)__popc(word));
  }
}

// Sorting of the work order on the device, one thread block per window of at
// most kSortWindow intervals: each short interval becomes the 64-bit word
// (INT32_MAX - key) << 32 | position, so that an ascending bitonic sort in
// shared memory orders by key descending and keeps the interval order among
// equal keys (the stable sort of the host path); long intervals (key -1) and
// the padding sort last and are dropped.
constexpr int kSortWindow = 4096;

__global__ void k_order_count(int64_t I, int64_t wiv, const int32_t* __restrict__ key, int32_t* __restrict__ cnt) {
  const int64_t w0 = (int64_t)blockIdx.x * wiv;
  const int64_t w1 = w0 + wiv < I ? w0 + wiv : I;
  int c = 0;
  for (int64_t it = w0 + threadIdx.x; it < w1; it += blockDim.x) c += key[it] >= 0 ? 1 : 0;
  c = __reduce_add_sync(0xffffffffu, (unsigned)c);
  __shared__ int part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
    cnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_order_sort(int64_t I, int64_t wiv, int P, const int32_t* __restrict__ key,
                                                     const int32_t* __restrict__ off, int32_t* __restrict__ order) {
  extern __shared__ unsigned long long sk[];  // P words, P = power of two >= wiv
  const int64_t w0 = (int64_t)blockIdx.x * wiv;
  const int64_t w1 = w0 + wiv < I ? w0 + wiv : I;
  const int nw = (int)(w1 - w0);
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    unsigned long long v = ~0ull;
    if (q < nw) {
      const int32_t k = key[w0 + q];
      if (k >= 0) v = ((unsigned long long)(uint32_t)(INT32_MAX - k) << 32) | (unsigned)q;
    }
    sk[q] = v;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = threadIdx.x; q < P; q += blockDim.x) {
        const int p = q ^ stride;
        if (p > q) {
          const bool up = (q & size) == 0;
          const unsigned long long a = sk[q], b = sk[p];
          if ((a > b) == up) {
            sk[q] = b;
            sk[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  const int32_t base = off[blockIdx.x];
  const int32_t valid = off[blockIdx.x + 1] - base;
  for (int q = threadIdx.x; q < valid; q += blockDim.x) order[base + q] = (int32_t)(w0 + (int64_t)(uint32_t)sk[q]);
}

}  // namespace

// Work order of the lane-per-row kernel (variants 9, 10, 13, 15): the short
// intervals, sorted by their longest row (descending, stable) inside windows
// of order_window rows (all intervals together when order_window <= 0), so
// that the 32/r intervals of one warp have rows of similar length and the
// warp's multiply-adds are fully packed. Small windows keep the rows that
// neighbouring warps read close together in memory (measured: one global
// sort, or handing whole thread blocks out heaviest first, is slower on
// power-law graphs than 1024-row windows). The storage is untouched; only the
// assignment of intervals to lanes changes.
spc5_status build_single_bits(spc5_matrix* h, cudaStream_t s) {
  if (h->single_bits || h->I == 0 || h->r != 1) return SPC5_OK;
  const int64_t words = (h->I + 31) / 32;
  uint32_t* d = nullptr;
  cudaError_t e = alloc_padded((void**)&d, sizeof(uint32_t) * (size_t)words, s);
  if (e != cudaSuccess) return cuda_fail(e, "single-value bits: allocation");
  DeviceBuf cnt;
  e = cnt.alloc(sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)((h->I + 255) / 256);
    if (h->mb == 1)
      k_single_bits<1><<<grid, 256, 0, s>>>(h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_masks,
                                             h->valptr, d, (unsigned long long*)cnt.p);
    else
      k_single_bits<2><<<grid, 256, 0, s>>>(h->I, h->long_blocks, h->long_values, h->block_rowptr, h->block_masks,
                                             h->valptr, d, (unsigned long long*)cnt.p);
    e = cudaGetLastError();
  }
  unsigned long long nset = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nset, cnt.p, sizeof(nset), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFreeAsync(d, s);
    return cuda_fail(e, "single-value bits");
  }
  h->single_bits = d;
  h->nsingle = (int64_t)nset;
  return SPC5_OK;
}

spc5_status build_order(spc5_matrix* h, cudaStream_t s) {
  if (h->order || h->I == 0) return SPC5_OK;
  const int64_t I = h->I;
  DeviceBuf keyd;
  cudaError_t e = keyd.alloc(sizeof(int32_t) * (size_t)I, s);
  if (e != cudaSuccess) return cuda_fail(e, "work order: scratch");
  switch (h->r) {
    case 1: launch_order_key<1>(h->c, h, (int32_t*)keyd.p, s); break;
    case 2: launch_order_key<2>(h->c, h, (int32_t*)keyd.p, s); break;
    case 4: launch_order_key<4>(h->c, h, (int32_t*)keyd.p, s); break;
    default: launch_order_key<8>(h->c, h, (int32_t*)keyd.p, s); break;
  }
  const int64_t wiv_d = h->order_window > 0 ? (h->order_window + h->r - 1) / h->r : I;
  if (wiv_d <= kSortWindow) {
    // windows small enough for one thread block each: sort on the device
    const int64_t nwin = (I + wiv_d - 1) / wiv_d;
    int P = 1;
    while (P < wiv_d) P <<= 1;
    DeviceBuf cnt, off;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cnt.alloc(sizeof(int32_t) * (size_t)nwin, s);
    if (e == cudaSuccess) e = off.alloc(sizeof(int32_t) * (size_t)(nwin + 1), s);
    if (e != cudaSuccess) return cuda_fail(e, "work order: scratch");
    k_order_count<<<(unsigned)nwin, 256, 0, s>>>(I, wiv_d, (const int32_t*)keyd.p, (int32_t*)cnt.p);
    int64_t total = 0;
    spc5_status st = scan_counts((const int32_t*)cnt.p, nwin, (int32_t*)off.p, &total, s);
    if (st != SPC5_OK) return st;
    int32_t* d = nullptr;
    if (total > 0) {
      e = alloc_padded((void**)&d, sizeof(int32_t) * (size_t)total, s);
      if (e != cudaSuccess) return cuda_fail(e, "work order: allocation");
      const size_t smem = sizeof(unsigned long long) * (size_t)P;
      if (smem > 48 * 1024) e = cudaFuncSetAttribute(k_order_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        k_order_sort<<<(unsigned)nwin, 1024, smem, s>>>(I, wiv_d, P, (const int32_t*)keyd.p, (const int32_t*)off.p, d);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        cudaFreeAsync(d, s);
        return cuda_fail(e, "work order: sort");
      }
    }
    h->order = d;
    h->norder = total;
    return SPC5_OK;
  }
  // larger windows (or all intervals together): stable sort on the host
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
      cudaFreeAsync(d, s);
      return cuda_fail(e, "work order: upload");
    }
    h->order = d;
  }
  h->norder = (int64_t)order.size();
  return SPC5_OK;
}

// ------------------------------------------------------------ assembly
// Checks of caller-built beta(r,c) arrays. status = min over bad items of
// (item * 8 + code); item = interval for the row pointer, block otherwise.
__global__ void k_asm_intervals(int64_t I, int64_t nb, const int32_t* __restrict__ brp,
                                unsigned long long* __restrict__ status) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  const int64_t a = brp[it], b = brp[it + 1];
  if (a < 0 || b < a || b > nb || (it == 0 && a != 0) || (it == I - 1 && b != nb))
    atomicMin(status, (unsigned long long)it * 8ull + (unsigned long long)SPC5_EINVAL);
}

// per block: column in range, no bit past column m - 1 or row n - 1, the next
// block of the interval starting at or after this one's window; cnt[b] = the
// block's stored values
template <int R>
__global__ void k_asm_blocks(int64_t n, int64_t m, int64_t I, int64_t nb, int c, int mb,
                             const int32_t* __restrict__ brp, const int32_t* __restrict__ bcol,
                             const uint8_t* __restrict__ bmask, int32_t* __restrict__ cnt,
                             unsigned long long* __restrict__ status) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  // interval of block b: the last interval whose first block is <= b
  int64_t lo = 0, hi = I;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (brp[mid] <= b) lo = mid; else hi = mid;
  }
  const int64_t it = lo;
  const int32_t col = bcol[b];
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  for (int q = 0; q < mb; ++q) w[q >> 2] |= (uint32_t)bmask[b * mb + q] << (8 * (q & 3));
  int code = 0, pc = 0;
  for (int i = 0; i < R; ++i) {
    const int p = i * c;
    const uint32_t bits = (w[p >> 5] >> (p & 31)) & (c == 32 ? 0xffffffffu : ((1u << c) - 1u));
    pc += __popc(bits);
    if (bits && it * R + i >= n) code = SPC5_ERANGE;                         // a row past n - 1
    if (bits && (int64_t)col + (31 - __clz(bits)) >= m) code = SPC5_ERANGE;  // a column past m - 1
  }
  if (col < 0 || col >= m) code = SPC5_ERANGE;
  if (b + 1 < brp[it + 1] && (int64_t)bcol[b + 1] < (int64_t)col + c) code = SPC5_EUNSORTED;  // windows overlap or go back
  cnt[b] = pc;
  if (code) atomicMin(status, (unsigned long long)b * 8ull + (unsigned long long)code);
}

// valptr[it] = values before interval it (from the block value prefix)
__global__ void k_asm_valptr(int64_t I, const int32_t* __restrict__ brp, const int32_t* __restrict__ bval,
                             int64_t* __restrict__ valptr, int32_t* __restrict__ counts) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it > I) return;
  valptr[it] = bval[brp[it]];
  if (it < I) counts[it] = brp[it + 1] - brp[it];
}

// segments of long intervals (blocks or values above the thresholds)
__global__ void k_asm_segments(int64_t I, int32_t long_blocks, int64_t long_values, int seg_blocks,
                               const int32_t* __restrict__ brp, const int32_t* __restrict__ bval,
                               const int64_t* __restrict__ valptr, int32_t* __restrict__ nseg) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  const int32_t nbk = brp[it + 1] - brp[it];
  const bool lng = nbk > long_blocks || valptr[it + 1] - valptr[it] > long_values;
  nseg[it] = lng ? (nbk + seg_blocks - 1) / seg_blocks : 0;
}

__global__ void k_asm_seg_fill(int64_t I, int seg_blocks, const int32_t* __restrict__ brp,
                               const int32_t* __restrict__ bval, const int32_t* __restrict__ segptr,
                               Segment* __restrict__ segs) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= I) return;
  const int32_t s0 = segptr[it], ns = segptr[it + 1] - s0;
  for (int32_t q = 0; q < ns; ++q) {
    Segment sg;
    sg.interval = (int32_t)it;
    sg.b_begin = brp[it] + q * seg_blocks;
    sg.b_end = min(sg.b_begin + seg_blocks, brp[it + 1]);
    sg.count = q == 0 ? ns : 0;
    sg.v_begin = bval[sg.b_begin];
    segs[s0 + q] = sg;
  }
}

spc5_status exclusive_scan_i32(const int32_t* in, int64_t L, int32_t* out, int64_t* total_host, cudaStream_t s) {
  return scan_counts(in, L, out, total_host, s);
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = handle_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 16, pool, s);
  return e;
}

void destroy_matrix(spc5_matrix* h) {
  h->arena_stream = nullptr;  // the caller synchronised the device; its stream may be gone
  free_matrix(h);
}

cudaError_t trim_pools() {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  cudaError_t e = cudaSuccess;
  for (int d = 0; d < kMaxPoolDevices; ++d)
    if (g_pools[d]) {
      const cudaError_t e2 = cudaMemPoolTrimTo(g_pools[d], 0);
      if (e == cudaSuccess) e = e2;
    }
  return e;
}

spc5_status assemble_impl(int64_t n, int64_t m, int64_t nnz, int64_t nb, int r, int c, spc5_dtype vt,
                          const int32_t* brp_in, const int32_t* bcol_in, const uint8_t* bmask_in, const void* vals_in,
                          const spc5_opts* opt, cudaStream_t s, spc5_matrix** out) {
  *out = nullptr;
  spc5_matrix* h = new spc5_matrix();
  h->arena_stream = s;  // failures free the arrays in this stream's order
  h->n = n;
  h->m = m;
  h->nnz = nnz;
  h->r = r;
  h->c = c;
  h->mb = mask_bytes(r, c);
  h->vt = vt;
  h->I = (n + r - 1) / r;
  h->nb = nb;
  int32_t user_long = 0;
  if (opt) {
    user_long = opt->long_blocks;
    if (opt->seg_blocks > 0) h->seg_blocks = opt->seg_blocks;
    h->variant = opt->variant;
    if (opt->order_window != 0) h->order_window = opt->order_window;
  }
  const int64_t I = h->I;
  auto bail = [&](spc5_status st) {
    free_matrix(h);
    return st;
  };
  cudaError_t e = alloc_padded((void**)&h->block_rowptr, sizeof(int32_t) * (size_t)(I + 1), s);
  if (e == cudaSuccess) e = alloc_padded((void**)&h->block_colidx, sizeof(int32_t) * (size_t)nb, s);
  if (e == cudaSuccess) e = alloc_padded((void**)&h->block_masks, (size_t)nb * (size_t)h->mb, s);
  if (e == cudaSuccess) e = alloc_padded(&h->values, value_size(vt) * (size_t)nnz, s);
  if (e == cudaSuccess) e = alloc_padded((void**)&h->valptr, sizeof(int64_t) * (size_t)(I + 1), s);
  if (e != cudaSuccess)
    return bail(e == cudaErrorMemoryAllocation ? fail(SPC5_ENOMEM, "assemble: out of device memory")
                                               : cuda_fail(e, "assemble: allocation"));
  e = cudaMemcpyAsync(h->block_rowptr, brp_in, sizeof(int32_t) * (size_t)(I + 1), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && nb > 0)
    e = cudaMemcpyAsync(h->block_colidx, bcol_in, sizeof(int32_t) * (size_t)nb, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && nb > 0)
    e = cudaMemcpyAsync(h->block_masks, bmask_in, (size_t)nb * (size_t)h->mb, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(h->values, vals_in, value_size(vt) * (size_t)nnz, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "assemble: copy"));
  // 1. checks
  DeviceBuf status, cnt, bval, counts, nseg, segptr;
  e = status.alloc(sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status.p, 0xff, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cnt.alloc(sizeof(int32_t) * (size_t)(nb + 1), s);
  if (e == cudaSuccess) e = bval.alloc(sizeof(int32_t) * (size_t)(nb + 1), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "assemble: scratch"));
  unsigned long long* sw = (unsigned long long*)status.p;
  if (I > 0) k_asm_intervals<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(I, nb, h->block_rowptr, sw);
  unsigned long long st_host = ~0ull;
  e = cudaMemcpyAsync(&st_host, sw, sizeof(st_host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "assemble: checks"));
  if (st_host != ~0ull)
    return bail(fail(SPC5_EINVAL, "assemble: block_rowptr entry " + std::to_string(st_host >> 3) +
                                      " (must rise from 0 to n_blocks)"));
  if (nb > 0) {
    const unsigned g = (unsigned)((nb + 255) / 256);
    switch (r) {
      case 1: k_asm_blocks<1><<<g, 256, 0, s>>>(n, m, I, nb, c, h->mb, h->block_rowptr, h->block_colidx, h->block_masks, (int32_t*)cnt.p, sw); break;
      case 2: k_asm_blocks<2><<<g, 256, 0, s>>>(n, m, I, nb, c, h->mb, h->block_rowptr, h->block_colidx, h->block_masks, (int32_t*)cnt.p, sw); break;
      case 4: k_asm_blocks<4><<<g, 256, 0, s>>>(n, m, I, nb, c, h->mb, h->block_rowptr, h->block_colidx, h->block_masks, (int32_t*)cnt.p, sw); break;
      default: k_asm_blocks<8><<<g, 256, 0, s>>>(n, m, I, nb, c, h->mb, h->block_rowptr, h->block_colidx, h->block_masks, (int32_t*)cnt.p, sw); break;
    }
  }
  e = cudaMemcpyAsync(&st_host, sw, sizeof(st_host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "assemble: checks"));
  if (st_host != ~0ull) {
    const int code = (int)(st_host & 7ull);
    const std::string what = code == SPC5_ERANGE ? "a column or row outside the matrix"
                                                 : "overlaps or precedes the previous block of its interval";
    return bail(fail((spc5_status)code, "assemble: block " + std::to_string(st_host >> 3) + ": " + what));
  }
  // 2. value offsets
  int64_t total = 0;
  spc5_status st = scan_counts((const int32_t*)cnt.p, nb, (int32_t*)bval.p, &total, s);
  if (st != SPC5_OK) return bail(st);
  if (total != nnz)
    return bail(fail(SPC5_EINVAL, "assemble: the masks hold " + std::to_string(total) + " entries, nnz is " +
                                      std::to_string(nnz)));
  e = counts.alloc(sizeof(int32_t) * (size_t)(I + 1), s);
  if (e == cudaSuccess) e = nseg.alloc(sizeof(int32_t) * (size_t)(I + 1), s);
  if (e == cudaSuccess) e = segptr.alloc(sizeof(int32_t) * (size_t)(I + 1), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "assemble: scratch"));
  k_asm_valptr<<<(unsigned)((I + 1 + 255) / 256), 256, 0, s>>>(I, h->block_rowptr, (const int32_t*)bval.p, h->valptr,
                                                               (int32_t*)counts.p);
  // 3. long intervals (same thresholds as the conversion)
  if (user_long > 0) {
    h->long_blocks = user_long;
  } else {
    const double mean = I > 0 ? (double)nb / (double)I : 0.0;
    const double lim = 4.0 * mean;
    h->long_blocks = lim > kLongBlocks ? (lim < (double)INT_MAX ? (int32_t)lim : INT_MAX) : kLongBlocks;
  }
  if (opt && opt->long_values > 0) {
    h->long_values = opt->long_values;
  } else {
    const double mean_v = I > 0 ? (double)nnz / (double)I : 0.0;
    const double lv = 8.0 * mean_v;
    h->long_values = lv > 2048.0 * r ? (int64_t)lv : (int64_t)2048 * r;
  }
  int64_t ns = 0;
  if (I > 0)
    k_asm_segments<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(I, h->long_blocks, h->long_values, h->seg_blocks,
                                                               h->block_rowptr, (const int32_t*)bval.p, h->valptr,
                                                               (int32_t*)nseg.p);
  st = scan_counts((const int32_t*)nseg.p, I, (int32_t*)segptr.p, &ns, s);
  if (st != SPC5_OK) return bail(st);
  h->nseg = ns;
  e = alloc_padded((void**)&h->segs, sizeof(Segment) * (size_t)ns, s);
  if (e == cudaSuccess) e = alloc_padded(&h->partials, (vt == SPC5_F64 ? 8 : 4) * (size_t)ns * (size_t)r, s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "assemble: segments"));
  if (ns > 0) {
    k_asm_seg_fill<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(I, h->seg_blocks, h->block_rowptr,
                                                               (const int32_t*)bval.p, (const int32_t*)segptr.p,
                                                               h->segs);
    int32_t* flag = (int32_t*)counts.p;
    int32_t* pos = (int32_t*)nseg.p;
    k_long_flags<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(I, (const int32_t*)segptr.p, flag);
    int64_t nlong = 0;
    st = scan_counts(flag, I, pos, &nlong, s);
    if (st != SPC5_OK) return bail(st);
    e = alloc_padded((void**)&h->seg_first, sizeof(int32_t) * (size_t)nlong, s);
    if (e == cudaSuccess) {
      k_seg_first<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(I, (const int32_t*)segptr.p, flag, pos, h->seg_first);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "assemble: long-interval list"));
    h->nlong = nlong;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "assemble"));
  if (ordered_variant(h->variant)) {
    spc5_status st2 = build_order(h, s);
    if (st2 != SPC5_OK) return bail(st2);
  }
  if (uses_single_bits(h->variant)) {
    spc5_status st2 = build_single_bits(h, s);
    if (st2 != SPC5_OK) return bail(st2);
  }
  *out = h;
  return SPC5_OK;
}

spc5_status convert_impl(int64_t n, int64_t m, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                         const void* values, spc5_dtype vt, int r, int c, const spc5_opts* opt, cudaStream_t s,
                         spc5_matrix** out) {
  *out = nullptr;
  spc5_matrix* h = new spc5_matrix();
  h->arena_stream = s;  // failures free the arrays in this stream's order
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
  e = status.alloc(sizeof(unsigned long long), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: status word"));
  e = cudaMemsetAsync(status.p, 0xff, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: status word"));
  if (n > 0) {
    k_validate_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nnz, rowptr, (unsigned long long*)status.p);
    const int64_t warps = (nnz + kValChunk - 1) / kValChunk;
    if (warps > 0)
      k_validate_cols<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(n, m, nnz, rowptr, colidx,
                                                                          (unsigned long long*)status.p);
  }
  // 2. count
  e = counts.alloc(sizeof(int32_t) * (size_t)(I + 1), s);
  if (e == cudaSuccess) e = nseg.alloc(sizeof(int32_t) * (size_t)(I + 1), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: counts"));
  unsigned long long st_host = ~0ull;
  e = cudaMemcpyAsync(&st_host, status.p, sizeof(st_host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && st_host != ~0ull) {
    // something is wrong: the row-by-row check names the first bad row and its code
    e = cudaMemsetAsync(status.p, 0xff, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
      k_validate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, m, nnz, rowptr, colidx, (unsigned long long*)status.p);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st_host, status.p, sizeof(st_host), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: validation"));
  if (st_host != ~0ull) {
    int code = (int)(st_host & 7ull);
    long long row = (long long)(st_host >> 3);
    const char* what = code == SPC5_EUNSORTED ? "columns out of order" : code == SPC5_EDUP ? "repeated column"
                       : code == SPC5_ERANGE  ? "column index out of range" : "bad row pointer";
    return bail(fail((spc5_status)code, std::string("convert: CSR row ") + std::to_string(row) + ": " + what));
  }
  e = alloc_padded((void**)&h->block_rowptr, sizeof(int32_t) * (size_t)(I + 1), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: block_rowptr"));
  int64_t nb = 0, ns = 0;
  spc5_status st = SPC5_OK;
  DeviceBuf marks, wcount, wprefix;  // r = 1: one block-start bit per entry, prefix of the word popcounts
  DeviceBuf hints;                   // rows of the entry chunks (r = 1 passes, r > 1 value pass)
  const int64_t eth = (nnz + kEntriesPerThread - 1) / kEntriesPerThread;
  const int64_t nwords = (nnz + 31) / 32;
  const int64_t nhint = (nnz + kHintChunk - 1) / kHintChunk;
  e = hints.alloc(sizeof(int64_t) * (size_t)(nhint + 2), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: row hints"));
  if (eth > 0) k_row_hints<<<(unsigned)((nhint + 1 + 255) / 256), 256, 0, s>>>(n, nnz, rowptr, (int64_t*)hints.p);
  if (r == 1) {
    e = marks.alloc(sizeof(uint32_t) * (size_t)(nwords + 1), s);
    if (e == cudaSuccess) e = wcount.alloc(sizeof(int32_t) * (size_t)(nwords + 1), s);
    if (e == cudaSuccess) e = wprefix.alloc(sizeof(int32_t) * (size_t)(nwords + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(marks.p, 0, sizeof(uint32_t) * (size_t)(nwords + 1), s);
    if (e != cudaSuccess)
      return bail(e == cudaErrorMemoryAllocation ? fail(SPC5_ENOMEM, "convert: out of device memory")
                                                 : cuda_fail(e, "convert: block marks"));
    if (eth > 0) {
      k_r1_flags<<<(unsigned)((eth + 255) / 256), 256, 0, s>>>(n, nnz, c, rowptr, colidx, (const int64_t*)hints.p,
                                                               (uint32_t*)marks.p);
    }
    if (nwords > 0)
      k_mark_counts<<<(unsigned)((nwords + 255) / 256), 256, 0, s>>>(nwords, (const uint32_t*)marks.p,
                                                                     (int32_t*)wcount.p);
    st = scan_counts((const int32_t*)wcount.p, nwords, (int32_t*)wprefix.p, &nb, s);
    if (st != SPC5_OK) return bail(st);
    if (n > 0)
      k_r1_rowptr<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(n, rowptr, nwords, (const uint32_t*)marks.p,
                                                                  (const int32_t*)wprefix.p, h->block_rowptr,
                                                                  (int32_t*)counts.p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(cuda_fail(e, "convert: block numbering"));
  } else {
    // 3. count, then scan
    count_r(r, n, I, c, rowptr, colidx, (int32_t*)counts.p, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(cuda_fail(e, "convert: count kernel"));
    st = scan_counts((const int32_t*)counts.p, I, h->block_rowptr, &nb, s);
    if (st != SPC5_OK) return bail(st);
  }
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
  if (opt && opt->long_values > 0) {
    h->long_values = opt->long_values;
  } else {
    // an interval is also long when it holds many more values than the mean
    const double mean_v = I > 0 ? (double)nnz / (double)I : 0.0;
    const double lv = 8.0 * mean_v;
    h->long_values = lv > 2048.0 * r ? (int64_t)lv : (int64_t)2048 * r;
  }
  if (I > 0)
    k_nseg<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(n, I, r, h->long_blocks, h->long_values, h->seg_blocks,
                                                      (const int32_t*)counts.p, rowptr, (int32_t*)nseg.p);
  DeviceBuf segptr;
  e = segptr.alloc(sizeof(int32_t) * (size_t)(I + 1), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "convert: segment pointers"));
  st = scan_counts((const int32_t*)nseg.p, I, (int32_t*)segptr.p, &ns, s);
  if (st != SPC5_OK) return bail(st);
  h->nb = nb;
  h->nseg = ns;

  // 4. arrays + fill
  e = alloc_arena(h, nb, nnz, ns, s);
  if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? fail(SPC5_ENOMEM, "convert: out of device memory")
                                                                    : cuda_fail(e, "convert: allocation"));
  const int32_t* sp = ns > 0 ? (const int32_t*)segptr.p : nullptr;
  if (r == 1) {
    if (eth > 0)
    {
      auto fill = [&](auto w) {
        using W = decltype(w);
        k_r1_fill<W><<<(unsigned)((eth + 255) / 256), 256, 0, s>>>(
            n, nnz, c, h->mb, h->seg_blocks, rowptr, colidx, (const int64_t*)hints.p, static_cast<const W*>(values),
            static_cast<W*>(h->values), nwords, (const uint32_t*)marks.p, (const int32_t*)wprefix.p,
            h->block_rowptr, sp, h->block_colidx, h->block_masks, h->segs);
      };
      switch (vt) {
        case SPC5_F64: fill(uint64_t{}); break;
        case SPC5_F32: fill(uint32_t{}); break;
        default: fill(uint16_t{}); break;
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(cuda_fail(e, "convert: fill"));
  } else {
    DeviceBuf bvo;  // value offset of each block inside its interval
    e = bvo.alloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1), s);
    if (e != cudaSuccess)
      return bail(e == cudaErrorMemoryAllocation ? fail(SPC5_ENOMEM, "convert: out of device memory")
                                                 : cuda_fail(e, "convert: block offsets"));
    launch_fill_r(r, n, I, c, h->mb, h->seg_blocks, rowptr, colidx, h->block_rowptr, sp, (int32_t*)bvo.p, h, s);
    switch (vt) {
      case SPC5_F64: launch_fill_values<uint64_t>(r, n, nnz, c, h->mb, rowptr, colidx, (const int64_t*)hints.p, values, (const int32_t*)bvo.p, h, s); break;
      case SPC5_F32: launch_fill_values<uint32_t>(r, n, nnz, c, h->mb, rowptr, colidx, (const int64_t*)hints.p, values, (const int32_t*)bvo.p, h, s); break;
      default: launch_fill_values<uint16_t>(r, n, nnz, c, h->mb, rowptr, colidx, (const int64_t*)hints.p, values, (const int32_t*)bvo.p, h, s); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(cuda_fail(e, "convert: fill"));
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
  if (uses_single_bits(h->variant)) {
    spc5_status st2 = build_single_bits(h, s);
    if (st2 != SPC5_OK) return bail(st2);
  }
  *out = h;
  return SPC5_OK;
}

}  // namespace spc5
