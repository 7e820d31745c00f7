// Batched SpMV: y_j = A_j x_j for many uneven matrices in one graph launch.
//
// Many small products launched one by one leave the GPU idle between tiny
// kernels. Here every short interval of every matrix belongs to a work item
// of 32/r consecutive intervals (one warp's worth, lane per row as in the
// single-matrix kernel). The items are grouped by (block shape, row decode):
// each matrix keeps its own shape and the decode of its tuned variant
// (chosen per matrix by spc5_tune or the caller's selector), and each group
// runs one kernel compiled for its shape and decode - one warp per item - so
// no group pays for the registers another decode needs. Long intervals are
// items of a second kind - one warp per segment, partials into the matrix's
// scratch - taken by persistent warps from a global counter (kGrab items per
// atomic), followed by one fix-up kernel over the long intervals. The group
// kernels and the segment kernel run on parallel branches (side streams
// joined by events); the whole product is captured once into a CUDA graph at
// batch creation, so a batched SpMV is one graph launch.
#include <algorithm>
#include <map>
#include <vector>

#include "spmv_beta.cuh"

namespace spc5 {
namespace {

struct MatDesc {  // one matrix of the batch (device copy)
  const int32_t* brp;
  const int32_t* bcol;
  const uint8_t* bmask;
  const void* val;
  const int64_t* valptr;
  const Segment* segs;
  void* partials;
  const void* x;
  void* y;
  const uint32_t* single;  // single-value class bits (variants 30 / 31), or NULL
  int64_t n, I, nseg, long_values;
  int32_t r, c, mb, long_blocks, log2r;
  int32_t dec;  // row decode of the matrix's tuned variant (see decode_of)
};

// items a warp takes per atomic on the shared counter: same-address atomics
// serialise (a few ns each), so one per 32-row item cost about a third of the
// batch on 256 matrices of ~3 M rows in total
constexpr int kGrab = 8;

// The decode of a matrix's short intervals, from its variant (the batch maps
// one lane to one row): 1 mask windows, 4 Algorithm 2's single-value test
// (r = 1: variants 30, 31 and the two-lane 33) with the mask windows for the
// other rows, 2 / 3 the unrolled bit positions one / two blocks per trip
// (variants 16/17, 18/19), 0 the flattened decode (variants 0-10).
inline int decode_of(int v, int r, int c, spc5_dtype vt) {
  if (v == 12 || v == 13 || v == 14 || v == 15) return 1;
  if ((v == 30 || v == 31 || v == 33) && r == 1) return 4;
  const int unrolled = c <= 8 ? 3 : 2;  // row_sum_e2 holds two blocks of at most 8 positions
  if (v == 16 || v == 17) return 2;
  if (v == 18 || v == 19) return unrolled;
  // the many-lane forms (two lanes per row, lanes per interval, the streaming
  // warp): the unrolled one-lane decode for the 4-byte types, the mask
  // windows for float64 (unrolled positions there cost float64 issue slots)
  if (v == 22 || v == 23 || (v >= 24 && v <= 29) || v == 32) return vt == SPC5_F64 ? 1 : unrolled;
  return 0;
}

struct Item {  // kind 0: intervals [i0, i0 + 32/r) of matrix mat; kind 1: segment i0 of mat
  int32_t mat;
  int32_t i0;
  int32_t kind;
  int32_t pad;
};

__device__ __forceinline__ uint32_t rb(const uint32_t (&w)[4], int p, int c) {
  return (w[p >> 5] >> (p & 31)) & ((1u << c) - 1u);
}

__device__ __forceinline__ int pb(const uint32_t (&w)[4], int p) {
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < (p >> 5)) cnt += __popc(w[q]);
  if (p & 31) cnt += __popc(w[p >> 5] & ((1u << (p & 31)) - 1u));
  return cnt;
}

__device__ __forceinline__ void ldmask(const uint8_t* __restrict__ m, int64_t b, int mb, uint32_t (&w)[4]) {
  w[0] = w[1] = w[2] = w[3] = 0u;
  switch (mb) {
    case 1: w[0] = __ldg(m + b); break;
    case 2: w[0] = __ldg(reinterpret_cast<const uint16_t*>(m) + b); break;
    case 4: w[0] = __ldg(reinterpret_cast<const uint32_t*>(m) + b); break;
    case 8: {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(m) + b);
      w[0] = v.x;
      w[1] = v.y;
      break;
    }
    default: {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(m) + b);
      w[0] = v.x;
      w[1] = v.y;
      w[2] = v.z;
      w[3] = v.w;
    }
  }
}

// one row of a short interval with the shape and decode known at compile time
template <int R, int C, class T, int DEC>
__device__ __forceinline__ typename T::A batch_row(const MatDesc& d, int64_t it, int i, int32_t b, int32_t bend,
                                                   int64_t v0) {
  const typename T::V* __restrict__ vrow = static_cast<const typename T::V*>(d.val) + v0;
  const typename T::X* __restrict__ x = static_cast<const typename T::X*>(d.x);
  if constexpr (DEC == 4) {
    if (d.single && ((__ldg(d.single + (it >> 5)) >> (it & 31)) & 1u)) {
      typename T::A acc = 0;
      const int32_t* __restrict__ crow = d.bcol + b;
      for (int32_t j = 0; j < bend - b; ++j) acc = fmadd<T>(T::val(vrow, j), T::xv(x, __ldg(crow + j)), acc);
      return acc;
    }
    return row_sum<R, C, T, 2, 1>(i, b, bend, vrow, d.bcol, d.bmask, x);
  } else {
    return row_sum<R, C, T, 2, DEC>(i, b, bend, vrow, d.bcol, d.bmask, x);
  }
}

// The unrolled-position decodes (2, 3) are left out here: with all twelve
// shapes inlined into the one persistent kernel they would set its register
// count (and occupancy) for every matrix; such matrices take the flattened
// decode in the batch.
template <int R, int C, class T>
__device__ __forceinline__ typename T::A batch_row_dec(const MatDesc& d, int64_t it, int i, int32_t b, int32_t bend,
                                                       int64_t v0) {
  if (d.dec == 1) return batch_row<R, C, T, 1>(d, it, i, b, bend, v0);
  if constexpr (R == 1)
    if (d.dec == 4) return batch_row<R, C, T, 4>(d, it, i, b, bend, v0);
  return batch_row<R, C, T, 0>(d, it, i, b, bend, v0);
}

template <class T>
__device__ __forceinline__ typename T::A batch_row_any(const MatDesc& d, int64_t it, int i, int32_t b, int32_t bend,
                                                       int64_t v0) {
#define SPC5_BCASE(RR, CC) \
  if (d.r == RR && d.c == CC) return batch_row_dec<RR, CC, T>(d, it, i, b, bend, v0);
  SPC5_BCASE(1, 4) SPC5_BCASE(1, 8) SPC5_BCASE(1, 16)
  SPC5_BCASE(2, 4) SPC5_BCASE(2, 8) SPC5_BCASE(2, 16)
  SPC5_BCASE(4, 4) SPC5_BCASE(4, 8) SPC5_BCASE(4, 16)
  SPC5_BCASE(8, 4) SPC5_BCASE(8, 8)
#undef SPC5_BCASE
  return batch_row_dec<8, 16, T>(d, it, i, b, bend, v0);
}

// One group: items of matrices with block shape R x C and row decode DEC,
// one warp per item (items[0 .. nitems) of this group).
template <class T, int R, int C, int DEC>
__global__ void __launch_bounds__(256) k_batch_rows(const MatDesc* __restrict__ mats, const Item* __restrict__ items,
                                                    int64_t nitems) {
  using X = typename T::X;
  using A = typename T::A;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nitems) return;  // whole warp
  const int lane = threadIdx.x & 31;
  const Item itm = items[w];
  const MatDesc& d = mats[itm.mat];
  const int64_t it = (int64_t)itm.i0 + lane / R;
  const int i = lane % R;
  if (it >= d.I) return;
  const int32_t b = __ldg(d.brp + it);
  const int32_t bend = __ldg(d.brp + it + 1);
  const int64_t v0 = __ldg(d.valptr + it);
  if (bend - b > d.long_blocks || __ldg(d.valptr + it + 1) - v0 > d.long_values) return;  // the segment path's
  const A acc = batch_row<R, C, T, DEC>(d, it, i, b, bend, v0);
  const int64_t row = it * R + i;
  if (row < d.n) static_cast<X*>(d.y)[row] = acc;
}

// launch of one group's kernel (shape and decode from the group's key)
template <class T>
cudaError_t launch_group(int r, int c, int dec, const MatDesc* mats, const Item* items, int64_t nitems,
                         cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const int threads = kSpmvThreads;
  const unsigned grid = (unsigned)((nitems * kWarp + threads - 1) / threads);
#define SPC5_GKERN(RR, CC, DD) k_batch_rows<T, RR, CC, DD><<<grid, threads, 0, s>>>(mats, items, nitems)
#define SPC5_GSHAPE(RR, CC)                                     \
  if (r == RR && c == CC) {                                     \
    if (dec == 1) {                                             \
      SPC5_GKERN(RR, CC, 1);                                    \
    } else if (dec == 2 || (dec == 3 && CC > 8)) {              \
      SPC5_GKERN(RR, CC, 2);                                    \
    } else if (dec == 3) {                                      \
      if constexpr (CC <= 8) SPC5_GKERN(RR, CC, 3);             \
    } else if (dec == 4) {                                      \
      if constexpr (RR == 1) SPC5_GKERN(RR, CC, 4);             \
      else SPC5_GKERN(RR, CC, 0);                               \
    } else {                                                    \
      SPC5_GKERN(RR, CC, 0);                                    \
    }                                                           \
    return cudaGetLastError();                                  \
  }
  SPC5_GSHAPE(1, 4) SPC5_GSHAPE(1, 8) SPC5_GSHAPE(1, 16)
  SPC5_GSHAPE(2, 4) SPC5_GSHAPE(2, 8) SPC5_GSHAPE(2, 16)
  SPC5_GSHAPE(4, 4) SPC5_GSHAPE(4, 8) SPC5_GSHAPE(4, 16)
  SPC5_GSHAPE(8, 4) SPC5_GSHAPE(8, 8) SPC5_GSHAPE(8, 16)
#undef SPC5_GSHAPE
#undef SPC5_GKERN
  return cudaErrorInvalidValue;
}

template <class T>
__global__ void __launch_bounds__(256) k_batch(const MatDesc* __restrict__ mats, const Item* __restrict__ items,
                                               int64_t nitems, unsigned long long* __restrict__ counter) {
  using V = typename T::V;
  using X = typename T::X;
  using A = typename T::A;
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long k0 = 0;
    if (lane == 0) k0 = atomicAdd(counter, (unsigned long long)kGrab);
    k0 = __shfl_sync(0xffffffffu, k0, 0);
    if (k0 >= (unsigned long long)nitems) break;
    const unsigned long long kend = k0 + kGrab < (unsigned long long)nitems ? k0 + kGrab : nitems;
    for (unsigned long long k = k0; k < kend; ++k) {
    const Item itm = items[k];
    const MatDesc& d = mats[itm.mat];
    const int r = d.r, c = d.c, mb = d.mb;
    const V* __restrict__ val = static_cast<const V*>(d.val);
    const X* __restrict__ x = static_cast<const X*>(d.x);
    if (itm.kind == 0) {
      const int64_t it = (int64_t)itm.i0 + (lane >> d.log2r);
      const int i = lane & (r - 1);
      if (it >= d.I) continue;
      const int32_t b = __ldg(d.brp + it);
      const int32_t bend = __ldg(d.brp + it + 1);
      const int64_t v0 = __ldg(d.valptr + it);
      if (bend - b > d.long_blocks || __ldg(d.valptr + it + 1) - v0 > d.long_values) continue;
      const A acc = batch_row_any<T>(d, it, i, b, bend, v0);
      const int64_t row = it * r + i;
      if (row < d.n) static_cast<X*>(d.y)[row] = acc;
    } else {
      // one warp per segment, cut into 32/r contiguous runs, lane = (run,
      // row), the same sums in the same order as k_spmv_segments
      const Segment sg = d.segs[itm.i0];
      const int S = kWarp >> d.log2r;
      const int slot = lane >> d.log2r, i = lane & (r - 1);
      const int32_t per = (sg.b_end - sg.b_begin + S - 1) / S;
      const int32_t rb0 = min(sg.b_begin + slot * per, sg.b_end);
      const int32_t re = min(rb0 + per, sg.b_end);
      int cnt = 0;
      for (int32_t b = rb0 + i; b < re; b += r) {
        uint32_t w[4];
        ldmask(d.bmask, b, mb, w);
        cnt += __popc(w[0]) + __popc(w[1]) + __popc(w[2]) + __popc(w[3]);
      }
      for (int dd = 1; dd < r; dd <<= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, dd);
      int incl = cnt;
      for (int dd = r; dd < kWarp; dd <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= dd) incl += t;
      }
      const V* __restrict__ vrun = val + sg.v_begin + (incl - cnt);
      A acc = 0;
      int32_t vbase = 0;
      for (int32_t b = rb0; b < re; ++b) {
        uint32_t w[4];
        ldmask(d.bmask, b, mb, w);
        uint32_t bits = rb(w, i * c, c);
        int32_t vo = vbase + pb(w, i * c);
        vbase += __popc(w[0]) + __popc(w[1]) + __popc(w[2]) + __popc(w[3]);
        if (!bits) continue;
        const int64_t col0 = __ldg(d.bcol + b);
        while (bits) {
          const int kb = __ffs(bits) - 1;
          bits &= bits - 1;
          acc = fma(T::val(vrun, vo++), T::xv(x, col0 + kb), acc);
        }
      }
      for (int dd = kWarp / 2; dd >= r; dd >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, dd);
      if (lane < r) static_cast<A*>(d.partials)[(int64_t)itm.i0 * r + lane] = acc;
    }
    }
  }
}

// one lane per long interval (matrix, first segment), long lists by the whole
// warp: the summation order of k_spmv_fixup
template <class T>
__global__ void __launch_bounds__(256) k_batch_fixup(const MatDesc* __restrict__ mats, const int2* __restrict__ firsts,
                                                     int64_t nfirst) {
  using X = typename T::X;
  using A = typename T::A;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >= nfirst) return;  // whole warp
  const bool have = e < nfirst;
  const int2 f = have ? firsts[e] : make_int2(0, 0);  // (matrix, first segment of the interval)
  const MatDesc& d = mats[f.x];
  const int32_t count = have ? d.segs[f.y].count : 0;
  const int32_t it = have ? d.segs[f.y].interval : 0;
  fixup_lane_interval<A, X, false>(have, f.y, count, it, d.r, d.n, static_cast<const A*>(d.partials),
                                   static_cast<X*>(d.y));
  unsigned big = __ballot_sync(0xffffffffu, have && count > kFixupSerial);
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const MatDesc& db = mats[__shfl_sync(0xffffffffu, f.x, src)];
    fixup_warp_interval<A, X, false>(__shfl_sync(0xffffffffu, f.y, src), __shfl_sync(0xffffffffu, count, src),
                                     __shfl_sync(0xffffffffu, it, src), db.r, db.n,
                                     static_cast<const A*>(db.partials), static_cast<X*>(db.y));
  }
}

}  // namespace
}  // namespace spc5

namespace spc5 {
namespace {
constexpr int kSide = 4;  // side streams the group kernels are spread over
struct Group {  // the items of one (block shape, decode): items_d[off .. off + cnt)
  int r, c, dec;
  int64_t off, cnt;
};
}  // namespace
}  // namespace spc5

struct spc5_batch_s {
  spc5_dtype vt = SPC5_F32;
  int count = 0;
  int64_t nitems = 0, nfirst = 0;
  int64_t seg_off = 0, nseg_items = 0;  // the segment items: items_d[seg_off .. seg_off + nseg_items)
  std::vector<spc5::Group> groups;
  spc5::MatDesc* mats_d = nullptr;
  spc5::Item* items_d = nullptr;
  int2* firsts_d = nullptr;  // (matrix, first segment) of every long interval
  unsigned long long* counter_d = nullptr;
  cudaStream_t side[spc5::kSide] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[spc5::kSide] = {};
  cudaGraphExec_t exec = nullptr;
  int blocks = 0;
};

namespace spc5 {

static void batch_free(spc5_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int q = 0; q < kSide; ++q) {
    if (b->side[q]) cudaStreamDestroy(b->side[q]);
    if (b->ev_join[q]) cudaEventDestroy(b->ev_join[q]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  cudaFree(b->mats_d);
  cudaFree(b->items_d);
  cudaFree(b->firsts_d);
  cudaFree(b->counter_d);
  delete b;
}

// the segments (persistent kernel, then the fix-up) on s, the groups on the
// side streams, forked from and joined back into s
template <class T>
cudaError_t batch_enqueue(spc5_batch_s* b, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->ev_fork, s);
  for (int q = 0; q < kSide && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(b->side[q], b->ev_fork, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counter_d, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (b->nseg_items > 0)
    k_batch<T><<<b->blocks, 256, 0, s>>>(b->mats_d, b->items_d + b->seg_off, b->nseg_items, b->counter_d);
  if (b->nfirst > 0)
    k_batch_fixup<T><<<(unsigned)((b->nfirst + 255) / 256), 256, 0, s>>>(b->mats_d, b->firsts_d, b->nfirst);
  e = cudaGetLastError();
  for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g) {
    const Group& gr = b->groups[g];
    e = launch_group<T>(gr.r, gr.c, gr.dec, b->mats_d, b->items_d + gr.off, gr.cnt, b->side[g % kSide]);
  }
  for (int q = 0; q < kSide && e == cudaSuccess; ++q) {
    e = cudaEventRecord(b->ev_join[q], b->side[q]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[q], 0);
  }
  return e;
}

cudaError_t batch_enqueue_any(spc5_batch_s* b, cudaStream_t s) {
  switch (b->vt) {
    case SPC5_F64: return batch_enqueue<F64>(b, s);
    case SPC5_F32: return batch_enqueue<F32>(b, s);
    default: return batch_enqueue<BF16>(b, s);
  }
}

spc5_status batch_create_impl(const spc5_handle* mats, const void* const* xs, void* const* ys, int count,
                              spc5_batch_s** out) {
  spc5_batch_s* b = new spc5_batch_s();
  b->count = count;
  b->vt = mats[0]->vt;
  std::vector<MatDesc> md((size_t)count);
  std::vector<Item> items, seg_items;
  std::map<int, std::vector<Item>> by_key;  // (r, c, decode) -> short-interval items
  std::vector<int2> firsts;
  std::vector<Segment> hsegs;
  for (int j = 0; j < count; ++j) {
    const spc5_matrix* h = mats[j];
    if (h->vt != b->vt) {
      batch_free(b);
      return fail(SPC5_EINVAL, "batch: all matrices must have the same value type");
    }
    MatDesc& d = md[(size_t)j];
    d.brp = h->block_rowptr;
    d.bcol = h->block_colidx;
    d.bmask = h->block_masks;
    d.val = h->values;
    d.valptr = h->valptr;
    d.segs = h->segs;
    d.partials = h->partials;
    d.x = xs[j];
    d.y = ys[j];
    d.n = h->n;
    d.I = h->I;
    d.nseg = h->nseg;
    d.long_values = h->long_values;
    d.r = h->r;
    d.c = h->c;
    d.mb = h->mb;
    d.long_blocks = h->long_blocks;
    d.log2r = h->r == 1 ? 0 : h->r == 2 ? 1 : h->r == 4 ? 2 : 3;
    d.dec = decode_of(h->variant, h->r, h->c, h->vt);
    d.single = d.dec == 4 ? h->single_bits : nullptr;
    const int S = kWarp / h->r;
    auto& list = by_key[(h->r * 32 + h->c) * 8 + d.dec];
    for (int64_t i0 = 0; i0 < h->I; i0 += S) list.push_back(Item{j, (int32_t)i0, 0, 0});
    if (h->nseg > 0) {
      hsegs.resize((size_t)h->nseg);
      cudaError_t e = cudaMemcpy(hsegs.data(), h->segs, sizeof(Segment) * (size_t)h->nseg, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch: segment table");
      }
    }
    for (int64_t q = 0; q < h->nseg; ++q) seg_items.push_back(Item{j, (int32_t)q, 1, 0});
    for (int64_t q = 0; q < h->nseg; ++q)
      if (hsegs[(size_t)q].count > 0) firsts.push_back(make_int2(j, (int)q));
  }
  // groups, largest first (the side streams start on the big ones), then the segments
  std::vector<std::pair<int, std::vector<Item>*>> keys;
  for (auto& kv : by_key) keys.push_back({kv.first, &kv.second});
  std::stable_sort(keys.begin(), keys.end(),
                   [](const auto& a, const auto& c) { return a.second->size() > c.second->size(); });
  for (auto& kv : keys) {
    const int key = kv.first;
    b->groups.push_back(Group{key / 256, (key / 8) % 32, key % 8, (int64_t)items.size(), (int64_t)kv.second->size()});
    items.insert(items.end(), kv.second->begin(), kv.second->end());
  }
  b->seg_off = (int64_t)items.size();
  b->nseg_items = (int64_t)seg_items.size();
  items.insert(items.end(), seg_items.begin(), seg_items.end());
  b->nitems = (int64_t)items.size();
  b->nfirst = (int64_t)firsts.size();
  cudaError_t e = cudaMalloc((void**)&b->mats_d, sizeof(MatDesc) * (size_t)count);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->items_d, sizeof(Item) * (items.size() + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->firsts_d, sizeof(int2) * (firsts.size() + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->counter_d, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpy(b->mats_d, md.data(), sizeof(MatDesc) * (size_t)count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(b->items_d, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !firsts.empty())
    e = cudaMemcpy(b->firsts_d, firsts.data(), sizeof(int2) * firsts.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "batch: descriptors");
  }
  // persistent grid: the CTAs resident at once (at most one item per warp)
  int per_sm = 8;
  {
    int v = 0;
    cudaError_t oe;
    switch (b->vt) {
      case SPC5_F64: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_batch<F64>, 256, 0); break;
      case SPC5_F32: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_batch<F32>, 256, 0); break;
      default: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_batch<BF16>, 256, 0); break;
    }
    if (oe == cudaSuccess && v > 0) per_sm = v;
  }
  int64_t blocks = (int64_t)sm_count() * per_sm;
  const int64_t need = (b->nseg_items + 8 * kGrab - 1) / (8 * kGrab);
  if (blocks > need) blocks = need > 0 ? need : 1;
  b->blocks = (int)blocks;
  for (int q = 0; q < kSide && e == cudaSuccess; ++q) {
    e = cudaStreamCreateWithFlags(&b->side[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "batch: streams");
  }
  // capture the whole batched product once; replays reuse it
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = batch_enqueue_any(b, cs);
    e = cudaStreamEndCapture(cs, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "batch: graph");
  }
  *out = b;
  return SPC5_OK;
}

}  // namespace spc5

using namespace spc5;

extern "C" {

spc5_status spc5_batch_create(const spc5_handle* mats, const void* const* x_d, void* const* y_d, int count,
                              spc5_batch* out) {
  if (!out) return fail(SPC5_EINVAL, "batch_create: NULL output");
  *out = nullptr;
  if (count < 1 || !mats || !x_d || !y_d) return fail(SPC5_EINVAL, "batch_create: empty batch or NULL array");
  for (int j = 0; j < count; ++j) {
    if (!mats[j]) return fail(SPC5_EINVAL, "batch_create: NULL handle");
    if ((mats[j]->m > 0 && !x_d[j]) || (mats[j]->n > 0 && !y_d[j])) return fail(SPC5_EINVAL, "batch_create: NULL vector");
    if (mats[j]->I > INT32_MAX || mats[j]->nseg > INT32_MAX / 8) return fail(SPC5_ERANGE, "batch_create: matrix too large");
  }
  spc5_batch_s* b = nullptr;
  spc5_status st = batch_create_impl(mats, x_d, y_d, count, &b);
  if (st != SPC5_OK) return st;
  *out = b;
  return SPC5_OK;
}

spc5_status spc5_batch_spmv(spc5_batch b, spc5_stream_t stream) {
  if (!b) return fail(SPC5_EINVAL, "batch_spmv: NULL batch");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch_spmv: graph launch");
  return SPC5_OK;
}

spc5_status spc5_batch_spmv_direct(spc5_batch b, spc5_stream_t stream) {
  if (!b) return fail(SPC5_EINVAL, "batch_spmv_direct: NULL batch");
  cudaError_t e = batch_enqueue_any(b, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch_spmv_direct: launch");
  return SPC5_OK;
}

spc5_status spc5_batch_destroy(spc5_batch b) {
  if (!b) return SPC5_OK;
  cudaError_t e = cudaDeviceSynchronize();
  batch_free(b);
  if (e != cudaSuccess) return cuda_fail(e, "batch_destroy: device synchronisation");
  return SPC5_OK;
}

}  // extern "C"
