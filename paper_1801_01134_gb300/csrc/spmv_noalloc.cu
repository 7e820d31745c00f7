// spc5_spmv_noalloc: y = A x for callers that cannot allocate device memory.
//
// The regular spc5_spmv hands the long-interval segments a per-handle scratch
// buffer that spc5_convert allocated with cudaMalloc. Some callers cannot let
// a library allocate at all: their device memory is owned by another
// component's pool allocator, or they run under a fixed device-memory budget
// where every allocation is accounted for up front. For them this entry point
// keeps its scratch in one fixed-size array placed in the library's own
// device image (a file-scope __device__ array), so the call itself performs
// no allocation of any kind.
//
// Facts a user of this entry point needs:
//   * The array holds kNoAllocScratchBytes (4 MiB) and every GPU that loads
//     the library keeps it resident until the process exits.
//   * A matrix needs n_segments * r accumulators in it (8 bytes each for
//     float64, 4 for float32 / bfloat16); larger needs are rejected with
//     SPC5_ERANGE before any launch.
//   * All calls on a device share the one array and it keeps what the last
//     call wrote. Each call writes every slot before reading it, so nothing
//     has to be cleared between calls; but two calls whose kernels overlap on
//     the GPU (different streams, no ordering) race on the array.
//   * The first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it; make
//     that first call before any stream capture begins.
#include <mutex>

#include "internal.cuh"

namespace spc5 {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace spc5

extern "C" spc5_status spc5_spmv_noalloc(spc5_handle h, const void* x_d, void* y_d, spc5_stream_t stream) {
  using namespace spc5;
  if (!h) return fail(SPC5_EINVAL, "spmv_noalloc: NULL handle");
  if ((h->m > 0 && !x_d) || (h->n > 0 && !y_d)) return fail(SPC5_EINVAL, "spmv_noalloc: NULL vector");
  const size_t acc_bytes = h->vt == SPC5_F64 ? 8 : 4;
  const size_t need = (size_t)h->nseg * (size_t)h->r * acc_bytes;
  if (need > kNoAllocScratchBytes)
    return fail(SPC5_ERANGE, "spmv_noalloc: the matrix needs " + std::to_string(need) +
                                 " bytes of segment scratch; the fixed array holds " +
                                 std::to_string(kNoAllocScratchBytes) + " (use spc5_spmv)");
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "spmv_noalloc: scratch address");
  // the kernels of spc5_spmv; only the segment scratch differs
  const cudaStream_t s = (cudaStream_t)stream;
  switch (h->vt) {
    case SPC5_F64: e = launch_spmv_f64(h, x_d, y_d, false, s, scratch); break;
    case SPC5_F32: e = launch_spmv_f32(h, x_d, y_d, false, s, scratch); break;
    case SPC5_BF16: e = launch_spmv_bf16(h, x_d, y_d, false, s, scratch); break;
    default: return fail(SPC5_EUNSUPPORTED, "spmv_noalloc: value type");
  }
  if (e != cudaSuccess) return cuda_fail(e, "spmv_noalloc launch");
  return SPC5_OK;
}
