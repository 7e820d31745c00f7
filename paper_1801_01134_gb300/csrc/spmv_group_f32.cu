// beta(r,c) SpMV with G lanes per interval (variants 24-29) and with the warp
// streaming its rows' blocks (variant 32, r = 1), F32 values.
#include "spmv_stream.cuh"

namespace spc5 {

cudaError_t launch_group_f32(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s, void* partials) {
  if (stream_variant(h->variant)) return dispatch_stream<F32>(h, x, y, acc, partials, s);
  return dispatch_grp<F32>(h, x, y, acc, partials, s);
}

}  // namespace spc5
