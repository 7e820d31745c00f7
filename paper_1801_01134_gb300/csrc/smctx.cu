// SM-limited streams: the GPU form of the paper's thread-count axis.
//
// The paper's parallel predictor records each kernel's performance for several
// numbers of threads and interpolates over (threads, Avg) (section
// "Performance prediction and optimal kernel selection", parallel part). On one
// GPU the matching axis is the number of SMs a product may use. A green
// context owns a partition of the SMs (a process-local partition of this
// context's work; it changes no device setting); kernels launched into a
// stream of that context run on its SMs only. spc5_sm_stream_create returns
// such a stream for a requested SM count, so that every library call
// (spc5_spmv, spc5_time_formats, ...) can run on a part of the GPU.
//
// The driver entry points are taken through cudaGetDriverEntryPointByVersion,
// so the library needs no link-time dependency on the driver library.
#include <cuda.h>

#include <map>
#include <mutex>

#include "internal.cuh"

namespace spc5 {
namespace {

using PFN_GetDevResource = CUresult (*)(CUdevice, CUdevResource*, CUdevResourceType);
using PFN_SmSplit = CUresult (*)(CUdevResource*, unsigned int*, const CUdevResource*, CUdevResource*, unsigned int,
                                 unsigned int);
using PFN_GenDesc = CUresult (*)(CUdevResourceDesc*, CUdevResource*, unsigned int);
using PFN_GreenCreate = CUresult (*)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned int);
using PFN_GreenDestroy = CUresult (*)(CUgreenCtx);
using PFN_GreenStream = CUresult (*)(CUstream*, CUgreenCtx, unsigned int, int);
using PFN_StreamDestroy = CUresult (*)(CUstream);
using PFN_DeviceGet = CUresult (*)(CUdevice*, int);

struct Driver {
  PFN_GetDevResource get_res = nullptr;
  PFN_SmSplit split = nullptr;
  PFN_GenDesc gen_desc = nullptr;
  PFN_GreenCreate green_create = nullptr;
  PFN_GreenDestroy green_destroy = nullptr;
  PFN_GreenStream green_stream = nullptr;
  PFN_StreamDestroy stream_destroy = nullptr;
  PFN_DeviceGet device_get = nullptr;
  bool ok = false;
};

std::mutex g_sm_mu;
Driver g_drv;
bool g_drv_tried = false;
struct SmStream {
  CUgreenCtx ctx;
  int sms;
};
std::map<cudaStream_t, SmStream> g_streams;

template <class F>
bool entry(const char* name, F* fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12080, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p)
    return false;
  *fn = reinterpret_cast<F>(p);
  return true;
}

bool load_driver() {
  if (g_drv_tried) return g_drv.ok;
  g_drv_tried = true;
  Driver d;
  d.ok = entry("cuDeviceGetDevResource", &d.get_res) && entry("cuDevSmResourceSplitByCount", &d.split) &&
         entry("cuDevResourceGenerateDesc", &d.gen_desc) && entry("cuGreenCtxCreate", &d.green_create) &&
         entry("cuGreenCtxDestroy", &d.green_destroy) && entry("cuGreenCtxStreamCreate", &d.green_stream) &&
         entry("cuStreamDestroy", &d.stream_destroy) && entry("cuDeviceGet", &d.device_get);
  g_drv = d;
  return d.ok;
}

spc5_status drv_fail(CUresult r, const char* what) {
  return fail(r == CUDA_ERROR_NOT_SUPPORTED ? SPC5_EUNSUPPORTED : SPC5_ECUDA,
              std::string(what) + ": driver error " + std::to_string((int)r));
}

}  // namespace
}  // namespace spc5

using namespace spc5;

extern "C" {

spc5_status spc5_sm_stream_create(int sms, spc5_stream_t* stream_out, int* sms_out) {
  if (!stream_out) return fail(SPC5_EINVAL, "sm_stream_create: NULL output");
  *stream_out = nullptr;
  if (sms < 1) return fail(SPC5_EINVAL, "sm_stream_create: sms < 1");
  std::lock_guard<std::mutex> lock(g_sm_mu);
  if (!load_driver()) return fail(SPC5_EUNSUPPORTED, "sm_stream_create: green contexts not available");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaFree(nullptr);  // the primary context exists before the green one
  if (e != cudaSuccess) return cuda_fail(e, "sm_stream_create");
  CUdevice cudev;
  CUresult r = g_drv.device_get(&cudev, dev);
  if (r != CUDA_SUCCESS) return drv_fail(r, "sm_stream_create: device");
  CUdevResource full{}, part{};
  r = g_drv.get_res(cudev, &full, CU_DEV_RESOURCE_TYPE_SM);
  if (r != CUDA_SUCCESS) return drv_fail(r, "sm_stream_create: SM resource");
  if ((unsigned)sms >= full.sm.smCount) {
    part = full;  // the whole GPU
  } else {
    unsigned int groups = 1;
    r = g_drv.split(&part, &groups, &full, nullptr, 0, (unsigned)sms);
    if (r != CUDA_SUCCESS || groups < 1) return drv_fail(r, "sm_stream_create: split");
  }
  CUdevResourceDesc desc;
  r = g_drv.gen_desc(&desc, &part, 1);
  if (r != CUDA_SUCCESS) return drv_fail(r, "sm_stream_create: descriptor");
  CUgreenCtx g;
  r = g_drv.green_create(&g, desc, cudev, CU_GREEN_CTX_DEFAULT_STREAM);
  if (r != CUDA_SUCCESS) return drv_fail(r, "sm_stream_create: green context");
  CUstream st;
  r = g_drv.green_stream(&st, g, CU_STREAM_NON_BLOCKING, 0);
  if (r != CUDA_SUCCESS) {
    g_drv.green_destroy(g);
    return drv_fail(r, "sm_stream_create: stream");
  }
  g_streams[(cudaStream_t)st] = SmStream{g, (int)part.sm.smCount};
  *stream_out = (spc5_stream_t)st;
  if (sms_out) *sms_out = (int)part.sm.smCount;
  return SPC5_OK;
}

spc5_status spc5_sm_stream_destroy(spc5_stream_t stream) {
  if (!stream) return SPC5_OK;
  std::lock_guard<std::mutex> lock(g_sm_mu);
  auto it = g_streams.find((cudaStream_t)stream);
  if (it == g_streams.end()) return fail(SPC5_EINVAL, "sm_stream_destroy: not a stream of spc5_sm_stream_create");
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  g_drv.stream_destroy((CUstream)stream);
  g_drv.green_destroy(it->second.ctx);
  g_streams.erase(it);
  if (e != cudaSuccess) return cuda_fail(e, "sm_stream_destroy: synchronisation");
  return SPC5_OK;
}

}  // extern "C"
