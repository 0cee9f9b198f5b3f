// SM partitions: streams whose kernels run on a fixed group of SMs (green
// contexts of the CUDA driver). They give the single-GPU analogue of the
// paper's weak-scaling experiment (Sec. 6: the work per processor held fixed
// while processors are added): a problem of P work units advanced on a
// partition of P SM groups.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <new>

#include "../../include/amrmhd.h"

namespace {

struct SmPartition {
  CUgreenCtx green = nullptr;
  CUstream stream = nullptr;
};

// The driver functions, resolved through the runtime (the library does not
// link the driver library, so it loads on machines without one).
struct Driver {
  CUresult (*device_get)(CUdevice*, int) = nullptr;
  CUresult (*get_dev_resource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*split_by_count)(CUdevResource*, unsigned int*, const CUdevResource*, CUdevResource*, unsigned int,
                             unsigned int) = nullptr;
  CUresult (*generate_desc)(CUdevResourceDesc*, CUdevResource*, unsigned int) = nullptr;
  CUresult (*green_create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned int) = nullptr;
  CUresult (*green_destroy)(CUgreenCtx) = nullptr;
  CUresult (*green_stream_create)(CUstream*, CUgreenCtx, unsigned int, int) = nullptr;
  CUresult (*stream_sync)(CUstream) = nullptr;
  CUresult (*stream_destroy)(CUstream) = nullptr;
  bool ok = false;
};

// the last failure of a partition call (step and code), for the caller's report
thread_local char g_err[160] = "";
void set_err(const char* what, int code) { snprintf(g_err, sizeof(g_err), "%s failed (code %d)", what, code); }

template <class F> bool entry(const char* name, F& fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  const cudaError_t e = cudaGetDriverEntryPointByVersion(name, &p, CUDART_VERSION, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
    snprintf(g_err, sizeof(g_err), "driver entry point %s not found (runtime %d, query %d)", name, (int)e, (int)q);
    return false;
  }
  fn = reinterpret_cast<F>(p);
  return true;
}

const Driver& driver() {
  static const Driver d = [] {
    Driver r;
    r.ok = entry("cuDeviceGet", r.device_get) && entry("cuDeviceGetDevResource", r.get_dev_resource) &&
           entry("cuDevSmResourceSplitByCount", r.split_by_count) &&
           entry("cuDevResourceGenerateDesc", r.generate_desc) && entry("cuGreenCtxCreate", r.green_create) &&
           entry("cuGreenCtxDestroy", r.green_destroy) && entry("cuGreenCtxStreamCreate", r.green_stream_create) &&
           entry("cuStreamSynchronize", r.stream_sync) && entry("cuStreamDestroy", r.stream_destroy);
    return r;
  }();
  return d;
}

}  // namespace

extern "C" amrmhd_status amrmhd_sm_partition_create(int32_t sm_count, void** stream, int32_t* sms, void** handle) {
  if (sm_count < 1 || !stream || !sms || !handle) return AMRMHD_EINVAL;
  *stream = nullptr;
  *handle = nullptr;
  // the runtime's primary context of the current device must exist first
  if (cudaFree(nullptr) != cudaSuccess) { set_err("cudaFree(0)", 0); return AMRMHD_ECUDA; }
  const Driver& D = driver();
  if (!D.ok) return AMRMHD_ECUDA;
  int dev_index = 0;
  if (cudaGetDevice(&dev_index) != cudaSuccess) { set_err("cudaGetDevice", 0); return AMRMHD_ECUDA; }
  CUdevice dev;
  CUresult r = D.device_get(&dev, dev_index);
  if (r != CUDA_SUCCESS) { set_err("cuDeviceGet", (int)r); return AMRMHD_ECUDA; }
  CUdevResource all;
  r = D.get_dev_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM);
  if (r != CUDA_SUCCESS) { set_err("cuDeviceGetDevResource", (int)r); return AMRMHD_ECUDA; }
  if ((unsigned)sm_count > all.sm.smCount) { set_err("SM count above the device's", (int)all.sm.smCount); return AMRMHD_EINVAL; }
  // one group of at least sm_count SMs (rounded up to the device's granularity)
  CUdevResource part, rest;
  unsigned int groups = 1;
  r = D.split_by_count(&part, &groups, &all, &rest, 0, (unsigned)sm_count);
  if (r != CUDA_SUCCESS || groups != 1) { set_err("cuDevSmResourceSplitByCount", (int)r); return AMRMHD_EINVAL; }
  CUdevResourceDesc desc;
  r = D.generate_desc(&desc, &part, 1);
  if (r != CUDA_SUCCESS) { set_err("cuDevResourceGenerateDesc", (int)r); return AMRMHD_ECUDA; }
  SmPartition* p = new (std::nothrow) SmPartition();
  if (!p) return AMRMHD_ENOMEM;
  r = D.green_create(&p->green, desc, dev, CU_GREEN_CTX_DEFAULT_STREAM);
  if (r != CUDA_SUCCESS) {
    set_err("cuGreenCtxCreate", (int)r);
    delete p;
    return AMRMHD_ECUDA;
  }
  r = D.green_stream_create(&p->stream, p->green, CU_STREAM_NON_BLOCKING, 0);
  if (r != CUDA_SUCCESS) {
    set_err("cuGreenCtxStreamCreate", (int)r);
    D.green_destroy(p->green);
    delete p;
    return AMRMHD_ECUDA;
  }
  *sms = (int32_t)part.sm.smCount;
  *stream = (void*)p->stream;
  *handle = (void*)p;
  return AMRMHD_OK;
}

extern "C" const char* amrmhd_sm_partition_error(void) { return g_err; }

extern "C" amrmhd_status amrmhd_sm_partition_destroy(void* handle) {
  if (!handle) return AMRMHD_EINVAL;
  SmPartition* p = (SmPartition*)handle;
  const Driver& D = driver();
  if (!D.ok) return AMRMHD_ECUDA;
  amrmhd_status st = AMRMHD_OK;
  if (p->stream && (D.stream_sync(p->stream) != CUDA_SUCCESS || D.stream_destroy(p->stream) != CUDA_SUCCESS))
    st = AMRMHD_ECUDA;
  if (p->green && D.green_destroy(p->green) != CUDA_SUCCESS) st = AMRMHD_ECUDA;
  delete p;
  return st;
}
