// SM partitions for serving: a CUDA green context owns a subset of the SMs, and kernels launched
// on a stream created from it run only on those SMs. A server gives its small graphs a partition
// of their own, so their short round kernels never wait for SM room held by the persistent round
// kernels of large graphs (stream priority orders waiting CTAs but does not preempt running ones).
// The driver's green-context calls are resolved through the runtime's driver entry points, so
// the library needs no link dependency on the driver API.
#include <cuda.h>
#include <new>

#include "alb_internal.cuh"

struct alb_partition_s {
  CUgreenCtx gc = nullptr;
  uint32_t sms = 0;
  int device = 0;
};

namespace {

using PfnDeviceGet = CUresult (*)(CUdevice*, int);
using PfnGetDevResource = CUresult (*)(CUdevice, CUdevResource*, CUdevResourceType);
using PfnSplitByCount = CUresult (*)(CUdevResource*, unsigned int*, const CUdevResource*, CUdevResource*,
                                     unsigned int, unsigned int);
using PfnGenerateDesc = CUresult (*)(CUdevResourceDesc*, CUdevResource*, unsigned int);
using PfnGreenCtxCreate = CUresult (*)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned int);
using PfnGreenCtxDestroy = CUresult (*)(CUgreenCtx);
using PfnGreenCtxStreamCreate = CUresult (*)(CUstream*, CUgreenCtx, unsigned int, int);

struct Driver {
  PfnDeviceGet device_get = nullptr;
  PfnGetDevResource get_dev_resource = nullptr;
  PfnSplitByCount split_by_count = nullptr;
  PfnGenerateDesc generate_desc = nullptr;
  PfnGreenCtxCreate green_create = nullptr;
  PfnGreenCtxDestroy green_destroy = nullptr;
  PfnGreenCtxStreamCreate green_stream_create = nullptr;
  bool ok = false;
};

template <class F>
bool entry(const char* name, F* fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  // the ABI versions of the declarations this file is compiled against
  if (cudaGetDriverEntryPointByVersion(name, &p, CUDART_VERSION, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *fn = reinterpret_cast<F>(p);
  return true;
}

const Driver& driver() {
  static const Driver d = [] {
    Driver x;
    x.ok = entry("cuDeviceGet", &x.device_get) && entry("cuDeviceGetDevResource", &x.get_dev_resource) &&
           entry("cuDevSmResourceSplitByCount", &x.split_by_count) &&
           entry("cuDevResourceGenerateDesc", &x.generate_desc) && entry("cuGreenCtxCreate", &x.green_create) &&
           entry("cuGreenCtxDestroy", &x.green_destroy) &&
           entry("cuGreenCtxStreamCreate", &x.green_stream_create);
    return x;
  }();
  return d;
}

alb_status make_partition(const Driver& d, CUdevice dev, int device, CUdevResource* res, alb_partition* out) {
  CUdevResourceDesc desc = nullptr;
  if (d.generate_desc(&desc, res, 1) != CUDA_SUCCESS) return ALB_ERR_CUDA;
  alb_partition p = new (std::nothrow) alb_partition_s();
  if (!p) return ALB_ERR_OOM;
  if (d.green_create(&p->gc, desc, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) {
    delete p;
    return ALB_ERR_CUDA;
  }
  p->sms = res->sm.smCount;
  p->device = device;
  *out = p;
  return ALB_OK;
}

}  // namespace

extern "C" alb_status alb_partition_split(int device, uint32_t sm_count, alb_partition* first,
                                          alb_partition* rest) {
  if (!first || !rest || sm_count == 0) return ALB_ERR_INVALID_ARG;
  *first = *rest = nullptr;
  if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) return ALB_ERR_CUDA;
  const Driver& d = driver();
  if (!d.ok) return ALB_ERR_UNSUPPORTED;
  CUdevice dev;
  if (d.device_get(&dev, device) != CUDA_SUCCESS) return ALB_ERR_CUDA;
  CUdevResource all{}, part{}, rem{};
  if (d.get_dev_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return ALB_ERR_UNSUPPORTED;
  if (sm_count >= all.sm.smCount) return ALB_ERR_INVALID_ARG;
  unsigned int groups = 1;
  if (d.split_by_count(&part, &groups, &all, &rem, 0, sm_count) != CUDA_SUCCESS) return ALB_ERR_INVALID_ARG;
  if (groups != 1 || part.sm.smCount == 0 || rem.sm.smCount == 0) return ALB_ERR_INVALID_ARG;
  alb_status rc = make_partition(d, dev, device, &part, first);
  if (rc != ALB_OK) return rc;
  rc = make_partition(d, dev, device, &rem, rest);
  if (rc != ALB_OK) {
    alb_partition_destroy(*first);
    *first = nullptr;
  }
  return rc;
}

extern "C" alb_status alb_partition_sms(alb_partition p, uint32_t* sms) {
  if (!p || !sms) return ALB_ERR_INVALID_ARG;
  *sms = p->sms;
  return ALB_OK;
}

extern "C" alb_status alb_partition_stream_create(alb_partition p, int priority, alb_stream* out) {
  if (!p || !out) return ALB_ERR_INVALID_ARG;
  *out = nullptr;
  const Driver& d = driver();
  if (!d.ok) return ALB_ERR_UNSUPPORTED;
  CUstream s = nullptr;
  if (d.green_stream_create(&s, p->gc, CU_STREAM_NON_BLOCKING, priority) != CUDA_SUCCESS) return ALB_ERR_CUDA;
  *out = (alb_stream)s;
  return ALB_OK;
}

extern "C" alb_status alb_partition_stream_destroy(alb_stream s) {
  if (!s) return ALB_ERR_INVALID_ARG;
  return cudaStreamDestroy((cudaStream_t)s) == cudaSuccess ? ALB_OK : ALB_ERR_CUDA;
}

extern "C" alb_status alb_partition_destroy(alb_partition p) {
  if (!p) return ALB_ERR_INVALID_ARG;
  const Driver& d = driver();
  alb_status rc = ALB_OK;
  if (p->gc && (!d.ok || d.green_destroy(p->gc) != CUDA_SUCCESS)) rc = ALB_ERR_CUDA;
  delete p;
  return rc;
}
