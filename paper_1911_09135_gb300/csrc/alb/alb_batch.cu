// Batched traversals: many sources over one graph.
#include "alb_device.cuh"

struct BatchWs {
  int unused = 0;
};

namespace alb {

alb_status free_batch(alb_graph g) {
  delete g->batch;
  g->batch = nullptr;
  return ALB_OK;
}

alb_status batch_stats(alb_graph, alb_stats*) { return ALB_OK; }

static alb_status run_batch(alb_graph g, App app, const uint32_t* hd_srcs, uint32_t k, uint32_t* out,
                            cudaStream_t s) {
  uint32_t* srcs = nullptr;
  bool own = false;
  if (is_device_ptr(hd_srcs)) {
    srcs = (uint32_t*)std::malloc(sizeof(uint32_t) * (k ? k : 1));
    own = true;
    ALB_CUDA_TRY(cudaMemcpy(srcs, hd_srcs, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
  } else {
    srcs = const_cast<uint32_t*>(hd_srcs);
  }
  alb_status rc = ALB_OK;
  for (uint32_t i = 0; i < k && rc == ALB_OK; ++i)
    if (srcs[i] >= g->n) rc = ALB_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < k && rc == ALB_OK; ++i)
    rc = run_traversal(g, app, srcs[i], 0u, out + (size_t)i * g->n, s);
  if (own) std::free(srcs);
  return rc;
}

}  // namespace alb

using namespace alb;

extern "C" alb_status alb_bfs_batch(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_out,
                                    alb_stream stream) {
  if (!g || (k && (!hd_srcs || !hd_out))) return ALB_ERR_INVALID_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  return run_batch(g, APP_BFS, hd_srcs, k, hd_out, (cudaStream_t)stream);
}

extern "C" alb_status alb_sssp_batch(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_out,
                                     alb_stream stream) {
  if (!g || (k && (!hd_srcs || !hd_out))) return ALB_ERR_INVALID_ARG;
  if (!g->has_w) return ALB_ERR_UNSUPPORTED;
  if ((uint64_t)g->max_w * (uint64_t)(g->n - 1) >= 0xFFFFFFFFull) return ALB_ERR_OVERFLOW;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  return run_batch(g, APP_SSSP, hd_srcs, k, hd_out, (cudaStream_t)stream);
}
