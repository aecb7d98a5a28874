// Autotuner for the load-balancing knobs: the huge-vertex threshold (Sec. 4.1 "Threshold"; the
// paper finds a wide flat range, Sec. 5.1 "Analyzing Threshold") and the TWC bin cut-offs.
// Coordinate search timed on the device: first the threshold over powers of 4 plus the paper's
// rule (threads of the LB kernel) and "never huge", then the CTA and warp cut-offs at the best
// threshold, then the round kernels' CTA size (128, 256, 512; Sec. 5.1 uses 2^8 threads). The
// fastest setting is left applied to that application on the handle.
#include <cfloat>
#include <vector>

#include "alb_device.cuh"

namespace alb {

static alb_status run_app(alb_graph g, alb_app app, uint32_t src, void* out, double* l1, uint32_t* it,
                          cudaStream_t s) {
  switch (app) {
    case ALB_APP_BFS: return alb_bfs(g, src, static_cast<uint32_t*>(out), s);
    case ALB_APP_SSSP: return alb_sssp(g, src, static_cast<uint32_t*>(out), s);
    case ALB_APP_CC: return alb_cc(g, static_cast<uint32_t*>(out), s);
    case ALB_APP_KCORE: return alb_kcore(g, 32u, static_cast<uint32_t*>(out), s);
    case ALB_APP_PAGERANK:
      return alb_pagerank(g, 0.85f, 1e-6, 1000u, static_cast<float*>(out), l1, it, s);
  }
  return ALB_ERR_INVALID_ARG;
}

// Mean device time of `reps` calls after one untimed call (which also builds the cached graph).
static alb_status time_app(alb_graph g, alb_app app, uint32_t src, void* out, double* l1, uint32_t* it,
                           uint32_t reps, cudaStream_t s, float* ms) {
  alb_status rc = run_app(g, app, src, out, l1, it, s);
  if (rc != ALB_OK) return rc;
  cudaEvent_t a, b;
  ALB_CUDA_TRY(cudaEventCreate(&a));
  ALB_CUDA_TRY(cudaEventCreate(&b));
  cudaEventRecord(a, s);
  for (uint32_t i = 0; i < reps && rc == ALB_OK; ++i) rc = run_app(g, app, src, out, l1, it, s);
  cudaEventRecord(b, s);
  cudaError_t e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != ALB_OK) return rc;
  if (e != cudaSuccess) return ALB_ERR_CUDA;
  rc = alb_sync(g);
  if (rc != ALB_OK) return rc;
  *ms = t / (float)(reps ? reps : 1);
  return ALB_OK;
}

}  // namespace alb

using namespace alb;

extern "C" alb_status alb_autotune(alb_graph g, alb_app app, uint32_t src, uint32_t reps,
                                   alb_params* best, float* best_ms, alb_stream stream) {
  if (!g || app < ALB_APP_BFS || app > ALB_APP_KCORE || reps == 0) return ALB_ERR_INVALID_ARG;
  if ((app == ALB_APP_BFS || app == ALB_APP_SSSP) && src >= g->n) return ALB_ERR_INVALID_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  void* out = nullptr;
  double* l1 = nullptr;
  uint32_t* it = nullptr;
  ALB_CUDA_TRY(cudaMalloc(&out, sizeof(uint32_t) * (size_t)g->n));
  if (cudaMalloc((void**)&l1, sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&it, sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(out);
    cudaFree(l1);
    return ALB_ERR_OOM;
  }
  alb_params start;
  alb_get_app_params(g, app, &start);
  alb_params cur = start, top = start;
  float top_ms = FLT_MAX;
  alb_status rc = ALB_OK;
  auto trial = [&](const alb_params& p) -> alb_status {
    alb_status r = alb_set_app_params(g, app, &p);
    if (r != ALB_OK) return r;
    float ms = 0.f;
    r = time_app(g, app, src, out, l1, it, reps, s, &ms);
    if (r != ALB_OK) return r;
    if (ms < top_ms) {
      top_ms = ms;
      top = p;
    }
    return ALB_OK;
  };
  // 1) threshold: the paper's rule, powers of 4 from 2^8 to 2^20, and "never huge" (TWC only)
  std::vector<int64_t> ts = {-1};
  for (int k = 8; k <= 20; k += 2) ts.push_back(int64_t(1) << k);
  ts.push_back(int64_t(1) << 40);
  for (int64_t t : ts) {
    cur = start;
    cur.hub_threshold = t;
    if ((rc = trial(cur)) != ALB_OK) break;
  }
  // 2) TWC cut-offs at the best threshold
  if (rc == ALB_OK) {
    const alb_params at = top;
    const uint32_t ctas[] = {128u, 256u, 512u, 1024u};
    const uint32_t warps[] = {16u, 32u, 64u};
    for (uint32_t cm : ctas) {
      for (uint32_t wm : warps) {
        if (wm > cm || (cm == at.twc_cta_min && wm == at.twc_warp_min)) continue;
        cur = at;
        cur.twc_cta_min = cm;
        cur.twc_warp_min = wm;
        if ((rc = trial(cur)) != ALB_OK) break;
      }
      if (rc != ALB_OK) break;
    }
  }
  // 3) CTA size of the round kernels at the best threshold and cut-offs (PageRank's kernels have
  //    a fixed CTA size)
  if (rc == ALB_OK && app != ALB_APP_PAGERANK) {
    const alb_params at = top;
    const uint32_t at_b = at.block_size ? at.block_size : (uint32_t)kBlock;
    for (uint32_t b : {128u, 256u, 512u}) {
      if (b == at_b) continue;
      cur = at;
      cur.block_size = b;
      if ((rc = trial(cur)) != ALB_OK) break;
    }
  }
  cudaFree(out);
  cudaFree(l1);
  cudaFree(it);
  alb_status rc2 = alb_set_app_params(g, app, rc == ALB_OK ? &top : &start);
  if (rc != ALB_OK) return rc;
  if (rc2 != ALB_OK) return rc2;
  if (best) *best = top;
  if (best_ms) *best_ms = top_ms;
  return ALB_OK;
}
