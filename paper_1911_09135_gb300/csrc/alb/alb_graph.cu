// Graph handles, parameters, statistics and the thin C ABI wrappers of
// include/alb.h (argument checks, host/device staging of buffers).
#include <cstring>
#include <new>

#include "alb_device.cuh"

namespace alb {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

alb_status setup_barrier() {
  ALB_CUDA_TRY(cudaDeviceSynchronize());
  return ALB_OK;
}

alb_status ensure_tmp(alb_graph g) {
  if (!g->tmp) {
    alb_status rc = setup_barrier();
    if (rc != ALB_OK) return rc;
    ALB_CUDA_TRY(cudaMalloc((void**)&g->tmp, sizeof(uint32_t) * (size_t)g->n));
  }
  return ALB_OK;
}

uint32_t effective_threshold(alb_graph g) { return g->threshold; }

struct ScanOut {
  uint32_t max_deg;
  uint32_t max_w;
  uint32_t bad;  // non-monotone offsets or index >= n
  uint32_t off0;
  uint32_t offn;
};

// One pass over the CSR: maximum degree and weight, and range checks, so that
// every later kernel may index with the graph's entries unchecked.
__global__ void k_scan_graph(const uint32_t* off, const uint32_t* idx, const uint32_t* w,
                             uint32_t n, uint64_t m, ScanOut* out) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t md = 0, mw = 0, bad = 0;
  for (uint64_t v = tid; v < n; v += stride) {
    const uint32_t a = off[v], b = off[v + 1];
    if (b < a) bad = 1;
    else md = max(md, b - a);
  }
  for (uint64_t e = tid; e < m; e += stride) {
    if (idx[e] >= n) bad = 1;
    if (w) mw = max(mw, w[e]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    md = max(md, __shfl_down_sync(kFull, md, o));
    mw = max(mw, __shfl_down_sync(kFull, mw, o));
    bad |= __shfl_down_sync(kFull, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (md) atomicMax(&out->max_deg, md);
    if (mw) atomicMax(&out->max_w, mw);
    if (bad) atomicOr(&out->bad, 1u);
  }
  if (tid == 0) {
    out->off0 = off[0];
    out->offn = off[n];
  }
}

static void free_graph_memory(alb_graph g) {
  if (!g->csr_refs || g->csr_refs->fetch_sub(1) == 1) {
    cudaFree(g->off);
    cudaFree(g->idx);
    cudaFree(g->w);
    delete g->csr_refs;
  }
  g->csr_refs = nullptr;
  cudaFree(g->F0);
  cudaFree(g->F1);
  cudaFree(g->hub_v);
  cudaFree(g->hub_p);
  cudaFree(g->pushed);
  cudaFree(g->tmp);
  cudaFree(g->st);
  cudaFree(g->args);
  cudaFree(g->chk);
  cudaFree(g->cta_twc);
  cudaFree(g->cta_lb);
  if (g->h_st) cudaFreeHost(g->h_st);
  cudaGetLastError();
}

// Launch configuration of application `app` for parameters p.
// Per-handle round workspace (two frontiers, huge worklist + prefix, push bitmaps, state).
static alb_status alloc_workspace(alb_graph g) {
  const size_t nb = sizeof(uint32_t) * (size_t)g->n;
  cudaError_t e = cudaMalloc((void**)&g->F0, nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->F1, nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->hub_v, nb + sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->hub_p, nb + sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->pushed, sizeof(uint32_t) * 2 * (((size_t)g->n + 31) / 32 + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->st, sizeof(RoundState));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->args, sizeof(CallArgs));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&g->h_st, sizeof(RoundState));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->chk, 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(g->chk, 0, 4 * sizeof(uint32_t));
  // the memset runs on the legacy stream, which callers' non-blocking streams do not wait for
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? ALB_ERR_OOM : ALB_ERR_CUDA;
  }
  return ALB_OK;
}

static void apply_launch_config(alb_graph g, int app, const alb_params& p) {
  alb_graph_s::AppCfg& c = g->cfg[app];
  c.p = p;
  c.block = p.block_size ? p.block_size : (uint32_t)kBlock;
  uint32_t occ_i = 1, occ_l = 1;
  occupancy(c.block, &occ_i, &occ_l);
  if (p.grid_blocks) {
    c.blocks = c.lb_blocks = p.grid_blocks;
  } else {
    c.blocks = (uint32_t)g->num_sms * occ_i;
    c.lb_blocks = (uint32_t)g->num_sms * occ_l;
  }
  if (p.hub_threshold < 0) c.threshold = c.lb_blocks * c.block;
  else c.threshold = p.hub_threshold > 0xFFFFFFFFll ? 0xFFFFFFFFu : (uint32_t)p.hub_threshold;
}

void select_cfg(alb_graph g, int app) {
  const alb_graph_s::AppCfg& c = g->cfg[app];
  g->params = c.p;
  g->blocks = c.blocks;
  g->lb_blocks = c.lb_blocks;
  g->threshold = c.threshold;
  g->block = c.block;
}

alb_status reset_cta_loads(alb_graph g, cudaStream_t s, uint32_t min_need) {
  // counters are sized for the largest grid any application of the handle may use
  uint32_t need = min_need;
  for (int a = 0; a < 5; ++a) {
    need = g->cfg[a].blocks > need ? g->cfg[a].blocks : need;
    need = g->cfg[a].lb_blocks > need ? g->cfg[a].lb_blocks : need;
  }
  need = need < 4096u ? 4096u : need;
  if (g->cta_cap < need) {
    // cached graphs hold the counters' addresses: drop them all before the arrays move
    ALB_CUDA_TRY(cudaDeviceSynchronize());
    free_traversal_graphs(g);
    free_pagerank(g);
    free_batch(g);
    cudaFree(g->cta_twc);
    cudaFree(g->cta_lb);
    g->cta_twc = g->cta_lb = nullptr;
    g->cta_cap = 0;
    ALB_CUDA_TRY(cudaMalloc((void**)&g->cta_twc, sizeof(unsigned long long) * need));
    ALB_CUDA_TRY(cudaMalloc((void**)&g->cta_lb, sizeof(unsigned long long) * need));
    g->cta_cap = need;
  }
  ALB_CUDA_TRY(cudaMemsetAsync(g->cta_twc, 0, sizeof(unsigned long long) * g->cta_cap, s));
  ALB_CUDA_TRY(cudaMemsetAsync(g->cta_lb, 0, sizeof(unsigned long long) * g->cta_cap, s));
  g->cta_n_twc = g->blocks;
  g->cta_n_lb = g->lb_blocks;
  return ALB_OK;
}

alb_status latch_from_state(alb_graph g, uint32_t status) {
  if (status & ST_ERR_SRC) g->latched = ALB_ERR_INVALID_ARG;
  else if (status & ST_ERR_INDEX) g->latched = ALB_ERR_DEVICE;
  else if (status & ST_ERR_ROUNDS) g->latched = ALB_ERR_TIMEOUT;
  return g->latched;
}

}  // namespace alb

using namespace alb;

extern "C" {

uint32_t alb_version(void) { return 10000u; }

uint32_t alb_checked_build(void) {
#ifdef ALB_CHECKED
  return 1u;
#else
  return 0u;
#endif
}

alb_status alb_get_cta_loads(alb_graph g, uint64_t* hd_twc, uint64_t* hd_lb, uint32_t cap,
                             uint32_t* n_twc, uint32_t* n_lb) {
  if (!g || !n_twc || !n_lb) return ALB_ERR_INVALID_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  ALB_CUDA_TRY(cudaStreamSynchronize(g->last_stream));
  *n_twc = g->cta_twc ? g->cta_n_twc : 0u;
  *n_lb = g->cta_lb ? g->cta_n_lb : 0u;
  if (hd_twc && *n_twc)
    ALB_CUDA_TRY(cudaMemcpy(hd_twc, g->cta_twc, sizeof(uint64_t) * (cap < *n_twc ? cap : *n_twc), cudaMemcpyDefault));
  if (hd_lb && *n_lb)
    ALB_CUDA_TRY(cudaMemcpy(hd_lb, g->cta_lb, sizeof(uint64_t) * (cap < *n_lb ? cap : *n_lb), cudaMemcpyDefault));
  return ALB_OK;
}

alb_status alb_debug_check(alb_graph g, uint32_t* out4) {
  if (!g || !out4) return ALB_ERR_INVALID_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  ALB_CUDA_TRY(cudaStreamSynchronize(g->last_stream));
  ALB_CUDA_TRY(cudaMemcpy(out4, g->chk, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return ALB_OK;
}

const char* alb_status_str(alb_status s) {
  switch (s) {
    case ALB_OK: return "ALB_OK";
    case ALB_ERR_INVALID_ARG: return "ALB_ERR_INVALID_ARG";
    case ALB_ERR_OOM: return "ALB_ERR_OOM";
    case ALB_ERR_CUDA: return "ALB_ERR_CUDA";
    case ALB_ERR_TIMEOUT: return "ALB_ERR_TIMEOUT";
    case ALB_ERR_OVERFLOW: return "ALB_ERR_OVERFLOW";
    case ALB_ERR_NOT_SYMMETRIC: return "ALB_ERR_NOT_SYMMETRIC";
    case ALB_ERR_UNSUPPORTED: return "ALB_ERR_UNSUPPORTED";
    case ALB_ERR_DEVICE: return "ALB_ERR_DEVICE";
  }
  return "ALB_ERR_UNKNOWN";
}

uint32_t alb_threshold_rule(uint32_t num_sms, uint32_t threads_per_sm) {
  const uint64_t t = (uint64_t)num_sms * threads_per_sm;
  return t > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)t;
}

alb_status alb_default_params(alb_params* p) {
  if (!p) return ALB_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->hub_threshold = -1;
  p->twc_warp_min = 32;
  p->twc_cta_min = (uint32_t)kBlock;
  p->grid_blocks = 0;
  p->distribution = 0;
  p->exec_mode = 0;
  p->max_rounds = 0;
  p->l2_persist_fraction = 0.f;
  p->profile = 0;
  p->block_size = (uint32_t)kBlock;
  return ALB_OK;
}

static bool params_valid(const alb_params* p) {
  if (p->distribution > 1 || p->exec_mode > 1 || p->profile > 1 || p->cta_stats > 1) return false;
  if (p->block_size != 0 && p->block_size != 128 && p->block_size != 256 && p->block_size != 512) return false;
  if (p->twc_warp_min > p->twc_cta_min) return false;
  if (p->grid_blocks > (1u << 20)) return false;
  if (!(p->l2_persist_fraction >= 0.f && p->l2_persist_fraction <= 1.f)) return false;
  return true;
}

alb_status alb_graph_create(uint32_t n, uint64_t m, const uint32_t* hd_offsets,
                            const uint32_t* hd_indices, const uint32_t* hd_weights,
                            uint32_t flags, alb_stream stream, alb_graph* out) {
  if (!out) return ALB_ERR_INVALID_ARG;
  *out = nullptr;
  if (n == 0 || n == 0xFFFFFFFFu || !hd_offsets || (m > 0 && !hd_indices)) return ALB_ERR_INVALID_ARG;
  if (m >= 0xFFFFFFFFull) return ALB_ERR_OVERFLOW;
  if (flags & ~(ALB_SYMMETRIC | ALB_VALIDATE)) return ALB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  alb_graph g = new (std::nothrow) alb_graph_s();
  if (!g) return ALB_ERR_OOM;
  auto fail = [&](alb_status rc) {
    free_graph_memory(g);
    delete g;
    return rc;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess) return fail(ALB_ERR_CUDA);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
    return fail(ALB_ERR_CUDA);
  g->num_sms = sms;
  g->n = n;
  g->m = m;
  g->flags = flags;
  g->has_w = hd_weights != nullptr || m == 0;  // a graph without edges has nothing to weigh
  const size_t nb = sizeof(uint32_t) * (size_t)n;
  const size_t mb = sizeof(uint32_t) * (size_t)(m ? m : 1);
  g->csr_refs = new (std::nothrow) std::atomic<int>(1);
  if (!g->csr_refs) return fail(ALB_ERR_OOM);
  cudaError_t e = cudaSuccess;
  e = cudaMalloc((void**)&g->off, nb + sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->idx, mb);
  if (e == cudaSuccess && g->has_w) e = cudaMalloc((void**)&g->w, mb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? ALB_ERR_OOM : ALB_ERR_CUDA);
  }
  alb_status wrc = alloc_workspace(g);
  if (wrc != ALB_OK) return fail(wrc);
  e = cudaMemcpyAsync(g->off, hd_offsets, nb + sizeof(uint32_t), cudaMemcpyDefault, s);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(g->idx, hd_indices, sizeof(uint32_t) * m, cudaMemcpyDefault, s);
  if (e == cudaSuccess && hd_weights && m)
    e = cudaMemcpyAsync(g->w, hd_weights, sizeof(uint32_t) * m, cudaMemcpyDefault, s);
  ScanOut* d_scan = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_scan, sizeof(ScanOut), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_scan, 0, sizeof(ScanOut), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ALB_ERR_CUDA);
  }
  k_scan_graph<<<(unsigned)sms * 4, 256, 0, s>>>(g->off, g->idx, g->w, n, m, d_scan);
  ScanOut h{};
  e = cudaMemcpyAsync(&h, d_scan, sizeof(ScanOut), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d_scan, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ALB_ERR_CUDA);
  }
  if (h.off0 != 0u || (uint64_t)h.offn != m) return fail(ALB_ERR_INVALID_ARG);
  if (h.bad) return fail(ALB_ERR_DEVICE);
  g->max_deg = h.max_deg;
  g->max_w = h.max_w;
  alb_params dp;
  alb_default_params(&dp);
  for (int a = 0; a < 5; ++a) apply_launch_config(g, a, dp);
  select_cfg(g, ALB_APP_BFS);
  g->last_stream = s;
  *out = g;
  return ALB_OK;
}

alb_status alb_graph_clone(alb_graph src, alb_graph* out) {
  if (!src || !out) return ALB_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(src->device) != cudaSuccess) return ALB_ERR_CUDA;
  alb_graph g = new (std::nothrow) alb_graph_s();
  if (!g) return ALB_ERR_OOM;
  g->device = src->device;
  g->n = src->n;
  g->m = src->m;
  g->flags = src->flags;
  g->has_w = src->has_w;
  g->max_w = src->max_w;
  g->max_deg = src->max_deg;
  g->off = src->off;
  g->idx = src->idx;
  g->w = src->w;
  g->csr_refs = src->csr_refs;
  g->csr_refs->fetch_add(1);
  g->num_sms = src->num_sms;
  for (int a = 0; a < 5; ++a) g->cfg[a] = src->cfg[a];
  select_cfg(g, ALB_APP_BFS);
  alb_status rc = alloc_workspace(g);
  if (rc != ALB_OK) {
    free_graph_memory(g);
    delete g;
    return rc;
  }
  *out = g;
  return ALB_OK;
}

alb_status alb_graph_destroy(alb_graph g) {
  if (!g) return ALB_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  // the handle may have queued work on several streams; none may still use what is freed
  cudaDeviceSynchronize();
  free_traversal_graphs(g);
  free_pagerank(g);
  free_batch(g);
  free_graph_memory(g);
  delete g;
  return ALB_OK;
}

alb_status alb_graph_trim(alb_graph g, uint64_t* freed_bytes) {
  if (!g) return ALB_ERR_INVALID_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  size_t before = 0, after = 0, total = 0;
  // the handle's calls may still run on several streams: nothing may use what is freed
  ALB_CUDA_TRY(cudaDeviceSynchronize());
  ALB_CUDA_TRY(cudaMemGetInfo(&before, &total));
  free_traversal_graphs(g);
  free_pagerank(g);
  free_batch(g);
  cudaFree(g->tmp);
  g->tmp = nullptr;
  cudaGetLastError();
  ALB_CUDA_TRY(cudaMemGetInfo(&after, &total));
  if (freed_bytes) *freed_bytes = after > before ? (uint64_t)(after - before) : 0u;
  return ALB_OK;
}

alb_status alb_set_params(alb_graph g, const alb_params* p) {
  if (!g || !p || !params_valid(p)) return ALB_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();  // cached graphs and workspaces are freed below
  free_traversal_graphs(g);
  free_pagerank(g);
  free_batch(g);
  for (int a = 0; a < 5; ++a) apply_launch_config(g, a, *p);
  select_cfg(g, ALB_APP_BFS);
  return ALB_OK;
}

alb_status alb_get_params(alb_graph g, alb_params* p) {
  if (!g || !p) return ALB_ERR_INVALID_ARG;
  *p = g->cfg[ALB_APP_BFS].p;
  return ALB_OK;
}

alb_status alb_set_app_params(alb_graph g, alb_app app, const alb_params* p) {
  if (!g || !p || app < ALB_APP_BFS || app > ALB_APP_KCORE || !params_valid(p)) return ALB_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();  // cached graphs and workspaces are freed below
  // only the cached work of this application depends on its parameters
  switch (app) {
    case ALB_APP_PAGERANK: free_pagerank(g); break;
    case ALB_APP_BFS: case ALB_APP_SSSP: free_batch(g); [[fallthrough]];
    default: {
      const int internal = app == ALB_APP_BFS ? APP_BFS : app == ALB_APP_SSSP ? APP_SSSP
                         : app == ALB_APP_CC ? APP_CC : APP_KCORE;
      if (g->exec[internal]) cudaGraphExecDestroy(g->exec[internal]);
      if (g->graph[internal]) cudaGraphDestroy(g->graph[internal]);
      g->exec[internal] = nullptr;
      g->graph[internal] = nullptr;
      if (app == ALB_APP_BFS) {  // the diagnostics run with the bfs configuration
        if (g->exec[APP_TRACE]) cudaGraphExecDestroy(g->exec[APP_TRACE]);
        g->exec[APP_TRACE] = nullptr;
      }
    }
  }
  apply_launch_config(g, app, *p);
  return ALB_OK;
}

alb_status alb_get_app_params(alb_graph g, alb_app app, alb_params* p) {
  if (!g || !p || app < ALB_APP_BFS || app > ALB_APP_KCORE) return ALB_ERR_INVALID_ARG;
  *p = g->cfg[app].p;
  return ALB_OK;
}

alb_status alb_sync(alb_graph g) {
  if (!g) return ALB_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  ALB_CUDA_TRY(cudaStreamSynchronize(g->last_stream));
  if (g->last_kind == 0) {
    ALB_CUDA_TRY(cudaMemcpy(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost));
    latch_from_state(g, g->h_st->status);
  } else if (g->last_kind == 1) {
    alb_stats tmp{};
    pr_stats(g, &tmp);
  } else if (g->last_kind == 2) {
    alb_stats tmp{};
    batch_stats(g, &tmp);
  }
  const alb_status rw = batch_sync_workers(g);
  alb_status rc = g->latched != ALB_OK ? g->latched : rw;
  g->latched = ALB_OK;
  return rc;
}

alb_status alb_get_stats(alb_graph g, alb_stats* out) {
  if (!g || !out) return ALB_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  ALB_CUDA_TRY(cudaStreamSynchronize(g->last_stream));
  alb_stats s = g->stats;
  s.hub_threshold = g->threshold;
  s.lb_threads = g->lb_blocks * g->block;
  s.grid_blocks = g->blocks;
  s.block_size = g->block;
  if (g->last_kind == 0) {
    ALB_CUDA_TRY(cudaMemcpy(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost));
    const RoundState& h = *g->h_st;
    s.rounds = h.round;
    s.hub_rounds = h.hub_rounds;
    s.max_hub_count = h.max_hub_count;
    s.edges_twc = h.edges_twc;
    s.edges_lb = h.edges_lb;
    s.pushes = h.pushes;
    latch_from_state(g, h.status);
  } else if (g->last_kind == 1) {
    alb_status rc = pr_stats(g, &s);
    if (rc != ALB_OK) return rc;
  } else if (g->last_kind == 2) {
    alb_status rc = batch_stats(g, &s);
    if (rc != ALB_OK) return rc;
  }
  *out = s;
  alb_status rc = g->latched;
  g->latched = ALB_OK;
  return rc;
}

static alb_status begin_call(alb_graph g, int app) {
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  select_cfg(g, app);
  if (!g->params.cta_stats) g->cta_n_twc = g->cta_n_lb = 0;  // this call is not instrumented
  g->stats.ms_inspect = g->stats.ms_lb = g->stats.ms_other = 0.0;
  g->stats.n_inspect = g->stats.n_lb = g->stats.n_other = 0;
  return ALB_OK;
}

alb_status alb_bfs(alb_graph g, uint32_t src, uint32_t* hd_levels, alb_stream stream) {
  if (!g || !hd_levels || src >= g->n) return ALB_ERR_INVALID_ARG;
  alb_status rc = begin_call(g, ALB_APP_BFS);
  if (rc != ALB_OK) return rc;
  return run_traversal(g, APP_BFS, src, 0u, hd_levels, (cudaStream_t)stream);
}

alb_status alb_sssp(alb_graph g, uint32_t src, uint32_t* hd_dist, alb_stream stream) {
  if (!g || !hd_dist || src >= g->n) return ALB_ERR_INVALID_ARG;
  if (!g->has_w) return ALB_ERR_UNSUPPORTED;
  if ((uint64_t)g->max_w * (uint64_t)(g->n - 1) >= 0xFFFFFFFFull) return ALB_ERR_OVERFLOW;
  alb_status rc = begin_call(g, ALB_APP_SSSP);
  if (rc != ALB_OK) return rc;
  return run_traversal(g, APP_SSSP, src, 0u, hd_dist, (cudaStream_t)stream);
}

alb_status alb_cc(alb_graph g, uint32_t* hd_labels, alb_stream stream) {
  if (!g || !hd_labels) return ALB_ERR_INVALID_ARG;
  if (!(g->flags & ALB_SYMMETRIC)) return ALB_ERR_NOT_SYMMETRIC;
  alb_status rc = begin_call(g, ALB_APP_CC);
  if (rc != ALB_OK) return rc;
  return run_traversal(g, APP_CC, 0u, 0u, hd_labels, (cudaStream_t)stream);
}

alb_status alb_kcore(alb_graph g, uint32_t k, uint32_t* hd_in_core, alb_stream stream) {
  if (!g || !hd_in_core) return ALB_ERR_INVALID_ARG;
  if (!(g->flags & ALB_SYMMETRIC)) return ALB_ERR_NOT_SYMMETRIC;
  alb_status rc = begin_call(g, ALB_APP_KCORE);
  if (rc != ALB_OK) return rc;
  return run_traversal(g, APP_KCORE, 0u, k, hd_in_core, (cudaStream_t)stream);
}

// Diagnostics: stage host buffers through stream-ordered device allocations.
struct Staged {
  void* d = nullptr;
  void* h = nullptr;
  size_t bytes = 0;
  bool owned = false;
};

static alb_status stage_in(Staged& b, const void* p, size_t bytes, cudaStream_t s) {
  b.bytes = bytes;
  if (is_device_ptr(p)) { b.d = const_cast<void*>(p); return ALB_OK; }
  ALB_CUDA_TRY(cudaMallocAsync(&b.d, bytes ? bytes : 4, s));
  b.owned = true;
  if (bytes) ALB_CUDA_TRY(cudaMemcpyAsync(b.d, p, bytes, cudaMemcpyHostToDevice, s));
  return ALB_OK;
}

static alb_status stage_out(Staged& b, void* p, size_t bytes, cudaStream_t s) {
  b.bytes = bytes;
  if (is_device_ptr(p)) { b.d = p; return ALB_OK; }
  b.h = p;
  ALB_CUDA_TRY(cudaMallocAsync(&b.d, bytes ? bytes : 4, s));
  b.owned = true;
  return ALB_OK;
}

static void unstage(Staged& b, cudaStream_t s) {
  if (b.h && b.bytes) cudaMemcpyAsync(b.h, b.d, b.bytes, cudaMemcpyDeviceToHost, s);
  if (b.owned) cudaFreeAsync(b.d, s);
  b.owned = false;
}

alb_status alb_inspect(alb_graph g, const uint32_t* hd_wl, uint32_t nf, uint8_t* hd_bin,
                       uint32_t* hd_work, uint32_t* hd_prefix, uint32_t* hd_counts,
                       alb_stream stream) {
  if (!g || (nf && (!hd_wl || !hd_bin)) || !hd_work || !hd_prefix || !hd_counts)
    return ALB_ERR_INVALID_ARG;
  alb_status rc = begin_call(g, ALB_APP_BFS);
  if (rc != ALB_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  Staged wl, bin, work, prefix, counts;
  if ((rc = stage_in(wl, hd_wl, sizeof(uint32_t) * nf, s)) != ALB_OK) return rc;
  if ((rc = stage_out(bin, hd_bin, nf, s)) != ALB_OK) return rc;
  if ((rc = stage_out(work, hd_work, sizeof(uint32_t) * (nf + 1), s)) != ALB_OK) return rc;
  if ((rc = stage_out(prefix, hd_prefix, sizeof(uint32_t) * (nf + 1), s)) != ALB_OK) return rc;
  if ((rc = stage_out(counts, hd_counts, sizeof(uint32_t) * 4, s)) != ALB_OK) return rc;
  rc = launch_inspect_only(g, (const uint32_t*)wl.d, nf, (uint8_t*)bin.d, (uint32_t*)work.d,
                           (uint32_t*)prefix.d, (uint32_t*)counts.d, s);
  unstage(bin, s);
  unstage(work, s);
  unstage(prefix, s);
  unstage(counts, s);
  unstage(wl, s);
  if (rc != ALB_OK) return rc;
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  ALB_CUDA_TRY(cudaMemcpy(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost));
  if (g->h_st->status & ST_ERR_INDEX) return ALB_ERR_INVALID_ARG;
  return ALB_OK;
}

alb_status alb_lb_trace(alb_graph g, const uint32_t* hd_work, const uint32_t* hd_prefix,
                        uint32_t nwork, uint32_t* hd_src, uint32_t* hd_dst, uint32_t* hd_thread,
                        alb_stream stream) {
  if (!g || !hd_prefix || (nwork && !hd_work) || nwork > g->n) return ALB_ERR_INVALID_ARG;
  alb_status rc = begin_call(g, ALB_APP_BFS);
  if (rc != ALB_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // total positions e = prefix[nwork], read on the host
  uint32_t e = 0;
  if (is_device_ptr(hd_prefix)) {
    ALB_CUDA_TRY(cudaMemcpyAsync(&e, hd_prefix + nwork, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    e = hd_prefix[nwork];
  }
  if (e && (!hd_src || !hd_dst || !hd_thread)) return ALB_ERR_INVALID_ARG;
  if ((rc = ensure_tmp(g)) != ALB_OK) return rc;
  Staged work, prefix, src, dst, thr;
  if ((rc = stage_in(work, hd_work, sizeof(uint32_t) * nwork, s)) != ALB_OK) return rc;
  if ((rc = stage_in(prefix, hd_prefix, sizeof(uint32_t) * (nwork + 1), s)) != ALB_OK) return rc;
  if ((rc = stage_out(src, hd_src, sizeof(uint32_t) * e, s)) != ALB_OK) return rc;
  if ((rc = stage_out(dst, hd_dst, sizeof(uint32_t) * e, s)) != ALB_OK) return rc;
  if ((rc = stage_out(thr, hd_thread, sizeof(uint32_t) * e, s)) != ALB_OK) return rc;
  rc = launch_lb_trace(g, (const uint32_t*)work.d, (const uint32_t*)prefix.d, nwork,
                       (uint32_t*)src.d, (uint32_t*)dst.d, (uint32_t*)thr.d, s);
  if (rc != ALB_OK) {
    src.h = dst.h = thr.h = nullptr;
  }
  unstage(src, s);
  unstage(dst, s);
  unstage(thr, s);
  unstage(work, s);
  unstage(prefix, s);
  if (rc != ALB_OK) return rc;
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  return ALB_OK;
}

}  // extern "C"
