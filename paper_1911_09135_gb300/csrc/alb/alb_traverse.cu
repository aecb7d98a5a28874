// Host engine of the data-driven traversals (bfs, sssp, cc, kcore): cached CUDA graphs with a
// device-side round loop, the host-driven loop, and the Algorithm 1 / Algorithm 2 diagnostics.
// The round kernels themselves are in alb_kernels.cuh.
#include "alb_kernels.cuh"

namespace alb {

// ---------------------------------------------- diagnostics: Algorithm 1 alone

__global__ void __launch_bounds__(kBlock) k_inspect_only(const uint32_t* off, uint32_t n,
    const uint32_t* wl, uint32_t nf, uint32_t threshold, uint32_t warp_min, uint32_t cta_min,
    uint8_t* bin, uint32_t* work, uint32_t* prefix, uint32_t* counts, RoundState* st) {
  for (uint64_t b = (uint64_t)blockIdx.x * kBlock; b < nf; b += (uint64_t)gridDim.x * kBlock) {
    const uint32_t i = (uint32_t)b + threadIdx.x;
    bool valid = i < nf;
    uint32_t v = 0u, deg = 0u;
    if (valid) {
      v = wl[i];
      if (v >= n) { atomicOr(&st->status, ST_ERR_INDEX); valid = false; }
      else deg = off[v + 1] - off[v];
    }
    const bool huge = valid && deg >= threshold;
    hub_append(huge, v, deg, work, prefix, &st->hub_packed);
    if (valid) {
      const uint8_t bb = huge ? 3 : (deg < warp_min ? 0 : (deg < cta_min ? 1 : 2));
      bin[i] = bb;
      atomicAdd(counts + bb, 1u);
    }
  }
  if (last_block_ticket(&st->done_inspect)) {
    const unsigned long long hp = __ldcg(&st->hub_packed);
    prefix[(uint32_t)(hp >> 32)] = (uint32_t)hp;
  }
}

// Check that a caller-supplied (work, prefix) pair matches the graph's degrees.
__global__ void k_check_work(const uint32_t* off, uint32_t n, const uint32_t* work,
                             const uint32_t* prefix, uint32_t nwork, uint32_t* bad) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nwork;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t u = work[j];
    if (u >= n || prefix[j + 1] < prefix[j] || prefix[j + 1] - prefix[j] != off[u + 1] - off[u])
      atomicOr(bad, 1u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && prefix[0] != 0u) atomicOr(bad, 1u);
}

__global__ void k_setup_trace(RoundState* st, const uint32_t* prefix, uint32_t nwork) {
  st->hub_packed = ((unsigned long long)nwork << 32) | prefix[nwork];
}

// ---------------------------------------------------------------- host side

static void* inspect_fn(App app, uint32_t B) {
  switch (app) {
    case APP_BFS: return inspect_for<BfsOp>(B);
    case APP_SSSP: return inspect_for<SsspOp>(B);
    case APP_CC: return inspect_for<CcOp>(B);
    case APP_KCORE: return inspect_for<KcoreOp>(B);
    default: return nullptr;
  }
}
static void* lb_fn(App app, uint32_t B) {
  switch (app) {
    case APP_BFS: return lb_for<BfsOp>(B);
    case APP_SSSP: return lb_for<SsspOp>(B);
    case APP_CC: return lb_for<CcOp>(B);
    case APP_KCORE: return lb_for<KcoreOp>(B);
    case APP_TRACE: return (void*)k_lb<BfsOp, true, kBlock>;
    default: return nullptr;
  }
}
static void* init_fn(App app) {
  switch (app) {
    case APP_BFS: return (void*)k_init<APP_BFS>;
    case APP_SSSP: return (void*)k_init<APP_SSSP>;
    case APP_CC: return (void*)k_init<APP_CC>;
    case APP_KCORE: return (void*)k_init<APP_KCORE>;
    default: return nullptr;
  }
}

// Resident CTAs per SM of the round kernels (the grid is persistent).
void occupancy(uint32_t B, uint32_t* inspect_per_sm, uint32_t* lb_per_sm) {
  int mi = 1 << 30, ml = 1 << 30;
  for (int a = APP_BFS; a <= APP_KCORE; ++a) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, inspect_fn((App)a, B), (int)B, 0) == cudaSuccess)
      mi = b < mi ? b : mi;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lb_fn((App)a, B), (int)B, 0) == cudaSuccess)
      ml = b < ml ? b : ml;
  }
  cudaGetLastError();
  *inspect_per_sm = (uint32_t)((mi >= 1 && mi < (1 << 30)) ? mi : 1);
  *lb_per_sm = (uint32_t)((ml >= 1 && ml < (1 << 30)) ? ml : 1);
}

TravCtx make_ctx(alb_graph g, bool use_graph, cudaGraphConditionalHandle hw,
                 cudaGraphConditionalHandle hi) {
  TravCtx c{};
  c.off = g->off;
  c.idx = g->idx;
  c.w = g->w;
  c.n = g->n;
  c.threshold = g->threshold;
  c.warp_min = g->params.twc_warp_min;
  c.cta_min = g->params.twc_cta_min;
  c.distribution = g->params.distribution;
  c.max_rounds = g->params.max_rounds ? g->params.max_rounds
                                      : (g->n < 0xFFFFFFFEu ? g->n + 1u : 0xFFFFFFFFu);
  c.use_graph = use_graph ? 1u : 0u;
  c.F0 = g->F0;
  c.F1 = g->F1;
  c.hub_v = g->hub_v;
  c.hub_p = g->hub_p;
  c.pushed = g->pushed;
  c.pw = (uint32_t)(((size_t)g->n + 31) / 32);
  c.st = g->st;
  c.args = g->args;
  c.h_while = hw;
  c.h_if = hi;
  c.m = (uint32_t)g->m;
  c.chk = g->chk;
  c.cta_twc = g->params.cta_stats ? g->cta_twc : nullptr;
  c.cta_lb = g->params.cta_stats ? g->cta_lb : nullptr;
  return c;
}

static alb_status add_kernel(cudaGraphNode_t* node, cudaGraph_t graph, const cudaGraphNode_t* dep,
                             size_t ndep, void* fn, uint32_t grid, TravCtx* c, uint32_t block = kBlock) {
  cudaKernelNodeParams kp{};
  void* kargs[] = {c};
  kp.func = fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = kargs;
  ALB_CUDA_TRY(cudaGraphAddKernelNode(node, graph, dep, ndep, &kp));
  return ALB_OK;
}

// memset(state) -> init -> while(frontier non-empty) { inspect -> if(work) { lb } } [-> kcore finish]
// L2 persistence for the label array (alb_params.l2_persist_fraction > 0, CUDA-graph mode): the
// labels live in the handle's own buffer, whose address the cached graph can hold, and are copied
// to the caller's buffer at the end of the call; the round kernels' nodes carry an access-policy
// window over that buffer whose hits persist in the L2 set-aside (a share of the device's
// persisting maximum, set for this process's context), while the streamed CSR goes through the
// rest of L2 as usual.
static bool persist_labels(const alb_graph g) {
  return g->params.l2_persist_fraction > 0.f && g->params.exec_mode == 0;
}

static alb_status label_window(alb_graph g, cudaAccessPolicyWindow* w) {
  int max_win = 0, max_persist = 0;
  ALB_CUDA_TRY(cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, g->device));
  ALB_CUDA_TRY(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, g->device));
  const size_t bytes = sizeof(uint32_t) * (size_t)g->n;
  const size_t win = bytes < (size_t)max_win ? bytes : (size_t)max_win;
  const size_t aside = (size_t)((double)g->params.l2_persist_fraction * (double)max_persist);
  size_t cur = 0;
  ALB_CUDA_TRY(cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
  if (cur < aside) ALB_CUDA_TRY(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, aside));
  w->base_ptr = g->tmp;
  w->num_bytes = win;
  // hits beyond the set-aside would evict each other: mark only that share of the window
  w->hitRatio = win ? (float)(aside < win ? (double)aside / (double)win : 1.0) : 0.f;
  w->hitProp = cudaAccessPropertyPersisting;
  w->missProp = cudaAccessPropertyStreaming;
  return ALB_OK;
}

static alb_status build_graph(alb_graph g, App app) {
  cudaGraph_t G = nullptr;
  ALB_CUDA_TRY(cudaGraphCreate(&G, 0));
  cudaGraphConditionalHandle hw, hi;
  alb_status rc = ALB_OK;
  auto fail = [&](alb_status s) { cudaGraphDestroy(G); return s; };
  if (cudaGraphConditionalHandleCreate(&hw, G, 1u, cudaGraphCondAssignDefault) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&hi, G, 0u, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(ALB_ERR_CUDA);
  TravCtx c = make_ctx(g, true, hw, hi);

  cudaGraphNode_t n_ms, n_init, n_while, n_insp, n_if, n_lb, n_fin;
  cudaMemsetParams ms{};
  ms.dst = g->st;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = sizeof(RoundState) / 4;
  ms.height = 1;
  if (cudaGraphAddMemsetNode(&n_ms, G, nullptr, 0, &ms) != cudaSuccess) return fail(ALB_ERR_CUDA);
  if ((rc = add_kernel(&n_init, G, &n_ms, 1, init_fn(app), g->blocks, &c)) != ALB_OK) return fail(rc);

  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  if (cudaGraphAddNode(&n_while, G, &n_init, nullptr, 1, &wp) != cudaSuccess) return fail(ALB_ERR_CUDA);
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  if ((rc = add_kernel(&n_insp, body, nullptr, 0, inspect_fn(app, g->block), g->blocks, &c, g->block)) != ALB_OK)
    return fail(rc);
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hi;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  if (cudaGraphAddNode(&n_if, body, &n_insp, nullptr, 1, &ip) != cudaSuccess) return fail(ALB_ERR_CUDA);
  cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
  if ((rc = add_kernel(&n_lb, ifbody, nullptr, 0, lb_fn(app, g->block), g->lb_blocks, &c, g->block)) != ALB_OK)
    return fail(rc);
  if (persist_labels(g)) {
    cudaKernelNodeAttrValue v{};
    if ((rc = label_window(g, &v.accessPolicyWindow)) != ALB_OK) return fail(rc);
    if (cudaGraphKernelNodeSetAttribute(n_insp, cudaKernelNodeAttributeAccessPolicyWindow, &v) != cudaSuccess ||
        cudaGraphKernelNodeSetAttribute(n_lb, cudaKernelNodeAttributeAccessPolicyWindow, &v) != cudaSuccess)
      return fail(ALB_ERR_CUDA);
  }
  if (app == APP_KCORE) {
    cudaKernelNodeParams kp{};
    const CallArgs* ca = g->args;
    uint32_t n = g->n;
    void* kargs[] = {(void*)&ca, (void*)&n};
    kp.func = (void*)k_kcore_finish;
    kp.gridDim = dim3(g->blocks);
    kp.blockDim = dim3(kBlock);
    kp.kernelParams = kargs;
    if (cudaGraphAddKernelNode(&n_fin, G, &n_while, 1, &kp) != cudaSuccess) return fail(ALB_ERR_CUDA);
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, G, 0) != cudaSuccess) {
    cudaGetLastError();
    return fail(ALB_ERR_CUDA);
  }
  g->graph[app] = G;
  g->exec[app] = ex;
  return ALB_OK;
}

alb_status free_traversal_graphs(alb_graph g) {
  for (int a = 0; a < APP_COUNT; ++a) {
    if (g->exec[a]) cudaGraphExecDestroy(g->exec[a]);
    if (g->graph[a]) cudaGraphDestroy(g->graph[a]);
    g->exec[a] = nullptr;
    g->graph[a] = nullptr;
  }
  return ALB_OK;
}

struct Timer {
  bool on;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  Timer(bool on_, cudaStream_t s_) : on(on_), s(s_) {
    if (on) { cudaEventCreate(&a); cudaEventCreate(&b); cudaEventRecord(a, s); }
  }
  float stop() {
    float ms = 0.f;
    if (on) {
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
    return ms;
  }
};

// Host-driven round loop (exec_mode 1): same kernels, the host reads the state
// after each kernel; with profile = 1 every kernel is timed with CUDA events.
static alb_status host_loop(alb_graph g, App app, cudaStream_t s) {
  TravCtx c = make_ctx(g, false, 0, 0);
  const bool prof = g->params.profile != 0;
  ALB_CUDA_TRY(cudaMemsetAsync(g->st, 0, sizeof(RoundState), s));
  {
    Timer t(prof, s);
    void* args[] = {&c};
    ALB_CUDA_TRY(cudaLaunchKernel(init_fn(app), dim3(g->blocks), dim3(kBlock), args, 0, s));
    g->stats.ms_other += t.stop();
    g->stats.n_other += 1;
  }
  for (;;) {
    {
      Timer t(prof, s);
      void* args[] = {&c};
      ALB_CUDA_TRY(cudaLaunchKernel(inspect_fn(app, g->block), dim3(g->blocks), dim3(g->block), args, 0, s));
      g->stats.ms_inspect += t.stop();
      g->stats.n_inspect += 1;
    }
    ALB_CUDA_TRY(cudaMemcpyAsync(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    if (g->h_st->hub_packed >> 32) {
      Timer t(prof, s);
      void* args[] = {&c};
      ALB_CUDA_TRY(cudaLaunchKernel(lb_fn(app, g->block), dim3(g->lb_blocks), dim3(g->block), args, 0, s));
      g->stats.ms_lb += t.stop();
      g->stats.n_lb += 1;
      ALB_CUDA_TRY(cudaMemcpyAsync(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost, s));
      ALB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    const RoundState& h = *g->h_st;
    if (h.status) break;
    if (h.fcount[h.round & 1u] == 0u) break;
  }
  if (app == APP_KCORE) {
    const CallArgs* ca = g->args;
    k_kcore_finish<<<g->blocks, kBlock, 0, s>>>(ca, g->n);
  }
  return ALB_OK;
}

alb_status run_traversal(alb_graph g, App app, uint32_t src, uint32_t k, uint32_t* out,
                         cudaStream_t s) {
  const bool dev = is_device_ptr(out);
  const bool persist = persist_labels(g);
  uint32_t* lab = out;
  if (!dev || persist) {
    alb_status rc = ensure_tmp(g);
    if (rc != ALB_OK) return rc;
    lab = g->tmp;
  }
  CallArgs ca{lab, src, k, nullptr, nullptr, nullptr};
  k_set_args<<<1, 1, 0, s>>>(g->args, ca);
  ALB_CUDA_TRY(cudaGetLastError());
  if (g->params.cta_stats) {
    alb_status rc = reset_cta_loads(g, s);
    if (rc != ALB_OK) return rc;
  }
  if (g->params.exec_mode == 0) {
    if (!g->exec[app]) {
      alb_status rc = setup_barrier();
      if (rc == ALB_OK) rc = build_graph(g, app);
      if (rc != ALB_OK) return rc;
    }
    ALB_CUDA_TRY(cudaGraphLaunch(g->exec[app], s));
  } else {
    alb_status rc = host_loop(g, app, s);
    if (rc != ALB_OK) return rc;
  }
  if (lab != out)
    ALB_CUDA_TRY(cudaMemcpyAsync(out, lab, sizeof(uint32_t) * g->n,
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  ALB_CUDA_TRY(cudaGetLastError());
  g->last_stream = s;
  g->last_kind = 0;
  return ALB_OK;
}

alb_status launch_inspect_only(alb_graph g, const uint32_t* d_wl, uint32_t nf, uint8_t* d_bin,
                               uint32_t* d_work, uint32_t* d_prefix, uint32_t* d_counts,
                               cudaStream_t s) {
  ALB_CUDA_TRY(cudaMemsetAsync(g->st, 0, sizeof(RoundState), s));
  ALB_CUDA_TRY(cudaMemsetAsync(d_counts, 0, 4 * sizeof(uint32_t), s));
  const uint32_t need = (nf + kBlock - 1) / kBlock;
  const uint32_t grid = need < g->blocks ? (need ? need : 1u) : g->blocks;
  k_inspect_only<<<grid, kBlock, 0, s>>>(g->off, g->n, d_wl, nf, g->threshold,
                                         g->params.twc_warp_min, g->params.twc_cta_min, d_bin,
                                         d_work, d_prefix, d_counts, g->st);
  ALB_CUDA_TRY(cudaGetLastError());
  g->last_stream = s;
  g->last_kind = 0;
  return ALB_OK;
}

alb_status launch_lb_trace(alb_graph g, const uint32_t* d_work, const uint32_t* d_prefix,
                           uint32_t nwork, uint32_t* d_src, uint32_t* d_dst, uint32_t* d_thread,
                           cudaStream_t s) {
  uint32_t* d_bad = nullptr;
  ALB_CUDA_TRY(cudaMallocAsync((void**)&d_bad, sizeof(uint32_t), s));
  ALB_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(uint32_t), s));
  k_check_work<<<g->blocks, kBlock, 0, s>>>(g->off, g->n, d_work, d_prefix, nwork, d_bad);
  uint32_t bad = 1;
  ALB_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFreeAsync(d_bad, s);
  if (bad) return ALB_ERR_INVALID_ARG;
  ALB_CUDA_TRY(cudaMemsetAsync(g->st, 0, sizeof(RoundState), s));
  ALB_CUDA_TRY(cudaMemcpyAsync(g->hub_v, d_work, sizeof(uint32_t) * nwork, cudaMemcpyDeviceToDevice, s));
  ALB_CUDA_TRY(cudaMemcpyAsync(g->hub_p, d_prefix, sizeof(uint32_t) * (nwork + 1),
                               cudaMemcpyDeviceToDevice, s));
  k_setup_trace<<<1, 1, 0, s>>>(g->st, d_prefix, nwork);
  CallArgs ca{g->tmp, 0u, 0u, d_src, d_dst, d_thread};
  k_set_args<<<1, 1, 0, s>>>(g->args, ca);
  TravCtx c = make_ctx(g, false, 0, 0);
  void* args[] = {&c};
  // the trace kernel is built for the default CTA size; its grid keeps the handle's thread count
  const uint32_t trace_grid = (uint32_t)(((uint64_t)g->lb_blocks * g->block + kBlock - 1) / kBlock);
  ALB_CUDA_TRY(cudaLaunchKernel(lb_fn(APP_TRACE, kBlock), dim3(trace_grid), dim3(kBlock), args, 0, s));
  ALB_CUDA_TRY(cudaGetLastError());
  g->last_stream = s;
  g->last_kind = 0;
  return ALB_OK;
}

}  // namespace alb

// ------------------------------------------------ BFS without any allocation
//
// alb_bfs_noalloc serves callers that cannot allocate device memory: code that
// runs while a CUDA graph is being captured on another stream, services whose
// device memory is entirely owned by another pool (a framework's caching
// allocator), and real-time loops where a cudaMalloc/cudaFree would block on
// the whole device. It runs the same BFS kernels as alb_bfs, with every scratch
// buffer (two frontiers, the huge worklist and its prefix sums, the round
// state) carved from one fixed-size __device__ array that lives in the module
// for as long as the library is loaded on a device.

#include <mutex>

namespace alb {

constexpr uint32_t kNoAllocMaxVertices = 1u << 20;
constexpr size_t kNoAllocVec = ((sizeof(uint32_t) * ((size_t)kNoAllocMaxVertices + 1) + 255) / 256) * 256;
constexpr size_t kNoAllocBits = ((sizeof(uint32_t) * ((size_t)kNoAllocMaxVertices / 32 + 1) + 255) / 256) * 256;
constexpr size_t kNoAllocBytes = 4 * kNoAllocVec + kNoAllocBits + 4 * 256;

// Shared by every call on a device: calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Result of the CSR check: bit kBadOrder for offsets that decrease (a malformed argument),
// bit kBadIndex for an index >= n (corrupt data); plus offsets[0] and offsets[n].
struct NoAllocCheck {
  uint32_t bad;
  uint32_t off0;
  uint32_t offn;
};
constexpr uint32_t kBadOrder = 1u, kBadIndex = 2u;

// One pass over the caller's CSR, so the traversal kernels never index out of range.
__global__ void k_noalloc_check(const uint32_t* off, const uint32_t* idx, uint32_t n, uint64_t m,
                                NoAllocCheck* out) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t bad = 0;
  for (uint64_t v = tid; v < n; v += stride)
    if (off[v + 1] < off[v]) bad |= kBadOrder;
  for (uint64_t e = tid; e < m; e += stride)
    if (idx[e] >= n) bad |= kBadIndex;
  if (bad) atomicOr(&out->bad, bad);
  if (tid == 0) {
    out->off0 = off[0];
    out->offn = off[n];
  }
}

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_base[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (host code cannot use the symbol itself: it names a host-side shadow).
static alb_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return ALB_ERR_CUDA; }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return ALB_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) { cudaGetLastError(); return ALB_ERR_CUDA; }
    g_noalloc_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_base[dev];
  return ALB_OK;
}

}  // namespace alb

extern "C" alb_status alb_bfs_noalloc(uint32_t n, uint64_t m, const uint32_t* d_offsets,
                                      const uint32_t* d_indices, uint32_t src, uint32_t* d_levels,
                                      alb_stream stream) {
  using namespace alb;
  if (n == 0 || n > kNoAllocMaxVertices) return ALB_ERR_INVALID_ARG;
  if (m >= 0xFFFFFFFFull) return ALB_ERR_OVERFLOW;
  if (!d_offsets || (m && !d_indices) || !d_levels || src >= n) return ALB_ERR_INVALID_ARG;
  if (!is_device_ptr(d_offsets) || (m && !is_device_ptr(d_indices)) || !is_device_ptr(d_levels))
    return ALB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  alb_status rc = noalloc_scratch(&base);
  if (rc != ALB_OK) return rc;
  uint32_t* F0 = reinterpret_cast<uint32_t*>(base);
  uint32_t* F1 = reinterpret_cast<uint32_t*>(base + kNoAllocVec);
  uint32_t* hub_v = reinterpret_cast<uint32_t*>(base + 2 * kNoAllocVec);
  uint32_t* hub_p = reinterpret_cast<uint32_t*>(base + 3 * kNoAllocVec);
  uint32_t* visited = reinterpret_cast<uint32_t*>(base + 4 * kNoAllocVec);  // bfs visited bitmap
  unsigned char* small = base + 4 * kNoAllocVec + kNoAllocBits;
  RoundState* st = reinterpret_cast<RoundState*>(small);
  CallArgs* args = reinterpret_cast<CallArgs*>(small + 256);
  NoAllocCheck* chk = reinterpret_cast<NoAllocCheck*>(small + 512);
  uint32_t* bounds = reinterpret_cast<uint32_t*>(small + 768);  // TravCtx::chk
  static_assert(sizeof(RoundState) <= 256 && sizeof(CallArgs) <= 256, "scratch layout");

  int dev = 0, sms = 0;
  ALB_CUDA_TRY(cudaGetDevice(&dev));
  ALB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint32_t occ_i = 1, occ_l = 1;
  occupancy(kBlock, &occ_i, &occ_l);
  const uint32_t blocks = (uint32_t)sms * occ_i, lb_blocks = (uint32_t)sms * occ_l;

  // validate the caller's CSR (this call's contents of the shared scratch start here)
  NoAllocCheck h{};
  ALB_CUDA_TRY(cudaMemsetAsync(chk, 0, sizeof(NoAllocCheck), s));
  k_noalloc_check<<<(unsigned)sms * 4, 256, 0, s>>>(d_offsets, d_indices, n, m, chk);
  ALB_CUDA_TRY(cudaGetLastError());
  ALB_CUDA_TRY(cudaMemcpyAsync(&h, chk, sizeof(h), cudaMemcpyDeviceToHost, s));
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.off0 != 0u || (uint64_t)h.offn != m || (h.bad & kBadOrder)) return ALB_ERR_INVALID_ARG;
  if (h.bad & kBadIndex) return ALB_ERR_DEVICE;

  TravCtx c{};
  c.off = d_offsets;
  c.idx = d_indices;
  c.w = nullptr;
  c.n = n;
  c.threshold = lb_blocks * (uint32_t)kBlock;  // the paper's rule: threads of the LB kernel
  c.warp_min = 32u;
  c.cta_min = (uint32_t)kBlock;
  c.distribution = 0u;
  c.max_rounds = n + 1u;
  c.use_graph = 0u;
  c.F0 = F0;
  c.F1 = F1;
  c.hub_v = hub_v;
  c.hub_p = hub_p;
  c.pushed = visited;  // cleared by the init kernel
  c.pw = (n + 31u) / 32u;
  c.st = st;
  c.args = args;
  c.m = (uint32_t)m;   // bound of the edge indices in the bounds-checked build
  c.chk = bounds;      // the bounds-checked build's record (never written by the regular build)

  CallArgs ca{d_levels, src, 0u, nullptr, nullptr, nullptr};
  k_set_args<<<1, 1, 0, s>>>(args, ca);
  ALB_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(RoundState), s));  // counters must start at zero
  ALB_CUDA_TRY(cudaMemsetAsync(bounds, 0, 4 * sizeof(uint32_t), s));
  void* kargs[] = {&c};
  ALB_CUDA_TRY(cudaLaunchKernel((void*)k_init<APP_BFS>, dim3(blocks), dim3(kBlock), kargs, 0, s));
  RoundState hs{};
  for (;;) {
    ALB_CUDA_TRY(cudaLaunchKernel((void*)k_inspect<BfsOp, kBlock>, dim3(blocks), dim3(kBlock), kargs, 0, s));
    ALB_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.hub_packed >> 32) {
      ALB_CUDA_TRY(cudaLaunchKernel((void*)k_lb<BfsOp, false, kBlock>, dim3(lb_blocks), dim3(kBlock), kargs, 0, s));
      ALB_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
      ALB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (hs.status & ST_ERR_ROUNDS) return ALB_ERR_TIMEOUT;
    if (hs.fcount[hs.round & 1u] == 0u) break;
  }
  uint32_t rec[4] = {0u, 0u, 0u, 0u};
  ALB_CUDA_TRY(cudaMemcpyAsync(rec, bounds, sizeof(rec), cudaMemcpyDeviceToHost, s));
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  if (rec[0] != 0u) return ALB_ERR_DEVICE;  // the bounds-checked build skipped an access
  return ALB_OK;
}
