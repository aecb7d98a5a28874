// Batched traversals.
//
// (1) Many sources on one graph (alb_bfs_batch, alb_sssp_batch). Sources run in groups of 32
//     that share every read of the CSR: a frontier vertex carries the set of sources (a 32-bit
//     mask) for which it is active, and the operator relaxes all of them along each edge it
//     reads. Labels of a group are kept vertex-major (lab[v * 32 + s]), so the 32 labels of a
//     vertex share one 128-byte line. The round kernels are the ALB kernels of every other
//     traversal (inspection + TWC, the cyclic LB kernel, the device-side round loop); only the
//     operator differs:
//       bfs : bit-parallel (a `seen` mask per vertex; one atomicOr discovers up to 32 sources),
//       sssp: per active source, the relaxation of Fig. 3 with atomicMin.
//     The per-round masks live in three 32-bit arrays used in rotation (read, written, cleared
//     for the round after next), so a mask is merged with one atomicOr.
// (2) Many small graphs (alb_bfs_multi, alb_sssp_multi): a traversal from a set of sources at
//     distance 0. Run on the disjoint union of many graphs with one source in each, it computes
//     every graph's own result in one launch sequence (components never interact).
#include <cstdlib>
#include <new>

#include "alb_kernels.cuh"

namespace alb {

struct BatchAux {
  uint32_t* lab;     // n x 32, vertex-major
  uint32_t* seen;    // n: sources that reached v (bfs)
  uint32_t* act[3];  // per-vertex source masks; round r reads act[r % 3], writes act[(r + 1) % 3]
                     // and clears act[(r + 2) % 3], which round r - 1 read and round r + 1 writes
};

__device__ __forceinline__ uint32_t* act_of(const BatchAux* x, uint32_t round) { return x->act[round % 3u]; }

// Sources for which v is active in round r (written during round r - 1).
__device__ __forceinline__ uint32_t act_mask(const BatchAux* x, uint32_t r, uint32_t v) {
  return act_of(x, r)[v];
}

// OR `bits` into v's mask for the next round; true for exactly one caller per vertex and round:
// the one that set its first bit (it appends the vertex to the next frontier). A plain read
// skips the atomic when every bit is already there (an entry only gains bits within a round,
// so a stale read can only under-report them). A single atomicOr per update: many relaxations
// of the same round often reach the same high-degree vertex, and a compare-and-swap loop there
// serialises into a retry storm that keeps one warp spinning while the SMs idle.
__device__ __forceinline__ bool act_or(uint32_t* p, uint32_t bits) {
  const uint32_t cur = *p;
  if ((cur & bits) == bits) return false;
  return atomicOr(p, bits) == 0u;
}

// Round r's clearing of the mask array round r + 1 writes (see BatchAux): a grid-stride loop of
// every CTA of the round's inspection kernel.
__device__ __forceinline__ void act_clear(const BatchAux* x, uint32_t r, uint32_t n) {
  uint32_t* c = act_of(x, r + 2u);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    c[i] = 0u;
}

// Multi-source bfs: sval is the vertex's source mask.
struct MsBfsOp {
  static constexpr bool kBatch = true;
  static constexpr bool kW = false;
  __device__ static void round_start(const OpArgs& a, uint32_t r) {
    act_clear(static_cast<const BatchAux*>(a.aux), r, a.n);
  }
  __device__ static uint32_t sval(const OpArgs& a, uint32_t v) {
    return act_mask(static_cast<const BatchAux*>(a.aux), a.next - 1u, v);
  }
  __device__ static bool apply(const OpArgs& a, uint32_t M, uint32_t dst, uint32_t) {
    const BatchAux* x = static_cast<const BatchAux*>(a.aux);
    if (!ALB_IN_RANGE(a.chk, CHK_ROW, dst, a.n)) return false;
    uint32_t nw = M & ~x->seen[dst];
    if (!nw) return false;
    nw &= ~atomicOr(x->seen + dst, nw);
    if (!nw) return false;
    uint32_t* row = x->lab + (size_t)dst * 32u;
    for (uint32_t b = nw; b; b &= b - 1u) row[__ffs(b) - 1] = a.next;
    return act_or(act_of(x, a.next) + dst, nw);
  }
};

// Multi-source sssp: sval is the vertex id (its mask and labels are read per edge; they are
// L1-resident while the vertex's edges are expanded). Per active source, the relaxation of
// Fig. 3. The atomicMin does not wait for its old value: the destination is marked for the next
// round whenever the pre-check saw an improvement, so the marked set contains every vertex
// whose label dropped (possibly a few more, which only costs a redundant visit).
struct MsSsspOp {
  static constexpr bool kBatch = true;
  static constexpr bool kW = true;
  __device__ static void round_start(const OpArgs& a, uint32_t r) {
    act_clear(static_cast<const BatchAux*>(a.aux), r, a.n);
  }
  __device__ static uint32_t sval(const OpArgs&, uint32_t v) { return v; }
  __device__ static bool apply(const OpArgs& a, uint32_t v, uint32_t dst, uint32_t w) {
    const BatchAux* x = static_cast<const BatchAux*>(a.aux);
    if (!ALB_IN_RANGE(a.chk, CHK_ROW, v, a.n) || !ALB_IN_RANGE(a.chk, CHK_ROW, dst, a.n)) return false;
    const uint32_t M = act_mask(x, a.next - 1u, v);
    const uint32_t* ru = x->lab + (size_t)v * 32u;
    uint32_t* rd = x->lab + (size_t)dst * 32u;
    uint32_t nb = 0u;
    // two sources per step, their four label loads issued together
    for (uint32_t b = M; b;) {
      const uint32_t s0 = __ffs(b) - 1;
      b &= b - 1u;
      const uint32_t s1 = b ? __ffs(b) - 1 : s0;
      b &= b - 1u;
      const uint32_t du0 = ru[s0], dv0 = rd[s0], du1 = ru[s1], dv1 = rd[s1];
      if ((uint64_t)du0 + w < (uint64_t)dv0) {
        atomicMin(rd + s0, du0 + w);
        nb |= 1u << s0;
      }
      if (s1 != s0 && (uint64_t)du1 + w < (uint64_t)dv1) {
        atomicMin(rd + s1, du1 + w);
        nb |= 1u << s1;
      }
    }
    return nb && act_or(act_of(x, a.next) + dst, nb);
  }
};

// ---- group kernels

// checked build: the group's pointers read from device memory must be set and aligned
__device__ __forceinline__ bool aux_ok(const TravCtx& c, const BatchAux* x) {
#ifdef ALB_CHECKED
  const uint64_t a = (uint64_t)x;
  if (!ALB_IN_RANGE(c.chk, CHK_PTR, (a == 0 || (a & 7)) ? 1u : 0u, 1u)) return false;
  const uint64_t l = (uint64_t)x->lab, s = (uint64_t)x->seen;
  const uint64_t p0 = (uint64_t)x->act[0], p1 = (uint64_t)x->act[1], p2 = (uint64_t)x->act[2];
  const bool bad = !l || (l & 3) || !s || (s & 3) || !p0 || (p0 & 3) || !p1 || (p1 & 3) || !p2 || (p2 & 3);
  return ALB_IN_RANGE(c.chk, CHK_PTR, bad ? 2u : 0u, 1u);
#else
  (void)c;
  (void)x;
  return true;
#endif
}

__global__ void __launch_bounds__(kBlock) k_batch_init(TravCtx c) {
  const BatchAux* x = static_cast<const BatchAux*>(c.args->aux);
  if (!aux_ok(c, x)) return;
  const uint64_t n = c.n;
  for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < n * 32u;
       i += (uint64_t)gridDim.x * kBlock)
    x->lab[i] = kInf;
  for (uint64_t v = (uint64_t)blockIdx.x * kBlock + threadIdx.x; v < n; v += (uint64_t)gridDim.x * kBlock) {
    x->seen[v] = 0u;
    x->act[0][v] = 0u;
    x->act[1][v] = 0u;
    x->act[2][v] = 0u;
  }
}

__global__ void k_batch_seed(TravCtx c) {
  const CallArgs* ca = c.args;
  const BatchAux* x = static_cast<const BatchAux*>(ca->aux);
  if (!aux_ok(c, x)) return;
  const uint32_t s = threadIdx.x;
  if (s < ca->nsrc) {
    const uint32_t v = ca->srcs[s], bit = 1u << s;
    if (v >= c.n) {  // only possible for sources passed in device memory
      atomicOr(&c.st->status, ST_ERR_SRC);
      return;
    }
    x->lab[(size_t)v * 32u + s] = 0u;
    atomicOr(x->seen + v, bit);
    if (act_or(x->act[0] + v, bit)) {
      const uint32_t slot = atomicAdd(&c.st->fcount[0], 1u);
      if (ALB_IN_RANGE(c.chk, CHK_PUSH, slot, c.n)) c.F0[slot] = v;
    }
  }
}

// lab (n x 32, vertex-major) -> out (nsrc x n, source-major), through a shared-memory tile.
__global__ void __launch_bounds__(kBlock) k_batch_out(TravCtx c) {
  __shared__ uint32_t tile[32][33];
  const CallArgs* ca = c.args;
  const BatchAux* x = static_cast<const BatchAux*>(ca->aux);
  if (!aux_ok(c, x)) return;
  const uint32_t n = c.n, ns = ca->nsrc;
  uint32_t* out = ca->lab;
  const uint32_t tx = threadIdx.x & 31u, ty = threadIdx.x >> 5;  // 32 x 8
  for (uint64_t v0 = (uint64_t)blockIdx.x * 32u; v0 < n; v0 += (uint64_t)gridDim.x * 32u) {
    for (uint32_t r = ty; r < 32u; r += 8u) {
      const uint64_t v = v0 + r;
      tile[r][tx] = v < n ? x->lab[v * 32u + tx] : 0u;
    }
    __syncthreads();
    for (uint32_t s = ty; s < ns; s += 8u) {
      const uint64_t v = v0 + tx;
      if (v < n) out[(size_t)s * n + v] = tile[tx][s];
    }
    __syncthreads();
  }
}

// ---- multi-source single-label kernels (many graphs as one disjoint union)

template <int APP>
__global__ void __launch_bounds__(kBlock) k_multi_init(TravCtx c) {
  uint32_t* lab = c.args->lab;
  for (uint64_t v = (uint64_t)blockIdx.x * kBlock + threadIdx.x; v < c.n; v += (uint64_t)gridDim.x * kBlock)
    lab[v] = kInf;
  // sssp: both push bitmaps start empty; bfs: the visited bitmap (the seed kernel sets the sources)
  const uint64_t words = APP == APP_SSSP ? 2ull * c.pw : (uint64_t)c.pw;
  if (c.pushed)
    for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < words; i += (uint64_t)gridDim.x * kBlock)
      c.pushed[i] = 0u;
}

template <int APP>
__global__ void k_multi_seed(TravCtx c) {
  const CallArgs* ca = c.args;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ca->nsrc; i += gridDim.x * blockDim.x) {
    const uint32_t v = ca->srcs[i];
    if (v >= c.n) {  // only possible for sources passed in device memory
      atomicOr(&c.st->status, ST_ERR_SRC);
      continue;
    }
    if (atomicCAS(ca->lab + v, kInf, 0u) == kInf) {
      if (APP == APP_BFS) atomicOr(c.pushed + (v >> 5), 1u << (v & 31u));  // visited
      const uint32_t slot = atomicAdd(&c.st->fcount[0], 1u);
      if (ALB_IN_RANGE(c.chk, CHK_PUSH, slot, c.n)) c.F0[slot] = v;
    }
  }
}

}  // namespace alb

// ---------------------------------------------------------------- host side

enum BatchKind { BK_MS_BFS = 0, BK_MS_SSSP = 1, BK_MULTI_BFS = 2, BK_MULTI_SSSP = 3, BK_COUNT = 4 };

// Groups of 32 sources in flight at once: the handle and up to kBatchWorkers - 1 worker clones
// (sharing its CSR, each with its own workspace and stream). One group's early and late rounds
// have small frontiers and leave most of the device idle; groups on several streams fill it.
constexpr uint32_t kBatchWorkers = 4;

struct BatchWs {
  alb_graph worker[kBatchWorkers - 1] = {};
  cudaStream_t wstream[kBatchWorkers - 1] = {};
  cudaEvent_t ev_start = nullptr;
  cudaEvent_t ev_done[kBatchWorkers - 1] = {};
  uint32_t nworkers = 0;       // created (and warmed)
  uint32_t used_workers = 0;   // used by the last call (alb_sync checks them)
  uint32_t* lab = nullptr;
  uint32_t* seen = nullptr;
  uint32_t* act = nullptr;  // 3 x n source masks (BatchAux::act)
  alb::BatchAux* aux = nullptr;
  uint32_t* srcs = nullptr;
  uint32_t cap_srcs = 0;
  uint32_t* tmp = nullptr;  // 32 x n staging for host outputs
  cudaGraph_t graph[BK_COUNT] = {};
  cudaGraphExec_t exec[BK_COUNT] = {};
};

namespace alb {

alb_status free_batch(alb_graph g) {
  BatchWs* b = g->batch;
  if (!b) return ALB_OK;
  for (uint32_t w = 0; w < kBatchWorkers - 1; ++w) {  // callers synchronise the device first
    if (b->worker[w]) alb_graph_destroy(b->worker[w]);
    if (b->wstream[w]) cudaStreamDestroy(b->wstream[w]);
    if (b->ev_done[w]) cudaEventDestroy(b->ev_done[w]);
  }
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  for (int i = 0; i < BK_COUNT; ++i) {
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
  }
  cudaFree(b->lab);
  cudaFree(b->seen);
  cudaFree(b->act);
  cudaFree(b->aux);
  cudaFree(b->srcs);  // callers synchronise the device before freeing a workspace
  cudaFree(b->tmp);
  cudaGetLastError();
  delete b;
  g->batch = nullptr;
  return ALB_OK;
}

alb_status batch_stats(alb_graph, alb_stats*) { return ALB_OK; }

// Status of the worker clones used by the last batch call (their round limits and checks).
alb_status batch_sync_workers(alb_graph g) {
  BatchWs* b = g->batch;
  alb_status rc = ALB_OK;
  if (!b) return rc;
  for (uint32_t w = 0; w < b->used_workers; ++w) {
    const alb_status r = alb_sync(b->worker[w]);
    if (rc == ALB_OK) rc = r;
  }
  b->used_workers = 0;
  return rc;
}

static __global__ void k_set_aux(BatchAux* dst, BatchAux v) { *dst = v; }

static alb_status ensure_batch(alb_graph g, bool group_arrays, uint32_t nsrc, cudaStream_t s) {
  if (!g->batch) g->batch = new (std::nothrow) BatchWs();
  BatchWs* b = g->batch;
  if (!b) return ALB_ERR_OOM;
  const size_t n = g->n;
  if (group_arrays && !b->lab) {
    alb_status rc = setup_barrier();
    if (rc != ALB_OK) return rc;
    ALB_CUDA_TRY(cudaMalloc((void**)&b->lab, sizeof(uint32_t) * n * 32u));
    ALB_CUDA_TRY(cudaMalloc((void**)&b->seen, sizeof(uint32_t) * n));
    ALB_CUDA_TRY(cudaMalloc((void**)&b->act, sizeof(uint32_t) * n * 3u));
    ALB_CUDA_TRY(cudaMalloc((void**)&b->aux, sizeof(BatchAux)));
    // written on the call's stream: the batch kernels queued after it read it
    BatchAux h{b->lab, b->seen, {b->act, b->act + n, b->act + 2 * n}};
    k_set_aux<<<1, 1, 0, s>>>(b->aux, h);
    ALB_CUDA_TRY(cudaGetLastError());
  }
  if (b->cap_srcs < nsrc) {
    // Stream-ordered: work already queued on s (an earlier batch's seed kernel) may still read
    // the old buffer, and a plain cudaFree need not wait for it.
    const uint32_t cap = nsrc < 1024u ? 1024u : nsrc;
    alb_status rc = setup_barrier();
    if (rc != ALB_OK) return rc;
    if (b->srcs) ALB_CUDA_TRY(cudaFreeAsync(b->srcs, s));
    b->srcs = nullptr;
    ALB_CUDA_TRY(cudaMallocAsync((void**)&b->srcs, sizeof(uint32_t) * cap, s));
    b->cap_srcs = cap;
  }
  return ALB_OK;
}

static alb_status add_node(cudaGraphNode_t* node, cudaGraph_t graph, const cudaGraphNode_t* dep,
                           size_t ndep, void* fn, uint32_t grid, uint32_t block, TravCtx* c) {
  cudaKernelNodeParams kp{};
  void* kargs[] = {c};
  kp.func = fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.kernelParams = kargs;
  ALB_CUDA_TRY(cudaGraphAddKernelNode(node, graph, dep, ndep, &kp));
  return ALB_OK;
}

// Kernels and grids of one batch kind on handle g: init, seed, the round kernels and their
// persistent grids (sized from the round kernels' own residency: the multi-source operators hold
// more registers than the single-source ones the handle's grids are sized for); the paper's
// threshold rule follows this LB grid.
struct BatchCfg {
  void *init, *seed, *insp, *lb;
  uint32_t seed_grid, seed_block, ib, lbb, threshold;
};

static BatchCfg batch_cfg(alb_graph g, BatchKind kind) {
  BatchCfg k{};
  k.seed_grid = 1;
  k.seed_block = 32;
  switch (kind) {
    case BK_MS_BFS:
      k.init = (void*)k_batch_init; k.seed = (void*)k_batch_seed;
      k.insp = inspect_for<MsBfsOp>(g->block); k.lb = lb_for<MsBfsOp>(g->block);
      break;
    case BK_MS_SSSP:
      k.init = (void*)k_batch_init; k.seed = (void*)k_batch_seed;
      k.insp = inspect_for<MsSsspOp>(g->block); k.lb = lb_for<MsSsspOp>(g->block);
      break;
    case BK_MULTI_BFS:
      k.init = (void*)k_multi_init<APP_BFS>; k.seed = (void*)k_multi_seed<APP_BFS>;
      k.insp = inspect_for<BfsOp>(g->block); k.lb = lb_for<BfsOp>(g->block);
      k.seed_grid = g->blocks; k.seed_block = kBlock;
      break;
    default:
      k.init = (void*)k_multi_init<APP_SSSP>; k.seed = (void*)k_multi_seed<APP_SSSP>;
      k.insp = inspect_for<SsspOp>(g->block); k.lb = lb_for<SsspOp>(g->block);
      k.seed_grid = g->blocks; k.seed_block = kBlock;
      break;
  }
  k.ib = g->blocks;
  k.lbb = g->lb_blocks;
  k.threshold = g->threshold;
  if (!g->params.grid_blocks) {
    int bi = 0, bl = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bi, k.insp, (int)g->block, 0) == cudaSuccess && bi > 0)
      k.ib = (uint32_t)g->num_sms * (uint32_t)bi;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, k.lb, (int)g->block, 0) == cudaSuccess && bl > 0)
      k.lbb = (uint32_t)g->num_sms * (uint32_t)bl;
    cudaGetLastError();
    if (g->params.hub_threshold < 0) k.threshold = k.lbb * g->block;
  }
  return k;
}

// memset(state) -> init -> seed -> while { inspect -> if (work) lb } [-> transpose]
static alb_status build_batch_graph(alb_graph g, BatchKind kind) {
  BatchWs* b = g->batch;
  cudaGraph_t G = nullptr;
  ALB_CUDA_TRY(cudaGraphCreate(&G, 0));
  auto fail = [&](alb_status s) { cudaGraphDestroy(G); return s; };
  cudaGraphConditionalHandle hw, hi;
  if (cudaGraphConditionalHandleCreate(&hw, G, 1u, cudaGraphCondAssignDefault) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&hi, G, 0u, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(ALB_ERR_CUDA);
  TravCtx c = make_ctx(g, true, hw, hi);
  const BatchCfg k = batch_cfg(g, kind);
  void *init = k.init, *seed = k.seed, *insp = k.insp, *lb = k.lb;
  const uint32_t seed_grid = k.seed_grid, seed_block = k.seed_block, ib = k.ib, lbb = k.lbb;
  c.threshold = k.threshold;
  cudaGraphNode_t n_ms, n_init, n_seed, n_while, n_insp, n_if, n_lb, n_out;
  cudaMemsetParams ms{};
  ms.dst = g->st;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = sizeof(RoundState) / 4;
  ms.height = 1;
  alb_status rc;
  if (cudaGraphAddMemsetNode(&n_ms, G, nullptr, 0, &ms) != cudaSuccess) return fail(ALB_ERR_CUDA);
  if ((rc = add_node(&n_init, G, &n_ms, 1, init, g->blocks, kBlock, &c)) != ALB_OK) return fail(rc);
  if ((rc = add_node(&n_seed, G, &n_init, 1, seed, seed_grid, seed_block, &c)) != ALB_OK) return fail(rc);
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  if (cudaGraphAddNode(&n_while, G, &n_seed, nullptr, 1, &wp) != cudaSuccess) return fail(ALB_ERR_CUDA);
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  if ((rc = add_node(&n_insp, body, nullptr, 0, insp, ib, g->block, &c)) != ALB_OK) return fail(rc);
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hi;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  if (cudaGraphAddNode(&n_if, body, &n_insp, nullptr, 1, &ip) != cudaSuccess) return fail(ALB_ERR_CUDA);
  if ((rc = add_node(&n_lb, ip.conditional.phGraph_out[0], nullptr, 0, lb, lbb, g->block, &c)) != ALB_OK)
    return fail(rc);
  if (kind == BK_MS_BFS || kind == BK_MS_SSSP) {
    if ((rc = add_node(&n_out, G, &n_while, 1, (void*)k_batch_out, g->blocks, kBlock, &c)) != ALB_OK)
      return fail(rc);
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, G, 0) != cudaSuccess) {
    cudaGetLastError();
    return fail(ALB_ERR_CUDA);
  }
  b->graph[kind] = G;
  b->exec[kind] = ex;
  return ALB_OK;
}

// Sources onto the device, stream-ordered and without a host round trip: host-memory sources are
// checked here; device-memory sources are checked by the seed kernels (a bad one is skipped and
// latched as ALB_ERR_INVALID_ARG, returned by alb_sync).
static alb_status stage_srcs(alb_graph g, const uint32_t* hd_srcs, uint32_t k, cudaStream_t s) {
  BatchWs* b = g->batch;
  if (!is_device_ptr(hd_srcs)) {
    for (uint32_t i = 0; i < k; ++i)
      if (hd_srcs[i] >= g->n) return ALB_ERR_INVALID_ARG;
  }
  ALB_CUDA_TRY(cudaMemcpyAsync(b->srcs, hd_srcs, sizeof(uint32_t) * k, cudaMemcpyDefault, s));
  return ALB_OK;
}

// The same launch sequence as the batch graph, driven by the host (exec_mode 1): one launch per
// kernel, the round state read after each round kernel; with profile = 1 every round kernel is
// timed with CUDA events. ncu profiles these launches, not kernels inside graphs with
// conditional nodes.
static alb_status batch_host_loop(alb_graph g, BatchKind kind, cudaStream_t s) {
  const BatchCfg k = batch_cfg(g, kind);
  TravCtx c = make_ctx(g, false, 0, 0);
  c.threshold = k.threshold;
  const bool prof = g->params.profile != 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof) { cudaEventCreate(&e0); cudaEventCreate(&e1); }
  auto launch = [&](void* fn, uint32_t grid, uint32_t block, double* ms, uint32_t* cnt) -> alb_status {
    void* args[] = {&c};
    if (prof && ms) cudaEventRecord(e0, s);
    ALB_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, s));
    if (prof && ms) {
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      *ms += t;
      *cnt += 1;
    }
    return ALB_OK;
  };
  alb_status rc = ALB_OK;
  ALB_CUDA_TRY(cudaMemsetAsync(g->st, 0, sizeof(RoundState), s));
  if ((rc = launch(k.init, g->blocks, kBlock, nullptr, nullptr)) != ALB_OK) return rc;
  if ((rc = launch(k.seed, k.seed_grid, k.seed_block, nullptr, nullptr)) != ALB_OK) return rc;
  for (;;) {
    if ((rc = launch(k.insp, k.ib, g->block, &g->stats.ms_inspect, &g->stats.n_inspect)) != ALB_OK) return rc;
    ALB_CUDA_TRY(cudaMemcpyAsync(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    if (g->h_st->hub_packed >> 32) {
      if ((rc = launch(k.lb, k.lbb, g->block, &g->stats.ms_lb, &g->stats.n_lb)) != ALB_OK) return rc;
      ALB_CUDA_TRY(cudaMemcpyAsync(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost, s));
      ALB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    const RoundState& h = *g->h_st;
    if (h.status || h.fcount[h.round & 1u] == 0u) break;
  }
  if (kind == BK_MS_BFS || kind == BK_MS_SSSP)
    if ((rc = launch((void*)k_batch_out, g->blocks, kBlock, nullptr, nullptr)) != ALB_OK) return rc;
  if (prof) { cudaEventDestroy(e0); cudaEventDestroy(e1); }
  ALB_CUDA_TRY(cudaGetLastError());
  return ALB_OK;
}

// One group of ns <= 32 sources (device list) on handle h and stream s, into dst (device).
static alb_status run_group_on(alb_graph h, BatchKind kind, const uint32_t* d_srcs, uint32_t ns, uint32_t* dst,
                               cudaStream_t s) {
  BatchWs* b = h->batch;
  CallArgs ca{dst, 0u, 0u, nullptr, nullptr, nullptr, b->aux, d_srcs, ns};
  k_set_args<<<1, 1, 0, s>>>(h->args, ca);
  ALB_CUDA_TRY(cudaGetLastError());
  ALB_CUDA_TRY(cudaGraphLaunch(b->exec[kind], s));
  h->last_stream = s;
  h->last_kind = 0;
  return ALB_OK;
}

// Create (once) and warm `want` worker clones for `kind`: their workspaces and CUDA graphs exist
// before any of them runs, and the device is idle while they are made (a first call that
// allocates and instantiates while other streams run is avoided, as for serving slots).
static alb_status ensure_workers(alb_graph g, BatchKind kind, int app, uint32_t want) {
  BatchWs* b = g->batch;
  bool made = false;
  for (uint32_t w = 0; w < want; ++w) {
    if (!b->worker[w]) {
      if (!made) ALB_CUDA_TRY(cudaDeviceSynchronize());
      made = true;
      alb_status rc = alb_graph_clone(g, &b->worker[w]);
      if (rc != ALB_OK) return rc;
      ALB_CUDA_TRY(cudaStreamCreateWithFlags(&b->wstream[w], cudaStreamNonBlocking));
      ALB_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_done[w], cudaEventDisableTiming));
    }
    alb_graph h = b->worker[w];
    select_cfg(h, app);
    if (!h->batch || !h->batch->lab || !h->batch->exec[kind]) {
      if (!made) ALB_CUDA_TRY(cudaDeviceSynchronize());
      made = true;
      alb_status rc = ensure_batch(h, true, 0u, b->wstream[w]);
      if (rc == ALB_OK && !h->batch->exec[kind]) rc = build_batch_graph(h, kind);
      if (rc != ALB_OK) return rc;
    }
  }
  if (!b->ev_start) ALB_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming));
  if (made) ALB_CUDA_TRY(cudaDeviceSynchronize());
  if (want > b->nworkers) b->nworkers = want;
  return ALB_OK;
}

static alb_status run_groups(alb_graph g, BatchKind kind, const uint32_t* hd_srcs, uint32_t k,
                             uint32_t* out, cudaStream_t s) {
  alb_status rc = ensure_batch(g, true, k, s);
  if (rc != ALB_OK) return rc;
  BatchWs* b = g->batch;
  if ((rc = stage_srcs(g, hd_srcs, k, s)) != ALB_OK) return rc;
  const bool host_loop = g->params.exec_mode == 1;
  if (!host_loop && !b->exec[kind] &&
      ((rc = setup_barrier()) != ALB_OK || (rc = build_batch_graph(g, kind)) != ALB_OK))
    return rc;
  const bool dev = is_device_ptr(out);
  const size_t n = g->n;
  const uint32_t ngroups = (k + 31u) / 32u;
  b->used_workers = 0;
  if (dev && ngroups > 1 && !host_loop) {
    // several groups with a device output: deal them over the handle and its worker clones
    const uint32_t W = ngroups < kBatchWorkers ? ngroups : kBatchWorkers;
    const int app = kind == BK_MS_BFS ? ALB_APP_BFS : ALB_APP_SSSP;
    alb_status rc2 = ensure_workers(g, kind, app, W - 1);
    if (rc2 != ALB_OK) return rc2;
    select_cfg(g, app);
    ALB_CUDA_TRY(cudaEventRecord(b->ev_start, s));
    for (uint32_t w = 0; w + 1 < W; ++w) ALB_CUDA_TRY(cudaStreamWaitEvent(b->wstream[w], b->ev_start, 0));
    for (uint32_t gi = 0; gi < ngroups; ++gi) {
      const uint32_t w = gi % W, g0 = 32u * gi;
      const uint32_t ns = (k - g0) < 32u ? (k - g0) : 32u;
      alb_graph h = w == 0 ? g : b->worker[w - 1];
      cudaStream_t hs = w == 0 ? s : b->wstream[w - 1];
      if ((rc2 = run_group_on(h, kind, b->srcs + g0, ns, out + (size_t)g0 * n, hs)) != ALB_OK) return rc2;
    }
    for (uint32_t w = 0; w + 1 < W; ++w) {
      ALB_CUDA_TRY(cudaEventRecord(b->ev_done[w], b->wstream[w]));
      ALB_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_done[w], 0));
    }
    b->used_workers = W - 1;
    g->last_stream = s;
    g->last_kind = 0;
    return ALB_OK;
  }
  if (!dev && !b->tmp) {
    if ((rc = setup_barrier()) != ALB_OK) return rc;
    ALB_CUDA_TRY(cudaMalloc((void**)&b->tmp, sizeof(uint32_t) * (size_t)g->n * 32u));
  }
  for (uint32_t g0 = 0; g0 < k; g0 += 32u) {
    const uint32_t ns = (k - g0) < 32u ? (k - g0) : 32u;
    uint32_t* dst = dev ? out + (size_t)g0 * n : b->tmp;
    CallArgs ca{dst, 0u, 0u, nullptr, nullptr, nullptr, b->aux, b->srcs + g0, ns};
    k_set_args<<<1, 1, 0, s>>>(g->args, ca);
    ALB_CUDA_TRY(cudaGetLastError());
    if (host_loop) {
      if ((rc = batch_host_loop(g, kind, s)) != ALB_OK) return rc;
    } else {
      ALB_CUDA_TRY(cudaGraphLaunch(b->exec[kind], s));
    }
    if (!dev)
      ALB_CUDA_TRY(cudaMemcpyAsync(out + (size_t)g0 * n, b->tmp, sizeof(uint32_t) * n * ns,
                                   cudaMemcpyDeviceToHost, s));
  }
  g->last_stream = s;
  g->last_kind = 0;
  return ALB_OK;
}

static alb_status run_multi(alb_graph g, BatchKind kind, const uint32_t* hd_srcs, uint32_t k,
                            uint32_t* out, cudaStream_t s) {
  alb_status rc = ensure_batch(g, false, k, s);
  if (rc != ALB_OK) return rc;
  BatchWs* b = g->batch;
  if ((rc = stage_srcs(g, hd_srcs, k, s)) != ALB_OK) return rc;
  const bool host_loop = g->params.exec_mode == 1;
  if (!host_loop && !b->exec[kind] &&
      ((rc = setup_barrier()) != ALB_OK || (rc = build_batch_graph(g, kind)) != ALB_OK))
    return rc;
  const bool dev = is_device_ptr(out);
  uint32_t* lab = out;
  if (!dev) {
    if ((rc = ensure_tmp(g)) != ALB_OK) return rc;
    lab = g->tmp;
  }
  CallArgs ca{lab, 0u, 0u, nullptr, nullptr, nullptr, nullptr, b->srcs, k};
  k_set_args<<<1, 1, 0, s>>>(g->args, ca);
  ALB_CUDA_TRY(cudaGetLastError());
  if (host_loop) {
    if ((rc = batch_host_loop(g, kind, s)) != ALB_OK) return rc;
  } else {
    ALB_CUDA_TRY(cudaGraphLaunch(b->exec[kind], s));
  }
  if (!dev) ALB_CUDA_TRY(cudaMemcpyAsync(out, lab, sizeof(uint32_t) * g->n, cudaMemcpyDeviceToHost, s));
  g->last_stream = s;
  g->last_kind = 0;
  return ALB_OK;
}

}  // namespace alb

using namespace alb;

// A batched call starts the per-kernel timers of alb_stats afresh (profile = 1, host loop).
static void begin_batch(alb_graph g, int app) {
  select_cfg(g, app);
  g->stats.ms_inspect = g->stats.ms_lb = g->stats.ms_other = 0.0;
  g->stats.n_inspect = g->stats.n_lb = g->stats.n_other = 0;
}

static alb_status sssp_ok(alb_graph g) {
  if (!g->has_w) return ALB_ERR_UNSUPPORTED;
  if ((uint64_t)g->max_w * (uint64_t)(g->n - 1) >= 0xFFFFFFFFull) return ALB_ERR_OVERFLOW;
  return ALB_OK;
}

extern "C" alb_status alb_bfs_batch(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_out,
                                    alb_stream stream) {
  if (!g || (k && (!hd_srcs || !hd_out))) return ALB_ERR_INVALID_ARG;
  if (k == 0) return ALB_OK;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  begin_batch(g, ALB_APP_BFS);
  return run_groups(g, BK_MS_BFS, hd_srcs, k, hd_out, (cudaStream_t)stream);
}

extern "C" alb_status alb_sssp_batch(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_out,
                                     alb_stream stream) {
  if (!g || (k && (!hd_srcs || !hd_out))) return ALB_ERR_INVALID_ARG;
  alb_status rc = sssp_ok(g);
  if (rc != ALB_OK) return rc;
  if (k == 0) return ALB_OK;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  begin_batch(g, ALB_APP_SSSP);
  return run_groups(g, BK_MS_SSSP, hd_srcs, k, hd_out, (cudaStream_t)stream);
}

extern "C" alb_status alb_bfs_multi(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_levels,
                                    alb_stream stream) {
  if (!g || !hd_srcs || !hd_levels || k == 0) return ALB_ERR_INVALID_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  begin_batch(g, ALB_APP_BFS);
  return run_multi(g, BK_MULTI_BFS, hd_srcs, k, hd_levels, (cudaStream_t)stream);
}

extern "C" alb_status alb_sssp_multi(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_dist,
                                     alb_stream stream) {
  if (!g || !hd_srcs || !hd_dist || k == 0) return ALB_ERR_INVALID_ARG;
  alb_status rc = sssp_ok(g);
  if (rc != ALB_OK) return rc;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  begin_batch(g, ALB_APP_SSSP);
  return run_multi(g, BK_MULTI_SSSP, hd_srcs, k, hd_dist, (cudaStream_t)stream);
}
