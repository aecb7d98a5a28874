// Internal declarations of libalb.so: device-side round state, the kernel
// context passed by value to every round kernel, and the host-side graph handle.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "alb.h"

namespace alb {

constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr int kBlock = 256;             // threads per CTA of every round kernel
constexpr int kWarps = kBlock / 32;
constexpr int kHubSmem = 2048;          // huge vertices the LB kernel stages in shared memory
constexpr uint32_t kFull = 0xFFFFFFFFu;

// Latched device error bits.
enum : uint32_t { ST_ERR_ROUNDS = 1u, ST_ERR_INDEX = 2u, ST_ERR_SRC = 4u };

enum App : int { APP_BFS = 0, APP_SSSP = 1, APP_CC = 2, APP_KCORE = 3, APP_TRACE = 4, APP_COUNT = 5 };

// Device-resident state of one traversal, zeroed before each call.
struct RoundState {
  uint32_t round;                  // current round r
  uint32_t fcount[2];              // frontier sizes, indexed by round parity
  uint32_t tile_next;              // dynamic tile counter of the inspection kernel
  unsigned long long hub_packed;   // (huge count << 32) | huge edge total, one atomic per warp
  uint32_t done_inspect;           // last-block tickets
  uint32_t done_lb;
  uint32_t status;                 // ST_ERR_* bits
  uint32_t all_active;             // round 0 of cc: the frontier is every vertex
  uint32_t hub_rounds;
  uint32_t max_hub_count;
  unsigned long long edges_twc;
  unsigned long long edges_lb;
  unsigned long long pushes;
};

// Per-call arguments, written on the stream by a one-thread kernel before the
// (cached) CUDA graph of the application is launched.
struct CallArgs {
  uint32_t* lab;      // labels being computed (levels, dist, labels, remaining degree)
  uint32_t src;
  uint32_t k;         // kcore
  uint32_t* trace_src;
  uint32_t* trace_dst;
  uint32_t* trace_thread;
  const void* aux;    // multi-source operators: their BatchAux
  const uint32_t* srcs;  // sources of a multi-source call
  uint32_t nsrc;
};

// Everything a round kernel needs, passed by value (fixed for a cached graph).
struct TravCtx {
  const uint32_t* off;
  const uint32_t* idx;
  const uint32_t* w;
  uint32_t n;
  uint32_t threshold;     // degree >= threshold: huge (Algorithm 1)
  uint32_t warp_min;      // TWC warp bin lower bound
  uint32_t cta_min;       // TWC CTA bin lower bound
  uint32_t distribution;  // 0 cyclic, 1 blocked (Algorithm 2)
  uint32_t max_rounds;
  uint32_t use_graph;     // conditional handles valid
  uint32_t m;             // CSR entries (bounds of the checked build)
  uint32_t* F0;           // frontier buffers (round parity 0 / 1)
  uint32_t* F1;
  uint32_t* hub_v;        // huge worklist "work"
  uint32_t* hub_p;        // exclusive prefix sum of huge degrees ("prefixWork")
  uint32_t* pushed;       // two bitmaps of pw words; bitmap r & 1 marks the vertices pushed in
                          // round r (dedup of next-frontier pushes, sssp and cc)
  uint32_t pw;            // words per bitmap: ceil(n / 32)
  RoundState* st;
  const CallArgs* args;
  cudaGraphConditionalHandle h_while;
  cudaGraphConditionalHandle h_if;
  uint32_t* chk;          // checked build: first failed bound (code, index, bound, count)
  unsigned long long* cta_twc;  // per-CTA edges expanded by the TWC kernel (cta_stats; else null)
  unsigned long long* cta_lb;   // per-CTA edges expanded by the LB kernel
};

// Codes recorded by the checked build (-DALB_CHECKED) when an index is out of range; the
// access is skipped instead of faulting.
enum : uint32_t {
  CHK_EDGE = 1,      // edge index >= m
  CHK_DST = 2,       // destination vertex >= n
  CHK_FRONTIER = 3,  // frontier entry >= n
  CHK_PUSH = 4,      // next-frontier slot >= n
  CHK_HUB = 5,       // huge-worklist slot > n
  CHK_ROW = 6,       // multi-source label row >= n
  CHK_SRC = 7,       // LB source index >= number of huge vertices
  CHK_STATE = 8,     // round state out of range (frontier size > n, huge count > n, edges > m)
  CHK_PTR = 9,       // a pointer read from device memory is null or misaligned
};

}  // namespace alb

// Host-side handle.
struct alb_graph_s {
  int device = 0;
  uint32_t n = 0;
  uint64_t m = 0;
  uint32_t flags = 0;
  bool has_w = false;
  uint32_t max_w = 0;
  uint32_t max_deg = 0;
  uint32_t* off = nullptr;
  uint32_t* idx = nullptr;
  uint32_t* w = nullptr;
  std::atomic<int>* csr_refs = nullptr;  // handles sharing off/idx/w (alb_graph_clone); the last frees them

  // per-application launch configuration (indexed by alb_app); the fields below hold the
  // configuration of the application being called (select_cfg copies it in)
  struct AppCfg {
    alb_params p{};
    uint32_t blocks = 0, lb_blocks = 0, threshold = 0, block = alb::kBlock;
  } cfg[5];
  alb_params params{};
  int num_sms = 0;
  uint32_t blocks = 0;        // CTAs of the inspection / init kernels (persistent grid)
  uint32_t lb_blocks = 0;     // CTAs of the LB kernel (its threads are the default threshold)
  uint32_t threshold = 0;     // effective huge threshold
  uint32_t block = alb::kBlock;  // threads per CTA of the round kernels

  // traversal workspace
  uint32_t* F0 = nullptr;
  uint32_t* F1 = nullptr;
  uint32_t* hub_v = nullptr;
  uint32_t* hub_p = nullptr;
  uint32_t* pushed = nullptr;       // 2 x ceil(n / 32) words (TravCtx::pushed)
  uint32_t* tmp = nullptr;        // n-entry scratch output when the caller's buffer is host memory
  alb::RoundState* st = nullptr;
  alb::CallArgs* args = nullptr;
  alb::RoundState* h_st = nullptr;  // pinned mirror
  uint32_t* chk = nullptr;          // 4 words: checked-build bound failures (never reset)
  unsigned long long* cta_twc = nullptr;  // per-CTA load counters (cta_stats)
  unsigned long long* cta_lb = nullptr;
  uint32_t cta_cap = 0;             // entries of each counter array
  uint32_t cta_n_twc = 0, cta_n_lb = 0;  // CTAs of the last instrumented call

  cudaGraph_t graph[alb::APP_COUNT] = {};
  cudaGraphExec_t exec[alb::APP_COUNT] = {};

  cudaStream_t last_stream = nullptr;
  int last_kind = -1;            // 0 traversal, 1 pagerank
  alb_status latched = ALB_OK;
  alb_stats stats{};

  // pagerank workspace (alb_pagerank.cu)
  struct PrWs* pr = nullptr;
  // batch workspace (alb_batch.cu)
  struct BatchWs* batch = nullptr;
};

namespace alb {

// ---- helpers shared by the host translation units -----------------------------------------
#define ALB_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) {                                                 \
      if (std::getenv("ALB_DEBUG"))                                          \
        std::fprintf(stderr, "libalb: %s failed: %s (%s:%d)\n", #expr,       \
                     cudaGetErrorString(_e), __FILE__, __LINE__);            \
      return (_e == cudaErrorMemoryAllocation) ? ALB_ERR_OOM : ALB_ERR_CUDA; \
    }                                                                        \
  } while (0)

bool is_device_ptr(const void* p);
// Set-up (a device allocation, a CUDA-graph instantiation, PageRank's per-graph inspection) runs
// with the device idle: this waits for all work on the device. A handle's first call of each kind
// calls it once, so no set-up ever overlaps kernels of other handles or streams.
alb_status setup_barrier();
alb_status ensure_tmp(alb_graph g);
alb_status traversal_status(alb_graph g);   // reads h_st after a sync
alb_status free_traversal_graphs(alb_graph g);
alb_status free_pagerank(alb_graph g);
alb_status free_batch(alb_graph g);
TravCtx make_ctx(alb_graph g, bool use_graph, cudaGraphConditionalHandle hw,
                 cudaGraphConditionalHandle hi);
alb_status run_traversal(alb_graph g, App app, uint32_t src, uint32_t k, uint32_t* out,
                         cudaStream_t s);
alb_status launch_lb_trace(alb_graph g, const uint32_t* d_work, const uint32_t* d_prefix,
                           uint32_t nwork, uint32_t* d_src, uint32_t* d_dst, uint32_t* d_thread,
                           cudaStream_t s);
alb_status launch_inspect_only(alb_graph g, const uint32_t* d_wl, uint32_t nf, uint8_t* d_bin,
                               uint32_t* d_work, uint32_t* d_prefix, uint32_t* d_counts,
                               cudaStream_t s);
// Resident CTAs per SM of the round kernels built for CTA size B (the least over the apps).
void occupancy(uint32_t B, uint32_t* inspect_per_sm, uint32_t* lb_per_sm);
alb_status pr_stats(alb_graph g, alb_stats* out);
alb_status batch_stats(alb_graph g, alb_stats* out);
alb_status batch_sync_workers(alb_graph g);  // status of the worker clones of the last batch call
alb_status latch_from_state(alb_graph g, uint32_t status);
uint32_t effective_threshold(alb_graph g);
void select_cfg(alb_graph g, int app);
// zero (and size, to at least min_need CTAs) the per-CTA counters
alb_status reset_cta_loads(alb_graph g, cudaStream_t s, uint32_t min_need = 0);

}  // namespace alb
