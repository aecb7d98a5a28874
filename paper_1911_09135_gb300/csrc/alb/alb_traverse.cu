// Data-driven traversals (bfs, sssp, cc, kcore) with the adaptive load balancer
// of arXiv:1911.09135, Sec. 4.
//
// One round = two kernels:
//   k_inspect  Algorithm 1 fused with TWC expansion (Sec. 3, Sec. 4.1): each CTA
//              takes tiles of the frontier, reads every vertex's degree, appends
//              huge vertices (degree >= threshold) to `work` together with their
//              slot of the exclusive prefix sum of huge degrees (one packed 64-bit
//              atomic per warp yields both the slot and the prefix, so prefixWork
//              needs no separate scan pass), and expands the rest at once: CTA bin
//              by the whole CTA, warp bin by one warp, thread bin by a CTA-wide
//              fine-grained gather over the small vertices' edges.
//   k_lb       Algorithm 2: the edges of all huge vertices are dealt cyclically
//              (position k goes to thread k mod p) or blocked over every thread
//              of the grid; the source of position k is found by binary search
//              of prefixWork (staged in shared memory).
// The LB kernel runs only when `work` is non-empty (a conditional graph node).
// Each round's last CTA closes the round on the device (last-block ticket) and
// sets the while-node condition, so whole traversals run without host syncs.
#include "alb_device.cuh"

namespace alb {

// ------------------------------------------------------------------ operators

struct OpArgs {
  uint32_t* lab;
  uint32_t* stamp;
  uint32_t next;  // round + 1
  uint32_t k;
};

// bfs (push): level[dst] = round + 1 if unvisited.
struct BfsOp {
  static constexpr bool kW = false;
  __device__ static uint32_t sval(const OpArgs&, uint32_t) { return 0u; }
  __device__ static bool want(const OpArgs&, uint32_t, uint32_t cur, uint32_t) { return cur == kInf; }
  __device__ static bool commit(const OpArgs& a, uint32_t, uint32_t dst, uint32_t) {
    return atomicCAS(a.lab + dst, kInf, a.next) == kInf;
  }
};

// sssp (push relaxation, Fig. 3): dist[dst] = min(dist[dst], dist[src] + w).
// A vertex whose distance drops is pushed once per round (round stamp).
struct SsspOp {
  static constexpr bool kW = true;
  __device__ static uint32_t sval(const OpArgs& a, uint32_t u) { return a.lab[u]; }
  __device__ static bool want(const OpArgs&, uint32_t sv, uint32_t cur, uint32_t w) {
    return (uint64_t)sv + w < (uint64_t)cur;
  }
  __device__ static bool commit(const OpArgs& a, uint32_t sv, uint32_t dst, uint32_t w) {
    const uint32_t nd = sv + w;
    const uint32_t old = atomicMin(a.lab + dst, nd);
    return nd < old && atomicMax(a.stamp + dst, a.next) < a.next;
  }
};

// cc (push min-label propagation): label[dst] = min(label[dst], label[src]).
struct CcOp {
  static constexpr bool kW = false;
  __device__ static uint32_t sval(const OpArgs& a, uint32_t u) { return a.lab[u]; }
  __device__ static bool want(const OpArgs&, uint32_t sv, uint32_t cur, uint32_t) { return sv < cur; }
  __device__ static bool commit(const OpArgs& a, uint32_t sv, uint32_t dst, uint32_t) {
    const uint32_t old = atomicMin(a.lab + dst, sv);
    return sv < old && atomicMax(a.stamp + dst, a.next) < a.next;
  }
};

// kcore (peeling): a removed vertex decrements each neighbour's remaining
// degree; the neighbour is removed (pushed) exactly when it drops from k to
// k - 1. Neighbours already below k are skipped (their membership is settled).
struct KcoreOp {
  static constexpr bool kW = false;
  __device__ static uint32_t sval(const OpArgs&, uint32_t) { return 0u; }
  __device__ static bool want(const OpArgs& a, uint32_t, uint32_t cur, uint32_t) { return cur >= a.k; }
  __device__ static bool commit(const OpArgs& a, uint32_t, uint32_t dst, uint32_t) {
    return atomicSub(a.lab + dst, 1u) == a.k;
  }
};

// Relax U edges per thread; all loads are issued before the atomics so each
// thread keeps U independent memory requests in flight. Warp-uniform callers.
template <class Op, int U>
__device__ __forceinline__ void relax(const TravCtx& c, const OpArgs& a, const uint32_t (&e)[U],
                                      const bool (&ok)[U], const uint32_t (&sv)[U], uint32_t* Fn,
                                      uint32_t* ncount) {
  uint32_t dst[U], wt[U], cur[U];
#pragma unroll
  for (int u = 0; u < U; ++u) dst[u] = ok[u] ? __ldcs(c.idx + e[u]) : 0u;  // streamed once: evict-first
#pragma unroll
  for (int u = 0; u < U; ++u) wt[u] = (Op::kW && ok[u]) ? __ldcs(c.w + e[u]) : 0u;
#pragma unroll
  for (int u = 0; u < U; ++u) cur[u] = ok[u] ? a.lab[dst[u]] : 0u;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const bool push = ok[u] && Op::want(a, sv[u], cur[u], wt[u]) && Op::commit(a, sv[u], dst[u], wt[u]);
    warp_append(push, dst[u], Fn, ncount);
  }
}

// Close round r (one thread of the last CTA): account, reset the per-round
// counters, advance the round and set the while condition.
__device__ void finish_round(const TravCtx& c) {
  RoundState* st = c.st;
  const uint32_t r = __ldcg(&st->round);
  const uint32_t cur = r & 1u;
  const uint32_t nextc = __ldcg(&st->fcount[cur ^ 1u]);
  const unsigned long long hp = __ldcg(&st->hub_packed);
  const uint32_t nh = (uint32_t)(hp >> 32);
  if (nh) {
    st->hub_rounds += 1u;
    if (nh > st->max_hub_count) st->max_hub_count = nh;
    st->edges_lb += (uint32_t)hp;
  }
  st->pushes += nextc;
  st->fcount[cur] = 0u;
  st->hub_packed = 0ull;
  st->tile_next = 0u;
  st->done_inspect = 0u;
  st->done_lb = 0u;
  st->all_active = 0u;
  st->round = r + 1u;
  bool go = nextc > 0u;
  if (go && r + 1u >= c.max_rounds) {
    st->status |= ST_ERR_ROUNDS;
    go = false;
  }
  __threadfence();
  if (c.use_graph) cudaGraphSetConditional(c.h_while, go ? 1u : 0u);
}

// Append huge vertices to `work` with their prefixWork entry: one 64-bit atomic
// per warp adds (count << 32 | degree sum), so slot order and prefix order agree.
__device__ __forceinline__ void hub_append(bool huge, uint32_t v, uint32_t deg, uint32_t* hub_v,
                                           uint32_t* hub_p, unsigned long long* packed) {
  const unsigned mask = __ballot_sync(kFull, huge);
  if (mask == 0) return;
  const uint32_t lane = lane_id();
  const uint32_t x = huge ? deg : 0u;
  const uint32_t incl = warp_inclusive_scan(x);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t leader = __ffs(mask) - 1;
  unsigned long long old = 0ull;
  if (lane == leader) old = atomicAdd(packed, ((unsigned long long)__popc(mask) << 32) | total);
  old = __shfl_sync(kFull, old, leader);
  if (huge) {
    const uint32_t slot = (uint32_t)(old >> 32) + __popc(mask & ((1u << lane) - 1u));
    hub_v[slot] = v;
    hub_p[slot] = (uint32_t)old + (incl - x);
  }
}

// ----------------------------------------------------- inspection + TWC kernel

template <class Op>
__global__ void __launch_bounds__(kBlock) k_inspect(TravCtx c) {
  __shared__ uint32_t s_cb[kBlock], s_cd[kBlock], s_cv[kBlock];       // CTA bin
  __shared__ uint32_t s_wb[kBlock], s_wd[kBlock], s_wv[kBlock];       // warp bin
  __shared__ uint32_t s_scan[kBlock + 1], s_sb[kBlock], s_sv[kBlock];  // thread bin
  __shared__ uint32_t s_warp[kWarps + 1];
  __shared__ uint32_t s_ncta, s_nwrp, s_tile;

  RoundState* st = c.st;
  const uint32_t r = st->round;
  const uint32_t cur = r & 1u;
  const bool all = st->all_active != 0u;
  const uint32_t nf = all ? c.n : st->fcount[cur];
  const uint32_t* F = cur ? c.F1 : c.F0;
  uint32_t* Fn = cur ? c.F0 : c.F1;
  uint32_t* ncount = &st->fcount[cur ^ 1u];
  const CallArgs* ca = c.args;
  const OpArgs a{ca->lab, c.stamp, r + 1u, ca->k};
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  unsigned long long twc_edges = 0ull;

  for (;;) {
    if (tid == 0) {
      s_tile = atomicAdd(&st->tile_next, 1u);
      s_ncta = 0u;
      s_nwrp = 0u;
    }
    __syncthreads();
    const uint64_t base = (uint64_t)s_tile * kBlock;
    if (base >= nf) break;  // CTA-uniform
    const uint32_t i = (uint32_t)base + tid;
    const bool valid = i < nf;
    uint32_t v = 0u, beg = 0u, deg = 0u, sv = 0u;
    if (valid) {
      v = all ? i : F[i];
      beg = c.off[v];
      deg = c.off[v + 1] - beg;
      sv = Op::sval(a, v);
    }
    const bool huge = valid && deg >= c.threshold;
    const bool cta = valid && !huge && deg >= c.cta_min;
    const bool wrp = valid && !huge && !cta && deg >= c.warp_min;
    const uint32_t sdeg = (valid && !huge && !cta && !wrp) ? deg : 0u;
    if (valid && !huge) twc_edges += deg;
    hub_append(huge, v, deg, c.hub_v, c.hub_p, &st->hub_packed);
    if (cta) {
      const uint32_t s = atomicAdd(&s_ncta, 1u);
      s_cb[s] = beg; s_cd[s] = deg; s_cv[s] = sv;
    }
    if (wrp) {
      const uint32_t s = atomicAdd(&s_nwrp, 1u);
      s_wb[s] = beg; s_wd[s] = deg; s_wv[s] = sv;
    }
    uint32_t stotal;
    const uint32_t ex = block_exclusive_scan<kBlock>(sdeg, s_warp, &stotal);
    s_scan[tid] = ex;
    s_sb[tid] = beg;
    s_sv[tid] = sv;
    if (tid == 0) s_scan[kBlock] = stotal;
    __syncthreads();

    // CTA bin: the whole CTA expands one vertex at a time.
    const uint32_t ncta = s_ncta;
    for (uint32_t j = 0; j < ncta; ++j) {
      const uint32_t b = s_cb[j], d = s_cd[j], svj = s_cv[j];
      for (uint32_t e0 = 0; e0 < d; e0 += kBlock * 4) {
        uint32_t e[4], s4[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t q = e0 + u * kBlock + tid;
          ok[u] = q < d; e[u] = b + q; s4[u] = svj;
        }
        relax<Op, 4>(c, a, e, ok, s4, Fn, ncount);
      }
    }
    // Warp bin: one warp per vertex.
    const uint32_t nw = s_nwrp;
    for (uint32_t j = warp; j < nw; j += kWarps) {
      const uint32_t b = s_wb[j], d = s_wd[j], svj = s_wv[j];
      for (uint32_t e0 = 0; e0 < d; e0 += 32 * 4) {
        uint32_t e[4], s4[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t q = e0 + u * 32 + lane;
          ok[u] = q < d; e[u] = b + q; s4[u] = svj;
        }
        relax<Op, 4>(c, a, e, ok, s4, Fn, ncount);
      }
    }
    // Thread bin: the small vertices' edges, gathered over the whole CTA
    // (consecutive threads take consecutive edges of the concatenated lists).
    const uint32_t S = s_scan[kBlock];
    uint32_t owner = 0u;
    for (uint32_t q0 = 0; q0 < S; q0 += kBlock * 2) {
      uint32_t e[2], s2[2];
      bool ok[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint32_t q = q0 + u * kBlock + tid;
        ok[u] = q < S;
        e[u] = 0u; s2[u] = 0u;
        if (ok[u]) {
          owner = upper_search(s_scan, owner, kBlock, q);
          e[u] = s_sb[owner] + (q - s_scan[owner]);
          s2[u] = s_sv[owner];
        }
      }
      relax<Op, 2>(c, a, e, ok, s2, Fn, ncount);
    }
    __syncthreads();
  }

  // statistics: one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) twc_edges += __shfl_down_sync(kFull, twc_edges, o);
  if (lane == 0 && twc_edges) atomicAdd(&st->edges_twc, twc_edges);

  if (last_block_ticket(&st->done_inspect)) {
    const unsigned long long hp = __ldcg(&st->hub_packed);
    const uint32_t nh = (uint32_t)(hp >> 32);
    if (c.use_graph) cudaGraphSetConditional(c.h_if, nh > 0u ? 1u : 0u);
    if (nh == 0u) finish_round(c);
  }
}

// ------------------------------------------------------------- LB kernel

struct TraceOp {};

template <class Op, bool kTrace>
__global__ void __launch_bounds__(kBlock) k_lb(TravCtx c) {
  constexpr int kStage = kHubSmem;
  __shared__ uint32_t s_p[kStage];
  __shared__ uint32_t s_base[kStage];
  __shared__ uint32_t s_val[kStage];
  __shared__ uint32_t s_src[kTrace ? kStage : 1];

  RoundState* st = c.st;
  const unsigned long long hp = st->hub_packed;
  const uint32_t nh = (uint32_t)(hp >> 32);
  const uint32_t e = (uint32_t)hp;
  const uint32_t r = st->round;
  const uint32_t cur = r & 1u;
  uint32_t* Fn = cur ? c.F0 : c.F1;
  uint32_t* ncount = &st->fcount[cur ^ 1u];
  const CallArgs* ca = c.args;
  const OpArgs a{ca->lab, c.stamp, r + 1u, ca->k};
  const uint32_t tid = threadIdx.x, lane = tid & 31u;

  const bool staged = nh <= (uint32_t)kStage;
  if (staged) {
    for (uint32_t j = tid; j < nh; j += kBlock) {
      const uint32_t u = c.hub_v[j], p = c.hub_p[j];
      s_p[j] = p;
      s_base[j] = c.off[u] - p;
      if constexpr (kTrace) s_src[j] = u;
      else s_val[j] = Op::sval(a, u);
    }
  }
  __syncthreads();
  const uint32_t* P = staged ? s_p : c.hub_p;

  // source lookup for position k; j only grows along a thread's positions
  uint32_t j = 0u, jc = kInf, base_c = 0u, val_c = 0u, src_c = 0u;
  auto resolve = [&](uint32_t k, uint32_t& edge, uint32_t& sv, uint32_t& src) {
    j = upper_search(P, j, nh, k);
    if (staged) {
      edge = k + s_base[j];
      if constexpr (kTrace) { src = s_src[j]; sv = 0u; }
      else { sv = s_val[j]; src = 0u; }
    } else {
      if (j != jc) {
        const uint32_t u = c.hub_v[j];
        base_c = c.off[u] - c.hub_p[j];
        if constexpr (!kTrace) val_c = Op::sval(a, u);
        src_c = u;
        jc = j;
      }
      edge = k + base_c; sv = val_c; src = src_c;
    }
  };

  const uint64_t p = (uint64_t)gridDim.x * kBlock;
  const uint64_t gt = (uint64_t)blockIdx.x * kBlock + tid;
  constexpr int U = 4;
  auto process = [&](const uint64_t (&k)[U], const bool (&ok)[U]) {
    uint32_t ed[U], sv[U], src[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ed[u] = 0u; sv[u] = 0u; src[u] = 0u;
      if (ok[u]) resolve((uint32_t)k[u], ed[u], sv[u], src[u]);
    }
    if constexpr (kTrace) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (ok[u]) {
          ca->trace_src[k[u]] = src[u];
          ca->trace_dst[k[u]] = c.idx[ed[u]];
          ca->trace_thread[k[u]] = (uint32_t)gt;
        }
      }
    } else {
      relax<Op, U>(c, a, ed, ok, sv, Fn, ncount);
    }
  };

  if (c.distribution == 0u) {
    // cyclic: thread gt takes positions gt, gt + p, gt + 2p, ... (Sec. 4.1)
    for (uint64_t k0 = gt - lane; k0 < e; k0 += p * U) {  // warp-uniform
      uint64_t k[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) { k[u] = k0 + lane + (uint64_t)u * p; ok[u] = k[u] < e; }
      process(k, ok);
    }
  } else {
    // blocked: thread gt takes [gt * C, min(e, (gt + 1) * C)), C = ceil(e / p)
    const uint64_t C = (e + p - 1) / p;
    const uint64_t lo = gt * C;
    const uint64_t hi = (lo + C < (uint64_t)e) ? lo + C : (uint64_t)e;
    for (uint64_t i0 = 0; i0 < C; i0 += U) {  // uniform trip count
      uint64_t k[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) { k[u] = lo + i0 + u; ok[u] = k[u] < hi; }
      process(k, ok);
    }
  }

  if (last_block_ticket(&st->done_lb)) {
    if constexpr (!kTrace) finish_round(c);
  }
}

// ------------------------------------------------------------- init kernels

template <int APP>
__global__ void __launch_bounds__(kBlock) k_init(TravCtx c) {
  const CallArgs* ca = c.args;
  uint32_t* lab = ca->lab;
  const uint32_t src = ca->src, k = ca->k, n = c.n;
  RoundState* st = c.st;
  for (uint64_t b = (uint64_t)blockIdx.x * kBlock; b < n; b += (uint64_t)gridDim.x * kBlock) {
    const uint32_t v = (uint32_t)b + threadIdx.x;
    const bool ok = v < n;
    if constexpr (APP == APP_BFS) {
      if (ok) lab[v] = (v == src) ? 0u : kInf;
    } else if constexpr (APP == APP_SSSP) {
      if (ok) { lab[v] = (v == src) ? 0u : kInf; c.stamp[v] = 0u; }
    } else if constexpr (APP == APP_CC) {
      if (ok) { lab[v] = v; c.stamp[v] = 0u; }
    } else if constexpr (APP == APP_KCORE) {
      uint32_t d = 0u;
      if (ok) { d = c.off[v + 1] - c.off[v]; lab[v] = d; }
      warp_append(ok && d < k, v, c.F0, &st->fcount[0]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if constexpr (APP == APP_BFS || APP == APP_SSSP) { c.F0[0] = src; st->fcount[0] = 1u; }
    if constexpr (APP == APP_CC) { st->all_active = 1u; st->fcount[0] = n; }
  }
}

// k-core output: remaining degree >= k  ->  1, else 0 (in place).
__global__ void k_kcore_finish(const CallArgs* ca, uint32_t n) {
  uint32_t* lab = ca->lab;
  const uint32_t k = ca->k;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    lab[v] = lab[v] >= k ? 1u : 0u;
}

__global__ void k_set_args(CallArgs* dst, CallArgs v) { *dst = v; }

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

static void* inspect_fn(App app) {
  switch (app) {
    case APP_BFS: return (void*)k_inspect<BfsOp>;
    case APP_SSSP: return (void*)k_inspect<SsspOp>;
    case APP_CC: return (void*)k_inspect<CcOp>;
    case APP_KCORE: return (void*)k_inspect<KcoreOp>;
    default: return nullptr;
  }
}
static void* lb_fn(App app) {
  switch (app) {
    case APP_BFS: return (void*)k_lb<BfsOp, false>;
    case APP_SSSP: return (void*)k_lb<SsspOp, false>;
    case APP_CC: return (void*)k_lb<CcOp, false>;
    case APP_KCORE: return (void*)k_lb<KcoreOp, false>;
    case APP_TRACE: return (void*)k_lb<BfsOp, true>;
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
void occupancy(uint32_t* inspect_per_sm, uint32_t* lb_per_sm) {
  int mi = 1 << 30, ml = 1 << 30;
  for (int a = APP_BFS; a <= APP_KCORE; ++a) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, inspect_fn((App)a), kBlock, 0) == cudaSuccess)
      mi = b < mi ? b : mi;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lb_fn((App)a), kBlock, 0) == cudaSuccess)
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
  c.stamp = g->stamp;
  c.st = g->st;
  c.args = g->args;
  c.h_while = hw;
  c.h_if = hi;
  return c;
}

static alb_status add_kernel(cudaGraphNode_t* node, cudaGraph_t graph, const cudaGraphNode_t* dep,
                             size_t ndep, void* fn, uint32_t grid, TravCtx* c) {
  cudaKernelNodeParams kp{};
  void* kargs[] = {c};
  kp.func = fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(kBlock);
  kp.sharedMemBytes = 0;
  kp.kernelParams = kargs;
  ALB_CUDA_TRY(cudaGraphAddKernelNode(node, graph, dep, ndep, &kp));
  return ALB_OK;
}

// memset(state) -> init -> while(frontier non-empty) { inspect -> if(work) { lb } } [-> kcore finish]
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
  if ((rc = add_kernel(&n_insp, body, nullptr, 0, inspect_fn(app), g->blocks, &c)) != ALB_OK)
    return fail(rc);
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hi;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  if (cudaGraphAddNode(&n_if, body, &n_insp, nullptr, 1, &ip) != cudaSuccess) return fail(ALB_ERR_CUDA);
  cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
  if ((rc = add_kernel(&n_lb, ifbody, nullptr, 0, lb_fn(app), g->lb_blocks, &c)) != ALB_OK)
    return fail(rc);
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
      ALB_CUDA_TRY(cudaLaunchKernel(inspect_fn(app), dim3(g->blocks), dim3(kBlock), args, 0, s));
      g->stats.ms_inspect += t.stop();
      g->stats.n_inspect += 1;
    }
    ALB_CUDA_TRY(cudaMemcpyAsync(g->h_st, g->st, sizeof(RoundState), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    if (g->h_st->hub_packed >> 32) {
      Timer t(prof, s);
      void* args[] = {&c};
      ALB_CUDA_TRY(cudaLaunchKernel(lb_fn(app), dim3(g->lb_blocks), dim3(kBlock), args, 0, s));
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
  uint32_t* lab = out;
  if (!dev) {
    alb_status rc = ensure_tmp(g);
    if (rc != ALB_OK) return rc;
    lab = g->tmp;
  }
  CallArgs ca{lab, src, k, nullptr, nullptr, nullptr};
  k_set_args<<<1, 1, 0, s>>>(g->args, ca);
  ALB_CUDA_TRY(cudaGetLastError());
  if (g->params.exec_mode == 0) {
    if (!g->exec[app]) {
      alb_status rc = build_graph(g, app);
      if (rc != ALB_OK) return rc;
    }
    ALB_CUDA_TRY(cudaGraphLaunch(g->exec[app], s));
  } else {
    alb_status rc = host_loop(g, app, s);
    if (rc != ALB_OK) return rc;
  }
  if (!dev) ALB_CUDA_TRY(cudaMemcpyAsync(out, lab, sizeof(uint32_t) * g->n, cudaMemcpyDeviceToHost, s));
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
  ALB_CUDA_TRY(cudaLaunchKernel(lb_fn(APP_TRACE), dim3(g->lb_blocks), dim3(kBlock), args, 0, s));
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
constexpr size_t kNoAllocBytes = 4 * kNoAllocVec + 3 * 256;

// Shared by every call on a device: calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocCheck {
  uint32_t bad;
  uint32_t off0;
  uint32_t offn;
};

// One pass over the caller's CSR, so the traversal kernels never index out of range.
__global__ void k_noalloc_check(const uint32_t* off, const uint32_t* idx, uint32_t n, uint64_t m,
                                NoAllocCheck* out) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t bad = 0;
  for (uint64_t v = tid; v < n; v += stride)
    if (off[v + 1] < off[v]) bad = 1;
  for (uint64_t e = tid; e < m; e += stride)
    if (idx[e] >= n) bad = 1;
  if (bad) atomicOr(&out->bad, 1u);
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
  RoundState* st = reinterpret_cast<RoundState*>(base + 4 * kNoAllocVec);
  CallArgs* args = reinterpret_cast<CallArgs*>(base + 4 * kNoAllocVec + 256);
  NoAllocCheck* chk = reinterpret_cast<NoAllocCheck*>(base + 4 * kNoAllocVec + 512);
  static_assert(sizeof(RoundState) <= 256 && sizeof(CallArgs) <= 256, "scratch layout");

  int dev = 0, sms = 0;
  ALB_CUDA_TRY(cudaGetDevice(&dev));
  ALB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint32_t occ_i = 1, occ_l = 1;
  occupancy(&occ_i, &occ_l);
  const uint32_t blocks = (uint32_t)sms * occ_i, lb_blocks = (uint32_t)sms * occ_l;

  // validate the caller's CSR (this call's contents of the shared scratch start here)
  NoAllocCheck h{};
  ALB_CUDA_TRY(cudaMemsetAsync(chk, 0, sizeof(NoAllocCheck), s));
  k_noalloc_check<<<(unsigned)sms * 4, 256, 0, s>>>(d_offsets, d_indices, n, m, chk);
  ALB_CUDA_TRY(cudaGetLastError());
  ALB_CUDA_TRY(cudaMemcpyAsync(&h, chk, sizeof(h), cudaMemcpyDeviceToHost, s));
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.off0 != 0u || (uint64_t)h.offn != m) return ALB_ERR_INVALID_ARG;
  if (h.bad) return ALB_ERR_DEVICE;

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
  c.stamp = nullptr;  // bfs needs no round stamps
  c.st = st;
  c.args = args;

  CallArgs ca{d_levels, src, 0u, nullptr, nullptr, nullptr};
  k_set_args<<<1, 1, 0, s>>>(args, ca);
  ALB_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(RoundState), s));  // counters must start at zero
  void* kargs[] = {&c};
  ALB_CUDA_TRY(cudaLaunchKernel((void*)k_init<APP_BFS>, dim3(blocks), dim3(kBlock), kargs, 0, s));
  RoundState hs{};
  for (;;) {
    ALB_CUDA_TRY(cudaLaunchKernel((void*)k_inspect<BfsOp>, dim3(blocks), dim3(kBlock), kargs, 0, s));
    ALB_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.hub_packed >> 32) {
      ALB_CUDA_TRY(cudaLaunchKernel((void*)k_lb<BfsOp, false>, dim3(lb_blocks), dim3(kBlock), kargs, 0, s));
      ALB_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
      ALB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (hs.status & ST_ERR_ROUNDS) return ALB_ERR_TIMEOUT;
    if (hs.fcount[hs.round & 1u] == 0u) break;
  }
  return ALB_OK;
}
