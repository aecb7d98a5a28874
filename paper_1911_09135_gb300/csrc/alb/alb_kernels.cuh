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
#pragma once

#include "alb_device.cuh"

namespace alb {

// ------------------------------------------------------------------ operators

struct OpArgs {
  uint32_t* lab;
  uint32_t* pushed;  // this round's push bitmap (sssp, cc); the visited bitmap (bfs)
  uint32_t next;     // round + 1
  uint32_t k;
  const void* aux;  // operator-specific state (the multi-source operators)
  uint32_t n;
  uint32_t* chk;    // checked build
};

// bfs (push): level[dst] = round + 1 if unvisited. Visited vertices are kept in a bitmap (one bit
// per vertex, set once for the whole traversal): the per-edge probe reads a bitmap word, which
// stays in L2 (2 MB at 2^24 vertices) where the 4-byte level array (64 MB) would compete with the
// streamed CSR, and the atomicOr that sets the bit claims the vertex, whose level is then a plain
// store.
struct BfsOp {
  static constexpr bool kBatch = false;
  static constexpr bool kW = false;
  static constexpr bool kVisited = true;
  __device__ static uint32_t sval(const OpArgs&, uint32_t) { return 0u; }
  __device__ static bool want(const OpArgs&, uint32_t, uint32_t cur, uint32_t) { return cur == kInf; }
  __device__ static bool commit(const OpArgs& a, uint32_t, uint32_t dst, uint32_t) {
    return atomicCAS(a.lab + dst, kInf, a.next) == kInf;
  }
  // U edges at once: the U CAS are issued before any result is used
  template <int U>
  __device__ static void commit_u(const OpArgs& a, const uint32_t (&)[U], const uint32_t (&dst)[U],
                                  const uint32_t (&)[U], const bool (&w)[U], bool (&push)[U]) {
    uint32_t old[U];
#pragma unroll
    for (int u = 0; u < U; ++u) old[u] = w[u] ? atomicCAS(a.lab + dst[u], kInf, a.next) : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) push[u] = w[u] && old[u] == kInf;
  }
};

// Push of a min operator's destination, at most once per round: the first thread to set the
// vertex's bit in this round's bitmap pushes it (a plain read of the word skips the atomic when
// the bit is already set). The bitmaps are 1/32 the size of a per-vertex round stamp, so they and
// the labels stay in L2 together.
__device__ __forceinline__ bool claim_push(const OpArgs& a, uint32_t dst) {
  const uint32_t bit = 1u << (dst & 31u);
  uint32_t* word = a.pushed + (dst >> 5);
  return !(*word & bit) && !(atomicOr(word, bit) & bit);
}

// The min operators' U-edge commit: U non-returning atomicMin, then U bitmap reads, then the
// atomicOr of the bits not yet set, then the push decisions; each group of memory operations is
// issued before any of its results is used.
template <int U, class Cand>
__device__ __forceinline__ void min_commit_u(const OpArgs& a, const uint32_t (&dst)[U], const bool (&w)[U],
                                             bool (&push)[U], Cand cand) {
#pragma unroll
  for (int u = 0; u < U; ++u) if (w[u]) atomicMin(a.lab + dst[u], cand(u));
  uint32_t wd[U];
#pragma unroll
  for (int u = 0; u < U; ++u) wd[u] = w[u] ? a.pushed[dst[u] >> 5] : 0xFFFFFFFFu;
  uint32_t old[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint32_t bit = 1u << (dst[u] & 31u);
    old[u] = (wd[u] & bit) ? bit : atomicOr(a.pushed + (dst[u] >> 5), bit);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) push[u] = w[u] && !(old[u] & (1u << (dst[u] & 31u)));
}

// sssp (push relaxation, Fig. 3): dist[dst] = min(dist[dst], dist[src] + w).
// The atomicMin does not wait for its old value: a destination whose pre-checked distance
// improves is pushed (once per round, by its bit in the round's push bitmap), so every vertex
// whose distance drops is in the next frontier.
struct SsspOp {
  static constexpr bool kBatch = false;
  static constexpr bool kW = true;
  static constexpr bool kPushBitmap = true;
  __device__ static uint32_t sval(const OpArgs& a, uint32_t u) { return a.lab[u]; }
  __device__ static bool want(const OpArgs&, uint32_t sv, uint32_t cur, uint32_t w) {
    return (uint64_t)sv + w < (uint64_t)cur;
  }
  __device__ static bool commit(const OpArgs& a, uint32_t sv, uint32_t dst, uint32_t w) {
    atomicMin(a.lab + dst, sv + w);
    return claim_push(a, dst);
  }
  template <int U>
  __device__ static void commit_u(const OpArgs& a, const uint32_t (&sv)[U], const uint32_t (&dst)[U],
                                  const uint32_t (&wt)[U], const bool (&w)[U], bool (&push)[U]) {
    min_commit_u<U>(a, dst, w, push, [&](int u) { return sv[u] + wt[u]; });
  }
};

// cc (push min-label propagation): label[dst] = min(label[dst], label[src]); the same
// non-blocking update and once-per-round push as sssp.
struct CcOp {
  static constexpr bool kBatch = false;
  static constexpr bool kW = false;
  static constexpr bool kPushBitmap = true;
  __device__ static uint32_t sval(const OpArgs& a, uint32_t u) { return a.lab[u]; }
  __device__ static bool want(const OpArgs&, uint32_t sv, uint32_t cur, uint32_t) { return sv < cur; }
  __device__ static bool commit(const OpArgs& a, uint32_t sv, uint32_t dst, uint32_t) {
    atomicMin(a.lab + dst, sv);
    return claim_push(a, dst);
  }
  template <int U>
  __device__ static void commit_u(const OpArgs& a, const uint32_t (&sv)[U], const uint32_t (&dst)[U],
                                  const uint32_t (&)[U], const bool (&w)[U], bool (&push)[U]) {
    min_commit_u<U>(a, dst, w, push, [&](int u) { return sv[u]; });
  }
};

// kcore (peeling): a removed vertex decrements each neighbour's remaining
// degree; the neighbour is removed (pushed) exactly when it drops from k to
// k - 1. Neighbours already below k are skipped (their membership is settled).
// Lanes of a warp that decrement the same vertex are combined into one
// atomicSub of their count (many peeled vertices share the same high-degree
// neighbours); the group whose subtraction crosses k pushes the vertex.
struct KcoreOp {
  static constexpr bool kBatch = false;
  static constexpr bool kAggregate = true;
  static constexpr bool kW = false;
  __device__ static uint32_t sval(const OpArgs&, uint32_t) { return 0u; }
  __device__ static bool want(const OpArgs& a, uint32_t, uint32_t cur, uint32_t) { return cur >= a.k; }
  __device__ static bool commit_n(const OpArgs& a, uint32_t dst, uint32_t cnt) {
    const uint32_t old = atomicSub(a.lab + dst, cnt);
    return old >= a.k && old - cnt < a.k;
  }
  __device__ static bool commit(const OpArgs& a, uint32_t, uint32_t dst, uint32_t) { return commit_n(a, dst, 1u); }
};

template <class Op, class = void>
struct uses_visited { static constexpr bool value = false; };
template <class Op>
struct uses_visited<Op, decltype(void(Op::kVisited))> { static constexpr bool value = Op::kVisited; };

// The bitmap an operator's OpArgs carries in round parity `cur`: the round's push bitmap, or the
// traversal-wide visited bitmap (bitmap 0).
template <class Op>
__device__ __forceinline__ uint32_t* op_bitmap(const TravCtx& c, uint32_t cur) {
  if (!c.pushed) return nullptr;
  return uses_visited<Op>::value ? c.pushed : c.pushed + (size_t)cur * c.pw;
}

template <class Op, class = void>
struct uses_push_bitmap { static constexpr bool value = false; };
template <class Op>
struct uses_push_bitmap<Op, decltype(void(Op::kPushBitmap))> { static constexpr bool value = Op::kPushBitmap; };

template <class Op, class = void>
struct aggregates { static constexpr bool value = false; };
template <class Op>
struct aggregates<Op, decltype(void(Op::kAggregate))> { static constexpr bool value = Op::kAggregate; };

// CTA-level aggregation of the counted updates (k-core) to high-degree targets. The graph's
// hubs receive most of the decrements (every small vertex has edges to them), and same-address
// atomics serialise in L2; warp aggregation rarely finds two lanes on the same hub. A CTA keeps
// an open-addressing table (key = target, value = pending count) in shared memory for targets
// whose remaining degree is >= kHotDeg and applies it with one atomic per target at the end of
// its round. A full probe window falls back to the direct atomic. k-core's result (the k-core)
// does not depend on the order of the decrements.
constexpr uint32_t kHotBits = 10;
constexpr uint32_t kHotSlots = 1u << kHotBits;
constexpr uint32_t kHotProbe = 4;
constexpr uint32_t kHotDeg = 1u << 16;
static_assert(kHotSlots % 512 == 0, "the table flush loop needs a uniform trip count at every CTA size");

__device__ __forceinline__ bool hot_add(uint32_t* key, uint32_t* cnt, uint32_t v, uint32_t n) {
  uint32_t s = (v * 2654435761u) >> (32 - kHotBits);
  for (uint32_t p = 0; p < kHotProbe; ++p, s = (s + 1u) & (kHotSlots - 1u)) {
    uint32_t k = ((volatile uint32_t*)key)[s];
    if (k == kInf) {
      k = atomicCAS(key + s, kInf, v);
      if (k == kInf) k = v;
    }
    if (k == v) {
      atomicAdd(cnt + s, n);
      return true;
    }
  }
  return false;
}

// Where pushes go: the next frontier (global) and, in the TWC kernel, a CTA staging buffer in
// shared memory. Every warp of every CTA appends to the same frontier counter, and same-address
// atomics serialise in L2, so the TWC kernel collects a tile's pushes in shared memory (one
// shared atomic per warp and step) and moves them to the frontier with one global atomic per
// tile. Pushes that do not fit in the buffer go to the frontier directly.
// Staging entries per CTA: the inspection kernel's tile buffer, and the LB kernel's: 2048, or one
// LB step of the CTA (B threads x 8 positions) if larger.
constexpr uint32_t kTilePushBuf = 2048;
template <int B>
constexpr uint32_t kPushBufOf = (uint32_t)B * 8u > 2048u ? (uint32_t)B * 8u : 2048u;

struct PushSink {
  uint32_t* Fn;      // next frontier
  uint32_t* ncount;  // its length
  uint32_t cap;      // its capacity (n)
  uint32_t* chk;
  uint32_t* sbuf;    // CTA staging buffer (shared memory), or null: push to Fn directly
  uint32_t* sn;      // entries claimed in it (may exceed scap; the excess went to Fn)
  uint32_t scap;     // entries of sbuf
};

// Warp-aggregated push of up to U values per lane (v[u] where pred[u]); every lane of the warp
// calls it.
template <int U>
__device__ __forceinline__ void push_n(const bool (&pred)[U], const uint32_t (&v)[U], const PushSink& k) {
  if (!k.sbuf) {
    warp_append_n<U>(pred, v, k.Fn, k.ncount, k.cap, k.chk);
    return;
  }
  uint32_t cnt = 0u;
#pragma unroll
  for (int u = 0; u < U; ++u) cnt += pred[u] ? 1u : 0u;
  const uint32_t incl = warp_inclusive_scan(cnt);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  if (total == 0u) return;
  uint32_t base = 0u, gbase = 0u;
  if (lane_id() == 0u) {
    base = atomicAdd(k.sn, total);
    const uint32_t end = base + total;
    if (end > k.scap) gbase = atomicAdd(k.ncount, end - (base > k.scap ? base : k.scap));
  }
  base = __shfl_sync(kFull, base, 0);
  gbase = __shfl_sync(kFull, gbase, 0);
  const uint32_t over0 = base > k.scap ? base : k.scap;  // first position sent to Fn
  uint32_t pos = base + incl - cnt;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (pred[u]) {
      if (pos < k.scap) {
        k.sbuf[pos] = v[u];
      } else {
        const uint32_t g = gbase + (pos - over0);
        if (ALB_IN_RANGE(k.chk, 4u, g, k.cap)) k.Fn[g] = v[u];
      }
      ++pos;
    }
  }
}

// Move the staged pushes to the frontier: one global atomic, coalesced stores. Called by every
// thread of the CTA after a barrier that follows the tile's last push.
__device__ __forceinline__ void push_flush(const PushSink& k, uint32_t* s_base) {
  const uint32_t nb = *k.sn < k.scap ? *k.sn : k.scap;
  if (nb == 0u) return;  // CTA-uniform
  if (threadIdx.x == 0) *s_base = atomicAdd(k.ncount, nb);
  __syncthreads();
  const uint32_t b = *s_base;
  for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
    const uint32_t g = b + j;
    if (ALB_IN_RANGE(k.chk, 4u, g, k.cap)) k.Fn[g] = k.sbuf[j];
  }
}

// Relax U edges per thread; all loads are issued before the atomics so each
// thread keeps U independent memory requests in flight. Warp-uniform callers.
// hot_key / hot_cnt: the CTA's aggregation table (counted operators; null = none).
template <class Op, int U>
__device__ __forceinline__ void relax(const TravCtx& c, const OpArgs& a, const uint32_t (&e)[U],
                                      const bool (&ok_in)[U], const uint32_t (&sv)[U], const PushSink& sink,
                                      uint32_t* hot_key = nullptr, uint32_t* hot_cnt = nullptr) {
  uint32_t dst[U], wt[U];
  bool ok[U];
#pragma unroll
  for (int u = 0; u < U; ++u) ok[u] = ok_in[u] && ALB_IN_RANGE(c.chk, CHK_EDGE, e[u], c.m);
#pragma unroll
  for (int u = 0; u < U; ++u) dst[u] = ok[u] ? __ldcs(c.idx + e[u]) : 0u;  // streamed once: evict-first
#pragma unroll
  for (int u = 0; u < U; ++u) ok[u] = ok[u] && ALB_IN_RANGE(c.chk, CHK_DST, dst[u], c.n);
#pragma unroll
  for (int u = 0; u < U; ++u) wt[u] = (Op::kW && ok[u]) ? __ldcs(c.w + e[u]) : 0u;
  if constexpr (Op::kBatch) {
    // multi-source operators do their own label reads (a row of sources per vertex)
    bool push[U];
#pragma unroll
    for (int u = 0; u < U; ++u) push[u] = ok[u] && Op::apply(a, sv[u], dst[u], wt[u]);
    push_n<U>(push, dst, sink);
  } else if constexpr (aggregates<Op>::value) {
    uint32_t cur[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cur[u] = ok[u] ? a.lab[dst[u]] : 0u;
    const uint32_t lane = lane_id();
    bool push[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool w = ok[u] && Op::want(a, sv[u], cur[u], wt[u]);
      const unsigned wm = __ballot_sync(kFull, w);
      push[u] = false;
      if (w) {
        const unsigned grp = __match_any_sync(wm, dst[u]);
        if ((int)lane == __ffs(grp) - 1) {
          const uint32_t cnt = (uint32_t)__popc(grp);
          if (!(hot_key && cur[u] >= kHotDeg && hot_add(hot_key, hot_cnt, dst[u], cnt)))
            push[u] = Op::commit_n(a, dst[u], cnt);
        }
      }
    }
    push_n<U>(push, dst, sink);
  } else if constexpr (uses_visited<Op>::value) {
    // probe the visited bitmap; the atomicOr that sets a bit claims the vertex (U of each issued
    // before any result is used), and the claimant stores the level
    uint32_t wd[U], old[U];
#pragma unroll
    for (int u = 0; u < U; ++u) wd[u] = ok[u] ? a.pushed[dst[u] >> 5] : 0xFFFFFFFFu;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t bit = 1u << (dst[u] & 31u);
      old[u] = (wd[u] & bit) ? bit : atomicOr(a.pushed + (dst[u] >> 5), bit);
    }
    bool push[U];
#pragma unroll
    for (int u = 0; u < U; ++u) push[u] = ok[u] && !(old[u] & (1u << (dst[u] & 31u)));
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (push[u]) a.lab[dst[u]] = a.next;
    push_n<U>(push, dst, sink);
  } else {
    uint32_t cur[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cur[u] = ok[u] ? a.lab[dst[u]] : 0u;
    bool w[U], push[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = ok[u] && Op::want(a, sv[u], cur[u], wt[u]);
    Op::template commit_u<U>(a, sv, dst, wt, w, push);
    push_n<U>(push, dst, sink);
  }
}

// Close round r (one thread of the last CTA): account, reset the per-round
// counters, advance the round and set the while condition.
static __device__ void finish_round(const TravCtx& c) {
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
static __device__ __forceinline__ void hub_append(bool huge, uint32_t v, uint32_t deg, uint32_t* hub_v,
                                           uint32_t* hub_p, unsigned long long* packed,
                                           uint32_t cap = 0xFFFFFFFFu, uint32_t* chk = nullptr) {
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
    if (ALB_IN_RANGE(chk, CHK_HUB, slot, cap)) {
      hub_v[slot] = v;
      hub_p[slot] = (uint32_t)old + (incl - x);
    }
  }
  (void)cap;
  (void)chk;
}

// ----------------------------------------------------- inspection + TWC kernel

// Resident CTAs per SM the round kernels are compiled for: 5 for the single-source operators
// (the register cap costs a few spilled bytes, the extra warps hide more of the per-edge
// latency chain: +8 % over bfs, sssp, cc and k-core on rmat24-hubs); 4 for the multi-source
// operators, which hold a row of labels per edge (5 spilled up to 272 bytes; with no minimum,
// ptxas gave them up to 118 registers and 2 CTAs per SM, 1.4x slower batches).
// Entries of the inspection kernel's thread-bin owner map: 16 edge positions per thread (12 for
// k-core at 512 threads, whose CTA table shares the 48 KB of static shared memory); positions
// beyond it are found by binary search of the bin's scan.
template <class Op, int B>
constexpr uint32_t kOwnerMapOf = (aggregates<Op>::value && B >= 512) ? 12u * B : 16u * B;

template <class Op, int B>
constexpr int round_kernel_min_blocks() { return (Op::kBatch ? 4 : 5) * kBlock / B; }

// CTA sizes the round kernels are built for (alb_params.block_size); kBlock is the default.
constexpr int kBlockSizes[] = {128, 256, 512};

// Edges relaxed per thread per step (memory requests a thread keeps in flight), per bin.
constexpr int kUCta = 8;     // CTA bin
constexpr int kUWarp = 8;    // warp bin
constexpr int kUThread = 4;  // thread bin (fine-grained gather)
constexpr int kULb = 8;      // LB kernel
constexpr int kUMs = 8;      // multi-source operators (every bin and the LB kernel)

template <class Op, int B>
__global__ void __launch_bounds__(B, (round_kernel_min_blocks<Op, B>())) k_inspect(TravCtx c) {
  constexpr int kNW = B / 32;  // warps of the CTA
  __shared__ uint32_t s_cb[B], s_cd[B], s_cv[B];       // CTA bin
  __shared__ uint32_t s_wb[B], s_wd[B], s_wv[B];       // warp bin
  __shared__ uint32_t s_scan[B + 1], s_sb[B], s_sv[B];  // thread bin
  __shared__ uint32_t s_warp[kNW + 1];
  __shared__ uint32_t s_ncta, s_nwrp, s_tile;
  constexpr int UC = Op::kBatch ? kUMs : kUCta;  // edges in flight per thread, per bin
  constexpr int UW = Op::kBatch ? kUMs : kUWarp;
  constexpr int UT = Op::kBatch ? (kUMs < kUThread ? kUMs : kUThread) : kUThread;
  __shared__ uint32_t s_push[kTilePushBuf];  // the tile's pushes (PushSink)
  constexpr uint32_t kMap = kOwnerMapOf<Op, B>;
  __shared__ uint16_t s_own[kMap];  // thread-bin edge position -> the thread (vertex) owning it
  __shared__ uint32_t s_npush, s_pbase;
  constexpr bool kHot = aggregates<Op>::value;
  constexpr uint32_t kHotN = kHot ? kHotSlots : 1u;
  __shared__ uint32_t s_hkey[kHotN], s_hcnt[kHotN];  // counted operators: CTA aggregation table
  uint32_t* hk = kHot ? s_hkey : nullptr;
  uint32_t* hc = kHot ? s_hcnt : nullptr;
  if constexpr (kHot) {
    for (uint32_t i = threadIdx.x; i < kHotSlots; i += B) { s_hkey[i] = kInf; s_hcnt[i] = 0u; }
  }  // visible after the tile loop's first barrier

  RoundState* st = c.st;
  const uint32_t r = st->round;
  const uint32_t cur = r & 1u;
  const bool all = st->all_active != 0u;
  uint32_t nf = all ? c.n : st->fcount[cur];
  if (!ALB_IN_RANGE(c.chk, CHK_STATE, nf, (uint64_t)c.n + 1u)) nf = 0u;
  const uint32_t* F = cur ? c.F1 : c.F0;
  uint32_t* Fn = cur ? c.F0 : c.F1;
  uint32_t* ncount = &st->fcount[cur ^ 1u];
  const CallArgs* ca = c.args;
  const OpArgs a{ca->lab, op_bitmap<Op>(c, cur), r + 1u, ca->k, ca->aux, c.n, c.chk};
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  unsigned long long twc_edges = 0ull;
  const PushSink sink{Fn, ncount, c.n, c.chk, s_push, &s_npush, kTilePushBuf};
  if constexpr (uses_push_bitmap<Op>::value) {
    // the other bitmap (last round's) is cleared for the next round
    if (c.pushed) {
      uint32_t* other = c.pushed + (size_t)(cur ^ 1u) * c.pw;
      for (uint32_t i = blockIdx.x * B + tid; i < c.pw; i += gridDim.x * B) other[i] = 0u;
    }
  }
  if constexpr (Op::kBatch) Op::round_start(a, r);  // multi-source operators' per-round state

  // Tiles of B frontier entries, taken dynamically. Tile t is made of the 32-entry chunks
  // t, t + T, ..., t + 7T (T tiles; warp w reads chunk t + wT, coalesced): vertices found
  // together (often of similar degree) spread over many tiles, so no tile holds a run of
  // CTA-bin vertices that would leave its CTA the last one running.
  const uint32_t ntiles = (uint32_t)(((uint64_t)nf + B - 1) / B);
  for (;;) {
    if (tid == 0) {
      s_tile = atomicAdd(&st->tile_next, 1u);
      s_ncta = 0u;
      s_nwrp = 0u;
      s_npush = 0u;
    }
    __syncthreads();
    if (s_tile >= ntiles) break;  // CTA-uniform
    const uint64_t i64 = ((uint64_t)s_tile + (uint64_t)warp * ntiles) * 32u + lane;
    const uint32_t i = (uint32_t)i64;
    bool valid = i64 < nf;
    uint32_t v = 0u, beg = 0u, deg = 0u, sv = 0u;
    if (valid) v = all ? i : F[i];
    if (valid && !ALB_IN_RANGE(c.chk, CHK_FRONTIER, v, c.n)) valid = false;
    if (valid) {
      beg = c.off[v];
      deg = c.off[v + 1] - beg;
      sv = Op::sval(a, v);
    }
    const bool huge = valid && deg >= c.threshold;
    const bool cta = valid && !huge && deg >= c.cta_min;
    const bool wrp = valid && !huge && !cta && deg >= c.warp_min;
    const uint32_t sdeg = (valid && !huge && !cta && !wrp) ? deg : 0u;
    if (valid && !huge) twc_edges += deg;
    hub_append(huge, v, deg, c.hub_v, c.hub_p, &st->hub_packed, c.n + 1u, c.chk);
    if (cta) {
      const uint32_t s = atomicAdd(&s_ncta, 1u);
      s_cb[s] = beg; s_cd[s] = deg; s_cv[s] = sv;
    }
    if (wrp) {
      const uint32_t s = atomicAdd(&s_nwrp, 1u);
      s_wb[s] = beg; s_wd[s] = deg; s_wv[s] = sv;
    }
    uint32_t stotal;
    const uint32_t ex = block_exclusive_scan<B>(sdeg, s_warp, &stotal);
    s_scan[tid] = ex;
    s_sb[tid] = beg;
    s_sv[tid] = sv;
    if (tid == 0) s_scan[B] = stotal;
    {
      // the thread bin's owner map: each small vertex marks its run of positions (the first kMap)
      const uint32_t end = ex + sdeg < kMap ? ex + sdeg : kMap;
      for (uint32_t q = ex; q < end; ++q) s_own[q] = (uint16_t)tid;
    }
    __syncthreads();

    // CTA bin: the whole CTA expands one vertex at a time.
    const uint32_t ncta = s_ncta;
    for (uint32_t j = 0; j < ncta; ++j) {
      const uint32_t b = s_cb[j], d = s_cd[j], svj = s_cv[j];
      for (uint32_t e0 = 0; e0 < d; e0 += B * UC) {
        uint32_t e[UC], s4[UC];
        bool ok[UC];
#pragma unroll
        for (int u = 0; u < UC; ++u) {
          const uint32_t q = e0 + u * B + tid;
          ok[u] = q < d; e[u] = b + q; s4[u] = svj;
        }
        relax<Op, UC>(c, a, e, ok, s4, sink, hk, hc);
      }
    }
    // Warp bin: one warp per vertex.
    const uint32_t nw = s_nwrp;
    for (uint32_t j = warp; j < nw; j += kNW) {
      const uint32_t b = s_wb[j], d = s_wd[j], svj = s_wv[j];
      for (uint32_t e0 = 0; e0 < d; e0 += 32 * UW) {
        uint32_t e[UW], s4[UW];
        bool ok[UW];
#pragma unroll
        for (int u = 0; u < UW; ++u) {
          const uint32_t q = e0 + u * 32 + lane;
          ok[u] = q < d; e[u] = b + q; s4[u] = svj;
        }
        relax<Op, UW>(c, a, e, ok, s4, sink, hk, hc);
      }
    }
    // Thread bin: the small vertices' edges, gathered over the whole CTA
    // (consecutive threads take consecutive edges of the concatenated lists).
    const uint32_t S = s_scan[B];
    uint32_t owner = 0u;
    for (uint32_t q0 = 0; q0 < S; q0 += B * UT) {
      uint32_t e[UT], s2[UT];
      bool ok[UT];
#pragma unroll
      for (int u = 0; u < UT; ++u) {
        const uint32_t q = q0 + u * B + tid;
        ok[u] = q < S;
        e[u] = 0u; s2[u] = 0u;
        if (ok[u]) {
          owner = q < kMap ? (uint32_t)s_own[q] : upper_search(s_scan, owner, B, q);
          e[u] = s_sb[owner] + (q - s_scan[owner]);
          s2[u] = s_sv[owner];
        }
      }
      relax<Op, UT>(c, a, e, ok, s2, sink, hk, hc);
    }
    __syncthreads();
    push_flush(sink, &s_pbase);
  }
  if constexpr (kHot) {
    // apply the CTA's pending counts: one atomic per target; the one that crosses k pushes it
    __syncthreads();
    for (uint32_t i = tid; i < kHotSlots; i += B) {  // same trip count in every thread
      const uint32_t v = s_hkey[i];
      const bool push = v != kInf && ALB_IN_RANGE(c.chk, CHK_DST, v, c.n) && Op::commit_n(a, v, s_hcnt[i]);
      warp_append(push, v, Fn, ncount, c.n, c.chk);
    }
  }

  // statistics: one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) twc_edges += __shfl_down_sync(kFull, twc_edges, o);
  if (lane == 0 && twc_edges) {
    atomicAdd(&st->edges_twc, twc_edges);
    if (c.cta_twc) atomicAdd(c.cta_twc + blockIdx.x, twc_edges);  // per-CTA load (cta_stats)
  }

  if (last_block_ticket(&st->done_inspect)) {
    const unsigned long long hp = __ldcg(&st->hub_packed);
    const uint32_t nh = (uint32_t)(hp >> 32);
    if (c.use_graph) cudaGraphSetConditional(c.h_if, nh > 0u ? 1u : 0u);
    if (nh == 0u) finish_round(c);
  }
}

// ------------------------------------------------------------- LB kernel

struct TraceOp {};

template <class Op, bool kTrace, int B>
__global__ void __launch_bounds__(B, (round_kernel_min_blocks<Op, B>())) k_lb(TravCtx c) {
  constexpr int kStage = kHubSmem;
  __shared__ uint32_t s_p[kStage];
  __shared__ uint32_t s_base[kStage];
  __shared__ uint32_t s_val[kStage];
  __shared__ uint32_t s_src[kTrace ? kStage : 1];
  __shared__ uint32_t s_push[kTrace ? 1 : kPushBufOf<B>];  // one step's pushes (PushSink)
  __shared__ uint32_t s_npush, s_pbase;

  RoundState* st = c.st;
  const unsigned long long hp = st->hub_packed;
  uint32_t nh = (uint32_t)(hp >> 32);
  uint32_t e = (uint32_t)hp;
  if (!ALB_IN_RANGE(c.chk, CHK_STATE, nh, (uint64_t)c.n + 1u) ||
      !ALB_IN_RANGE(c.chk, CHK_STATE, e, (uint64_t)c.m + 1u)) {
    nh = 0u;
    e = 0u;
  }
  const uint32_t r = st->round;
  const uint32_t cur = r & 1u;
  uint32_t* Fn = cur ? c.F0 : c.F1;
  uint32_t* ncount = &st->fcount[cur ^ 1u];
  const CallArgs* ca = c.args;
  const OpArgs a{ca->lab, op_bitmap<Op>(c, cur), r + 1u, ca->k, ca->aux, c.n, c.chk};
  const uint32_t tid = threadIdx.x, lane = tid & 31u;
  // a step of the CTA is B x U positions, at most one push each: the buffer never overflows
  static_assert(kTrace || B * (Op::kBatch ? kUMs : kULb) <= kPushBufOf<B>,
                "one LB step's pushes must fit the CTA buffer");
  const PushSink sink{Fn, ncount, c.n, c.chk, kTrace ? nullptr : s_push, &s_npush, kPushBufOf<B>};
  if (threadIdx.x == 0) s_npush = 0u;

  const bool staged = nh <= (uint32_t)kStage;
  if (staged) {
    for (uint32_t j = tid; j < nh; j += B) {
      uint32_t u = c.hub_v[j];
      const uint32_t p = c.hub_p[j];
      if (!ALB_IN_RANGE(c.chk, CHK_FRONTIER, u, c.n)) u = 0u;
      s_p[j] = p;
      s_base[j] = c.off[u] - p;
      if constexpr (kTrace) s_src[j] = u;
      else s_val[j] = Op::sval(a, u);
    }
  }
  __syncthreads();
  const uint32_t* P = staged ? s_p : c.hub_p;

  // source lookup for position k, from j0 (P[j0] <= k); a thread's positions only grow
  uint32_t j = 0u, jc = kInf, base_c = 0u, val_c = 0u, src_c = 0u;
  auto resolve = [&](uint32_t k, uint32_t j0, uint32_t& edge, uint32_t& sv, uint32_t& src) {
    j = advance_search(P, j0 > j ? j0 : j, nh, k);
    if (!ALB_IN_RANGE(c.chk, CHK_SRC, j, nh)) j = 0u;
    if (staged) {
      edge = k + s_base[j];
      if constexpr (kTrace) { src = s_src[j]; sv = 0u; }
      else { sv = s_val[j]; src = 0u; }
    } else {
      if (j != jc) {
        uint32_t u = c.hub_v[j];
        if (!ALB_IN_RANGE(c.chk, CHK_FRONTIER, u, c.n)) u = 0u;
        base_c = c.off[u] - c.hub_p[j];
        if constexpr (!kTrace) val_c = Op::sval(a, u);
        src_c = u;
        jc = j;
      }
      edge = k + base_c; sv = val_c; src = src_c;
    }
  };

  const uint64_t p = (uint64_t)gridDim.x * B;
  const uint64_t gt = (uint64_t)blockIdx.x * B + tid;
  constexpr int U = Op::kBatch ? kUMs : kULb;
  unsigned long long lb_edges = 0ull;  // positions this thread processed (cta_stats)
  // Cyclic distribution: in every step the CTA's B threads take B consecutive positions per
  // slot u (c0 + u p + tid), which span one or two huge vertices, while a thread's own positions
  // are p apart and cross many when the huge vertices average fewer than p edges. Then U lanes
  // of warp 0 search prefixWork once per step for the CTA's first position of each slot (s_jw[u],
  // between the step's barriers) and each thread steps forward from there, instead of every
  // thread binary-searching every position (threshold 4096 on rmat24-hubs: cc 10.4 -> 8.4 ms).
  // With a few very large huge vertices a thread's own search is one step, and it is kept.
  __shared__ uint32_t s_jw[U];
  const bool shared_search = !kTrace && c.distribution == 0u && (uint64_t)e < p * (uint64_t)nh;
  auto slot_starts = [&](uint64_t c0) {  // warp 0 only; c0 = the CTA's first position of the step
    if (tid < (uint32_t)U) {
      const uint64_t kc = c0 + (uint64_t)tid * p;
      const uint32_t prev = s_jw[tid];
      s_jw[tid] = kc < e ? upper_search(P, prev, nh, (uint32_t)kc) : prev;
    }
  };
  auto process = [&](const uint64_t (&k)[U], const bool (&ok)[U]) {
    uint32_t ed[U], sv[U], src[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ed[u] = 0u; sv[u] = 0u; src[u] = 0u;
      if (ok[u]) {
        resolve((uint32_t)k[u], shared_search ? s_jw[u] : 0u, ed[u], sv[u], src[u]);
        ++lb_edges;
      }
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
      relax<Op, U>(c, a, ed, ok, sv, sink);
    }
  };

  // after each CTA-uniform step: the step's staged pushes go to the frontier in one atomic (and,
  // between the two barriers, the next step's slot starts are found)
  auto flush = [&](uint64_t next_c0) {
    if constexpr (!kTrace) {
      __syncthreads();
      push_flush(sink, &s_pbase);
      if (threadIdx.x == 0) s_npush = 0u;  // every thread read the count inside push_flush
      if (shared_search) slot_starts(next_c0);
      __syncthreads();
    }
  };
  if (c.distribution == 0u) {
    // cyclic: thread gt takes positions gt, gt + p, gt + 2p, ... (Sec. 4.1)
    const uint64_t cta0 = (uint64_t)blockIdx.x * B;
    if (shared_search) {
      if (tid < (uint32_t)U) s_jw[tid] = 0u;  // P[0] = 0 <= every position
      slot_starts(cta0);                       // each lane reads and writes its own entry
      __syncthreads();
    }
    for (uint64_t c0 = cta0; c0 < e; c0 += p * U) {  // CTA-uniform
      const uint64_t k0 = c0 + (gt - cta0) - lane;
      uint64_t k[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) { k[u] = k0 + lane + (uint64_t)u * p; ok[u] = k[u] < e; }
      process(k, ok);
      flush(c0 + p * U);
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
      flush(0u);
    }
  }

  if (c.cta_lb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lb_edges += __shfl_down_sync(kFull, lb_edges, o);
    if (lane == 0 && lb_edges) atomicAdd(c.cta_lb + blockIdx.x, lb_edges);
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
      if (ok) lab[v] = (v == src) ? 0u : kInf;
    } else if constexpr (APP == APP_CC) {
      if (ok) lab[v] = v;
    } else if constexpr (APP == APP_KCORE) {
      uint32_t d = 0u;
      if (ok) { d = c.off[v + 1] - c.off[v]; lab[v] = d; }
      warp_append(ok && d < k, v, c.F0, &st->fcount[0], c.n, c.chk);
    }
  }
  if constexpr (APP == APP_SSSP || APP == APP_CC) {  // both push bitmaps start empty
    for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < 2ull * c.pw; i += (uint64_t)gridDim.x * kBlock)
      c.pushed[i] = 0u;
  }
  if constexpr (APP == APP_BFS) {  // the visited bitmap starts with the source alone
    for (uint64_t i = (uint64_t)blockIdx.x * kBlock + threadIdx.x; i < c.pw; i += (uint64_t)gridDim.x * kBlock)
      c.pushed[i] = (i == (src >> 5)) ? 1u << (src & 31u) : 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if constexpr (APP == APP_BFS || APP == APP_SSSP) { c.F0[0] = src; st->fcount[0] = 1u; }
    if constexpr (APP == APP_CC) { st->all_active = 1u; st->fcount[0] = n; }
  }
}

// k-core output: remaining degree >= k  ->  1, else 0 (in place).
static __global__ void k_kcore_finish(const CallArgs* ca, uint32_t n) {
  uint32_t* lab = ca->lab;
  const uint32_t k = ca->k;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    lab[v] = lab[v] >= k ? 1u : 0u;
}

static __global__ void k_set_args(CallArgs* dst, CallArgs v) { *dst = v; }

// The round kernels of operator Op built for CTA size B (128, 256 or 512; anything else: kBlock).
template <class Op>
static inline void* inspect_for(uint32_t B) {
  switch (B) {
    case 128: return (void*)k_inspect<Op, 128>;
    case 512: return (void*)k_inspect<Op, 512>;
    default: return (void*)k_inspect<Op, kBlock>;
  }
}
template <class Op, bool kTrace = false>
static inline void* lb_for(uint32_t B) {
  switch (B) {
    case 128: return (void*)k_lb<Op, kTrace, 128>;
    case 512: return (void*)k_lb<Op, kTrace, 512>;
    default: return (void*)k_lb<Op, kTrace, kBlock>;
  }
}

}  // namespace alb
