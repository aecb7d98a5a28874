// PageRank with the adaptive load balancer (arXiv:1911.09135, Sec. 5 "pr":
// pull over incoming edges; on a symmetric graph the CSR rows are the in-edge
// lists). pr is topology-driven: every vertex is active in every iteration, so
// the inspection of Algorithm 1 runs once per graph and its bins are reused:
//   - huge vertices (degree >= threshold): their in-edges are dealt cyclically
//     over every thread of the grid (Algorithm 2); each warp covers 32
//     consecutive positions and reduces them per source vertex, writing one
//     partial per (32-position chunk, vertex) pair into its own slot; a second
//     kernel sums each vertex's partials in chunk order;
//   - CTA / warp / thread bins: one CTA / warp / thread forms a vertex's sum. Each bin is cut
//     into one contiguous range per CTA of the pull kernel with equal cost (degree + a per-vertex
//     constant), computed once per graph, so every CTA takes the same share of every bin and no
//     CTA is a straggler.
// All sums have a fixed order and the assignment is static, so the result is bit-reproducible. Values and
// sums are FP32; the L1 change that decides convergence is summed in FP64.
//
// Recurrence (N = n, deg = out-degree, D_t = mass on degree-0 vertices):
//   x_0 = 1/N,  x_{t+1}[v] = (1-d)/N + d * (sum_{u->v} x_t[u]/deg(u) + D_t/N).
#include <new>
#include <vector>

#include "alb_device.cuh"

namespace alb {

constexpr uint32_t kPartChunk = 4096;  // vertices per CTA in the stable partition
constexpr uint32_t kFinTask = 4096;    // hub partial slots per first-level reduction task
constexpr uint32_t kFinDirect = 256;   // shorter slot runs are summed by the hub's own warp
constexpr uint32_t kPullItemCost = 3;  // per-vertex work of the pull in edge units (row bounds, x, x and x/deg stores)
constexpr uint32_t kCutPer = 16;       // items per thread in the cost scan of the CTA cut
constexpr uint32_t kCutChunk = kBlock * kCutPer;
constexpr uint32_t kPullWaves = 8;     // pull CTAs = resident CTAs x this: the block scheduler then
                                       // evens out the SMs' finishing times

struct PrState {
  uint32_t iter;
  uint32_t status;
  double l1;
  float dangling;  // D_t of the current iterate
  float pad;
};

struct PrArgs {
  float* rank;
  float damping;
  double tol;
  uint32_t max_iter;
  double* l1_out;      // device pointer or null
  uint32_t* iters_out; // device pointer or null
};

struct PrCtx {
  const uint32_t* off;
  const uint32_t* idx;
  uint32_t n;
  uint32_t nh, nc, nw, ns;     // bin sizes
  const uint32_t* hubs;        // bin lists, each in vertex order
  const uint32_t* ctas;
  const uint32_t* warps;
  const uint32_t* smalls;
  const uint32_t* pull_cut;    // bin k's range of pull CTA b: items [cut[k(G+1)+b], cut[k(G+1)+b+1])
  const uint32_t* hub_p;       // exclusive prefix of hub degrees (nh + 1)
  uint32_t e;                  // hub edges
  float* x[2];
  float* cb[2];                // x / deg (0 for deg 0)
  float* part;                 // hub partial slots
  double* l1_part;             // per pull-CTA, then per hub
  float* dang_part;
  uint32_t pull_blocks;
  uint32_t ntask;              // hub-sum tasks (runs of <= kFinTask slots of one hub)
  const uint32_t* task_start;
  const uint32_t* task_len;
  const uint32_t* hub_t0;      // tasks of hub j: [hub_t0[j], hub_t0[j+1])
  float* part2;
  unsigned long long* cta_twc; // per-CTA edges (cta_stats; else null)
  unsigned long long* cta_lb;
  uint32_t cta_cap;            // entries of each counter array
  PrState* st;
  const PrArgs* args;
  cudaGraphConditionalHandle h_while;
  uint32_t use_graph;
};

}  // namespace alb

struct PrWs {
  bool ready = false;
  uint32_t nh = 0, nc = 0, nw = 0, ns = 0, e = 0, zero_deg = 0;
  uint32_t* lists = nullptr;   // n entries: hubs | ctas | warps | smalls
  uint32_t* hub_p = nullptr;
  uint32_t* cnt = nullptr;     // per-partition-block bin counts
  float* x0 = nullptr;
  float* x1 = nullptr;
  float* c0 = nullptr;
  float* c1 = nullptr;
  float* part = nullptr;
  double* l1_part = nullptr;
  float* dang_part = nullptr;
  uint32_t pull_blocks = 0, hub_blocks = 0, ntask = 0;
  uint32_t* task_start = nullptr;
  uint32_t* task_len = nullptr;
  uint32_t* hub_t0 = nullptr;
  float* part2 = nullptr;
  uint32_t* pull_cut = nullptr;
  alb::PrState* st = nullptr;
  alb::PrState* h_st = nullptr;
  alb::PrArgs* args = nullptr;
  float* tmp_rank = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace alb {

__device__ __forceinline__ uint32_t pr_bin(uint32_t deg, uint32_t t, uint32_t wmin, uint32_t cmin) {
  if (deg >= t) return 0u;    // huge
  if (deg >= cmin) return 1u; // CTA
  if (deg >= wmin) return 2u; // warp
  return 3u;                  // thread
}

// ---- one-time inspection: stable partition of all vertices into the 4 bins

__global__ void __launch_bounds__(kBlock) k_pr_count(const uint32_t* off, uint32_t n, uint32_t t,
                                                     uint32_t wmin, uint32_t cmin, uint32_t* cnt) {
  __shared__ uint32_t s[5];
  if (threadIdx.x < 5) s[threadIdx.x] = 0u;
  __syncthreads();
  const uint64_t lo = (uint64_t)blockIdx.x * kPartChunk;
  const uint64_t hi = lo + kPartChunk < n ? lo + kPartChunk : n;
  uint32_t c[5] = {0, 0, 0, 0, 0};
  for (uint64_t v = lo + threadIdx.x; v < hi; v += kBlock) {
    const uint32_t d = off[v + 1] - off[v];
    c[pr_bin(d, t, wmin, cmin)]++;
    if (d == 0) c[4]++;
  }
  for (int b = 0; b < 5; ++b) if (c[b]) atomicAdd(&s[b], c[b]);
  __syncthreads();
  if (threadIdx.x < 5) cnt[blockIdx.x * 5 + threadIdx.x] = s[threadIdx.x];
}

// Exclusive scan of the per-block counts of each bin: CTA b scans bin b (carried CTA scans).
__global__ void __launch_bounds__(kBlock) k_pr_scan_counts(uint32_t* cnt, uint32_t nblk, uint32_t* totals) {
  __shared__ uint32_t s_warp[kWarps + 1];
  __shared__ uint32_t s_carry;
  const uint32_t b = blockIdx.x;
  if (threadIdx.x == 0) s_carry = 0u;
  __syncthreads();
  for (uint32_t i0 = 0; i0 < nblk; i0 += kBlock) {
    const uint32_t i = i0 + threadIdx.x;
    const uint32_t c = i < nblk ? cnt[i * 5 + b] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<kBlock>(c, s_warp, &tot);
    if (i < nblk) cnt[i * 5 + b] = s_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[b] = s_carry;
}

__global__ void __launch_bounds__(kBlock) k_pr_scatter(const uint32_t* off, uint32_t n, uint32_t t,
    uint32_t wmin, uint32_t cmin, const uint32_t* cnt, uint32_t* lists, uint32_t nh, uint32_t nc,
    uint32_t nw) {
  __shared__ uint32_t s_warp[kWarps + 1];
  __shared__ uint32_t s_base[4];
  const uint32_t bin_start[4] = {0u, nh, nh + nc, nh + nc + nw};
  if (threadIdx.x < 4) s_base[threadIdx.x] = bin_start[threadIdx.x] + cnt[blockIdx.x * 5 + threadIdx.x];
  __syncthreads();
  const uint64_t lo = (uint64_t)blockIdx.x * kPartChunk;
  const uint64_t hi = lo + kPartChunk < n ? lo + kPartChunk : n;
  for (uint64_t b0 = lo; b0 < hi; b0 += kBlock) {
    const uint64_t v = b0 + threadIdx.x;
    const bool ok = v < hi;
    const uint32_t bin = ok ? pr_bin(off[v + 1] - off[v], t, wmin, cmin) : 4u;
    for (uint32_t b = 0; b < 4; ++b) {
      uint32_t tot;
      const uint32_t rank = block_exclusive_scan<kBlock>(bin == b ? 1u : 0u, s_warp, &tot);
      if (bin == b) lists[s_base[b] + rank] = (uint32_t)v;
      __syncthreads();
      if (threadIdx.x == 0) s_base[b] += tot;
      __syncthreads();
    }
  }
}

// prefix[j] = sum of degrees of hubs[0..j), prefix[nh] = e (one CTA, carried scan).
__global__ void k_pr_hub_prefix(const uint32_t* off, const uint32_t* hubs, uint32_t nh,
                                uint32_t* prefix) {
  __shared__ uint32_t s_warp[kWarps + 1];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0u;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nh; b0 += kBlock) {
    const uint32_t j = b0 + threadIdx.x;
    const uint32_t d = j < nh ? off[hubs[j] + 1] - off[hubs[j]] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<kBlock>(d, s_warp, &tot);
    if (j < nh) prefix[j] = s_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) prefix[nh] = s_carry;
}

// ---- one-time cost-balanced cut of the non-hub vertices over the pull kernel's CTAs

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long x) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  return x;
}

// Exclusive scan over the CTA (every thread calls it); *total receives the CTA sum.
__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long x, unsigned long long* total) {
  __shared__ unsigned long long s_w[kWarps + 1];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned long long incl = warp_incl_scan_u64(x);
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long t = lane < (uint32_t)kWarps ? s_w[lane] : 0ull;
    const unsigned long long ti = warp_incl_scan_u64(t);
    if (lane < (uint32_t)kWarps) s_w[lane] = ti - t;
    if (lane == 31) s_w[kWarps] = ti;
  }
  __syncthreads();
  const unsigned long long r = s_w[warp] + incl - x;
  *total = s_w[kWarps];
  __syncthreads();
  return r;
}

// Cost of non-hub item i (degree + kPullItemCost) and its inclusive prefix within its chunk of
// kCutChunk items; chunk sums to csum.
__global__ void __launch_bounds__(kBlock) k_pr_cost_scan(const uint32_t* off, const uint32_t* items, uint32_t nn,
                                                         unsigned long long* pre, unsigned long long* csum) {
  const uint64_t i0 = (uint64_t)blockIdx.x * kCutChunk + (uint64_t)threadIdx.x * kCutPer;
  uint32_t cost[kCutPer];
  unsigned long long sum = 0ull;
#pragma unroll
  for (uint32_t u = 0; u < kCutPer; ++u) {
    const uint64_t i = i0 + u;
    cost[u] = 0u;
    if (i < nn) {
      const uint32_t v = items[i];
      cost[u] = off[v + 1] - off[v] + kPullItemCost;
    }
    sum += cost[u];
  }
  unsigned long long tot;
  unsigned long long run = block_excl_scan_u64(sum, &tot);
#pragma unroll
  for (uint32_t u = 0; u < kCutPer; ++u) {
    run += cost[u];
    if (i0 + u < nn) pre[i0 + u] = run;
  }
  if (threadIdx.x == 0) csum[blockIdx.x] = tot;
}

// Exclusive scan of the chunk sums (one CTA, carried); coff[nchunk] = total cost.
__global__ void __launch_bounds__(kBlock) k_pr_scan_chunks(const unsigned long long* csum, uint32_t nchunk,
                                                           unsigned long long* coff) {
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0ull;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nchunk; b0 += kBlock) {
    const uint32_t b = b0 + threadIdx.x;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan_u64(b < nchunk ? csum[b] : 0ull, &tot);
    if (b < nchunk) coff[b] = s_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) coff[nchunk] = s_carry;
}

__device__ __forceinline__ unsigned long long cost_before(const unsigned long long* pre,
                                                          const unsigned long long* coff, uint32_t i) {
  return i == 0 ? 0ull : coff[(i - 1) / kCutChunk] + pre[i - 1];
}

// For bin k (items [s_k, e_k): CTA bin, warp bin, thread bin) and b = 0..G,
// cut[k(G+1) + b] = number of items whose inclusive cost prefix is <= P(s_k) + floor(C_k * b / G)
// (P = exclusive prefix, C_k = the bin's cost): CTA b takes the bin's items whose cost ends in
// (T_b, T_{b+1}], so its share of every bin is within one item's cost of C_k / G.
__global__ void __launch_bounds__(kBlock) k_pr_cuts(const unsigned long long* pre, const unsigned long long* coff,
                                                    uint32_t nchunk, uint32_t nn, uint32_t nc, uint32_t nw,
                                                    uint32_t G, uint32_t* cut) {
  const uint32_t t = blockIdx.x * kBlock + threadIdx.x;
  if (t >= 3u * (G + 1u)) return;
  const uint32_t k = t / (G + 1u), b = t - k * (G + 1u);
  const uint32_t s_k = k == 0 ? 0u : (k == 1 ? nc : nc + nw);
  const uint32_t e_k = k == 0 ? nc : (k == 1 ? nc + nw : nn);
  const unsigned long long P0 = cost_before(pre, coff, s_k), Ck = cost_before(pre, coff, e_k) - P0;
  const unsigned long long T = P0 + (Ck / G) * b + ((Ck % G) * b) / G;
  if (b == 0) { cut[t] = s_k; return; }
  if (b == G) { cut[t] = e_k; return; }
  const unsigned long long total = coff[nchunk];
  if (T >= total) { cut[t] = nn; return; }
  uint32_t lo = 0, hi = nchunk;  // largest chunk k with coff[k] <= T (coff[0] = 0 <= T < coff[nchunk])
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (coff[mid] <= T) lo = mid; else hi = mid;
  }
  const unsigned long long r = T - coff[lo];
  uint32_t a = lo * kCutChunk;  // first item of the chunk whose in-chunk prefix exceeds r
  uint32_t z = (uint64_t)(lo + 1) * kCutChunk < nn ? (lo + 1) * kCutChunk : nn;
  while (a < z) {
    const uint32_t mid = a + ((z - a) >> 1);
    if (pre[mid] <= r) a = mid + 1; else z = mid;
  }
  cut[t] = a;
}

// ---- iteration kernels

__global__ void __launch_bounds__(kBlock) k_pr_init(PrCtx c, float dangling0) {
  const float x0 = 1.0f / (float)c.n;
  for (uint64_t v = (uint64_t)blockIdx.x * kBlock + threadIdx.x; v < c.n; v += (uint64_t)gridDim.x * kBlock) {
    const uint32_t d = c.off[v + 1] - c.off[v];
    c.x[0][v] = x0;
    c.cb[0][v] = d ? x0 / (float)d : 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c.st->iter = 0u;
    c.st->dangling = dangling0;
    c.st->l1 = 0.0;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Writes x_{t+1}[v], its contribution, and accumulates |x_{t+1} - x_t| and the new
// dangling mass in the calling thread's accumulators.
__device__ __forceinline__ void pr_update(const PrCtx& c, uint32_t v, uint32_t deg, float s,
                                          float base, float d, uint32_t par, double& l1, float& dang) {
  const float xn = base + d * s;
  c.x[par ^ 1u][v] = xn;
  c.cb[par ^ 1u][v] = deg ? xn / (float)deg : 0.0f;
  l1 += fabs((double)xn - (double)c.x[par][v]);
  if (deg == 0) dang += xn;
}

template <int BLOCK>
__device__ __forceinline__ void block_reduce_store(double l1, float dang, double* l1_out, float* dang_out) {
  __shared__ double s_l1[BLOCK / 32];
  __shared__ float s_d[BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l1 += __shfl_xor_sync(kFull, l1, o);
    dang += __shfl_xor_sync(kFull, dang, o);
  }
  const uint32_t warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { s_l1[warp] = l1; s_d[warp] = dang; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    float b = 0.0f;
    for (int w = 0; w < BLOCK / 32; ++w) { a += s_l1[w]; b += s_d[w]; }
    *l1_out = a;
    *dang_out = b;
  }
}

// Sum of x/deg over the in-edges idx[b + o], idx[b + o + S], ... (< deg) of one vertex, in that
// order. U index loads are issued before their U dependent gathers, so a thread keeps U requests
// in flight; the index stream is read once (evict-first), the gathers go through the read-only path.
// kComp (the CTA bin): the U values of a step are added pairwise and the step sums are
// accumulated with Kahan's compensation. A thread of a CTA-bin vertex adds up to
// (threshold / block) terms, and a plain FP32 running sum over tens of thousands of them drifts
// beyond the accuracy PageRank needs; a warp- or thread-bin thread adds at most 8 and keeps the
// plain sum.
template <int U, bool kComp>
__device__ __forceinline__ float strided_sum(const uint32_t* __restrict__ idx, const float* __restrict__ cb,
                                             uint32_t b, uint32_t deg, uint32_t o, uint32_t S) {
  float s = 0.0f, comp = 0.0f;
  for (uint32_t e0 = o; e0 < deg; e0 += S * U) {
    uint32_t id[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t e = e0 + (uint32_t)u * S;
      id[u] = e < deg ? __ldcs(idx + b + e) : kInf;
    }
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = id[u] != kInf ? __ldg(cb + id[u]) : 0.0f;
    if constexpr (kComp) {
#pragma unroll
      for (int w = 1; w < U; w <<= 1) {
#pragma unroll
        for (int u = 0; u + w < U; u += 2 * w) v[u] += v[u + w];
      }
      const float y = v[0] - comp;
      const float t = s + y;
      comp = (t - s) - y;
      s = t;
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) s += v[u];
    }
  }
  (void)comp;
  return s;
}

constexpr uint32_t kCtaBatch = 32;  // CTA-bin vertices per barrier

// CTA, warp and thread bins. Static assignment (CTA b always takes the same cost-balanced range
// of items, and within it the same warp / thread takes the same vertex), fixed reduction order,
// so sums and partials are reproducible.
__global__ void __launch_bounds__(kBlock, 8) k_pr_pull(PrCtx c) {
  __shared__ float s_part[kCtaBatch][kWarps + 1];
  const PrArgs* pa = c.args;
  const float d = pa->damping;
  const uint32_t par = c.st->iter & 1u;
  const float N = (float)c.n;
  const float base = (1.0f - d) / N + d * (c.st->dangling / N);
  const float* __restrict__ cb = c.cb[par];
  const uint32_t* __restrict__ idx = c.idx;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  double l1 = 0.0;
  float dang = 0.0f;
  unsigned long long edges = 0ull;  // this thread's share of the CTA's load (cta_stats)
  // this CTA's range of each bin (bins back to back: CTA bin [0, nc), warp bin [nc, nc + nw),
  // thread bin after)
  const uint32_t* items = c.ctas;
  const uint32_t* cut = c.pull_cut + blockIdx.x;
  const uint32_t G1 = gridDim.x + 1u;
  // CTA bin: every warp sums a strided slice of a vertex's edges; the 8 warp sums of each of a
  // batch of 32 vertices are combined after one barrier
  const uint32_t c_end = cut[1];
  for (uint32_t q = cut[0]; q < c_end; q += kCtaBatch) {
#pragma unroll 1
    for (uint32_t i = 0; i < kCtaBatch; ++i) {
      const uint32_t j = q + i;
      if (j >= c_end) break;  // CTA-uniform
      const uint32_t v = items[j];
      const uint32_t b = c.off[v], deg = c.off[v + 1] - b;
      float sv = strided_sum<4, true>(idx, cb, b, deg, tid, kBlock);
      sv = warp_sum(sv);
      if (lane == 0) s_part[i][warp] = sv;
    }
    __syncthreads();
    if (tid < kCtaBatch) {
      const uint32_t j = q + tid;
      if (j < c_end) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += s_part[tid][w];
        const uint32_t v = items[j];
        const uint32_t deg = c.off[v + 1] - c.off[v];
        pr_update(c, v, deg, t, base, d, par, l1, dang);
        edges += deg;
      }
    }
    __syncthreads();
  }
  // warp bin: one warp per vertex
  const uint32_t w_end = cut[G1 + 1];
  for (uint32_t j = cut[G1] + warp; j < w_end; j += kWarps) {
    const uint32_t v = items[j];
    const uint32_t b = c.off[v], deg = c.off[v + 1] - b;
    float sv = warp_sum(strided_sum<4, false>(idx, cb, b, deg, lane, 32));
    if (lane == 0) {
      pr_update(c, v, deg, sv, base, d, par, l1, dang);
      edges += deg;
    }
  }
  // thread bin: one thread per vertex, its edges in order, 8 loads in flight
  const uint32_t t_end = cut[2 * G1 + 1];
  for (uint32_t j = cut[2 * G1] + tid; j < t_end; j += kBlock) {
    const uint32_t v = items[j];
    const uint32_t b = c.off[v], deg = c.off[v + 1] - b;
    pr_update(c, v, deg, strided_sum<8, false>(idx, cb, b, deg, 0, 1), base, d, par, l1, dang);
    edges += deg;
  }
  if (c.cta_twc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) edges += __shfl_down_sync(kFull, edges, o);
    if (lane == 0 && edges && blockIdx.x < c.cta_cap) atomicAdd(c.cta_twc + blockIdx.x, edges);
  }
  block_reduce_store<kBlock>(l1, dang, c.l1_part + blockIdx.x, c.dang_part + blockIdx.x);
}

// Huge vertices, cyclic over all threads (Algorithm 2): thread gt takes positions gt, gt + p, ...
// four per iteration. Each warp covers 32 consecutive positions; their values are reduced per
// source vertex (segmented scan) and each segment's sum is written to the slot
// (position / 32) + source index, unique per (chunk, vertex) pair.
__global__ void __launch_bounds__(kBlock) k_pr_hub(PrCtx c) {
  __shared__ uint32_t s_p[kHubSmem];
  __shared__ uint32_t s_base[kHubSmem];
  const uint32_t nh = c.nh, e = c.e;
  const bool staged = nh <= (uint32_t)kHubSmem;
  if (staged) {
    for (uint32_t j = threadIdx.x; j < nh; j += kBlock) {
      const uint32_t p = c.hub_p[j];
      s_p[j] = p;
      s_base[j] = c.off[c.hubs[j]] - p;
    }
  }
  __syncthreads();
  const uint32_t* P = staged ? s_p : c.hub_p;
  const float* __restrict__ cb = c.cb[c.st->iter & 1u];
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t p = (uint64_t)gridDim.x * kBlock;
  const uint64_t gt = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  constexpr int U = 4;
  uint32_t j = 0u;
  unsigned long long edges = 0ull;  // positions this thread took (cta_stats)
  for (uint64_t k0 = gt - lane; k0 < e; k0 += p * U) {  // warp-uniform
    uint32_t jj[U], id[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t k = k0 + (uint64_t)u * p + lane;
      jj[u] = kInf;
      id[u] = kInf;
      if (k < e) {
        j = advance_search(P, j, nh, (uint32_t)k);
        jj[u] = j;
        const uint32_t base = staged ? s_base[j] : c.off[c.hubs[j]] - c.hub_p[j];
        id[u] = __ldcs(c.idx + (uint32_t)k + base);
        ++edges;
      }
    }
    float val[U];
#pragma unroll
    for (int u = 0; u < U; ++u) val[u] = id[u] != kInf ? __ldg(cb + id[u]) : 0.0f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t slot0 = (uint32_t)((k0 + (uint64_t)u * p) >> 5);
      const uint32_t j0 = __shfl_sync(kFull, jj[u], 0);
      if (__all_sync(kFull, jj[u] == j0) && j0 != kInf) {
        // the usual case: all 32 positions belong to one huge vertex, one sum
        const float t = warp_sum(val[u]);
        if (lane == 0) c.part[slot0 + j0] = t;
        continue;
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(kFull, val[u], o);
        const uint32_t jy = __shfl_up_sync(kFull, jj[u], o);
        if (lane >= (uint32_t)o && jy == jj[u]) val[u] += y;
      }
      const uint32_t jn = __shfl_down_sync(kFull, jj[u], 1);
      const bool tail = jj[u] != kInf && (lane == 31 || jn != jj[u]);
      if (tail) c.part[slot0 + jj[u]] = val[u];
    }
  }
  if (c.cta_lb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) edges += __shfl_down_sync(kFull, edges, o);
    if (lane == 0 && edges && blockIdx.x < c.cta_cap) atomicAdd(c.cta_lb + blockIdx.x, edges);
  }
}

// First level of the hub sums: one CTA per task (a run of at most kFinTask slots of one hub),
// fixed-order sum into part2[task].
__global__ void __launch_bounds__(kBlock) k_pr_hub_fin1(PrCtx c) {
  __shared__ float s_red[kWarps];
  for (uint32_t t = blockIdx.x; t < c.ntask; t += gridDim.x) {
    const uint32_t s0 = c.task_start[t], len = c.task_len[t];
    float s = 0.0f;
    for (uint32_t i = threadIdx.x; i < len; i += kBlock) s += c.part[s0 + i];
    s = warp_sum(s);
    if ((threadIdx.x & 31u) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = 0.0f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) a += s_red[w];
      c.part2[t] = a;
    }
    __syncthreads();
  }
}

// One warp per huge vertex: the sum of its tasks' partials (or, for a short slot run, of the
// slots themselves) in a fixed order, then the update.
__global__ void __launch_bounds__(kBlock) k_pr_hub_fin(PrCtx c) {
  const PrArgs* pa = c.args;
  const float d = pa->damping;
  const uint32_t par = c.st->iter & 1u;
  const float N = (float)c.n;
  const float base = (1.0f - d) / N + d * (c.st->dangling / N);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = (blockIdx.x * kBlock + threadIdx.x) >> 5, nwarps = (gridDim.x * kBlock) >> 5;
  for (uint32_t j = gw; j < c.nh; j += nwarps) {
    const uint32_t v = c.hubs[j];
    const uint32_t p0 = c.hub_p[j], p1 = c.hub_p[j + 1];
    const uint32_t t0 = c.hub_t0[j], t1 = c.hub_t0[j + 1];
    float s = 0.0f;
    if (t1 > t0) {
      for (uint32_t t = t0 + lane; t < t1; t += 32) s += c.part2[t];
    } else if (p1 > p0) {
      const uint32_t w0 = p0 >> 5, w1 = (p1 - 1) >> 5;
      for (uint32_t w = w0 + lane; w <= w1; w += 32) s += c.part[w + j];
    }
    s = warp_sum(s);
    double l1 = 0.0;
    float dang = 0.0f;
    if (lane == 0) {
      pr_update(c, v, p1 - p0, s, base, d, par, l1, dang);
      c.l1_part[c.pull_blocks + j] = l1;
      c.dang_part[c.pull_blocks + j] = dang;
    }
  }
}

// Reduce the partials in a fixed order, advance the iteration, set the loop condition.
__global__ void k_pr_finalize(PrCtx c) {
  __shared__ double s_l1[kWarps];
  __shared__ float s_d[kWarps];
  const uint32_t np = c.pull_blocks + c.nh;
  double l1 = 0.0;
  float dg = 0.0f;
  for (uint32_t i = threadIdx.x; i < np; i += kBlock) { l1 += c.l1_part[i]; dg += c.dang_part[i]; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l1 += __shfl_xor_sync(kFull, l1, o);
    dg += __shfl_xor_sync(kFull, dg, o);
  }
  if ((threadIdx.x & 31) == 0) { s_l1[threadIdx.x >> 5] = l1; s_d[threadIdx.x >> 5] = dg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    float b = 0.0f;
    for (int w = 0; w < kWarps; ++w) { a += s_l1[w]; b += s_d[w]; }
    PrState* st = c.st;
    const PrArgs* pa = c.args;
    st->l1 = a;
    st->dangling = b;
    st->iter += 1u;
    const bool go = !(a < pa->tol) && st->iter < pa->max_iter;
    if (c.use_graph) cudaGraphSetConditional(c.h_while, go ? 1u : 0u);
  }
}

__global__ void k_pr_output(PrCtx c) {
  const PrArgs* pa = c.args;
  const uint32_t par = c.st->iter & 1u;
  const float* x = c.x[par];
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < c.n;
       v += (uint64_t)gridDim.x * blockDim.x)
    pa->rank[v] = x[v];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (pa->l1_out) *pa->l1_out = c.st->l1;
    if (pa->iters_out) *pa->iters_out = c.st->iter;
  }
}

__global__ void k_pr_set_args(PrArgs* dst, PrArgs v) { *dst = v; }

// ---------------------------------------------------------------- host side

alb_status free_pagerank(alb_graph g) {
  PrWs* w = g->pr;
  if (!w) return ALB_OK;
  if (w->exec) cudaGraphExecDestroy(w->exec);
  if (w->graph) cudaGraphDestroy(w->graph);
  cudaFree(w->lists); cudaFree(w->hub_p); cudaFree(w->cnt);
  cudaFree(w->x0); cudaFree(w->x1); cudaFree(w->c0); cudaFree(w->c1);
  cudaFree(w->part); cudaFree(w->l1_part); cudaFree(w->dang_part);
  cudaFree(w->task_start); cudaFree(w->task_len); cudaFree(w->hub_t0); cudaFree(w->part2);
  cudaFree(w->pull_cut);
  cudaFree(w->st); cudaFree(w->args); cudaFree(w->tmp_rank);
  if (w->h_st) cudaFreeHost(w->h_st);
  cudaGetLastError();
  delete w;
  g->pr = nullptr;
  return ALB_OK;
}

static PrCtx pr_ctx(alb_graph g, bool use_graph, cudaGraphConditionalHandle hw) {
  PrWs* w = g->pr;
  PrCtx c{};
  c.off = g->off;
  c.idx = g->idx;
  c.n = g->n;
  c.nh = w->nh; c.nc = w->nc; c.nw = w->nw; c.ns = w->ns;
  c.hubs = w->lists;
  c.ctas = w->lists + w->nh;
  c.warps = w->lists + w->nh + w->nc;
  c.smalls = w->lists + w->nh + w->nc + w->nw;
  c.pull_cut = w->pull_cut;
  c.hub_p = w->hub_p;
  c.e = w->e;
  c.x[0] = w->x0; c.x[1] = w->x1;
  c.cb[0] = w->c0; c.cb[1] = w->c1;
  c.part = w->part;
  c.l1_part = w->l1_part;
  c.dang_part = w->dang_part;
  c.pull_blocks = w->pull_blocks;
  c.ntask = w->ntask;
  c.task_start = w->task_start;
  c.task_len = w->task_len;
  c.hub_t0 = w->hub_t0;
  c.part2 = w->part2;
  c.cta_twc = g->params.cta_stats ? g->cta_twc : nullptr;
  c.cta_lb = g->params.cta_stats ? g->cta_lb : nullptr;
  c.cta_cap = g->cta_cap;
  c.st = w->st;
  c.args = w->args;
  c.h_while = hw;
  c.use_graph = use_graph ? 1u : 0u;
  return c;
}

// Grids of the pull and hub kernels. The pull kernel needs little shared memory: the rest of the
// SM's on-chip memory goes to L1, which caches the popular entries of the x/deg gathers. The hub
// kernel is persistent (one wave); the pull kernel runs kPullWaves waves of its static ranges.
static alb_status pr_grids(alb_graph g, uint32_t* pull, uint32_t* hub) {
  ALB_CUDA_TRY(cudaFuncSetAttribute(k_pr_pull, cudaFuncAttributePreferredSharedMemoryCarveout, 5));
  int occ = 0;
  ALB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pr_pull, kBlock, 0));
  *pull = g->params.grid_blocks ? g->params.grid_blocks
                                : (uint32_t)g->num_sms * (uint32_t)(occ > 0 ? occ : 1) * kPullWaves;
  occ = 0;
  ALB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pr_hub, kBlock, 0));
  *hub = g->params.grid_blocks ? g->params.grid_blocks : (uint32_t)g->num_sms * (uint32_t)(occ > 0 ? occ : 1);
  return ALB_OK;
}

// One-time setup per graph and parameters: bins, hub prefix, buffers.
static alb_status pr_setup(alb_graph g, cudaStream_t s) {
  if (g->pr && g->pr->ready) return ALB_OK;
  {
    alb_status rb = setup_barrier();
    if (rb != ALB_OK) return rb;
  }
  if (!g->pr) g->pr = new (std::nothrow) PrWs();
  PrWs* w = g->pr;
  if (!w) return ALB_ERR_OOM;
  const uint32_t n = g->n;
  const size_t nb = sizeof(float) * (size_t)n;
  const uint32_t nblk = (n + kPartChunk - 1) / kPartChunk;
  ALB_CUDA_TRY(cudaMalloc((void**)&w->lists, sizeof(uint32_t) * (size_t)n));
  ALB_CUDA_TRY(cudaMalloc((void**)&w->cnt, sizeof(uint32_t) * (5 * (size_t)nblk + 5)));
  ALB_CUDA_TRY(cudaMalloc((void**)&w->x0, nb));
  ALB_CUDA_TRY(cudaMalloc((void**)&w->x1, nb));
  ALB_CUDA_TRY(cudaMalloc((void**)&w->c0, nb));
  ALB_CUDA_TRY(cudaMalloc((void**)&w->c1, nb));
  ALB_CUDA_TRY(cudaMalloc((void**)&w->st, sizeof(PrState)));
  ALB_CUDA_TRY(cudaMalloc((void**)&w->args, sizeof(PrArgs)));
  ALB_CUDA_TRY(cudaMallocHost((void**)&w->h_st, sizeof(PrState)));
  const uint32_t t = g->threshold, wmin = g->params.twc_warp_min, cmin = g->params.twc_cta_min;
  uint32_t* totals = w->cnt + 5 * (size_t)nblk;
  k_pr_count<<<nblk, kBlock, 0, s>>>(g->off, n, t, wmin, cmin, w->cnt);
  k_pr_scan_counts<<<5, kBlock, 0, s>>>(w->cnt, nblk, totals);
  uint32_t h[5];
  ALB_CUDA_TRY(cudaMemcpyAsync(h, totals, sizeof(h), cudaMemcpyDeviceToHost, s));
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  w->nh = h[0]; w->nc = h[1]; w->nw = h[2]; w->ns = h[3]; w->zero_deg = h[4];
  k_pr_scatter<<<nblk, kBlock, 0, s>>>(g->off, n, t, wmin, cmin, w->cnt, w->lists, w->nh, w->nc, w->nw);
  ALB_CUDA_TRY(cudaMalloc((void**)&w->hub_p, sizeof(uint32_t) * ((size_t)w->nh + 1)));
  k_pr_hub_prefix<<<1, kBlock, 0, s>>>(g->off, w->lists, w->nh, w->hub_p);
  ALB_CUDA_TRY(cudaMemcpyAsync(&w->e, w->hub_p + w->nh, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  ALB_CUDA_TRY(cudaStreamSynchronize(s));
  const size_t slots = (size_t)(w->e / 32u) + 1 + w->nh;
  ALB_CUDA_TRY(cudaMalloc((void**)&w->part, sizeof(float) * slots));
  {
    alb_status rg = pr_grids(g, &w->pull_blocks, &w->hub_blocks);
    if (rg != ALB_OK) return rg;
  }
  ALB_CUDA_TRY(cudaMalloc((void**)&w->l1_part, sizeof(double) * ((size_t)w->pull_blocks + w->nh)));
  // cost-balanced cut of the non-hub items over the pull CTAs (scratch freed before returning)
  {
    const uint32_t nn = n - w->nh;
    const uint32_t nchunk = (uint32_t)(((uint64_t)nn + kCutChunk - 1) / kCutChunk);
    ALB_CUDA_TRY(cudaMalloc((void**)&w->pull_cut, sizeof(uint32_t) * 3 * ((size_t)w->pull_blocks + 1)));
    unsigned long long* scratch = nullptr;
    ALB_CUDA_TRY(cudaMalloc((void**)&scratch, sizeof(unsigned long long) * ((size_t)nn + 2 * (size_t)nchunk + 1)));
    unsigned long long* pre = scratch;
    unsigned long long* csum = scratch + nn;
    unsigned long long* coff = csum + nchunk;
    if (nchunk) k_pr_cost_scan<<<nchunk, kBlock, 0, s>>>(g->off, w->lists + w->nh, nn, pre, csum);
    k_pr_scan_chunks<<<1, kBlock, 0, s>>>(csum, nchunk, coff);
    const uint32_t ncut = 3u * (w->pull_blocks + 1u);
    k_pr_cuts<<<(ncut + kBlock - 1) / kBlock, kBlock, 0, s>>>(pre, coff, nchunk, nn, w->nc, w->nw,
                                                              w->pull_blocks, w->pull_cut);
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return ALB_ERR_CUDA;
  }
  ALB_CUDA_TRY(cudaMalloc((void**)&w->dang_part, sizeof(float) * ((size_t)w->pull_blocks + w->nh)));
  // hub-sum tasks: each hub's slot run [w0 + j, w1 + j] cut into pieces of <= kFinTask slots;
  // runs of <= kFinDirect slots are summed directly by the hub's warp
  {
    std::vector<uint32_t> hp((size_t)w->nh + 1);
    ALB_CUDA_TRY(cudaMemcpyAsync(hp.data(), w->hub_p, sizeof(uint32_t) * hp.size(), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<uint32_t> ts, tl, t0((size_t)w->nh + 1, 0u);
    for (uint32_t j = 0; j < w->nh; ++j) {
      t0[j] = (uint32_t)ts.size();
      if (hp[j + 1] <= hp[j]) continue;
      const uint32_t w0 = hp[j] >> 5, w1 = (hp[j + 1] - 1) >> 5, L = w1 - w0 + 1;
      if (L <= kFinDirect) continue;
      for (uint32_t o = 0; o < L; o += kFinTask) {
        ts.push_back(w0 + j + o);
        tl.push_back(L - o < kFinTask ? L - o : kFinTask);
      }
    }
    t0[w->nh] = (uint32_t)ts.size();
    w->ntask = (uint32_t)ts.size();
    ALB_CUDA_TRY(cudaMalloc((void**)&w->hub_t0, sizeof(uint32_t) * t0.size()));
    // stream-ordered with the kernels that read them (the caller's stream may not block on the
    // legacy default stream), and complete before the host vectors go out of scope
    ALB_CUDA_TRY(cudaMemcpyAsync(w->hub_t0, t0.data(), sizeof(uint32_t) * t0.size(), cudaMemcpyHostToDevice, s));
    const size_t nt = ts.size() ? ts.size() : 1;
    ALB_CUDA_TRY(cudaMalloc((void**)&w->task_start, sizeof(uint32_t) * nt));
    ALB_CUDA_TRY(cudaMalloc((void**)&w->task_len, sizeof(uint32_t) * nt));
    ALB_CUDA_TRY(cudaMalloc((void**)&w->part2, sizeof(float) * nt));
    if (!ts.empty()) {
      ALB_CUDA_TRY(cudaMemcpyAsync(w->task_start, ts.data(), sizeof(uint32_t) * ts.size(), cudaMemcpyHostToDevice, s));
      ALB_CUDA_TRY(cudaMemcpyAsync(w->task_len, tl.data(), sizeof(uint32_t) * tl.size(), cudaMemcpyHostToDevice, s));
    }
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
  }
  ALB_CUDA_TRY(cudaGetLastError());
  w->ready = true;
  return ALB_OK;
}

static uint32_t pr_fin_blocks(const PrWs* w) {
  const uint32_t b = (w->nh * 32u + kBlock - 1) / kBlock;
  return b == 0 ? 1u : (b < w->pull_blocks ? b : w->pull_blocks);
}

static alb_status pr_add_kernel(cudaGraphNode_t* node, cudaGraph_t graph, const cudaGraphNode_t* dep,
                                size_t ndep, void* fn, uint32_t grid, void** args) {
  cudaKernelNodeParams kp{};
  kp.func = fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(kBlock);
  kp.kernelParams = args;
  ALB_CUDA_TRY(cudaGraphAddKernelNode(node, graph, dep, ndep, &kp));
  return ALB_OK;
}

static alb_status pr_build_graph(alb_graph g) {
  PrWs* w = g->pr;
  cudaGraph_t G = nullptr;
  ALB_CUDA_TRY(cudaGraphCreate(&G, 0));
  auto fail = [&](alb_status s) { cudaGraphDestroy(G); return s; };
  cudaGraphConditionalHandle hw;
  if (cudaGraphConditionalHandleCreate(&hw, G, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(ALB_ERR_CUDA);
  PrCtx c = pr_ctx(g, true, hw);
  float dang0 = (float)w->zero_deg / (float)g->n;
  void* a_init[] = {&c, &dang0};
  void* a_c[] = {&c};
  cudaGraphNode_t n_init, n_while, n_pull, n_hub, n_fin, n_final, n_out;
  alb_status rc;
  if ((rc = pr_add_kernel(&n_init, G, nullptr, 0, (void*)k_pr_init, g->blocks, a_init)) != ALB_OK)
    return fail(rc);
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  if (cudaGraphAddNode(&n_while, G, &n_init, nullptr, 1, &wp) != cudaSuccess) return fail(ALB_ERR_CUDA);
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  // the hub branch (LB kernel and its sums) reads only x_t and writes only the hubs' entries and
  // slots, so it runs beside the pull kernel and fills its tail; both join before the finalize
  if ((rc = pr_add_kernel(&n_pull, body, nullptr, 0, (void*)k_pr_pull, w->pull_blocks, a_c)) != ALB_OK)
    return fail(rc);
  cudaGraphNode_t joins[2] = {n_pull, nullptr};
  size_t njoin = 1;
  if (w->nh) {
    if ((rc = pr_add_kernel(&n_hub, body, nullptr, 0, (void*)k_pr_hub, w->hub_blocks, a_c)) != ALB_OK)
      return fail(rc);
    cudaGraphNode_t last = n_hub;
    if (w->ntask) {
      cudaGraphNode_t n_fin1;
      const uint32_t b1 = w->ntask < w->pull_blocks ? w->ntask : w->pull_blocks;
      if ((rc = pr_add_kernel(&n_fin1, body, &last, 1, (void*)k_pr_hub_fin1, b1, a_c)) != ALB_OK)
        return fail(rc);
      last = n_fin1;
    }
    if ((rc = pr_add_kernel(&n_fin, body, &last, 1, (void*)k_pr_hub_fin, pr_fin_blocks(w), a_c)) != ALB_OK)
      return fail(rc);
    joins[njoin++] = n_fin;
  }
  if ((rc = pr_add_kernel(&n_final, body, joins, njoin, (void*)k_pr_finalize, 1, a_c)) != ALB_OK)
    return fail(rc);
  if ((rc = pr_add_kernel(&n_out, G, &n_while, 1, (void*)k_pr_output, g->blocks, a_c)) != ALB_OK)
    return fail(rc);
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, G, 0) != cudaSuccess) {
    cudaGetLastError();
    return fail(ALB_ERR_CUDA);
  }
  w->graph = G;
  w->exec = ex;
  return ALB_OK;
}

static alb_status pr_host_loop(alb_graph g, cudaStream_t s, uint32_t max_iter, double tol) {
  PrWs* w = g->pr;
  PrCtx c = pr_ctx(g, false, 0);
  float dang0 = (float)w->zero_deg / (float)g->n;
  k_pr_init<<<g->blocks, kBlock, 0, s>>>(c, dang0);
  const bool prof = g->params.profile != 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (prof) { cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2); }
  while (max_iter > 0) {
    if (prof) cudaEventRecord(e0, s);
    k_pr_pull<<<w->pull_blocks, kBlock, 0, s>>>(c);
    if (prof) cudaEventRecord(e1, s);
    if (w->nh) {
      k_pr_hub<<<w->hub_blocks, kBlock, 0, s>>>(c);
      if (prof) cudaEventRecord(e2, s);
      if (w->ntask) k_pr_hub_fin1<<<w->ntask < w->pull_blocks ? w->ntask : w->pull_blocks, kBlock, 0, s>>>(c);
      k_pr_hub_fin<<<pr_fin_blocks(w), kBlock, 0, s>>>(c);
    }
    k_pr_finalize<<<1, kBlock, 0, s>>>(c);
    ALB_CUDA_TRY(cudaGetLastError());
    ALB_CUDA_TRY(cudaMemcpyAsync(w->h_st, w->st, sizeof(PrState), cudaMemcpyDeviceToHost, s));
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    if (prof) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      g->stats.ms_inspect += ms; g->stats.n_inspect += 1;
      if (w->nh) { cudaEventElapsedTime(&ms, e1, e2); g->stats.ms_lb += ms; g->stats.n_lb += 1; }
    }
    if (w->h_st->l1 < tol || w->h_st->iter >= max_iter) break;
  }
  if (prof) { cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2); }
  k_pr_output<<<g->blocks, kBlock, 0, s>>>(c);
  ALB_CUDA_TRY(cudaGetLastError());
  return ALB_OK;
}

alb_status pr_stats(alb_graph g, alb_stats* out) {
  PrWs* w = g->pr;
  if (!w || !w->st) return ALB_OK;
  ALB_CUDA_TRY(cudaMemcpy(w->h_st, w->st, sizeof(PrState), cudaMemcpyDeviceToHost));
  out->rounds = w->h_st->iter;
  out->pr_l1 = w->h_st->l1;
  out->hub_rounds = w->nh ? w->h_st->iter : 0u;
  out->max_hub_count = w->nh;
  out->edges_lb = (uint64_t)w->e * w->h_st->iter;
  out->edges_twc = (g->m - w->e) * (uint64_t)w->h_st->iter;
  out->pushes = 0;
  return ALB_OK;
}

}  // namespace alb

using namespace alb;

extern "C" alb_status alb_pagerank(alb_graph g, float damping, double tol, uint32_t max_iter,
                                   float* hd_rank, double* hd_l1, uint32_t* hd_iters,
                                   alb_stream stream) {
  if (!g || !hd_rank || !(damping >= 0.0f && damping <= 1.0f) || !(tol >= 0.0)) return ALB_ERR_INVALID_ARG;
  if (!(g->flags & ALB_SYMMETRIC)) return ALB_ERR_NOT_SYMMETRIC;
  if (cudaSetDevice(g->device) != cudaSuccess) return ALB_ERR_CUDA;
  select_cfg(g, ALB_APP_PAGERANK);
  g->stats.ms_inspect = g->stats.ms_lb = g->stats.ms_other = 0.0;
  g->stats.n_inspect = g->stats.n_lb = g->stats.n_other = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (!g->params.cta_stats) g->cta_n_twc = g->cta_n_lb = 0;  // this call is not instrumented
  if (g->params.cta_stats) {  // before the setup: the counters' addresses go into the cached graph
    uint32_t pull = 0, hub = 0;
    alb_status rc0 = g->pr && g->pr->ready ? ALB_OK : pr_grids(g, &pull, &hub);
    if (rc0 == ALB_OK && g->pr && g->pr->ready) { pull = g->pr->pull_blocks; hub = g->pr->hub_blocks; }
    if (rc0 == ALB_OK) rc0 = reset_cta_loads(g, s, pull > hub ? pull : hub);
    if (rc0 != ALB_OK) return rc0;
  }
  alb_status rc = pr_setup(g, s);
  if (rc != ALB_OK) return rc;
  PrWs* w = g->pr;
  if (g->params.cta_stats) {
    g->cta_n_twc = w->pull_blocks;
    g->cta_n_lb = w->nh ? w->hub_blocks : 0u;
  }
  const bool dev_rank = is_device_ptr(hd_rank);
  float* rank = hd_rank;
  if (!dev_rank) {
    if (!w->tmp_rank) {
      if ((rc = setup_barrier()) != ALB_OK) return rc;
      ALB_CUDA_TRY(cudaMalloc((void**)&w->tmp_rank, sizeof(float) * (size_t)g->n));
    }
    rank = w->tmp_rank;
  }
  const bool dev_l1 = hd_l1 && is_device_ptr(hd_l1);
  const bool dev_it = hd_iters && is_device_ptr(hd_iters);
  PrArgs a{rank, damping, tol, max_iter, dev_l1 ? hd_l1 : nullptr, dev_it ? hd_iters : nullptr};
  k_pr_set_args<<<1, 1, 0, s>>>(w->args, a);
  ALB_CUDA_TRY(cudaMemsetAsync(w->st, 0, sizeof(PrState), s));
  if (max_iter == 0) {
    // no iteration: the output is the starting vector
    PrCtx c = pr_ctx(g, false, 0);
    k_pr_init<<<g->blocks, kBlock, 0, s>>>(c, (float)w->zero_deg / (float)g->n);
    k_pr_output<<<g->blocks, kBlock, 0, s>>>(c);
  } else if (g->params.exec_mode == 0) {
    if (!w->exec) {
      rc = setup_barrier();
      if (rc == ALB_OK) rc = pr_build_graph(g);
      if (rc != ALB_OK) return rc;
    }
    ALB_CUDA_TRY(cudaGraphLaunch(w->exec, s));
  } else {
    rc = pr_host_loop(g, s, max_iter, tol);
    if (rc != ALB_OK) return rc;
  }
  if (!dev_rank) ALB_CUDA_TRY(cudaMemcpyAsync(hd_rank, rank, sizeof(float) * g->n, cudaMemcpyDeviceToHost, s));
  g->last_stream = s;
  g->last_kind = 1;
  if ((hd_l1 && !dev_l1) || (hd_iters && !dev_it)) {
    ALB_CUDA_TRY(cudaStreamSynchronize(s));
    ALB_CUDA_TRY(cudaMemcpy(w->h_st, w->st, sizeof(PrState), cudaMemcpyDeviceToHost));
    if (hd_l1 && !dev_l1) *hd_l1 = w->h_st->l1;
    if (hd_iters && !dev_it) *hd_iters = w->h_st->iter;
  }
  ALB_CUDA_TRY(cudaGetLastError());
  return ALB_OK;
}
