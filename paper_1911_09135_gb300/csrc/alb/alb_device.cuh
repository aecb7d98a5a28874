// Device helpers shared by the round kernels: warp-aggregated appends, warp and
// block scans, and the last-block ticket used to finish a round on the device.
#pragma once

#include "alb_internal.cuh"

namespace alb {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Bounds checks of the checked build: an index outside [0, bound) records (code, index,
// bound) once in chk and counts every failure in chk[3]; the caller skips the access.
#ifdef ALB_CHECKED
__device__ __forceinline__ bool in_range(uint32_t* chk, uint32_t code, uint64_t idx, uint64_t bound) {
  if (idx < bound) return true;
  if (chk) {
    if (atomicCAS(chk, 0u, code) == 0u) {
      chk[1] = (uint32_t)idx;
      chk[2] = (uint32_t)bound;
    }
    atomicAdd(chk + 3, 1u);
  }
  return false;
}
#define ALB_IN_RANGE(chk, code, idx, bound) ::alb::in_range((chk), (code), (uint64_t)(idx), (uint64_t)(bound))
#else
#define ALB_IN_RANGE(chk, code, idx, bound) true
#endif

// Warp-aggregated append of `v` for every lane with `pred`: one atomicAdd on
// `count` per warp (ballot + popc), lanes write consecutive slots. Every lane of
// the warp must call it (the callers keep their loops warp-uniform).
__device__ __forceinline__ void warp_append(bool pred, uint32_t v, uint32_t* buf, uint32_t* count,
                                            uint32_t cap = 0xFFFFFFFFu, uint32_t* chk = nullptr) {
  const unsigned mask = __ballot_sync(kFull, pred);
  if (mask == 0) return;
  const uint32_t lane = lane_id();
  const uint32_t leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
  base = __shfl_sync(kFull, base, leader);
  const uint32_t slot = base + __popc(mask & ((1u << lane) - 1u));
  if (pred && ALB_IN_RANGE(chk, 4u, slot, cap)) buf[slot] = v;
  (void)cap;
  (void)chk;
}

// Inclusive warp scan (Kogge-Stone over shuffles).
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  return x;
}

// Warp-aggregated append of up to U values per lane (v[u] where pred[u]): a scan of the lanes'
// counts, one atomicAdd on `count` per warp for all of them, each lane writes its run of slots.
// Every lane of the warp must call it.
template <int U>
__device__ __forceinline__ void warp_append_n(const bool (&pred)[U], const uint32_t (&v)[U], uint32_t* buf,
                                              uint32_t* count, uint32_t cap = 0xFFFFFFFFu,
                                              uint32_t* chk = nullptr) {
  uint32_t cnt = 0u;
#pragma unroll
  for (int u = 0; u < U; ++u) cnt += pred[u] ? 1u : 0u;
  const uint32_t incl = warp_inclusive_scan(cnt);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  if (total == 0u) return;
  uint32_t base = 0u;
  if (lane_id() == 0u) base = atomicAdd(count, total);
  uint32_t slot = __shfl_sync(kFull, base, 0) + incl - cnt;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (pred[u]) {
      if (ALB_IN_RANGE(chk, 4u, slot, cap)) buf[slot] = v[u];
      ++slot;
    }
  }
  (void)cap;
  (void)chk;
}

// Exclusive scan over the CTA; *total receives the CTA sum. Uses s_warp[kWarps]
// and synchronises the CTA (every thread must call it).
template <int BLOCK>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp, uint32_t* total) {
  constexpr int W = BLOCK / 32;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t incl = warp_inclusive_scan(x);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < (uint32_t)W ? s_warp[lane] : 0u;
    const uint32_t ti = warp_inclusive_scan(t);
    if (lane < (uint32_t)W) s_warp[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) s_warp[W] = ti;
  }
  __syncthreads();
  const uint32_t res = s_warp[warp] + incl - x;
  *total = s_warp[W];
  __syncthreads();
  return res;
}

// Last-block ticket: every CTA calls this once at its end (all threads). Returns
// true in exactly one thread of the CTA that arrives last; that thread then
// sees every other CTA's writes (fence before the ticket, L2 reads after).
__device__ __forceinline__ bool last_block_ticket(uint32_t* counter) {
  __shared__ uint32_t s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
    if (s_last) __threadfence();
  }
  __syncthreads();
  return s_last && threadIdx.x == 0;
}

// Largest j in [lo, hi) with P[j] <= k, given P[lo] <= k and (implicitly) P[hi] > k.
__device__ __forceinline__ uint32_t upper_search(const uint32_t* P, uint32_t lo, uint32_t hi, uint32_t k) {
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (P[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

// upper_search for a caller whose k only grows (the LB kernels' positions): the next position
// usually falls in the same entry or the next one, so two linear steps are tried before the
// binary search.
__device__ __forceinline__ uint32_t advance_search(const uint32_t* P, uint32_t lo, uint32_t hi, uint32_t k) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (lo + 1 >= hi || P[lo + 1] > k) return lo;
    ++lo;
  }
  return upper_search(P, lo, hi, k);
}

}  // namespace alb
