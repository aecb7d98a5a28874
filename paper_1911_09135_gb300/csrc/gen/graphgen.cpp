// Seeded synthetic graph generator (host, C++/OpenMP).
//
// Produces the CSR inputs that both the CUDA path and the CPU oracle consume.
// It contains none of the traversal arithmetic: it only draws edges, removes
// self-loops and duplicate entries, optionally adds reverse edges, and
// attaches per-edge weights.
//
// Randomness is counter-based (SplitMix64, Steele, Lea and Flood, OOPSLA 2014:
// state_k = key + k * 0x9E3779B97F4A7C15, output = mix(state_k)), so every
// edge sample is a pure function of (seed, sample index) and the CSR that comes
// out is identical for any number of threads and on any host.
//
// RMAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each sample descends `scale`
// levels of the adjacency matrix, picking quadrant (0,0),(0,1),(1,0),(1,1) with
// probabilities a, b, c, 1-a-b-c. No noise and no vertex relabelling are
// applied, so low vertex ids carry the highest degrees.
//
// Injected hubs: `n_hubs` distinct vertex ids are drawn uniformly; hub j gets
// `hub_degree` distinct targets (never itself), taken as the first values of a
// seeded bijection of [0, n) (a 4-round Feistel network with cycle walking),
// i.e. a uniform sample without replacement.

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#include <omp.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// k-th output of the SplitMix64 stream whose state starts at `key`.
inline uint64_t splitmix_at(uint64_t key, uint64_t k) { return mix64(key + (k + 1) * kGamma); }

struct Rmat {
  uint32_t scale;
  uint64_t key;
  uint32_t ta, tab, tabc;  // cumulative quadrant thresholds in units of 2^-32
  inline void sample(uint64_t i, uint32_t* u_out, uint32_t* v_out) const {
    const uint32_t words = (scale + 1) / 2;  // two 32-bit draws per 64-bit word
    uint32_t u = 0, v = 0;
    for (uint32_t w = 0; w < words; ++w) {
      const uint64_t r64 = splitmix_at(key, i * words + w);
      for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t level = 2 * w + h;
        if (level >= scale) break;
        const uint32_t r = h ? (uint32_t)(r64 >> 32) : (uint32_t)r64;
        uint32_t bu, bv;
        if (r < ta) { bu = 0; bv = 0; }
        else if (r < tab) { bu = 0; bv = 1; }
        else if (r < tabc) { bu = 1; bv = 0; }
        else { bu = 1; bv = 1; }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
      }
    }
    *u_out = u;
    *v_out = v;
  }
};

inline uint32_t prob_to_u32(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return 0xFFFFFFFFu;
  return (uint32_t)(p * 4294967296.0);
}

// Bijection of [0, n) from a Feistel network over 2^bits >= n (bits even),
// extended to [0, n) by cycle walking.
struct Feistel {
  uint32_t half_bits;
  uint64_t half_mask;
  uint64_t n;
  uint64_t keys[4];
  Feistel(uint64_t n_, uint64_t key) : n(n_) {
    uint32_t bits = 2;
    while ((1ull << bits) < n_) bits += 2;
    half_bits = bits / 2;
    half_mask = (1ull << half_bits) - 1;
    for (int r = 0; r < 4; ++r) keys[r] = splitmix_at(key, (uint64_t)r);
  }
  inline uint64_t round_trip(uint64_t x) const {
    uint64_t l = x >> half_bits, r = x & half_mask;
    for (int k = 0; k < 4; ++k) {
      const uint64_t f = mix64(keys[k] ^ r) & half_mask;
      const uint64_t nl = r;
      r = l ^ f;
      l = nl;
    }
    return (l << half_bits) | r;
  }
  inline uint64_t operator()(uint64_t x) const {
    uint64_t y = round_trip(x);
    while (y >= n) y = round_trip(y);
    return y;
  }
};

}  // namespace

extern "C" {

typedef struct {
  uint32_t scale;       // n = 2^scale vertices
  uint32_t symmetrize;  // 1: add the reverse of every edge
  uint64_t nsamples;    // RMAT edge samples drawn (edge factor * n)
  uint64_t seed;
  double a, b, c;       // RMAT quadrant probabilities, d = 1 - a - b - c
  uint32_t n_hubs;      // injected hub vertices
  uint32_t hub_degree;  // distinct targets per hub (< n)
  uint32_t weighted;    // 1: attach weights uniform in [wmin, wmax]
  uint32_t wmin, wmax;
  int32_t nthreads;     // <= 0: OpenMP default
} gg_rmat_params;

typedef struct gg_csr_s {
  uint32_t n;
  uint64_t m;
  uint32_t* off;  // n + 1
  uint32_t* idx;  // m
  uint32_t* w;    // m or NULL
  uint32_t* hubs; // n_hubs injected hub ids (draw order)
  uint32_t n_hubs;
} gg_csr;

enum { GG_OK = 0, GG_ERR_ARG = 1, GG_ERR_OOM = 2, GG_ERR_OVERFLOW = 3 };

void gg_free(gg_csr* g) {
  if (!g) return;
  std::free(g->off);
  std::free(g->idx);
  std::free(g->w);
  std::free(g->hubs);
  std::free(g);
}

uint32_t gg_n(const gg_csr* g) { return g ? g->n : 0; }
uint64_t gg_m(const gg_csr* g) { return g ? g->m : 0; }
uint32_t gg_num_hubs(const gg_csr* g) { return g ? g->n_hubs : 0; }

int gg_copy(const gg_csr* g, uint32_t* off, uint32_t* idx, uint32_t* w, uint32_t* hubs) {
  if (!g) return GG_ERR_ARG;
  if (off) std::memcpy(off, g->off, sizeof(uint32_t) * ((size_t)g->n + 1));
  if (idx && g->m) std::memcpy(idx, g->idx, sizeof(uint32_t) * g->m);
  if (w && g->w && g->m) std::memcpy(w, g->w, sizeof(uint32_t) * g->m);
  if (hubs && g->n_hubs) std::memcpy(hubs, g->hubs, sizeof(uint32_t) * g->n_hubs);
  return GG_OK;
}

// Weight of the undirected pair {u, v}: the same value in both directions.
uint32_t gg_edge_weight(uint64_t seed, uint32_t u, uint32_t v, uint32_t wmin, uint32_t wmax) {
  const uint32_t lo = u < v ? u : v, hi = u < v ? v : u;
  const uint64_t h = mix64(mix64(seed ^ 0xA5A5A5A5DEADBEEFull) + (((uint64_t)lo << 32) | hi));
  const uint64_t span = (uint64_t)wmax - wmin + 1;
  return wmin + (uint32_t)(h % span);
}

int gg_rmat(const gg_rmat_params* p, gg_csr** out) {
  if (!p || !out) return GG_ERR_ARG;
  *out = nullptr;
  if (p->scale > 31) return GG_ERR_ARG;
  if (p->weighted && (p->wmin > p->wmax)) return GG_ERR_ARG;
  const uint64_t n = 1ull << p->scale;
  if (p->n_hubs > n) return GG_ERR_ARG;
  if (p->n_hubs && (uint64_t)p->hub_degree >= n) return GG_ERR_ARG;
  // The thread count never changes the output; it is set on every call so one
  // call's choice does not carry over to the next.
  omp_set_num_threads(p->nthreads > 0 ? p->nthreads : omp_get_num_procs());

  Rmat rm;
  rm.scale = p->scale;
  rm.key = mix64(p->seed * 0x2545F4914F6CDD1Dull + 0x1234567ull);
  rm.ta = prob_to_u32(p->a);
  rm.tab = prob_to_u32(p->a + p->b);
  rm.tabc = prob_to_u32(p->a + p->b + p->c);

  gg_csr* g = (gg_csr*)std::calloc(1, sizeof(gg_csr));
  if (!g) return GG_ERR_OOM;
  g->n = (uint32_t)n;

  // Hub ids: sequential draws, duplicates rejected.
  std::vector<uint32_t> hub_ids;
  const uint64_t hub_key = mix64(p->seed ^ 0x7F4A7C159E3779B9ull);
  for (uint64_t k = 0; hub_ids.size() < p->n_hubs; ++k) {
    const uint32_t h = (uint32_t)(splitmix_at(hub_key, k) % n);
    if (std::find(hub_ids.begin(), hub_ids.end(), h) == hub_ids.end()) hub_ids.push_back(h);
  }
  g->n_hubs = p->n_hubs;
  if (p->n_hubs) {
    g->hubs = (uint32_t*)std::malloc(sizeof(uint32_t) * p->n_hubs);
    if (!g->hubs) { gg_free(g); return GG_ERR_OOM; }
    std::copy(hub_ids.begin(), hub_ids.end(), g->hubs);
  }
  // Hub targets: first hub_degree values of a per-hub bijection of [0, n), the hub itself skipped.
  std::vector<std::vector<uint32_t>> hub_tgt(p->n_hubs);
  for (uint32_t j = 0; j < p->n_hubs; ++j) {
    Feistel perm(n, splitmix_at(hub_key, 1000003ull + j));
    std::vector<uint32_t>& t = hub_tgt[j];
    t.resize((size_t)p->hub_degree + 1);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < (int64_t)p->hub_degree + 1; ++x) t[x] = (uint32_t)perm((uint64_t)x);
    auto it = std::find(t.begin(), t.begin() + p->hub_degree, hub_ids[j]);
    if (it != t.begin() + p->hub_degree) t.erase(it);
    t.resize(p->hub_degree);
  }

  // Pass 1: count raw entries per source row.
  std::vector<std::atomic<uint64_t>> cnt(n);
  for (uint64_t i = 0; i < n; ++i) cnt[i].store(0, std::memory_order_relaxed);
  const bool sym = p->symmetrize != 0;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)p->nsamples; ++i) {
    uint32_t u, v;
    rm.sample((uint64_t)i, &u, &v);
    if (u == v) continue;
    cnt[u].fetch_add(1, std::memory_order_relaxed);
    if (sym) cnt[v].fetch_add(1, std::memory_order_relaxed);
  }
  for (uint32_t j = 0; j < p->n_hubs; ++j) {
    const uint32_t h = hub_ids[j];
    cnt[h].fetch_add(p->hub_degree, std::memory_order_relaxed);
    if (sym) {
      const std::vector<uint32_t>& t = hub_tgt[j];
#pragma omp parallel for schedule(static)
      for (int64_t x = 0; x < (int64_t)t.size(); ++x) cnt[t[x]].fetch_add(1, std::memory_order_relaxed);
    }
  }
  std::vector<uint64_t> start(n + 1);
  start[0] = 0;
  for (uint64_t i = 0; i < n; ++i) start[i + 1] = start[i] + cnt[i].load(std::memory_order_relaxed);
  const uint64_t raw = start[n];

  // Pass 2: scatter destinations into their rows (order inside a row is fixed later by sorting).
  uint32_t* buf = (uint32_t*)std::malloc(sizeof(uint32_t) * (raw ? raw : 1));
  if (!buf) { gg_free(g); return GG_ERR_OOM; }
  for (uint64_t i = 0; i < n; ++i) cnt[i].store(start[i], std::memory_order_relaxed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)p->nsamples; ++i) {
    uint32_t u, v;
    rm.sample((uint64_t)i, &u, &v);
    if (u == v) continue;
    buf[cnt[u].fetch_add(1, std::memory_order_relaxed)] = v;
    if (sym) buf[cnt[v].fetch_add(1, std::memory_order_relaxed)] = u;
  }
  for (uint32_t j = 0; j < p->n_hubs; ++j) {
    const uint32_t h = hub_ids[j];
    const std::vector<uint32_t>& t = hub_tgt[j];
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < (int64_t)t.size(); ++x) {
      buf[cnt[h].fetch_add(1, std::memory_order_relaxed)] = t[x];
      if (sym) buf[cnt[t[x]].fetch_add(1, std::memory_order_relaxed)] = h;
    }
  }
  hub_tgt.clear();

  // Sort and deduplicate each row.
  std::vector<uint64_t> deg(n);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t u = 0; u < (int64_t)n; ++u) {
    uint32_t* b = buf + start[u];
    uint32_t* e = buf + start[u + 1];
    std::sort(b, e);
    deg[u] = (uint64_t)(std::unique(b, e) - b);
  }
  uint64_t m = 0;
  for (uint64_t u = 0; u < n; ++u) m += deg[u];
  if (m >= 0xFFFFFFFFull) { std::free(buf); gg_free(g); return GG_ERR_OVERFLOW; }
  g->m = m;
  g->off = (uint32_t*)std::malloc(sizeof(uint32_t) * (n + 1));
  g->idx = (uint32_t*)std::malloc(sizeof(uint32_t) * (m ? m : 1));
  if (!g->off || !g->idx) { std::free(buf); gg_free(g); return GG_ERR_OOM; }
  g->off[0] = 0;
  for (uint64_t u = 0; u < n; ++u) g->off[u + 1] = g->off[u] + (uint32_t)deg[u];
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t u = 0; u < (int64_t)n; ++u)
    std::memcpy(g->idx + g->off[u], buf + start[u], sizeof(uint32_t) * deg[u]);
  std::free(buf);

  if (p->weighted) {
    g->w = (uint32_t*)std::malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!g->w) { gg_free(g); return GG_ERR_OOM; }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t u = 0; u < (int64_t)n; ++u)
      for (uint32_t e = g->off[u]; e < g->off[u + 1]; ++e)
        g->w[e] = gg_edge_weight(p->seed, (uint32_t)u, g->idx[e], p->wmin, p->wmax);
  }
  *out = g;
  return GG_OK;
}

}  // extern "C"
