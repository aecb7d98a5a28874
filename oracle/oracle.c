/*
 * CPU oracle for the ALB graph analytics path (arXiv:1911.09135).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * definition that the CUDA path is checked against. Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may load it; the
 * library never does. It shares no code, header or table with the CUDA path.
 *
 * Plain serial C99 (the PageRank pull loop may use OpenMP: every vertex's sum
 * is still formed sequentially in CSR order, so the result does not depend on
 * the thread count). Graphs are CSR: the out-neighbours of u are
 * idx[off[u] .. off[u+1]). Unreached vertices get UINT32_MAX (BFS, SSSP).
 *
 * Contents and where each one comes from in the paper:
 *   oracle_bfs        - bfs (Sec. 5 applications): level = hop distance from src.
 *   oracle_sssp       - sssp, the relaxation operator of Sec. 4.3 (Fig. 3); reached
 *                       exactly by Dijkstra's algorithm (binary heap, 64-bit sums).
 *   oracle_cc         - cc (Sec. 5): component label = smallest vertex id (union-find).
 *   oracle_pagerank   - pr (Sec. 5, pull over incoming edges): Jacobi power iteration in
 *                       FP64, damping d, dangling mass spread uniformly, L1 stopping rule.
 *   oracle_kcore      - kcore (Sec. 5): membership in the k-core, by peeling.
 *   oracle_inspect    - Algorithm 1 (inspection): huge / CTA / warp / thread bins and the
 *                       exclusive prefix sum of huge degrees ("prefixWork", Sec. 4.1).
 *   oracle_lb_edges   - Algorithm 2 (execution): the edges thread T_i is given under the
 *                       cyclic or blocked distribution, each source found by binary
 *                       search of prefixWork (Sec. 4.1 "Distribution", "Search").
 *   oracle_check_bfs  - exact certificate of BFS levels, usable at any graph size.
 *   oracle_check_sssp - exact certificate of shortest-path distances (weights >= 1).
 *
 * Every function is pinned by tests against something other than itself
 * (brute force, library routines, closed forms, invariants, planted errors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_INF 0xFFFFFFFFu

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_OOM = 2, OR_ERR_OVERFLOW = 3, OR_ERR_CHECK = 4 };

/* ---------------------------------------------------------------- bfs */

/* Breadth-first search from src with a FIFO queue: level[v] is the number of
 * edges on a shortest path src -> v, UINT32_MAX if v is unreachable. */
int oracle_bfs(uint32_t n, const uint32_t* off, const uint32_t* idx, uint32_t src,
               uint32_t* level) {
  if (src >= n) return OR_ERR_ARG;
  uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  if (!queue) return OR_ERR_OOM;
  for (uint32_t v = 0; v < n; ++v) level[v] = ORACLE_INF;
  size_t head = 0, tail = 0;
  level[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    uint32_t u = queue[head++];
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = idx[e];
      if (level[v] == ORACLE_INF) {
        level[v] = level[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return OR_OK;
}

/* --------------------------------------------------------------- sssp */

/* Binary min-heap of (distance, vertex) with lazy deletion. */
typedef struct { uint64_t d; uint32_t v; } heap_item;

static void heap_push(heap_item* h, size_t* size, heap_item it) {
  size_t i = (*size)++;
  h[i] = it;
  while (i > 0) {
    size_t parent = (i - 1) / 2;
    if (h[parent].d <= h[i].d) break;
    heap_item t = h[parent]; h[parent] = h[i]; h[i] = t;
    i = parent;
  }
}

static heap_item heap_pop(heap_item* h, size_t* size) {
  heap_item top = h[0];
  h[0] = h[--(*size)];
  size_t i = 0;
  for (;;) {
    size_t l = 2 * i + 1, r = l + 1, s = i;
    if (l < *size && h[l].d < h[s].d) s = l;
    if (r < *size && h[r].d < h[s].d) s = r;
    if (s == i) break;
    heap_item t = h[s]; h[s] = h[i]; h[i] = t;
    i = s;
  }
  return top;
}

/* Dijkstra's algorithm from src; distances are accumulated in 64 bits and the
 * result must fit below UINT32_MAX (the unreached marker). */
int oracle_sssp(uint32_t n, const uint32_t* off, const uint32_t* idx, const uint32_t* w,
                uint32_t src, uint32_t* dist) {
  if (src >= n || !w) return OR_ERR_ARG;
  uint64_t* d = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  uint8_t* done = (uint8_t*)calloc(n ? n : 1, 1);
  size_t cap = (size_t)off[n] + 1;
  heap_item* heap = (heap_item*)malloc(sizeof(heap_item) * cap);
  if (!d || !done || !heap) { free(d); free(done); free(heap); return OR_ERR_OOM; }
  for (uint32_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
  size_t size = 0;
  d[src] = 0;
  heap_item first = {0, src};
  heap_push(heap, &size, first);
  while (size > 0) {
    heap_item it = heap_pop(heap, &size);
    uint32_t u = it.v;
    if (done[u] || it.d != d[u]) continue;
    done[u] = 1;
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = idx[e];
      uint64_t nd = d[u] + (uint64_t)w[e];
      if (nd < d[v]) {
        d[v] = nd;
        heap_item nx = {nd, v};
        heap_push(heap, &size, nx);
      }
    }
  }
  int rc = OR_OK;
  for (uint32_t v = 0; v < n; ++v) {
    if (d[v] == UINT64_MAX) dist[v] = ORACLE_INF;
    else if (d[v] >= ORACLE_INF) { dist[v] = ORACLE_INF; rc = OR_ERR_OVERFLOW; }
    else dist[v] = (uint32_t)d[v];
  }
  free(d); free(done); free(heap);
  return rc;
}

/* ----------------------------------------------------------------- cc */

static uint32_t uf_find(uint32_t* parent, uint32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]]; /* path halving */
    x = parent[x];
  }
  return x;
}

/* Connected components of an undirected graph given as a symmetric CSR:
 * label[v] = the smallest vertex id in v's component. Union-find with union by
 * size, then a pass that takes each root's minimum member. */
int oracle_cc(uint32_t n, const uint32_t* off, const uint32_t* idx, uint32_t* label) {
  uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
  uint32_t* size = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
  uint32_t* minid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
  if (!parent || !size || !minid) { free(parent); free(size); free(minid); return OR_ERR_OOM; }
  for (uint32_t v = 0; v < n; ++v) { parent[v] = v; size[v] = 1; minid[v] = ORACLE_INF; }
  for (uint32_t u = 0; u < n; ++u) {
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t a = uf_find(parent, u), b = uf_find(parent, idx[e]);
      if (a == b) continue;
      if (size[a] < size[b]) { uint32_t t = a; a = b; b = t; }
      parent[b] = a;
      size[a] += size[b];
    }
  }
  for (uint32_t v = 0; v < n; ++v) {
    uint32_t r = uf_find(parent, v);
    if (v < minid[r]) minid[r] = v;
  }
  for (uint32_t v = 0; v < n; ++v) label[v] = minid[uf_find(parent, v)];
  free(parent); free(size); free(minid);
  return OR_OK;
}

/* ----------------------------------------------------------- pagerank */

/* PageRank by Jacobi power iteration in FP64 (pr pulls over incoming edges,
 * Sec. 5). With N = n, out-degree deg(u) and damping d:
 *   x_0[v]     = 1/N
 *   D_t        = sum of x_t[u] over vertices with deg(u) = 0 (dangling mass)
 *   x_{t+1}[v] = (1-d)/N + d * ( sum_{u -> v} x_t[u]/deg(u) + D_t/N )
 * iterated until ||x_{t+1} - x_t||_1 < tol or max_iter iterations. The last
 * iterate is returned with the number of iterations and its L1 change.
 * assume_symmetric = 1 uses the CSR itself as the in-edge lists (a symmetric
 * graph); otherwise the transpose is built here. */
int oracle_pagerank(uint32_t n, const uint32_t* off, const uint32_t* idx, double d, double tol,
                    uint32_t max_iter, int assume_symmetric, int nthreads, double* x_out,
                    uint32_t* iters_out, double* l1_out) {
  if (n == 0) { if (iters_out) *iters_out = 0; if (l1_out) *l1_out = 0.0; return OR_OK; }
  const uint64_t m = off[n];
  const uint32_t* in_off = off;
  const uint32_t* in_idx = idx;
  uint32_t* t_off = NULL;
  uint32_t* t_idx = NULL;
  if (!assume_symmetric) {
    t_off = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
    t_idx = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    uint32_t* cur = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    if (!t_off || !t_idx || !cur) { free(t_off); free(t_idx); free(cur); return OR_ERR_OOM; }
    for (uint64_t e = 0; e < m; ++e) t_off[idx[e] + 1]++;
    for (uint32_t v = 0; v < n; ++v) t_off[v + 1] += t_off[v];
    for (uint32_t v = 0; v < n; ++v) cur[v] = t_off[v];
    for (uint32_t u = 0; u < n; ++u)
      for (uint32_t e = off[u]; e < off[u + 1]; ++e) t_idx[cur[idx[e]]++] = u;
    free(cur);
    in_off = t_off;
    in_idx = t_idx;
  }
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* xn = (double*)malloc(sizeof(double) * (size_t)n);
  double* contrib = (double*)malloc(sizeof(double) * (size_t)n);
  if (!x || !xn || !contrib) {
    free(x); free(xn); free(contrib); free(t_off); free(t_idx);
    return OR_ERR_OOM;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const double N = (double)n;
  for (uint32_t v = 0; v < n; ++v) x[v] = 1.0 / N;
  uint32_t it = 0;
  double l1 = 0.0;
  while (it < max_iter) {
    double dangling = 0.0;
    for (uint32_t u = 0; u < n; ++u) {
      uint32_t deg = off[u + 1] - off[u];
      if (deg == 0) { contrib[u] = 0.0; dangling += x[u]; }
      else contrib[u] = x[u] / (double)deg;
    }
    const double base = (1.0 - d) / N + d * dangling / N;
#pragma omp parallel for schedule(static)
    for (int64_t vv = 0; vv < (int64_t)n; ++vv) {
      uint32_t v = (uint32_t)vv;
      double s = 0.0;
      for (uint32_t e = in_off[v]; e < in_off[v + 1]; ++e) s += contrib[in_idx[e]];
      xn[v] = base + d * s;
    }
    l1 = 0.0;
    for (uint32_t v = 0; v < n; ++v) l1 += fabs(xn[v] - x[v]);
    double* t = x; x = xn; xn = t;
    ++it;
    if (l1 < tol) break;
  }
  memcpy(x_out, x, sizeof(double) * (size_t)n);
  if (iters_out) *iters_out = it;
  if (l1_out) *l1_out = l1;
  free(x); free(xn); free(contrib); free(t_off); free(t_idx);
  return OR_OK;
}

/* -------------------------------------------------------------- kcore */

/* k-core membership by peeling: repeatedly remove a vertex whose count of
 * remaining neighbour entries is below k, until none is left. in_core[v] = 1
 * for the survivors (the maximal subgraph in which every vertex keeps >= k
 * neighbour entries), 0 otherwise. Degrees count CSR entries of the symmetric
 * graph, so on a simple graph this is the usual k-core. */
int oracle_kcore(uint32_t n, const uint32_t* off, const uint32_t* idx, uint32_t k,
                 uint32_t* in_core) {
  uint32_t* deg = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
  uint8_t* removed = (uint8_t*)calloc(n ? n : 1, 1);
  uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
  if (!deg || !removed || !queue) { free(deg); free(removed); free(queue); return OR_ERR_OOM; }
  size_t head = 0, tail = 0;
  for (uint32_t v = 0; v < n; ++v) {
    deg[v] = off[v + 1] - off[v];
    if (deg[v] < k) { removed[v] = 1; queue[tail++] = v; }
  }
  while (head < tail) {
    uint32_t u = queue[head++];
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = idx[e];
      if (removed[v]) continue;
      deg[v]--;
      if (deg[v] < k) { removed[v] = 1; queue[tail++] = v; }
    }
  }
  for (uint32_t v = 0; v < n; ++v) in_core[v] = removed[v] ? 0u : 1u;
  free(deg); free(removed); free(queue);
  return OR_OK;
}

/* ------------------------------------------------- inspection (Alg. 1) */

/* Algorithm 1: for each active vertex of the worklist, read its out-degree; a
 * degree >= threshold sends it to the huge worklist `work`, otherwise it goes to
 * a TWC bin: thread if degree < warp_min, warp if degree < cta_min, else CTA.
 * bin[i] (for wl[i]) is 0 thread, 1 warp, 2 CTA, 3 huge. work keeps worklist
 * order, and prefix[0..nwork] is the exclusive prefix sum of the huge degrees
 * (prefix[nwork] = total huge edges e). counts[0..3] are the bin sizes. */
int oracle_inspect(uint32_t n, const uint32_t* off, const uint32_t* wl, uint32_t nf,
                   uint32_t threshold, uint32_t warp_min, uint32_t cta_min, uint32_t* work,
                   uint64_t* prefix, uint8_t* bin, uint32_t* counts) {
  uint32_t nwork = 0;
  counts[0] = counts[1] = counts[2] = counts[3] = 0;
  prefix[0] = 0;
  for (uint32_t i = 0; i < nf; ++i) {
    uint32_t v = wl[i];
    if (v >= n) return OR_ERR_ARG;
    uint32_t degree = off[v + 1] - off[v];
    uint8_t b;
    if (degree >= threshold) {
      b = 3;
      work[nwork] = v;
      prefix[nwork + 1] = prefix[nwork] + degree;
      ++nwork;
    } else if (degree < warp_min) {
      b = 0;
    } else if (degree < cta_min) {
      b = 1;
    } else {
      b = 2;
    }
    bin[i] = b;
    counts[b]++;
  }
  return OR_OK;
}

/* ------------------------------------------------- execution (Alg. 2) */

/* Largest j in [0, nwork) with prefix[j] <= k (binary search of prefixWork). */
static uint32_t prefix_search(const uint64_t* prefix, uint32_t nwork, uint64_t k) {
  uint32_t lo = 0, hi = nwork; /* invariant: prefix[lo] <= k < prefix[hi] */
  while (hi - lo > 1) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (prefix[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

/* Algorithm 2 for one thread T_i of p: the edge positions it is given in the
 * concatenated edge list of the huge vertices (total e = prefix[nwork]):
 *   cyclic  (policy 0): k = i, i + p, i + 2p, ... < e
 *   blocked (policy 1): k in [i*c, min(e, (i+1)*c)) with c = ceil(e/p)
 * For each k the source is work[j] with j found by binary search of prefix, the
 * edge is off[src] + (k - prefix[j]) and its destination idx[edge]. Writes up to
 * max_out (k, src, dst) triples and returns how many positions the thread has. */
int64_t oracle_lb_edges(const uint32_t* off, const uint32_t* idx, const uint32_t* work,
                        const uint64_t* prefix, uint32_t nwork, uint64_t p, uint64_t i,
                        int policy, uint64_t* k_out, uint32_t* src_out, uint32_t* dst_out,
                        int64_t max_out) {
  if (p == 0 || i >= p || nwork == 0) return 0;
  const uint64_t e = prefix[nwork];
  uint64_t begin, step, end;
  if (policy == 0) {
    begin = i; step = p; end = e;
  } else {
    uint64_t c = (e + p - 1) / p;
    begin = i * c; step = 1; end = (i + 1) * c < e ? (i + 1) * c : e;
  }
  int64_t count = 0;
  for (uint64_t k = begin; k < end; k += step) {
    if (count < max_out) {
      uint32_t j = prefix_search(prefix, nwork, k);
      uint32_t src = work[j];
      uint64_t edge = (uint64_t)off[src] + (k - prefix[j]);
      k_out[count] = k;
      src_out[count] = src;
      dst_out[count] = idx[edge];
    }
    ++count;
  }
  return count;
}

/* ------------------------------------------------------- certificates */

/* Exact check of BFS levels from src, valid at any size:
 *  (1) level[src] = 0 and no other vertex has level 0;
 *  (2) along every edge u -> v with level[u] finite: level[v] <= level[u] + 1;
 *  (3) every reached v != src has an in-neighbour u with level[u] + 1 = level[v].
 * (2) bounds each level above by the hop distance, (3) below; so they hold only
 * for the true BFS levels. Returns 0 if all hold, else 1 + the first failing
 * vertex in *bad. */
int oracle_check_bfs(uint32_t n, const uint32_t* off, const uint32_t* idx, uint32_t src,
                     const uint32_t* level, int64_t* bad) {
  *bad = -1;
  if (src >= n) return OR_ERR_ARG;
  uint8_t* has_pred = (uint8_t*)calloc(n ? n : 1, 1);
  if (!has_pred) return OR_ERR_OOM;
  int rc = OR_OK;
  if (level[src] != 0) { *bad = src; rc = OR_ERR_CHECK; }
  for (uint32_t u = 0; u < n && rc == OR_OK; ++u) {
    if (u != src && level[u] == 0) { *bad = u; rc = OR_ERR_CHECK; break; }
    if (level[u] == ORACLE_INF) continue;
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = idx[e];
      if (level[v] == ORACLE_INF || level[v] > level[u] + 1) { *bad = v; rc = OR_ERR_CHECK; break; }
      if (level[v] == level[u] + 1) has_pred[v] = 1;
    }
  }
  for (uint32_t v = 0; v < n && rc == OR_OK; ++v) {
    if (v != src && level[v] != ORACLE_INF && !has_pred[v]) { *bad = v; rc = OR_ERR_CHECK; }
  }
  free(has_pred);
  return rc;
}

/* Exact check of single-source shortest-path distances for weights >= 1:
 *  (1) dist[src] = 0;
 *  (2) along every edge u -> v with dist[u] finite: dist[v] <= dist[u] + w;
 *  (3) every reached v != src has an in-neighbour u with dist[u] + w = dist[v].
 * (2) gives dist <= true distance; (3) with positive weights gives a path of
 * length dist[v] back to src, so dist >= true distance. */
int oracle_check_sssp(uint32_t n, const uint32_t* off, const uint32_t* idx, const uint32_t* w,
                      uint32_t src, const uint32_t* dist, int64_t* bad) {
  *bad = -1;
  if (src >= n || !w) return OR_ERR_ARG;
  uint8_t* has_pred = (uint8_t*)calloc(n ? n : 1, 1);
  if (!has_pred) return OR_ERR_OOM;
  int rc = OR_OK;
  if (dist[src] != 0) { *bad = src; rc = OR_ERR_CHECK; }
  for (uint32_t u = 0; u < n && rc == OR_OK; ++u) {
    if (dist[u] == ORACLE_INF) continue;
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = idx[e];
      if (w[e] == 0) { *bad = v; rc = OR_ERR_ARG; break; }
      uint64_t nd = (uint64_t)dist[u] + w[e];
      if (dist[v] == ORACLE_INF || (uint64_t)dist[v] > nd) { *bad = v; rc = OR_ERR_CHECK; break; }
      if ((uint64_t)dist[v] == nd) has_pred[v] = 1;
    }
  }
  for (uint32_t v = 0; v < n && rc == OR_OK; ++v) {
    if (v != src && dist[v] != ORACLE_INF && !has_pred[v]) { *bad = v; rc = OR_ERR_CHECK; }
  }
  free(has_pred);
  return rc;
}
