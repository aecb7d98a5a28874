/*
 * alb.h - C ABI of libalb.so: the adaptive load balancer (ALB) for graph
 * analytics of Jatala et al., "An Adaptive Load Balancer For Graph Analytics on
 * GPUs" (arXiv:1911.09135), for one NVIDIA GB300 (sm_103a).
 *
 * Every traversal runs in bulk-synchronous rounds over a sparse frontier of
 * active vertices (Sec. 2). Each round:
 *   - inspection (Algorithm 1, Sec. 4.1) reads each active vertex's degree and
 *     sends degree >= threshold to the huge worklist `work`, appending each one
 *     together with its slot of the exclusive prefix sum of huge degrees
 *     ("prefixWork", Sec. 4.1 "Search"); the other vertices are expanded at once
 *     by thread, warp or CTA according to their degree (TWC, Sec. 3);
 *   - if `work` is non-empty (and only then, Sec. 5.1 "Thread Block Load
 *     Distribution"), the execution kernel (Algorithm 2) spreads the edges of
 *     all huge vertices over every thread of the grid, cyclically by default
 *     (Sec. 4.1 "Distribution"), finding each edge's source by binary search of
 *     prefixWork;
 *   - the operator (Sec. 2, Fig. 3) is applied along every expanded edge and
 *     the vertices it activates form the next frontier.
 * The loop runs on the device (a CUDA graph with a conditional while node), so
 * a call makes no host round trip per round.
 *
 * Conventions for every call:
 *   - Pointers named d_* must be device memory (or managed). Pointers named
 *     hd_* may be host or device memory; the library detects which. Arrays are
 *     plain uint32_t / float / double in native order, no padding.
 *   - Work is enqueued on `stream` (a cudaStream_t cast to void*, NULL = the
 *     legacy default stream) and is asynchronous: results are valid once the
 *     stream has been synchronised or alb_sync() returned ALB_OK. When an
 *     output is host memory the library copies into it on the same stream.
 *   - Calls on one alb_graph must be ordered (same stream, or externally
 *     synchronised): a handle owns one workspace and is not thread-safe.
 *     Different handles are independent. The first call of each kind on a
 *     handle allocates its workspace and instantiates a CUDA graph; it first
 *     waits for the whole device to be idle (cudaDeviceSynchronize), so no
 *     set-up ever overlaps running kernels. Make those first calls (warm the
 *     handle) before running several handles concurrently on different streams,
 *     or the other streams stall while one handle sets up.
 *   - Argument errors are returned synchronously and enqueue nothing. Errors
 *     detected on the device (round limit exceeded, corrupt CSR) are latched in
 *     the handle and returned by alb_sync() and alb_get_stats().
 *   - Unreached vertices get ALB_UNREACHED (BFS, SSSP).
 */
#ifndef ALB_H_
#define ALB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ALB_UNREACHED 0xFFFFFFFFu

typedef struct alb_graph_s* alb_graph; /* opaque, library-owned */
typedef void* alb_stream;              /* a cudaStream_t */

typedef enum {
  ALB_OK = 0,
  ALB_ERR_INVALID_ARG = 1,   /* bad pointer, size, vertex id or parameter */
  ALB_ERR_OOM = 2,           /* device or pinned-host allocation failed */
  ALB_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  ALB_ERR_TIMEOUT = 4,       /* the round limit (alb_params.max_rounds) was reached */
  ALB_ERR_OVERFLOW = 5,      /* m >= 2^32, or max_weight * (n - 1) does not fit below 2^32 - 1 */
  ALB_ERR_NOT_SYMMETRIC = 6, /* cc / kcore / pagerank need a graph created with ALB_SYMMETRIC */
  ALB_ERR_UNSUPPORTED = 7,   /* e.g. sssp on a graph without weights */
  ALB_ERR_DEVICE = 8         /* a device-side check failed (an index out of range in the CSR) */
} alb_status;

typedef enum {
  ALB_APP_BFS = 0,
  ALB_APP_SSSP = 1,
  ALB_APP_CC = 2,
  ALB_APP_PAGERANK = 3, /* d = 0.85, tol = 1e-6 */
  ALB_APP_KCORE = 4     /* k = 32 */
} alb_app;

/* Flags of alb_graph_create. */
#define ALB_SYMMETRIC 0x1u /* the CSR holds both directions of every edge (undirected graph) */
#define ALB_VALIDATE  0x2u /* check on the device that every index is < n and offsets are monotone */

/* Tuning knobs (Sec. 4.1 "Threshold", Sec. 3 "TWC"). alb_default_params()
 * fills the defaults; alb_set_params() applies them to one handle. */
typedef struct {
  /* Degree at or above which an active vertex is huge and goes to the LB
   * kernel. < 0 (default): the number of threads the LB kernel launches, the
   * paper's rule (Sec. 4.1; 163840 on its V100, Sec. 5). 0 sends every active
   * vertex to the LB kernel; a value above the maximum degree disables it
   * (plain TWC). */
  int64_t hub_threshold;
  uint32_t twc_warp_min;   /* degree >= this goes to the warp bin (default 32) */
  uint32_t twc_cta_min;    /* degree >= this goes to the CTA bin (default 256, the CTA size) */
  uint32_t grid_blocks;    /* CTAs of every round kernel; 0 = SMs x resident CTAs per SM of each kernel
                            * (PageRank's pull kernel: 8 such waves) */
  uint32_t distribution;   /* LB edge distribution: 0 cyclic (default), 1 blocked (Sec. 4.1) */
  uint32_t exec_mode;      /* 0: device-side round loop in a CUDA graph (default); 1: host loop
                            * (one launch per kernel, the round state read by the host after each;
                            * batched calls then run their groups one after another) */
  uint32_t max_rounds;     /* 0: n + 1 (enough for every app); ALB_ERR_TIMEOUT when reached */
  float l2_persist_fraction; /* > 0 (CUDA-graph mode): the labels get an L2 access-policy window
                              * whose hits persist in this share of the device's persisting L2
                              * maximum (set for the calling process's context); the labels are
                              * then computed in the handle's buffer and copied to the output.
                              * 0 = off (default) */
  uint32_t profile;        /* 1: time every kernel launch with CUDA events (host loop only) */
  uint32_t cta_stats;      /* 1: count the edges each CTA expands (alb_get_cta_loads) */
  uint32_t block_size;     /* threads per CTA of the round kernels (inspection + TWC, LB kernel):
                            * 128, 256 (default; the paper's 2^8, Sec. 5.1) or 512; 0 = 256.
                            * The LB kernel's thread count, and so the default threshold, follows
                            * it. PageRank's kernels keep 256. */
} alb_params;

/* Counters of the last completed call on a handle. */
typedef struct {
  uint32_t rounds;         /* rounds (PageRank: iterations) */
  uint32_t hub_rounds;     /* rounds in which the LB kernel ran */
  uint32_t max_hub_count;  /* largest huge worklist of any round */
  uint32_t hub_threshold;  /* effective threshold */
  uint32_t lb_threads;     /* threads the LB kernel launches (p in Sec. 4.2) */
  uint32_t grid_blocks;    /* CTAs of the round kernels */
  uint32_t block_size;     /* threads per CTA */
  uint32_t reserved;
  uint64_t edges_twc;      /* CSR entries expanded by the TWC part of inspection */
  uint64_t edges_lb;       /* CSR entries expanded by the LB kernel */
  uint64_t pushes;         /* vertices appended to next frontiers */
  double pr_l1;            /* PageRank: L1 change of the last iteration */
  /* profile = 1 only: summed device time (ms) and launch counts per kernel */
  double ms_inspect, ms_lb, ms_other;
  uint32_t n_inspect, n_lb, n_other, reserved2;
} alb_stats;

/* ---------------------------------------------------------------- graphs */

/* Create a graph from CSR arrays (Sec. 4.1 "Search": CSR keeps only each
 * edge's destination; sources are found by search). hd_offsets[n+1] and
 * hd_indices[m] (and hd_weights[m], may be NULL) may be host or device
 * memory; they are copied into library-owned device memory on `stream`, so
 * the caller may free them once the stream has synchronised. The out-edges of
 * u are hd_indices[hd_offsets[u] .. hd_offsets[u+1]). m must be < 2^32.
 * Returns ALB_ERR_INVALID_ARG for n == 0, NULL arrays, or hd_offsets[n] != m
 * (checked after the copy, synchronising the stream), ALB_ERR_OVERFLOW for
 * m >= 2^32, ALB_ERR_DEVICE if ALB_VALIDATE finds an index >= n. */
alb_status alb_graph_create(uint32_t n, uint64_t m, const uint32_t* hd_offsets,
                            const uint32_t* hd_indices, const uint32_t* hd_weights,
                            uint32_t flags, alb_stream stream, alb_graph* out);

/* A second handle on the same device graph: it shares the CSR (no copy) and the parameters
 * of `src` at the time of the call, and owns a separate workspace, so calls on the two handles
 * may run concurrently on different streams (e.g. several server slots on one large graph).
 * The CSR is freed with the last handle that uses it. */
alb_status alb_graph_clone(alb_graph src, alb_graph* out);

/* Free a graph and its workspace (waits for the whole device first). */
alb_status alb_graph_destroy(alb_graph g);

/* Release what the handle's calls allocated on first use and kept for the next call: the
 * multi-source batch workspace and its worker clones, PageRank's per-graph inspection and
 * vectors, the staging buffer of host outputs and every cached CUDA graph. The CSR and the round
 * workspace stay, so the handle remains usable; the next call of each kind allocates again. A
 * server uses it to give device memory back to other graphs under memory pressure. The paper has
 * no counterpart (it runs one query at a time). Waits for the whole device first; *freed_bytes
 * (may be NULL) receives the growth of the device's free memory. */
alb_status alb_graph_trim(alb_graph g, uint64_t* freed_bytes);

/* alb_set_params applies p to every application of the handle; alb_get_params returns the
 * bfs parameters. Per-application parameters: see alb_set_app_params below. Setting
 * parameters drops cached work and waits for the whole device first. */
alb_status alb_default_params(alb_params* p);
alb_status alb_set_params(alb_graph g, const alb_params* p);
alb_status alb_get_params(alb_graph g, alb_params* p);

/* ----------------------------------------------------------- applications */

/* Breadth-first search (Sec. 5 "bfs", push): hd_levels[v] = hops from src,
 * ALB_UNREACHED if none. hd_levels has n entries. */
alb_status alb_bfs(alb_graph g, uint32_t src, uint32_t* hd_levels, alb_stream stream);

/* Single-source shortest paths (Sec. 5 "sssp"; the relaxation operator of
 * Sec. 4.3, Fig. 3: dist[v] = min(dist[v], dist[u] + w(u,v)), applied
 * data-driven until no distance changes). Needs weights; hd_dist has n entries.
 * ALB_ERR_OVERFLOW if max_weight * (n - 1) could reach 2^32 - 1. */
alb_status alb_sssp(alb_graph g, uint32_t src, uint32_t* hd_dist, alb_stream stream);

/* Connected components (Sec. 5 "cc", push label propagation): hd_labels[v] =
 * the smallest vertex id of v's component. Needs ALB_SYMMETRIC. */
alb_status alb_cc(alb_graph g, uint32_t* hd_labels, alb_stream stream);

/* PageRank (Sec. 5 "pr", pull over incoming edges; for a symmetric graph these
 * are the CSR rows). FP32 with FP32 sums, deterministic order:
 *   x_0 = 1/n;  x_{t+1}[v] = (1-d)/n + d * (sum_{u->v} x_t[u]/deg(u) + D_t/n),
 * D_t = sum of x_t over vertices of degree 0; stops when the FP64 L1 change
 * ||x_{t+1} - x_t||_1 < tol or after max_iter iterations. hd_rank[n] receives
 * the last iterate; hd_l1 (1 double) and hd_iters (1 uint32) may be NULL.
 * Needs ALB_SYMMETRIC. */
alb_status alb_pagerank(alb_graph g, float damping, double tol, uint32_t max_iter,
                        float* hd_rank, double* hd_l1, uint32_t* hd_iters, alb_stream stream);

/* k-core (Sec. 5 "kcore"): hd_in_core[v] = 1 if v belongs to the k-core (the
 * maximal subgraph in which every vertex keeps >= k neighbour entries), else 0.
 * Peels vertices whose remaining degree drops below k. Needs ALB_SYMMETRIC. */
alb_status alb_kcore(alb_graph g, uint32_t k, uint32_t* hd_in_core, alb_stream stream);

/* ---------------------------------------------------------------- batches */

/* Many sources over one graph: source s's result goes to hd_out[s * n .. (s+1) * n)
 * (source-major), identical per source to alb_bfs / alb_sssp. Sources run in groups of 32
 * that share every CSR read: a frontier vertex carries the set of sources for which it is
 * active and each expanded edge is relaxed for all of them (bit-parallel for bfs). The
 * rounds use the same inspection, TWC and cyclic LB kernels (Algorithms 1 and 2). hd_srcs
 * has k entries (repeats allowed); each must be < n: sources in host memory are checked at
 * once (ALB_ERR_INVALID_ARG, nothing enqueued); sources in device memory are checked on the
 * device, an invalid one is skipped and ALB_ERR_INVALID_ARG is returned by alb_sync. Sources
 * in pinned host memory are copied asynchronously: keep them unchanged until the stream has
 * passed the call. Workspace:
 * 32 labels, a seen mask and three round masks per vertex (144 bytes x n), allocated on first use.
 * With more than 32 sources and a device output, the groups run concurrently: the handle takes
 * one and up to three worker clones of it (sharing its CSR; each with its own round and batch
 * workspace, CUDA graphs and stream, about 170 bytes x n) the others. The workers are made and
 * warmed on the first such call with the device idle (cudaDeviceSynchronize), kept until the
 * parameters change or the handle is destroyed, and joined to `stream` by events; alb_sync
 * reports their errors. A host output keeps the groups on `stream`, one after another. */
alb_status alb_bfs_batch(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_out,
                         alb_stream stream);
alb_status alb_sssp_batch(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_out,
                          alb_stream stream);

/* One traversal from a set of sources at distance 0: hd_levels[v] (hd_dist[v]) = distance from
 * the nearest of hd_srcs[0..k). On a graph that is the disjoint union of many graphs with one
 * source in each, this computes every graph's own bfs (sssp) in one launch sequence, which is
 * how many small graphs are batched. Sources are checked as for alb_bfs_batch. */
alb_status alb_bfs_multi(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_levels,
                         alb_stream stream);
alb_status alb_sssp_multi(alb_graph g, const uint32_t* hd_srcs, uint32_t k, uint32_t* hd_dist,
                          alb_stream stream);

/* -------------------------------------------------------------- autotuner */


/* Parameters of one application only (what alb_autotune sets); the diagnostics and the
 * batched / multi-source bfs (sssp) calls use the bfs (sssp) parameters. */
alb_status alb_set_app_params(alb_graph g, alb_app app, const alb_params* p);
alb_status alb_get_app_params(alb_graph g, alb_app app, alb_params* p);

/* Pick the load-balancing knobs for one application on this graph by timing it on the device
 * (Sec. 4.1 "Threshold": the best threshold depends on the hardware; Sec. 5.1 finds a wide
 * flat range). Coordinate search: the threshold over {threads of the LB kernel, 2^8, 2^10, ...,
 * 2^20, never huge}, then twc_cta_min in {128, 256, 512, 1024} x twc_warp_min in {16, 32, 64}
 * at the best threshold, then block_size in {128, 256, 512} (not for PageRank); each setting is
 * timed as the mean of `reps` calls after one warm-up call. The fastest setting is applied to that application (alb_set_app_params) and returned
 * in *best (may be NULL) with
 * its time in *best_ms (may be NULL). src is used by bfs and sssp. Synchronises `stream`.
 * Results of every setting are identical (only the schedule changes). */
alb_status alb_autotune(alb_graph g, alb_app app, uint32_t src, uint32_t reps, alb_params* best,
                        float* best_ms, alb_stream stream);

/* ------------------------------------------------------------ diagnostics */

/* Algorithm 1 alone, on the device, for an explicit worklist hd_wl[nf]:
 * hd_bin[i] = 0 thread, 1 warp, 2 CTA, 3 huge for hd_wl[i]; the huge vertices
 * are written to hd_work[0..v) in device append order with hd_prefix[0..v]
 * their exclusive prefix sum of degrees (hd_prefix[v] = total huge edges);
 * hd_counts[4] = bin sizes. hd_work and hd_prefix need nf + 1 entries. */
alb_status alb_inspect(alb_graph g, const uint32_t* hd_wl, uint32_t nf, uint8_t* hd_bin,
                       uint32_t* hd_work, uint32_t* hd_prefix, uint32_t* hd_counts,
                       alb_stream stream);

/* Algorithm 2's edge assignment as performed by the LB kernel itself: for the
 * huge worklist hd_work[nwork] with exclusive prefix hd_prefix[nwork+1], every
 * position k < e = hd_prefix[nwork] of the concatenated edge list is processed
 * by the kernel, which records hd_src[k], hd_dst[k] and the global thread id
 * hd_thread[k] that handled it. Uses the handle's distribution and grid. */
alb_status alb_lb_trace(alb_graph g, const uint32_t* hd_work, const uint32_t* hd_prefix,
                        uint32_t nwork, uint32_t* hd_src, uint32_t* hd_dst, uint32_t* hd_thread,
                        alb_stream stream);

/* The paper's default threshold rule (Sec. 4.1, Sec. 5): the number of
 * threads launched = SMs x resident threads per SM (80 x 2048 = 163840 on V100). */
uint32_t alb_threshold_rule(uint32_t num_sms, uint32_t threads_per_sm);

/* ------------------------------------------------------ allocation-free */

/* Largest graph alb_bfs_noalloc accepts. */
#define ALB_NOALLOC_MAX_VERTICES (1u << 20)

/* BFS for callers that cannot allocate device memory: for instance code running
 * while another stream captures a CUDA graph, a service whose device memory is
 * all owned by another allocator, or a latency-bound loop that must not block
 * the device in cudaMalloc/cudaFree. The paper has no counterpart: this is a
 * packaging of the same bfs path (same kernels and results as alb_bfs with
 * default parameters). It needs no alb_graph and never allocates: its scratch
 * (frontiers, huge worklist and prefix sums, visited bitmap, round state; about 16.9 MB) is one
 * fixed array in the library's device image, held on every GPU that loads the
 * library until the process exits.
 *   n <= ALB_NOALLOC_MAX_VERTICES, else ALB_ERR_INVALID_ARG (nothing enqueued);
 *   d_offsets[n+1], d_indices[m], d_levels[n] must be device memory.
 * The CSR is checked on the device first: ALB_ERR_INVALID_ARG if offsets[0] != 0,
 * offsets[n] != m or the offsets decrease anywhere; ALB_ERR_DEVICE if an index is
 * >= n. Nothing is traversed after a failed check. In the bounds-checked build
 * (libalb_checked.so) an access the round kernels had to skip is reported as
 * ALB_ERR_DEVICE at the end of the call. The call synchronises `stream` once per
 * round and returns after d_levels is complete.
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture begins. Every call on a device shares
 * the one array and overwrites it, so calls whose work overlaps on the GPU
 * (other threads, other streams) race and must be serialised by the caller. */
alb_status alb_bfs_noalloc(uint32_t n, uint64_t m, const uint32_t* d_offsets,
                           const uint32_t* d_indices, uint32_t src, uint32_t* d_levels,
                           alb_stream stream);

/* Wait for the handle's last call and return any latched device error. */
alb_status alb_sync(alb_graph g);

/* Counters of the last call (synchronises like alb_sync). */
alb_status alb_get_stats(alb_graph g, alb_stats* out);

/* Static string for a status code. */
const char* alb_status_str(alb_status s);

/* Per-CTA load of the last call made with cta_stats = 1 (the measure behind the paper's
 * thread-block load distributions, Sec. 3 Fig. 1 and Sec. 5.1 Fig. 4): hd_twc[b] = edges CTA b of
 * the TWC part expanded (the inspection kernel of bfs/sssp/cc/kcore; PageRank's pull kernel), and
 * hd_lb[b] = edges CTA b of the LB kernel expanded, summed over the call's rounds. At most cap
 * entries are written to each (host or device memory); *n_twc / *n_lb receive the number of
 * CTAs (0 if the last call was not instrumented). Synchronises the handle's last stream. */
alb_status alb_get_cta_loads(alb_graph g, uint64_t* hd_twc, uint64_t* hd_lb, uint32_t cap,
                             uint32_t* n_twc, uint32_t* n_lb);

/* Bounds-checked build. libalb_checked.so (built with -DALB_CHECKED) tests every CSR, frontier,
 * worklist and label-row index a round kernel uses; an index out of range is skipped and
 * recorded instead of being accessed. alb_debug_check copies the handle's record (first
 * failing code, its index and bound, number of failures; all zero when none failed, and
 * always zero in the regular build) after synchronising the handle's last stream.
 * alb_checked_build returns 1 in the checked build, 0 otherwise. */
alb_status alb_debug_check(alb_graph g, uint32_t* out4);
uint32_t alb_checked_build(void);

/* ------------------------------------------------------- SM partitions (serving) */

/* An SM partition: a CUDA green context owning a subset of the device's SMs. Kernels launched on
 * a stream created from it (every call of this library takes the stream) run only on its SMs.
 * A server gives small graphs a partition of their own, so their short round kernels do not wait
 * for SM room held by large graphs' persistent round kernels. There is no counterpart in the
 * paper, which runs one query at a time. Device memory is shared with the rest of the process.
 * Returns ALB_ERR_UNSUPPORTED where the driver has no green contexts. */
typedef struct alb_partition_s* alb_partition; /* opaque, library-owned */

/* Split device `device` into *first with sm_count SMs (rounded up to the device's partition
 * granularity, 8 SMs on GB300) and *rest with the remaining SMs. sm_count must leave SMs for
 * *rest (ALB_ERR_INVALID_ARG otherwise; nothing is created). */
alb_status alb_partition_split(int device, uint32_t sm_count, alb_partition* first, alb_partition* rest);
/* SMs the partition owns. */
alb_status alb_partition_sms(alb_partition p, uint32_t* sms);
/* A non-blocking stream of the partition with the given priority (lower = higher, as
 * cudaStreamCreateWithPriority); destroy it with alb_partition_stream_destroy before the
 * partition. */
alb_status alb_partition_stream_create(alb_partition p, int priority, alb_stream* out);
alb_status alb_partition_stream_destroy(alb_stream s);
/* Destroys the partition (its streams must be destroyed and their work complete). */
alb_status alb_partition_destroy(alb_partition p);

/* Library version: major * 10000 + minor * 100 + patch. */
uint32_t alb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ALB_H_ */
