/*
 * srk.h -- C ABI of the GB300 single-source SimRank library.
 *
 * The library computes the sqrt(c)-walk Monte Carlo estimate of single-source
 * SimRank described in "Massively Parallel Single-Source SimRanks in o(log n)
 * Rounds" (Luo and Zhu, arXiv 2304.04015), on one CUDA device (sm_103a).
 * The paper's MPC rounds become kernel phases on one stream:
 *   a1  sample-count table (Algorithm 1 lines 3-5, Algorithm 2 line 2, Lemma 7)
 *   a2  source walks of fixed lengths (Algorithm 1 lines 4-7, Section 4.1(a))
 *   a3  one uniform shuffle of the source's walks (Section 4.1(b), 5.2)
 *   a4  target walks, meeting detection and weighted counting (Section 4.2,
 *       Lemma 2, Lemma 3, Algorithm 2, Section 5.5)
 *   a5  scores s~(s,u) = sum of weights / z (Algorithm 2 line 10)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Graph: an in-neighbour CSR.  row_ptr has n+1 int32 entries, row_ptr[0] = 0,
 *   row_ptr[n] = m, non-decreasing; col has m int32 entries in [0, n), and
 *   col[row_ptr[v] .. row_ptr[v+1]) lists I(v), the in-neighbours of v
 *   (Eq. 1).  A walk moves from v to a uniform member of I(v), i.e. along a
 *   reversed edge (the graph G-bar of Lemma 2).  The list order matters only
 *   for reproducibility: the k-th entry is chosen by index.
 * Random numbers (Salmon et al., SC'11): walk steps use Philox2x32-10 with
 *   the 32-bit walk key kappa(seed, q) = h32(q ^ (mix64(seed) mod 2^32))
 *   (mix64: SplitMix64's output function; h32: the "lowbias32" finalizer;
 *   q = the query source s); step i >= 1 of walk replica r from node v takes
 *   word (i-1) & 1 of the block with counter (((i-1) >> 1) 2^24 + r, v), and
 *   the in-neighbour index below d is Lemire's bounded draw of that word
 *   (floor(w d / 2^32), accepted when w d mod 2^32 >= 2^32 mod d; a rejected
 *   word, probability < d / 2^32, is replaced by floor(R d / 2^64) from the
 *   block whose counter has the top bit of word (i-1) & 1 set), so every walk
 *   is reproducible on its own and every index is uniform up to d / 2^64.
 *   The source's Fisher-Yates draws use Philox4x32-10 keyed by
 *   (seed mod 2^32, seed >> 32).
 * Errors: every function returns SRK_OK (0) or a negative code; the message
 *   of the last failure on the calling thread is srk_last_error().  On error
 *   no output is guaranteed to be written.
 * Pointers: unless a flag says otherwise, an output pointer may be host or
 *   device memory (the library asks CUDA which).  With host output pointers
 *   the call copies results back and synchronises the stream before it
 *   returns; with device pointers it only enqueues work on `cuda_stream`
 *   (a cudaStream_t; NULL = the legacy default stream).
 * Determinism: identical graph, source, c, eps, seed and options give
 *   bit-identical counts, weight sums and scores, whatever the launch shape.
 * Threads: queries only read the graph, so concurrent queries on different
 *   streams are safe.  Each call allocates its scratch from a library-owned
 *   stream-ordered pool on the stream it runs on.
 */
#ifndef SRK_H
#define SRK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define SRK_OK        0
#define SRK_EINVAL   (-1)  /* an argument is out of range or malformed */
#define SRK_ENOMEM   (-2)  /* a device or host allocation failed */
#define SRK_ECUDA    (-3)  /* a CUDA runtime call or a kernel launch failed */
#define SRK_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define SRK_ENOTSUP  (-5)  /* the request is valid but not supported */

/* srk_opts.flags */
#define SRK_OPT_NO_GRAPH 1  /* srk_multi_source: enqueue launches directly
                               instead of through a captured CUDA graph */
#define SRK_OPT_WARMUP_RULE 2  /* sample counts of the warm-up algorithm
                                  (Section 3): z = ln(2 n^2) / (2 eps^2),
                                  L = floor(3 ln(n / eps) / ln(1/sqrt c));
                                  p and q are then not used */
#define SRK_OPT_LITERAL_SHUFFLE 4  /* single-source only: shuffle every
                                  target's walks too, by a keyed per-target
                                  permutation pi_u (unbalanced 4-round Feistel
                                  with hash round functions), as Section 5.2
                                  shuffles every node's walks.  Per target the
                                  pairing stays a uniform bijection (the
                                  source's shuffle is uniform); pi_u is only
                                  pseudo-random, so the independence of the
                                  pairings across targets that Section 5.2
                                  has is approximated, not reproduced.  About
                                  3.6x slower than the default pairing */

#define SRK_OPT_SHARED_WALKS 8  /* target walks keyed by (node, replica) alone:
                                  walk r of target u draws its steps under the
                                  walk key kappa(seed, 0xFFFFFFFE) instead of
                                  kappa(seed, s), so every
                                  node's walks are the same for all sources,
                                  as Algorithm 1 draws each node's walks once.
                                  Each (s, u) estimate keeps its law; estimates
                                  of different sources share target walks.
                                  srk_multi_source then walks each target once
                                  for all sources of a batch (up to 64 at a
                                  time); its results equal those of
                                  srk_single_source with this flag */

/* srk_graph_load flags. */
#define SRK_DEVICE_PTRS 1  /* row_ptr/col/edge_w are device pointers, borrowed */
#define SRK_VALIDATE    2  /* accepted; the CSR invariants are always checked */
#define SRK_ADJ_NARROW  4  /* force 4-byte adjacency entries (see srk_graph_load) */
#define SRK_ADJ_WIDE    8  /* force 8-byte adjacency entries (see srk_graph_load) */
#define SRK_ADJ_CSR    16  /* walks read row_ptr and col directly (see srk_graph_load) */

/* Upper bounds of this build. */
#define SRK_MAX_LEN   255          /* largest truncation length L */
#define SRK_MAX_WALKS (1 << 24)    /* largest N_tot, walks per node */

typedef struct srk_graph srk_graph;
typedef struct srk_linear_ctx srk_linear_ctx;

/* Per-query statistics (host memory), filled when srk_opts.stats != NULL. */
typedef struct srk_stats {
    double  z;              /* expected number of walk samples (Alg. 2 line 2) */
    int32_t L;              /* truncation length */
    int32_t n_walks;        /* N_tot = sum_l N_l, walks per node and pairs per target */
    int32_t n_active_pairs; /* pairs whose both walks take >= 1 step */
    int32_t batch_shape;    /* srk_multi_source: index of the persistent kernel's
                               launch shape the autotuner chose; else -1 */
    uint64_t source_steps;  /* steps taken by the source's walks */
    uint64_t target_steps;  /* target-walk steps taken over all targets (with
                               SRK_OPT_SHARED_WALKS in srk_multi_source: the
                               steps of the shared walks) */
    int64_t graph_updates;  /* srk_multi_source: batches launched by updating
                               the graph handle's cached CUDA-graph executable
                               instead of instantiating one (this call) */
} srk_stats;

/* Query options; pass NULL for the paper's defaults. */
typedef struct srk_opts {
    double   z_override;   /* > 0: use as z instead of ln(2n^q)/(2(eps-3/n^p)^2);
                              eps is then not used.  0: the paper's z; NaN,
                              negative or infinite: SRK_EINVAL */
    int32_t  L_override;   /* >= 0: truncation length instead of
                              floor(p ln n / ln(1/sqrt(c))); < 0: paper */
    int32_t  flags;        /* SRK_OPT_* bits (SRK_OPT_NO_GRAPH: multi-source only) */
    double   p;            /* threshold knob of Appendix B.5, >= 1 (0 means 1) */
    double   q;            /* failure knob of Appendix B.5, >= 1 (0 means 1) */
    uint32_t *step_counts; /* NULL or n entries (host or device memory):
                              target-walk steps taken per target */
    srk_stats *stats;      /* NULL or host pointer; forces a stream sync */
    void     *timing_events; /* NULL or a host array of two cudaEvent_t: [0] is
                              recorded on the query's stream just before the
                              target-walk kernel (step a4), [1] just after */
    int32_t  target_begin; /* with target_end: compute and write only the
                              targets u in [target_begin, target_end); 0, 0 =
                              all.  The paper's owner rule (Section 5.5): a
                              query split by node range across devices */
    int32_t  target_end;
} srk_opts;

/*
 * srk_graph_load -- make a graph resident on the current CUDA device.
 *   row_ptr, col : the in-neighbour CSR described above (n+1 and m entries).
 *   n            : number of nodes, 1 <= n < 2^31.
 *   m            : number of edges, 0 <= m < 2^31 (int32 offsets).
 *   flags        : SRK_DEVICE_PTRS: the arrays live on the current device and
 *                  are borrowed; the caller keeps them alive and unchanged
 *                  until srk_graph_free.  Otherwise they are host arrays and
 *                  are copied.  SRK_VALIDATE is accepted and implied.
 *                  SRK_ADJ_NARROW / SRK_ADJ_WIDE / SRK_ADJ_CSR force the
 *                  adjacency layout the walks read: a packed copy with
 *                  4-byte entries carrying a degree code of 32 - b bits,
 *                  2^b >= n + m + H, where the H nodes whose degree the code
 *                  cannot hold keep their degree in a header (n + m + H
 *                  words plus n positions; SRK_EINVAL if n + m + H >= 2^31);
 *                  a packed copy with 8-byte entries carrying the full
 *                  degree (2 (n + m) words); or row_ptr and col themselves
 *                  (no copy).  By default: 4-byte entries while
 *                  n + m <= 2^28, 8-byte entries beyond.  Results do not
 *                  depend on the layout; giving more than one of the flags
 *                  is SRK_EINVAL.
 * The CSR invariants (row_ptr[0] = 0, row_ptr[n] = m, row_ptr non-decreasing,
 * 0 <= col < n) are always checked on the device before the handle is
 * returned; a violation returns SRK_EINVAL.  The walk kernels rely on them.
 *   edge_w       : NULL, or m FP32 edge weights aligned with col (used by the
 *                  linearised form); copied unless SRK_DEVICE_PTRS.
 *   out          : receives the handle.
 * Storage follows the paper's reversed graph G-bar (Algorithm 1 lines 1-2):
 * walks read in-neighbour lists.  The call is synchronous.
 */
int srk_graph_load(const int32_t *row_ptr, const int32_t *col, int32_t n,
                   int64_t m, int flags, const float *edge_w, srk_graph **out);

/* srk_graph_free -- release a handle and the device memory it owns.
 * Waits for the device; NULL is accepted. */
int srk_graph_free(srk_graph *g);

/* srk_graph_info -- n and m of a loaded graph (either pointer may be NULL). */
int srk_graph_info(const srk_graph *g, int32_t *n, int64_t *m);

/* srk_graph_layout -- the adjacency layout the walks read (see srk_graph_load):
 * *layout = SRK_ADJ_NARROW, SRK_ADJ_WIDE or SRK_ADJ_CSR. */
int srk_graph_layout(const srk_graph *g, int32_t *layout);

/*
 * srk_single_source -- estimate s~(s, u) for every node u (Algorithms 1, 2).
 *   s     : query source, 0 <= s < n.
 *   c     : SimRank decay factor, 0 < c < 1 (walks continue w.p. sqrt(c)).
 *   eps   : absolute error target, 3/n^p < eps < 1 (Theorem 6); z =
 *           ln(2n^q) / (2 (eps - 3/n^p)^2) walk samples per node.
 *   seed  : 64-bit seed of every random draw of the query.
 *   opt   : NULL or options (see srk_opts).
 *   scores      : n FP64 outputs, s~(s, u) = W_u 2^-32 / z, s~(s, s) = 1, and
 *                 0 for a node without in-neighbours.
 *   meet_counts : NULL or n uint32 outputs, meeting walk pairs per target.
 *   weight_sums : NULL or n uint64 outputs, W_u = sum over meeting pairs of
 *                 round(a(l1) a(l2) 2^32), a(l) = |Z_l| / |Z^_l| (Lemma 7).
 *   cuda_stream : stream to run on (see Pointers).
 * Walk lengths: N_l = ceil(z sqrt(c)^l (1 - sqrt(c))) walks of length l for
 * l = 0..L, L = floor(p ln n / ln(1/sqrt c)).  The source's N_tot walks are
 * shuffled by one Fisher-Yates permutation; pair j joins source walk sigma(j)
 * with target walk j (with SRK_OPT_LITERAL_SHUFFLE, target u's walk pi_u(j),
 * pi_u a keyed permutation of its own).  A pair meets when both walks are at
 * the same node at
 * the same step i >= 1; it counts once.  A walk stops early at a node without
 * in-neighbours.  Returns SRK_EINVAL for s, c, eps, p, q out of range, or
 * when L > SRK_MAX_LEN, N_tot > SRK_MAX_WALKS or sum_l l N_l >= 2^31.
 */
int srk_single_source(const srk_graph *g, int32_t s, double c, double eps,
                      uint64_t seed, const srk_opts *opt, double *scores,
                      uint32_t *meet_counts, uint64_t *weight_sums,
                      void *cuda_stream);

/*
 * srk_multi_source -- k independent single-source queries, batched.
 *   sources : k source nodes (host memory).
 *   eps     : k error targets (host memory), one per source, so the sources'
 *             walk budgets N_tot differ.
 *   scores  : k x n FP64 outputs (host or device), row i for sources[i].
 *   meet_counts : NULL or k x n uint32 outputs.
 * Results equal k calls of srk_single_source with the same seed (each walk's
 * key is derived from its source).  The sources run in batches sized by
 * a scratch budget (a quarter of free device memory, at most 8 GiB, or the
 * byte count in the environment variable SRK_BATCH_BYTES): one
 * launch per source-side phase for the whole batch, then one persistent
 * launch over the batch's (source, target) work items, captured in a CUDA
 * graph unless opt->flags has SRK_OPT_NO_GRAPH.  Sources none of whose walk
 * pairs can meet (e.g. no in-neighbours) and targets without in-neighbours
 * produce no work items; their scores are written directly.  The persistent
 * kernel's launch shape is picked per graph by timing the candidate shapes on
 * the first items of the first call (kept in the handle).  The call
 * synchronises the stream at the end of every batch.  With
 * SRK_OPT_SHARED_WALKS the batches hold up to 64 sources, grouped by walk
 * budget with the sources without in-neighbours last (the call first reads
 * the sources' in-degrees from the device CSR, synchronising the stream);
 * rows still land in the caller's order.  opt->step_counts must
 * be NULL, and target ranges and SRK_OPT_LITERAL_SHUFFLE are refused
 * (SRK_EINVAL); opt->stats, if set, receives totals over all sources.
 */
int srk_multi_source(const srk_graph *g, const int32_t *sources, int32_t k,
                     double c, const double *eps, uint64_t seed,
                     const srk_opts *opt, double *scores,
                     uint32_t *meet_counts, void *cuda_stream);

/*
 * srk_multi_source_topk -- srk_multi_source with a sparse output: for each
 * source, its `top` most similar targets.  Section 5.5 ends with every
 * machine holding the scores s~(s, u) of its targets; for many sources the
 * dense k x n matrix is too large to keep (4,096 sources of a 16.8M-node
 * graph: 550 GB), so this call keeps per source only
 *   top_nodes  : k x top int32 (device): row i lists the targets u != s_i of
 *                largest s~(s_i, u), score descending, ties by smaller id;
 *                -1 after the last nonzero score;
 *   top_scores : k x top FP64 (device): their scores (0 after the last);
 *   top_count  : NULL or k int32 (device): entries filled, min(top, nnz);
 *   nnz        : NULL or k int64 (device): targets with a nonzero score.
 * The scores are exactly those of srk_multi_source (same options, including
 * SRK_OPT_SHARED_WALKS).  Sources run in chunks whose dense rows fit a
 * scratch budget (an eighth of free device memory, at most 16 GiB, or the
 * byte count in SRK_TOPK_ROWS_BYTES; a multiple of 64 rows when 64 or more
 * fit); with SRK_OPT_SHARED_WALKS the chunks take the sources with
 * in-neighbours by eps, descending, and the others last (sources outside
 * [0, n) are refused, SRK_EINVAL).  Each chunk's rows are selected on the
 * device by a radix select over the scores' bit patterns.  1 <= top <= 4096
 * (SRK_EINVAL otherwise); host output pointers are refused (SRK_EINVAL).
 */
int srk_multi_source_topk(const srk_graph *g, const int32_t *sources, int32_t k,
                          double c, const double *eps, uint64_t seed,
                          const srk_opts *opt, int32_t top, int32_t *top_nodes,
                          double *top_scores, int32_t *top_count, int64_t *nnz,
                          void *cuda_stream);

/*
 * srk_linear_fwd -- truncated linearised single-source SimRank (Appendix A:
 * S = c P^T S P + D, truncated to L + 1 terms, as in the DISK discussion):
 *     s_out = sum_{t=0}^{L} c^t (P^T)^t D P^t e_s,   D = (1 - c) I,
 * with P the column-normalised in-edge weight matrix,
 * P[u][a] = w(u -> a) / sum_{u' in I(a)} w(u' -> a).  D = (1 - c) I is a
 * simplification: the paper's D is a correction matrix that is estimated.
 *   g      : the graph; its in-lists give the edges (edge e = entry e of col).
 *   edge_w : m positive finite FP32 weights aligned with col (device memory),
 *            or NULL for the weights given to srk_graph_load (or when m = 0).
 *   s, c   : source (0 <= s < n) and decay (0 < c < 1).
 *   L      : last term, 0 <= L <= SRK_MAX_LEN.
 *   s_out  : n FP32 outputs (device memory).
 *   ctx    : NULL, or receives the context the backward needs (device
 *            memory for P, the vectors P^t e_s and the partial sums, about
 *            (2L + 5) n + 2m words); release it with srk_linear_ctx_free.
 *            The context refers to g, which must outlive it.
 *   cuda_stream : stream to run on; the call synchronises it (to report
 *            non-positive weights as SRK_EINVAL).
 * The first call on a graph also builds and keeps in the handle a transpose
 * of the graph (out-lists in edge order) and the edges' owners, about
 * 3m + 3n words, released by srk_graph_free.  Arithmetic is FP32; P v and
 * P^T v are gathers along out-lists and in-lists, every sum taken in a fixed
 * order, so results are bitwise reproducible.
 */
int srk_linear_fwd(const srk_graph *g, const float *edge_w, int32_t s, double c,
                   int32_t L, float *s_out, srk_linear_ctx **ctx, void *cuda_stream);

/*
 * srk_linear_bwd -- gradient of a loss w.r.t. the edge weights, by the adjoint
 * of the forward recursions.
 *   ctx    : from srk_linear_fwd (not freed here; one backward at a time).
 *   grad_s : n FP32, dLoss/ds_out (device memory).
 *   grad_w : m FP32 outputs, dLoss/dw_e (device memory; may be NULL when m = 0).  Because P is
 *            invariant to scaling a node's in-weights, sum_{e in I(a)} w_e
 *            grad_w[e] = 0 for every node a (up to rounding).
 * Enqueues work on cuda_stream without synchronising.
 */
int srk_linear_bwd(srk_linear_ctx *ctx, const float *grad_s, float *grad_w,
                   void *cuda_stream);

/* srk_linear_ctx_free -- release a context (waits for the device); NULL ok. */
int srk_linear_ctx_free(srk_linear_ctx *ctx);

/*
 * srk_single_source_noalloc -- srk_single_source that allocates nothing.
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory while they issue queries (an application whose
 * own allocator owns the device budget, a serving thread that must not block
 * on or fail in the driver's allocator).  Load the graph once beforehand
 * (SRK_DEVICE_PTRS borrows the caller's arrays); this call then makes no
 * cudaMalloc, cudaFree, cudaMallocAsync or other allocating call.
 *   Arguments and results are those of srk_single_source, except: scores,
 *   meet_counts, weight_sums and opt->step_counts must be device memory
 *   (SRK_EINVAL otherwise), and the query's scratch must fit in
 *   SRK_NOALLOC_SCRATCH_BYTES (about 4 N_tot (L + 18) bytes; SRK_EINVAL with
 *   the needed size otherwise).
 *   Scratch: one static device array of SRK_NOALLOC_SCRATCH_BYTES, held on
 *   every GPU where the library's module is loaded until the process exits.
 *   Its address is looked up by the first call in each CUDA context of a
 *   device (make that first call before any stream capture; a context that
 *   replaced an earlier one, e.g. after cudaDeviceReset, gets a fresh
 *   lookup).  Every call reuses the array and
 *   clears what must start at zero; calls that overlap on the GPU (e.g. on
 *   two streams) race on it and must be serialised by the caller.
 */
#define SRK_NOALLOC_SCRATCH_BYTES (16u << 20)
int srk_single_source_noalloc(const srk_graph *g, int32_t s, double c,
                              double eps, uint64_t seed, const srk_opts *opt,
                              double *scores, uint32_t *meet_counts,
                              uint64_t *weight_sums, void *cuda_stream);

/*
 * srk_probe_gather -- measurement utility (the paper has no counterpart): the
 * random-gather roofline a walk step is measured against.  Enqueues one kernel
 * on `cuda_stream` in which every thread of a full-occupancy grid performs
 * `iters` rounds of four independent random 4-byte loads from `data` (device,
 * n int32 entries, 1 <= n < 2^32), indices from per-thread linear congruential
 * generators seeded by `seed`.  `sink` (device, one uint64) keeps the loads
 * alive; `loads` (host, may be NULL) receives the number of loads issued.  The
 * caller times the launch (e.g. with CUDA events) and divides.
 */
int srk_probe_gather(const int32_t *data, int64_t n, int64_t iters, uint32_t seed,
                     unsigned long long *sink, int64_t *loads, void *cuda_stream);

/*
 * srk_probe_gather_ex -- srk_probe_gather with the PTX cache operator of the
 * loads chosen by `cache_op` (one of SRK_PROBE_*), to show whether a cache
 * hint changes the random-gather ceiling.  SRK_EINVAL for an unknown value.
 */
#define SRK_PROBE_DEFAULT 0  /* ld.global */
#define SRK_PROBE_CG      1  /* ld.global.cg: cache in L2, not L1 */
#define SRK_PROBE_NC      2  /* ld.global.nc: read-only data path */
#define SRK_PROBE_CA      3  /* ld.global.ca: cache at all levels */
int srk_probe_gather_ex(const int32_t *data, int64_t n, int64_t iters, uint32_t seed,
                        int32_t cache_op, unsigned long long *sink, int64_t *loads,
                        void *cuda_stream);

/*
 * srk_pool_stats -- what the library's stream-ordered memory pool of `device`
 * holds (a measurement utility; the paper has no counterpart).  Queries take
 * their scratch from this pool and return it when they finish.
 *   reserved:  bytes of device memory backing the pool now;
 *   used:      bytes handed out to queries in flight now;
 *   used_high: the largest `used` since the pool was created or the mark was
 *              last reset.
 * Any output pointer may be NULL.  reset_high != 0 resets the mark to the
 * current use after reading it.  SRK_EINVAL for a device outside
 * [0, device count), SRK_ECUDA when the pool cannot be created or read.
 */
int srk_pool_stats(int32_t device, uint64_t *reserved, uint64_t *used, uint64_t *used_high,
                   int reset_high);

/*
 * Query server (no counterpart in the paper; the serving configuration):
 * resident graphs, memory-based admission, worker threads with one CUDA
 * stream each, latency statistics.
 *
 * srk_server_create -- graphs: n_graphs loaded handles (they must outlive the
 *   server); mem_budget: device bytes that admitted, unfinished requests may
 *   hold (each request holds its query scratch plus its n-entry score vector);
 *   n_workers: worker threads / streams (1..64); latency_target_ms: 0 for
 *   memory-only admission and first-in-first-out service, else a target for
 *   the estimated time to finish all admitted work including the new request,
 *   with shortest-estimated-work-first service.  The estimate of a request
 *   is (nodes with in-neighbours) x N_tot x (walk steps per pair) / (walk
 *   steps per second), 0 when the source has no in-neighbours; both figures
 *   are kept per graph, measured at creation by four queries with z = 256
 *   from evenly spaced nodes with in-neighbours, and refined by every
 *   completed request (exponential averages).  Copies each graph's row_ptr
 *   to the host once.
 * srk_server_submit -- enqueue one srk_single_source query on graph index
 *   `graph`.  The request is admitted if the memory it needs fits in what the
 *   budget leaves (and, with a latency target, its estimated finish fits the
 *   target); otherwise it is shed (*admitted = 0; not an error).
 *   host_scores: NULL, or n host doubles that receive the scores before the
 *   request counts as completed (caller keeps them alive until then).  tag is
 *   reserved for the caller.  Invalid arguments return SRK_EINVAL.
 * srk_server_drain -- wait until every admitted request has completed.
 * srk_server_stats -- counters and the latency (submission to scores on the
 *   host) percentiles of completed requests.
 * srk_server_destroy -- finish queued requests, stop the workers, free.
 */
typedef struct srk_server srk_server;
typedef struct srk_server_report {
    uint64_t submitted, admitted, shed, completed, failed;
    uint64_t target_steps;   /* walk steps of completed requests */
    uint64_t reserved_peak;  /* most device memory held by admitted requests */
    double p50_ms, p99_ms, mean_ms, max_ms;
    double wall_s;           /* first submission to last completion */
    double queries_per_s;    /* completed / wall_s */
} srk_server_report;

int srk_server_create(const srk_graph *const *graphs, int32_t n_graphs,
                      uint64_t mem_budget, int32_t n_workers, double latency_target_ms,
                      srk_server **out);
int srk_server_submit(srk_server *srv, int32_t graph, int32_t s, double c, double eps,
                      uint64_t seed, double *host_scores, uint64_t tag, int32_t *admitted);
int srk_server_drain(srk_server *srv);
int srk_server_stats(srk_server *srv, srk_server_report *report);
int srk_server_destroy(srk_server *srv);

/* Message of the last failure on this thread ("" if none). */
const char *srk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SRK_H */
