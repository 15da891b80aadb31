// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "srk.h"

struct srk_graph {
  int32_t n = 0;
  int64_t m = 0;
  int device = 0;
  const int32_t *row_ptr = nullptr;  // device, n+1
  const int32_t *col = nullptr;      // device, m
  const float *edge_w = nullptr;     // device, m or null
  // Packed adjacency (owned, n + m + H words, H the hubs below).  Node v's
  // identity inside the walk kernels is its position npos[v].  A node of
  // in-degree d < deg_max = 2^(32-pos_bits) - 1 has the word d at its
  // position and its list right after it; a hub (d >= deg_max) has two words
  // {d, offset of its list} at position 2r of the hub region at the front,
  // r its rank by how often walks visit it (so the hot headers share
  // sectors), and its list after the other nodes'.  The other nodes' words
  // follow in the order of expected visits per list entry (build_narrow).  Entry k of v's list holds
  // the k-th in-neighbour y as (min(|I(y)|, deg_max) << pos_bits) | npos[y],
  // so a walk step learns the next node's degree from the entry it reads and
  // reads a header only at a hub.
  // Wide layout (layout = 1, chosen when n + m needs more than 28 bits or
  // forced by SRK_ADJ_WIDE): 2 (n + m) words forming 8-byte entries at
  // positions v + row_ptr[v], adj[pos(v)] = {0, |I(v)|} and entries
  // {pos(y), |I(y)|}, so a step never reads a header.  CSR layout (layout =
  // 2, only when forced by SRK_ADJ_CSR): no packed copy; nodes are their ids
  // and a step reads row_ptr and col.
  uint32_t *adj = nullptr;
  int32_t *npos = nullptr;  // narrow layout: positions, n (owned)
  int32_t n_hubs = 0;       // narrow layout: H
  int32_t pos_bits = 1;     // positions < 2^pos_bits
  int layout = 0;        // 0 narrow, 1 wide, 2 CSR (no packed adjacency; walks read row_ptr/col)
  // Nodes with at least one in-neighbour, ascending (owned): the only targets
  // whose score can be nonzero.
  int32_t *act = nullptr;
  int32_t n_act = 0;
  // Launch shape of the batched target kernel chosen by the autotuner
  // (-1: not tuned yet).
  int batch_cfg = -1;
  // Executable of the last captured batch (srk_multi_source with a CUDA
  // graph), updated in place for the next batch of the same shape.
  cudaGraphExec_t batch_exec = nullptr;
  // Topology of the linearised form (edge owners, a transpose, list size
  // classes), built by the first srk_linear_fwd on the graph.
  struct srk_lin_topo *lin = nullptr;
  int32_t *own_row_ptr = nullptr;    // owned copies (null when borrowed)
  int32_t *own_col = nullptr;
  float *own_w = nullptr;
};

namespace srk {

// The output function of SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) and
// the 32-bit finalizer "lowbias32" (C. Wellons, 2018); both are bijections.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
__host__ __device__ __forceinline__ uint32_t h32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

// Key word of the shared target walks (SRK_OPT_SHARED_WALKS) in place of a
// source (sources are below 2^31, so it names none).
constexpr uint32_t kSharedWalkKey = 0xFFFFFFFEu;

// The 32-bit Philox2x32-10 key of a query's walks: h32(q ^ low half of
// mix64(seed)), q the source (its source walks, and its target walks by
// default) or kSharedWalkKey (the shared target walks).  Injective in q for a
// given seed, since h32 is a bijection.
__host__ __device__ __forceinline__ uint32_t walk_key(uint64_t seed, uint32_t q) {
  return h32(q ^ (uint32_t)mix64(seed));
}

// Sample-count table of one query (Algorithm 1 lines 3-5, Algorithm 2 line 2,
// Lemma 7).  Passed by value as a kernel parameter (stays below 4 KB).
struct QueryTab {
  int32_t s, n, L, N_tot;
  uint32_t key0, key1;  // the seed's halves (Fisher-Yates draws, literal shuffle)
  uint32_t skey, tkey;  // walk keys of the source walks and of the target walks
  int32_t literal;  // 1: literal target shuffle (SRK_OPT_LITERAL_SHUFFLE)
  int32_t shared;   // 1: shared target walks (SRK_OPT_SHARED_WALKS)
  double z;
  int32_t P[SRK_MAX_LEN + 2];  // stratum prefix: walk r has length l iff P[l] <= r < P[l+1]
  double a[SRK_MAX_LEN + 1];   // rounding weight a(l) = |Z_l| / |Z^_l|
};
static_assert(sizeof(QueryTab) <= 4096, "kernel parameter too large");

// Fills `t`; returns SRK_OK or SRK_EINVAL (message set).
int build_table(int32_t n, int32_t s, double c, double eps, uint64_t seed,
                const srk_opts *opt, QueryTab *t);

// Sets the thread's last-error message (printf-style) and returns `code`.
int fail(int code, const char *fmt, ...);
// Maps a CUDA error to SRK_ECUDA / SRK_ENOMEM with a message.
int cuda_fail(cudaError_t e, const char *what);
void clear_error();

// Library-owned stream-ordered pool of the given device.
cudaMemPool_t pool(int device);
// True when p is device or managed memory visible to the current device.
bool is_device_ptr(const void *p);

// RAII guard that makes `dev` current and restores the previous device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
      cudaSetDevice(prev);
  }
};

// SM count of the current device (cached per device).
int sm_count(int device);

// Scratch of one query, carved from one device block (srk_query.cu).
struct Workspace {
  int32_t *spos, *seff, *kdraw, *grp_cnt, *rank, *grp_off, *items, *first,
      *succ, *sigma, *pair_j, *Hc, *small;
  unsigned long long *pair_w;
  size_t bytes;
};

// Device outputs of one query (null = not wanted, except scores).
struct Outputs {
  double *scores;
  uint32_t *counts;
  unsigned long long *wsums;
  uint32_t *steps;
};

// Carves `base` (or only sizes the plan when base is null); returns the
// number of bytes one query of table `t` needs.
size_t plan(const QueryTab &t, Workspace *w, char *base);
// Enqueues steps a2-a5 on `st`; `timing` (may be null) gets two events
// recorded around the target-walk kernel.
int enqueue_query(const srk_graph *g, const QueryTab &t, const Workspace &w,
                  const Outputs &o, cudaStream_t st, const cudaEvent_t *timing,
                  int32_t u_begin, int32_t u_end);
// [*b, *e): the targets a query computes, from its options (SRK_EINVAL when
// the range is malformed).
int target_range(const srk_graph *g, const srk_opts *opt, int32_t *b, int32_t *e);
// Exclusive scan of cnt[0..N) into off[0..N] (one block of 1024 threads).
__global__ void k_scan(const int32_t *__restrict__ cnt, int32_t *__restrict__ off,
                       int32_t N);


// In-degrees of k sources (ids already checked against n), read from the
// device CSR on stream st (synchronises st).  SRK_OK or an error code.
int source_in_degrees(const srk_graph *g, const int32_t *sources, int32_t k, cudaStream_t st,
                      std::vector<int32_t> *deg);

// Releases the graph's linear topology, if built (srk_linear.cu).
void free_lin_topo(srk_graph *g);

// Copies the query counters into `stats` (synchronises `st`).
int read_stats(const QueryTab &t, const Workspace &w, cudaStream_t st,
               srk_stats *stats, bool accumulate);

}  // namespace srk
