// Single- and multi-source queries: the sqrt(c)-walk Monte Carlo estimator of
// arXiv 2304.04015 as kernel phases on one stream.
//
//   a2  k_source_walks   N_tot fixed-length walks from s (Algorithm 1 lines
//                        4-7) and the Fisher-Yates draws of the shuffle
//   a3  k_fy_rank .. k_pairs
//                        the Fisher-Yates permutation sigma (Section 4.1(b),
//                        Section 5.2), resolved in parallel (see k_pairs), and
//                        each pair's step cap min(l2, steps of source walk)
//       k_rows, k_hit_table
//                        pairs sorted by cap (descending) and the step-major
//                        hit table: row i holds, for every pair that can still
//                        meet at step i, the source walk's node at step i
//   a4+a5 k_target_walks the hot loop: every target walks its pairs, detects
//                        the first meeting (Lemma 2, Algorithm 2, Section 5.5)
//                        and writes count, weight sum and score
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "srk_device.cuh"
#include "srk_internal.h"

namespace srk {

// ---------------------------------------------------------------- step a2 --
// Walk r of the source has length l = stratum(r).  Step i >= 1 moves to
// I(x)[k], k the bounded draw below |I(x)| from word (i-1)&1 of the
// Philox2x32-10 block (((i-1)>>1) << 24 | r, s) under the source's walk key
// (step_entry); it stops early at a node with no in-neighbours.  Walks run
// on the graph's adjacency layout (a packed copy
// in which nodes are identified by their position, or the CSR itself).  The
// same thread computes Fisher-Yates draw t = r, k_t = floor(R * (t+1) / 2^64)
// with R from counter (t>>1, ~0, ~0, s).
template <int kLayout>
__global__ void __launch_bounds__(256)
k_source_walks(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
               const uint32_t *__restrict__ adj, const int32_t *__restrict__ npos, int pos_bits,
               const __grid_constant__ QueryTab tab,
               int32_t *__restrict__ spos, int32_t *__restrict__ seff,
               int32_t *__restrict__ kdraw, int32_t *__restrict__ grp_cnt,
               int32_t *__restrict__ small_base) {
  __shared__ int32_t P[SRK_MAX_LEN + 2];
  for (int i = threadIdx.x; i <= tab.L + 1; i += blockDim.x) P[i] = tab.P[i];
  __syncthreads();
  const RoundKeys rk = round_keys(tab.key0, tab.key1);
  const int Ls = tab.L > 0 ? tab.L : 1;
  const uint32_t s = (uint32_t)tab.s;
  const auto G = adj_view<kLayout>(adj, npos, pos_bits, row_ptr, col);
  uint32_t deg_s = 0;
  const int32_t b_s = node_start(G, row_ptr, tab.s, deg_s);
  unsigned long long steps = 0;
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < tab.N_tot;
       r += gridDim.x * blockDim.x) {
    grp_cnt[r] = 0;
    kdraw[r] = (r >= 1) ? fy_draw(rk, s, r) : 0;
    const int len = stratum_of(P, tab.L, r);
    const int eff = source_walk(tab.skey, G, s, b_s, deg_s, r, len, spos + (int64_t)r * Ls);
    seff[r] = eff;
    steps += (unsigned long long)eff;
  }
  // source-step total (one atomic per warp)
  for (int off = 16; off > 0; off >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, off);
  if ((threadIdx.x & 31) == 0 && steps)
    atomicAdd(small_view(small_base).ctr + 1, steps);
}

// ---------------------------------------------------------------- step a3 --
// The permutation sigma of the sequential Fisher-Yates loop "for t = N-1
// down to 1: swap(sigma[t], sigma[k_t])" is resolved in parallel.  Position
// t >= 1 is final after step t and receives the value that position k_t held
// just before step t.  Position p (p <= t) was last written before step t by
// the step t' = min{t' > t : k_t' = p}, which moved in the value position t'
// held before step t'; if no such step exists it still holds p.  Following
// these links gives sigma[t] (sigma[0]: the value of position 0 after all
// steps).  Steps are grouped by k (counting sort) to find the links.

__global__ void k_fy_rank(const int32_t *__restrict__ kdraw, int32_t *grp_cnt,
                          int32_t *__restrict__ rank, int32_t N) {
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += gridDim.x * blockDim.x)
    if (t >= 1) rank[t] = atomicAdd(&grp_cnt[kdraw[t]], 1);
}

// Exclusive scan of cnt[0..N) into off[0..N], one block of 1024 threads.
__global__ void __launch_bounds__(1024)
k_scan(const int32_t *__restrict__ cnt, int32_t *__restrict__ off, int32_t N) {
  __shared__ int32_t warp_sum[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < N; base += 4096) {
    const int64_t i0 = base + 4 * (int64_t)threadIdx.x;
    int32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (i0 + k < N) ? cnt[i0 + k] : 0;
    const int32_t local = v[0] + v[1] + v[2] + v[3];
    int32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int32_t ws = warp_sum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sum[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    int32_t run = carry + (wid ? warp_sum[wid - 1] : 0) + incl - local;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i0 + k < N) off[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = run;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[N] = carry;
}

__global__ void k_fy_scatter(const int32_t *__restrict__ kdraw,
                             const int32_t *__restrict__ off,
                             const int32_t *__restrict__ rank,
                             int32_t *__restrict__ items, int32_t N) {
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += gridDim.x * blockDim.x)
    if (t >= 1) items[off[kdraw[t]] + rank[t]] = t;
}

// Per group q = {t : k_t = q}: sort ascending, first[q] = its smallest step,
// succ[t] = the next larger step of t's group (-1 for the largest).
__global__ void k_fy_groups(const int32_t *__restrict__ off,
                            int32_t *__restrict__ items,
                            int32_t *__restrict__ first,
                            int32_t *__restrict__ succ, int32_t N) {
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < N;
       q += gridDim.x * blockDim.x) {
    const int32_t b = off[q], e = off[q + 1];
    for (int32_t i = b + 1; i < e; ++i) {  // insertion sort (groups are tiny)
      const int32_t x = items[i];
      int32_t k = i - 1;
      while (k >= b && items[k] > x) { items[k + 1] = items[k]; --k; }
      items[k + 1] = x;
    }
    first[q] = (e > b) ? items[b] : -1;
    for (int32_t i = b; i < e; ++i) succ[items[i]] = (i + 1 < e) ? items[i + 1] : -1;
  }
}

// sigma[j] by following the links, then the pair's step cap
// cap_j = min(l2 = stratum(j), steps taken by source walk sigma[j]);
// pairs with cap >= 1 are counted per cap value.
__global__ void __launch_bounds__(256)
k_pairs(const __grid_constant__ QueryTab tab, const int32_t *__restrict__ kdraw,
        const int32_t *__restrict__ first, const int32_t *__restrict__ succ,
        const int32_t *__restrict__ seff, int32_t *__restrict__ sigma,
        int32_t *__restrict__ small_base) {
  __shared__ int32_t P[SRK_MAX_LEN + 2];
  __shared__ int32_t hist[SRK_MAX_LEN + 2];
  for (int i = threadIdx.x; i <= tab.L + 1; i += blockDim.x) {
    P[i] = tab.P[i];
    hist[i] = 0;
  }
  __syncthreads();
  const int32_t N = tab.N_tot;
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < N;
       j += gridDim.x * blockDim.x) {
    const int32_t p = resolve_sigma(j, kdraw, first, succ, N);
    sigma[j] = p;
    // literal mode: the target walk is pi_u(j), so only the source bounds the cap
    const int32_t cap = tab.literal ? seff[p] : min(stratum_of(P, tab.L, j), seff[p]);
    if (cap >= 1) atomicAdd(&hist[cap], 1);
  }
  __syncthreads();
  Small sm = small_view(small_base);
  for (int i = threadIdx.x; i <= tab.L + 1; i += blockDim.x)
    if (hist[i]) atomicAdd(&sm.cap_hist[i], hist[i]);
}

// Hit-table geometry: pairs sorted by cap, descending.  Row i (i = 1..L) has
// cnt[i] = #pairs with cap >= i entries and starts at R[i].
// Also finds [act_lo, act_hi), the part of the ascending active-target list
// `act` inside [u_begin, u_end): the target kernel's work counter starts at
// act_lo, and act_hi is stored in the word after it.
__global__ void k_rows(int L, int32_t *__restrict__ small_base, const int32_t *__restrict__ act,
                       int32_t n_act, int32_t n, int32_t u_begin, int32_t u_end) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Small sm = small_view(small_base);
  int32_t *bounds = reinterpret_cast<int32_t *>(sm.ctr + 2);  // counter, act_hi
  auto lower_bound = [&](int32_t v) {  // first index with act[index] >= v
    int32_t lo = 0, hi = n_act;
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo) / 2;
      if (act[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  bounds[0] = u_begin == 0 ? 0 : lower_bound(u_begin);
  bounds[1] = u_end == n ? n_act : lower_bound(u_end);
  int32_t c = 0;
  sm.cnt[L + 1] = 0;
  for (int i = L; i >= 1; --i) {
    sm.cursor[i] = c;  // cap-i pairs follow all pairs with a larger cap
    c += sm.cap_hist[i];
    sm.cnt[i] = c;
  }
  int32_t r = 0;
  for (int i = 1; i <= L + 1; ++i) {
    sm.R[i] = r;
    if (i <= L) r += sm.cnt[i];
  }
  sm.cnt[0] = c;
  sm.R[0] = 0;
}

// Places every pair with cap >= 1 in its cap group and fills its column of the
// hit table with the source walk's nodes at steps 1..cap.  The pair's Lemma 7
// weight is round(a(l1) a(l2) 2^32) with l1 the source walk's length.
__global__ void __launch_bounds__(256)
k_hit_table(const __grid_constant__ QueryTab tab, const int32_t *__restrict__ sigma,
            const int32_t *__restrict__ seff, const int32_t *__restrict__ spos,
            int32_t *__restrict__ small_base, int32_t *__restrict__ pair_j,
            unsigned long long *__restrict__ pair_w, int32_t *__restrict__ Hc) {
  __shared__ int32_t P[SRK_MAX_LEN + 2];
  __shared__ int32_t R[SRK_MAX_LEN + 2];
  Small sm = small_view(small_base);
  for (int i = threadIdx.x; i <= tab.L + 1; i += blockDim.x) {
    P[i] = tab.P[i];
    R[i] = sm.R[i];
  }
  __syncthreads();
  const int Ls = tab.L > 0 ? tab.L : 1;
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < tab.N_tot;
       j += gridDim.x * blockDim.x) {
    const int32_t w = sigma[j];
    const int l2 = stratum_of(P, tab.L, j);
    const int32_t cap = tab.literal ? seff[w] : min(l2, seff[w]);
    if (cap < 1) continue;
    const int l1 = stratum_of(P, tab.L, w);
    const int32_t a = atomicAdd(&sm.cursor[cap], 1);
    pair_j[a] = j;
    // literal mode keeps l1: the weight needs the target walk's length
    pair_w[a] = tab.literal ? (unsigned long long)l1
                            : __double2ull_rn(tab.a[l1] * tab.a[l2] * 4294967296.0);
    const int32_t *src = spos + (int64_t)w * Ls;
    for (int i = 1; i <= cap; ++i) Hc[R[i] + a] = src[i - 1];
  }
}

// -------------------------------------------------------------- steps a4-a5 --
// Each warp takes targets u from a global counter.  Its 32 lanes walk the
// target's pairs a = 0, 1, ... of the cap-sorted list; a lane whose walk ends
// takes the next unassigned pair at once (lane refill), so walks that end
// early (cap, meeting, no in-neighbours) do not idle the warp.  Walks run on
// the packed adjacency: from a node at position p with degree d, a step reads
// entry adj[p + 1 + index], which holds the next node's position and, unless
// that node's degree is large, its degree as well.  Pair a (original index
// j) walks from u: one Philox2x32-10 block, counter (((i-1)>>1) << 24 | j, u)
// under the target walks' key, serves the odd step i (word 0) and the even
// step i+1 (word 1).  A step moves to I(x)[k], k the bounded draw below |I(x)|
// (step_entry); the walk meets when its node equals row i of
// the hit table, ends after cap steps (a >= cnt[i+1]) or at a node without
// in-neighbours.  The first meeting adds 1 to the count and the pair's weight
// to W_u.  The warp then reduces and writes count, W and s~(s,u) = W 2^-32 / z
// (s~(s,s) = 1).
struct TargetArgs {
  const int32_t *row_ptr;  // CSR offsets (wide and CSR layouts locate nodes by them)
  const int32_t *col;      // in-neighbour lists (CSR layout)
  const uint32_t *adj;     // packed adjacency (see srk_internal.h)
  const int32_t *npos;     // 4-byte-entry layout: node positions
  int32_t pos_bits;
  int32_t n, s, L;
  uint32_t walk_key;       // walk key of the target walks (the source's or the shared one)
  uint32_t key0, key1;
  double z;
  const int32_t *small_base;
  const int32_t *pair_j;
  const unsigned long long *pair_w;
  const int32_t *Hc;
  double *scores;
  uint32_t *counts;
  unsigned long long *wsums;
  uint32_t *steps_per_target;
  unsigned long long *steps_total;
  int32_t *target_counter;  // next index into act (from act_lo), then act_hi
  const int32_t *act;       // the targets with in-neighbours, ascending
  int32_t u_begin, u_end;   // targets computed: [u_begin, u_end)
  int32_t N_tot;            // literal mode: the permutation's domain
};

// Literal mode also needs the stratum prefix and the Lemma 7 weights.
struct LiteralArgs {
  int32_t P[SRK_MAX_LEN + 2];
  double a[SRK_MAX_LEN + 1];
};

// 8 blocks of 256 threads per SM (32 registers): the kernel is bound by the
// rate of scattered L1 misses, and full occupancy keeps the most misses in
// flight.  kLiteral: the literal target shuffle (walk_target_literal).
template <bool kLiteral, int kLayout>
__global__ void __launch_bounds__(256, 8)
k_target_walks(const __grid_constant__ TargetArgs A, const __grid_constant__ LiteralArgs X) {
  __shared__ int2 rc[SRK_MAX_LEN + 3];  // {R[i], cnt[i+1]}, one load per step
  __shared__ int32_t Psh[kLiteral ? SRK_MAX_LEN + 2 : 1];
  {
    const Small sm = small_view(const_cast<int32_t *>(A.small_base));
    for (int i = threadIdx.x; i <= A.L + 2; i += blockDim.x) {
      rc[i] = make_int2((i <= A.L + 1) ? sm.R[i] : 0,
                        (i + 1 <= A.L + 1) ? sm.cnt[i + 1] : 0);  // cnt[L+1] = cnt[L+2] = 0
      if (kLiteral && i <= A.L + 1) Psh[i] = X.P[i];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t lanes_below = (1u << lane) - 1u;
  const auto G = adj_view<kLayout>(A.adj, A.npos, A.pos_bits, A.row_ptr, A.col);
  PairSet S;
  S.rc = rc;
  S.pair_j = A.pair_j;
  S.pair_w = A.pair_w;
  S.Hc = A.Hc;
  S.n_pairs = rc[0].y;  // cnt[1]
  S.key = A.walk_key;
  FeistelShape fs;
  if constexpr (kLiteral)
    fs = feistel_shape(A.N_tot, ((uint64_t)A.key1 << 32) | A.key0, (uint32_t)A.s);
  unsigned long long warp_steps = 0;
  // the active targets act[counter .. act_hi) (k_rows set the counter to the
  // range's first index and act_hi beside it); the outputs of the others
  // were cleared before the launch, and s's score is 1
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.s >= A.u_begin && A.s < A.u_end)
    A.scores[A.s] = 1.0;
  if (S.n_pairs == 0) return;  // no pair can meet: every output is zero
  for (;;) {
    int32_t u = -1;
    if (lane == 0) {
      const int32_t q = atomicAdd(A.target_counter, 1);
      if (q < A.target_counter[1]) u = A.act[q];
    }
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u < 0) break;
    uint32_t c = 0, st = 0;
    unsigned long long W = 0;
    uint32_t deg_u = 0;
    const int32_t b_u = node_start(G, A.row_ptr, u, deg_u);
    if (u != A.s && deg_u > 0) {
      if (kLiteral)
        walk_target_literal(G, S, fs, Psh, A.L, X.a, (uint32_t)u, b_u, deg_u,
                            lanes_below, c, W, st);
      else
        walk_target(G, S, (uint32_t)u, b_u, deg_u, c, W, st);
    }
    for (int off = 16; off > 0; off >>= 1) {
      c += __shfl_xor_sync(0xffffffffu, c, off);
      st += __shfl_xor_sync(0xffffffffu, st, off);
      W += __shfl_xor_sync(0xffffffffu, W, off);
    }
    if (lane == 0) {
      A.scores[u] = (u == A.s) ? 1.0 : (double)W * 2.3283064365386963e-10 / A.z;
      if (A.counts) A.counts[u] = c;
      if (A.wsums) A.wsums[u] = W;
      if (A.steps_per_target) A.steps_per_target[u] = st;
      warp_steps += st;
    }
  }
  if (lane == 0 && warp_steps) atomicAdd(A.steps_total, warp_steps);
}

// ------------------------------------------------------------ host side --

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t plan(const QueryTab &t, Workspace *w, char *base) {
  const size_t N = (size_t)t.N_tot;
  const size_t Ls = (size_t)(t.L > 0 ? t.L : 1);
  size_t hc = 0;
  for (int l = 1; l <= t.L; ++l) hc += (size_t)l * (size_t)(t.P[l + 1] - t.P[l]);
  if (hc == 0) hc = 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  w->spos = (int32_t *)take(4 * N * Ls);
  w->seff = (int32_t *)take(4 * N);
  w->kdraw = (int32_t *)take(4 * N);
  w->grp_cnt = (int32_t *)take(4 * N);
  w->rank = (int32_t *)take(4 * N);
  w->grp_off = (int32_t *)take(4 * (N + 1));
  w->items = (int32_t *)take(4 * N);
  w->first = (int32_t *)take(4 * N);
  w->succ = (int32_t *)take(4 * N);
  w->sigma = (int32_t *)take(4 * N);
  w->pair_j = (int32_t *)take(4 * N);
  w->pair_w = (unsigned long long *)take(8 * N);
  w->Hc = (int32_t *)take(4 * hc);
  w->small = (int32_t *)take(kSmallBytes);
  w->bytes = off;
  return off;
}

static int grid_for(int64_t work, int threads, int device) {
  const int64_t want = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count(device) * 8;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

static int target_grid(int device) {
  static int blocks_per_sm[64] = {};
  int b = (device >= 0 && device < 64) ? blocks_per_sm[device] : 0;
  if (!b) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_target_walks<false, kNarrow>, 256, 0) !=
            cudaSuccess || b < 1)
      b = 1;
    if (device >= 0 && device < 64) blocks_per_sm[device] = b;
  }
  return sm_count(device) * b;
}

// Enqueues one query on `st` with device-resident outputs `o`.  Workspace
// `w` (already carved) must hold plan(t) bytes.
int enqueue_query(const srk_graph *g, const QueryTab &t, const Workspace &w,
                  const Outputs &o, cudaStream_t st, const cudaEvent_t *timing,
                  int32_t u_begin, int32_t u_end) {
  const int dev = g->device;
  const int N = t.N_tot;
  const int gN = grid_for(N, 256, dev);
  cudaError_t e = cudaMemsetAsync(w.small, 0, kSmallBytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "clearing query counters");
  if (g->layout == kWide)
    k_source_walks<kWide><<<gN, 256, 0, st>>>(g->row_ptr, g->col, g->adj, g->npos, g->pos_bits, t,
                                              w.spos, w.seff, w.kdraw, w.grp_cnt, w.small);
  else if (g->layout == kCsr)
    k_source_walks<kCsr><<<gN, 256, 0, st>>>(g->row_ptr, g->col, g->adj, g->npos, g->pos_bits, t,
                                             w.spos, w.seff, w.kdraw, w.grp_cnt, w.small);
  else
    k_source_walks<kNarrow><<<gN, 256, 0, st>>>(g->row_ptr, g->col, g->adj, g->npos, g->pos_bits, t,
                                                w.spos, w.seff, w.kdraw, w.grp_cnt, w.small);
  k_fy_rank<<<gN, 256, 0, st>>>(w.kdraw, w.grp_cnt, w.rank, N);
  k_scan<<<1, 1024, 0, st>>>(w.grp_cnt, w.grp_off, N);
  k_fy_scatter<<<gN, 256, 0, st>>>(w.kdraw, w.grp_off, w.rank, w.items, N);
  k_fy_groups<<<gN, 256, 0, st>>>(w.grp_off, w.items, w.first, w.succ, N);
  k_pairs<<<gN, 256, 0, st>>>(t, w.kdraw, w.first, w.succ, w.seff, w.sigma, w.small);
  k_rows<<<1, 32, 0, st>>>(t.L, w.small, g->act, g->n_act, g->n, u_begin, u_end);
  // targets without in-neighbours have zero outputs (and s, if it is one of
  // them, the score 1 the kernel writes): clear the range, then walk only
  // the active targets
  const size_t nr = (size_t)(u_end - u_begin);
  if (nr > 0) {
    e = cudaMemsetAsync(o.scores + u_begin, 0, sizeof(double) * nr, st);
    if (e == cudaSuccess && o.counts)
      e = cudaMemsetAsync(o.counts + u_begin, 0, sizeof(uint32_t) * nr, st);
    if (e == cudaSuccess && o.wsums)
      e = cudaMemsetAsync(o.wsums + u_begin, 0, sizeof(unsigned long long) * nr, st);
    if (e == cudaSuccess && o.steps)
      e = cudaMemsetAsync(o.steps + u_begin, 0, sizeof(uint32_t) * nr, st);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the outputs of the target range");
  }
  k_hit_table<<<gN, 256, 0, st>>>(t, w.sigma, w.seff, w.spos, w.small, w.pair_j,
                                  w.pair_w, w.Hc);
  TargetArgs A;
  A.row_ptr = g->row_ptr;
  A.col = g->col;
  A.adj = g->adj;
  A.npos = g->npos;
  A.pos_bits = g->pos_bits;
  A.n = g->n;
  A.s = t.s;
  A.walk_key = t.tkey;
  A.L = t.L;
  A.key0 = t.key0;
  A.key1 = t.key1;
  A.z = t.z;
  A.small_base = w.small;
  A.pair_j = w.pair_j;
  A.pair_w = w.pair_w;
  A.Hc = w.Hc;
  A.scores = o.scores;
  A.counts = o.counts;
  A.wsums = o.wsums;
  A.steps_per_target = o.steps;
  A.steps_total = small_view(w.small).ctr;
  A.target_counter = reinterpret_cast<int32_t *>(small_view(w.small).ctr + 2);
  A.act = g->act;
  A.u_begin = u_begin;
  A.u_end = u_end;
  A.N_tot = t.N_tot;
  LiteralArgs X;
  if (t.literal) {
    memcpy(X.P, t.P, sizeof X.P);
    memcpy(X.a, t.a, sizeof X.a);
  } else {
    memset(&X, 0, sizeof X);
  }
  if (timing) cudaEventRecord(timing[0], st);
  const int tg = target_grid(dev);
  switch (g->layout * 2 + (t.literal ? 1 : 0)) {
    case 2 * kWide: k_target_walks<false, kWide><<<tg, 256, 0, st>>>(A, X); break;
    case 2 * kWide + 1: k_target_walks<true, kWide><<<tg, 256, 0, st>>>(A, X); break;
    case 2 * kCsr: k_target_walks<false, kCsr><<<tg, 256, 0, st>>>(A, X); break;
    case 2 * kCsr + 1: k_target_walks<true, kCsr><<<tg, 256, 0, st>>>(A, X); break;
    case 2 * kNarrow + 1: k_target_walks<true, kNarrow><<<tg, 256, 0, st>>>(A, X); break;
    default: k_target_walks<false, kNarrow><<<tg, 256, 0, st>>>(A, X); break;
  }
  if (timing) cudaEventRecord(timing[1], st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return SRK_OK;
}

// The target range of a query from its options: [0, n) by default.
int target_range(const srk_graph *g, const srk_opts *opt, int32_t *b, int32_t *e) {
  *b = 0;
  *e = g->n;
  if (opt && (opt->target_begin != 0 || opt->target_end != 0)) {
    if (opt->target_begin < 0 || opt->target_begin > opt->target_end ||
        opt->target_end > g->n)
      return fail(SRK_EINVAL, "target range [%d, %d) outside [0, %d]", opt->target_begin,
                  opt->target_end, g->n);
    *b = opt->target_begin;
    *e = opt->target_end;
  }
  return SRK_OK;
}

// Reads back the counters of the small block into `stats` (synchronous).
int read_stats(const QueryTab &t, const Workspace &w, cudaStream_t st,
               srk_stats *stats, bool accumulate) {
  unsigned long long ctr[2] = {0, 0};
  int32_t active = 0;
  cudaError_t e = cudaMemcpyAsync(ctr, small_view(w.small).ctr, sizeof ctr,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&active, small_view(w.small).cnt + 1, sizeof active,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reading query statistics");
  if (!accumulate) {
    memset(stats, 0, sizeof *stats);
    stats->batch_shape = -1;
  }
  stats->z = t.z;
  stats->L = t.L;
  stats->n_walks = t.N_tot;
  stats->n_active_pairs += active;
  stats->target_steps += ctr[0];
  stats->source_steps += ctr[1];
  return SRK_OK;
}

}  // namespace srk

using namespace srk;

extern "C" int srk_single_source(const srk_graph *g, int32_t s, double c,
                                 double eps, uint64_t seed, const srk_opts *opt,
                                 double *scores, uint32_t *meet_counts,
                                 uint64_t *weight_sums, void *cuda_stream) {
  clear_error();
  if (!g) return fail(SRK_EINVAL, "null graph");
  if (!scores) return fail(SRK_EINVAL, "scores is null");
  if (opt && (opt->flags & ~(SRK_OPT_WARMUP_RULE | SRK_OPT_LITERAL_SHUFFLE |
                             SRK_OPT_SHARED_WALKS)))
    return fail(SRK_EINVAL, "unsupported opts.flags 0x%x", opt->flags);
  QueryTab t;
  int rc = build_table(g->n, s, c, eps, seed, opt, &t);
  if (rc) return rc;
  int32_t u_begin = 0, u_end = g->n;
  rc = target_range(g, opt, &u_begin, &u_end);
  if (rc) return rc;
  DeviceGuard guard(g->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)g->n;
  uint32_t *step_counts = opt ? opt->step_counts : nullptr;
  const bool d_scores = is_device_ptr(scores);
  const bool d_counts = !meet_counts || is_device_ptr(meet_counts);
  const bool d_wsums = !weight_sums || is_device_ptr(weight_sums);
  const bool d_steps = !step_counts || is_device_ptr(step_counts);
  Workspace w;
  size_t ws = plan(t, &w, nullptr);
  const size_t o_scores = ws;
  if (!d_scores) ws += align_up(8 * n);
  const size_t o_counts = ws;
  if (!d_counts) ws += align_up(4 * n);
  const size_t o_wsums = ws;
  if (!d_wsums) ws += align_up(8 * n);
  const size_t o_steps = ws;
  if (!d_steps) ws += align_up(4 * n);
  cudaMemPool_t mp = pool(g->device);
  if (!mp) return fail(SRK_ECUDA, "cannot create the device memory pool");
  char *base = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void **)&base, ws, mp, st);
  if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
  plan(t, &w, base);
  Outputs o;
  o.scores = d_scores ? scores : (double *)(base + o_scores);
  o.counts = d_counts ? meet_counts : (uint32_t *)(base + o_counts);
  o.wsums = d_wsums ? (unsigned long long *)weight_sums
                    : (unsigned long long *)(base + o_wsums);
  o.steps = d_steps ? step_counts : (uint32_t *)(base + o_steps);
  rc = enqueue_query(g, t, w, o, st,
                     opt ? (const cudaEvent_t *)opt->timing_events : nullptr, u_begin, u_end);
  bool host_out = !d_scores || !d_counts || !d_wsums || !d_steps;
  if (!rc) {  // host outputs: copy back the computed range only
    const size_t b = (size_t)u_begin, cnt = (size_t)(u_end - u_begin);
    if (!d_scores)
      e = cudaMemcpyAsync(scores + b, o.scores + b, 8 * cnt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !d_counts)
      e = cudaMemcpyAsync(meet_counts + b, o.counts + b, 4 * cnt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !d_wsums)
      e = cudaMemcpyAsync(weight_sums + b, o.wsums + b, 8 * cnt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !d_steps)
      e = cudaMemcpyAsync(step_counts + b, o.steps + b, 4 * cnt, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "copying results to the host");
  }
  if (!rc && opt && opt->stats) rc = read_stats(t, w, st, opt->stats, false);
  cudaFreeAsync(base, st);
  if (!rc && host_out) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "srk_single_source");
  }
  return rc;
}
