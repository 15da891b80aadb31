// srk_multi_source: many single-source queries with uneven walk budgets.
//
// The sources are processed in batches sized by a memory budget.  Each batch
// runs the source-side steps a2-a3 of all its sources with one launch per
// phase (thread g of a phase finds its source by a binary search over the
// prefix of the sources' walk counts), then one persistent launch walks every
// (source, target) work item: a warp takes items from a global counter in
// source-major order and walks the target's pairs exactly as the
// single-source kernel does (walk_target in srk_device.cuh), so the results
// are identical to srk_single_source.  Sources whose walks never leave the
// source (no pair can meet) are short-circuited: their score rows are
// prefilled (1 at the source, 0 elsewhere) and they contribute no items, and
// neither do targets without in-neighbours.  A batch's launches are captured
// in a CUDA graph and launched as one.  The persistent kernel's launch shape
// (block size x blocks per SM) is chosen per graph by timing the candidates
// on the first items of the first batch (autotuner).  With shared target walks
// (SRK_OPT_SHARED_WALKS) the batches hold up to 64 sources and the target
// walks run once for all of them (kb_shared_walks, below).
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "srk_device.cuh"
#include "srk_internal.h"

namespace srk {

// One source of a batch, as the batched kernels see it (device memory).
struct BatchSrc {
  Workspace w;            // the source's scratch (see plan())
  const QueryTab *tab;    // the source's table (device copy)
  double *scores;         // output row, n entries
  uint32_t *counts;       // output row or null
  unsigned long long *steps;  // target-walk steps of this source (one counter)
  unsigned long long *wj;     // shared walks: quantised Lemma 7 weight of pair j
  int32_t s, L, N_tot;
  double z;
};

struct BatchArgs {
  const BatchSrc *src;
  const int64_t *walk_off;  // prefix of N_tot over the batch, k+1 entries
  int32_t k;
  int64_t total_walks;
  const int32_t *row_ptr;
  const int32_t *col;
  const uint32_t *adj;
  const int32_t *npos;
  int32_t pos_bits;
  uint32_t key0, key1;
  uint32_t shared_key;  // walk key of the shared target walks
  uint4 *M;       // shared walks: M[(i-1) Jmax + j] (.x, .y) bit b = pair j of batch
                  // source b may still meet at step i (cap_b(j) >= i); (.z, .w) = the
                  // 64-bit signature of those sources' nodes at step i (bit
                  // node_hash(node) per node); Lmax + 1 rows
  uint4 *T;       // shared walks: the meeting tables, one per (step i, pair j) with
                  // j >= Pmin_i (below, no pair of the batch reaches step i) at
                  // T + ((rowbase[i] + j) << tbits): 2^tbits slots {node + 1,
                  // (.y, .z) the sources b with cap_b(j) >= i whose walk
                  // sigma_b(j) is at that node at step i}, empty slots 0,
                  // linear probing from slot_of(node)
  const int64_t *rowbase;  // shared walks: rowbase[i] = tables before step i - Pmin_i
  int32_t tbits;  // shared walks: log2 of the slots per table (>= 2 k)
  int32_t Jmax;   // shared walks: the largest N_tot of the batch
  int32_t Lmax;   // shared walks: the largest L of the batch
};

__device__ __forceinline__ int find_source(const int64_t *off, int k, int64_t g) {
  int lo = 0, hi = k - 1;  // last i with off[i] <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

#define SRK_BATCH_LOOP(A, ...)                                                   \
  for (int64_t g_ = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;              \
       g_ < (A).total_walks; g_ += (int64_t)gridDim.x * blockDim.x) {            \
    const int i_ = find_source((A).walk_off, (A).k, g_);                         \
    const BatchSrc &S_ = (A).src[i_];                                            \
    const int32_t r_ = (int32_t)(g_ - (A).walk_off[i_]);                         \
    __VA_ARGS__                                                                  \
  }

// a2: source walks and Fisher-Yates draws of every source of the batch.
template <int kLayout>
__global__ void __launch_bounds__(256) kb_source_walks(const __grid_constant__ BatchArgs A) {
  const RoundKeys rk = round_keys(A.key0, A.key1);
  const auto G = adj_view<kLayout>(A.adj, A.npos, A.pos_bits, A.row_ptr, A.col);
  SRK_BATCH_LOOP(A, {
    const QueryTab &t = *S_.tab;
    const uint32_t s = (uint32_t)S_.s;
    uint32_t deg_s = 0;
    const int32_t b_s = node_start(G, A.row_ptr, S_.s, deg_s);
    const int Ls = S_.L > 0 ? S_.L : 1;
    S_.w.grp_cnt[r_] = 0;
    S_.w.kdraw[r_] = (r_ >= 1) ? fy_draw(rk, s, r_) : 0;
    const int len = stratum_of(t.P, S_.L, r_);
    const int eff = source_walk(t.skey, G, s, b_s, deg_s, r_, len,
                                S_.w.spos + (int64_t)r_ * Ls);
    S_.w.seff[r_] = eff;
    atomicAdd(small_view(S_.w.small).ctr + 1, (unsigned long long)eff);
  })
}

__global__ void kb_fy_rank(const __grid_constant__ BatchArgs A) {
  SRK_BATCH_LOOP(A, {
    if (r_ >= 1) S_.w.rank[r_] = atomicAdd(&S_.w.grp_cnt[S_.w.kdraw[r_]], 1);
  })
}

// Exclusive scan of each source's group counts: block b scans source b.
__global__ void __launch_bounds__(1024) kb_scan(const __grid_constant__ BatchArgs A) {
  __shared__ int32_t warp_sum[32];
  __shared__ int32_t carry;
  const BatchSrc &S = A.src[blockIdx.x];
  const int32_t N = S.N_tot;
  const int32_t *cnt = S.w.grp_cnt;
  int32_t *off = S.w.grp_off;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < N; base += 4096) {
    const int64_t i0 = base + 4 * (int64_t)threadIdx.x;
    int32_t v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (i0 + q < N) ? cnt[i0 + q] : 0;
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
      warp_sum[lane] = ws;
    }
    __syncthreads();
    int32_t run = carry + (wid ? warp_sum[wid - 1] : 0) + incl - local;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (i0 + q < N) off[i0 + q] = run;
      run += v[q];
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = run;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[N] = carry;
}

__global__ void kb_fy_scatter(const __grid_constant__ BatchArgs A) {
  SRK_BATCH_LOOP(A, {
    if (r_ >= 1) S_.w.items[S_.w.grp_off[S_.w.kdraw[r_]] + S_.w.rank[r_]] = r_;
  })
}

__global__ void kb_fy_groups(const __grid_constant__ BatchArgs A) {
  SRK_BATCH_LOOP(A, {
    const int32_t b = S_.w.grp_off[r_], e = S_.w.grp_off[r_ + 1];
    int32_t *items = S_.w.items;
    for (int32_t x = b + 1; x < e; ++x) {  // insertion sort (groups are tiny)
      const int32_t y = items[x];
      int32_t q = x - 1;
      while (q >= b && items[q] > y) { items[q + 1] = items[q]; --q; }
      items[q + 1] = y;
    }
    S_.w.first[r_] = (e > b) ? items[b] : -1;
    for (int32_t x = b; x < e; ++x) S_.w.succ[items[x]] = (x + 1 < e) ? items[x + 1] : -1;
  })
}

__global__ void kb_pairs(const __grid_constant__ BatchArgs A) {
  SRK_BATCH_LOOP(A, {
    const int32_t p = resolve_sigma(r_, S_.w.kdraw, S_.w.first, S_.w.succ, S_.N_tot);
    S_.w.sigma[r_] = p;
    const int32_t cap = min(stratum_of(S_.tab->P, S_.L, r_), S_.w.seff[p]);
    if (cap >= 1) atomicAdd(&small_view(S_.w.small).cap_hist[cap], 1);
  })
}

// Row geometry of every source (one thread per source), as in k_rows, and
// the list of sources with at least one pair.
__global__ void kb_rows(const __grid_constant__ BatchArgs A, int32_t *act_src,
                        int32_t *n_act_src) {
  if (blockIdx.x != 0) return;
  for (int i = threadIdx.x; i < A.k; i += blockDim.x) {
    const Small sm = small_view(A.src[i].w.small);
    const int L = A.src[i].L;
    int32_t c = 0;
    sm.cnt[L + 1] = 0;
    for (int q = L; q >= 1; --q) {
      sm.cursor[q] = c;
      c += sm.cap_hist[q];
      sm.cnt[q] = c;
    }
    int32_t r = 0;
    for (int q = 1; q <= L + 1; ++q) {
      sm.R[q] = r;
      if (q <= L) r += sm.cnt[q];
    }
    sm.cnt[0] = c;
    sm.R[0] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // in source order, so the items stay source-major
    int32_t m = 0;
    for (int i = 0; i < A.k; ++i)
      if (small_view(A.src[i].w.small).cnt[1] > 0) act_src[m++] = i;
    *n_act_src = m;
  }
}

__global__ void kb_hit_table(const __grid_constant__ BatchArgs A) {
  SRK_BATCH_LOOP(A, {
    const int32_t j = r_;
    const int32_t w = S_.w.sigma[j];
    const int l2 = stratum_of(S_.tab->P, S_.L, j);
    const int32_t cap = min(l2, S_.w.seff[w]);
    if (cap >= 1) {
      const Small sm = small_view(S_.w.small);
      const int l1 = stratum_of(S_.tab->P, S_.L, w);
      const int32_t a = atomicAdd(&sm.cursor[cap], 1);
      S_.w.pair_j[a] = j;
      S_.w.pair_w[a] = __double2ull_rn(S_.tab->a[l1] * S_.tab->a[l2] * 4294967296.0);
      const int Ls = S_.L > 0 ? S_.L : 1;
      const int32_t *sp = S_.w.spos + (int64_t)w * Ls;
      for (int q = 1; q <= cap; ++q) S_.w.Hc[sm.R[q] + a] = sp[q - 1];
    }
  })
}

// Every output row: 1 at the source, 0 elsewhere (the rows of items walked
// later are overwritten per target).
__global__ void kb_prefill(const BatchSrc *__restrict__ src, int32_t k, int32_t n) {
  const int64_t total = (int64_t)k * n;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(g / n);
    const int32_t u = (int32_t)(g - (int64_t)i * n);
    src[i].scores[u] = (u == src[i].s) ? 1.0 : 0.0;
    if (src[i].counts) src[i].counts[u] = 0;
  }
}

// a4-a5 for every (active source, target with in-neighbours) item, source-
// major.  Items at or beyond `item_limit` are not walked (autotuner trials).
// Each warp keeps its current source's context in shared memory: the pair
// list pointers and the rows cnt[0..L+2], R[0..L+2] (dynamic shared memory,
// 2 (Lmax + 3) words per warp), so the walk loop holds no per-source state
// in registers.
template <int kBlock, int kMinBlocks, int kLayout>
__global__ void __launch_bounds__(kBlock, kMinBlocks)
kb_target_walks(const __grid_constant__ BatchArgs A, const int32_t *__restrict__ act,
                int32_t n_act, const int32_t *__restrict__ act_src,
                const int32_t *__restrict__ n_act_src_p,
                unsigned long long *__restrict__ item_counter, int64_t item_limit,
                int32_t row_words) {
  extern __shared__ int32_t rows[];
  __shared__ PairSet ctx[kBlock / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const auto G = adj_view<kLayout>(A.adj, A.npos, A.pos_bits, A.row_ptr, A.col);
  int2 *my_rc = reinterpret_cast<int2 *>(rows + (2 * wib) * row_words);
  const int64_t n_items = (int64_t)(*n_act_src_p) * n_act;
  const int64_t limit = item_limit < n_items ? item_limit : n_items;
  int cur = -1;
  unsigned long long acc = 0;  // steps of source `cur` by this warp (lane 0)
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(item_counter, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if ((int64_t)item >= limit) break;
    const int q = (int)((int64_t)item / n_act);
    const int32_t u = act[(int64_t)item - (int64_t)q * n_act];
    const int i = act_src[q];
    if (i != cur) {
      if (lane == 0 && cur >= 0 && acc) atomicAdd(A.src[cur].steps, acc);
      acc = 0;
      cur = i;
      const BatchSrc &B = A.src[i];
      const Small sm = small_view(B.w.small);
      __syncwarp();
      for (int x = lane; x <= B.L + 2; x += 32)
        my_rc[x] = make_int2((x <= B.L + 1) ? sm.R[x] : 0, (x + 1 <= B.L + 1) ? sm.cnt[x + 1] : 0);
      if (lane == 0) {
        PairSet &S = ctx[wib];
        S.rc = my_rc;
        S.pair_j = B.w.pair_j;
        S.pair_w = B.w.pair_w;
        S.Hc = B.w.Hc;
        S.n_pairs = sm.cnt[1];
        S.key = B.tab->tkey;
      }
      __syncwarp();
    }
    if (u == A.src[i].s) continue;  // prefilled with 1
    uint32_t c = 0, st = 0;
    unsigned long long W = 0;
    uint32_t deg_u = 0;
    const int32_t b_u = node_start(G, A.row_ptr, u, deg_u);
    walk_target(G, ctx[wib], (uint32_t)u, b_u, deg_u, c, W, st);
    for (int off = 16; off > 0; off >>= 1) {
      c += __shfl_xor_sync(0xffffffffu, c, off);
      st += __shfl_xor_sync(0xffffffffu, st, off);
      W += __shfl_xor_sync(0xffffffffu, W, off);
    }
    if (lane == 0) {
      const BatchSrc &B = A.src[i];
      B.scores[u] = (double)W * 2.3283064365386963e-10 / B.z;
      if (B.counts) B.counts[u] = c;
      acc += st;
    }
  }
  if (lane == 0 && cur >= 0 && acc) atomicAdd(A.src[cur].steps, acc);
}

// ------------------------------------------------------------------------
// Shared target walks (SRK_OPT_SHARED_WALKS).  Target walk j of u no longer
// depends on the source, so one walk serves pair j of every source of the
// batch: it goes on while some source's pair j can still meet (it has not met
// and its cap is not reached) and stops at a node without in-neighbours.  For
// source b the pair meets at the first step i <= cap_b(j) where the walk is
// at the node of source b's walk sigma_b(j) at step i, exactly as
// srk_single_source with the same flag decides it.  Those nodes of all the
// batch's sources sit in one small hash table per (step, pair), so a walk
// tests every pending source with one lookup of its own node (one sector,
// rarely two).  Batches hold at most 64 sources (one mask bit each).

// One of 64 bits for a node: the signature of a (step, pair) has the bits of
// the pending sources' nodes there, so a walk whose node's bit is clear
// meets no source there.
__device__ __forceinline__ uint32_t node_hash(int32_t x) {
  return ((uint32_t)x * 0x9E3779B9u) >> 26;
}
// Is the bit of node x set in the signature (sig.x: bits 0-31, sig.y: 32-63)?
__device__ __forceinline__ bool sig_has(uint2 sig, int32_t x) {
  const uint32_t h = node_hash(x);
  return ((h < 32 ? sig.x : sig.y) >> (h & 31)) & 1u;
}
// The first slot of node x in a meeting table of 2^tbits slots.
__device__ __forceinline__ uint32_t slot_of(int32_t x, int tbits) {
  return ((uint32_t)x * 0x85EBCA6Bu) >> (32 - tbits);
}

// Per source and pair j: the pair's weight, its bit in the step masks, its
// node's bit in the step signatures and its bit in the meeting tables of
// steps 1..cap(j) (source walk sigma(j)).  A table holds at most k nodes in
// 2^tbits >= 2k slots, so an insertion always finds its node or a free slot.
__global__ void kb_hitj(const __grid_constant__ BatchArgs A) {
  SRK_BATCH_LOOP(A, {
    const int32_t j = r_;
    const int32_t w = S_.w.sigma[j];
    const int l2 = stratum_of(S_.tab->P, S_.L, j);
    const int32_t cap = min(l2, S_.w.seff[w]);
    const int l1 = stratum_of(S_.tab->P, S_.L, w);
    S_.wj[j] = cap >= 1 ? __double2ull_rn(S_.tab->a[l1] * S_.tab->a[l2] * 4294967296.0) : 0ull;
    const int Ls = S_.L > 0 ? S_.L : 1;
    const int32_t *sp = S_.w.spos + (int64_t)w * Ls;
    const uint32_t bit = 1u << (i_ & 31);  // in word .x (sources 0-31) or .y (32-63)
    const bool high = i_ >= 32;
    const uint32_t smask = (1u << A.tbits) - 1u;
    for (int q = 1; q <= cap; ++q) {
      const int32_t node = sp[q - 1];
      uint4 *cell = &A.M[(int64_t)(q - 1) * A.Jmax + j];
      const uint32_t h = node_hash(node);
      atomicOr(high ? &cell->y : &cell->x, bit);
      atomicOr(h < 32 ? &cell->z : &cell->w, 1u << (h & 31));
      uint4 *tab = A.T + ((A.rowbase[q] + j) << A.tbits);
      const uint32_t key = (uint32_t)node + 1u;
      uint32_t sl = slot_of(node, A.tbits);
      for (uint32_t probe = 0; probe <= smask; ++probe, sl = (sl + 1u) & smask) {
        const uint32_t prev = atomicCAS(&tab[sl].x, 0u, key);
        if (prev == 0u || prev == key) {
          atomicOr(high ? &tab[sl].z : &tab[sl].y, bit);
          break;
        }
      }
    }
  })
}

// The batch's sources as the shared-walk kernel reads them (shared memory).
struct ShSrc {
  const unsigned long long *wj;
  double *scores;
  uint32_t *counts;
  double z;
  int32_t N, s;
};

// The meeting test after a step: a stepping lane whose node x has its bit
// in the step's signature looks x up in the step's meeting table (tab); the
// pending sources among the slot's are those that meet here.  Their counts
// and weight sums go to the warp's shared words cnt[b], wsum[b] (atomics:
// lanes of a warp can meet the same source at once).  Returns them.
__device__ __forceinline__ unsigned long long shared_meet(
    const ShSrc *src, const uint4 *tab, int tbits, bool stepped, int32_t x,
    unsigned long long pend, uint2 sig, int32_t j, uint32_t *cnt, unsigned long long *wsum) {
  unsigned long long hits = 0ull;
  if (stepped && pend != 0ull && sig_has(sig, x)) {
    const uint32_t smask = (1u << tbits) - 1u, key = (uint32_t)x + 1u;
    uint32_t sl = slot_of(x, tbits);
    for (uint32_t probe = 0; probe <= smask; ++probe, sl = (sl + 1u) & smask) {
      const uint4 e = tab[sl];
      if (e.x == key) {
        hits = (((unsigned long long)e.z << 32) | e.y) & pend;
        break;
      }
      if (e.x == 0u) break;
    }
    for (unsigned long long m = hits; m; m &= m - 1) {
      const int b = __ffsll((long long)m) - 1;
      atomicAdd(&cnt[b], 1u);
      atomicAdd(&wsum[b], src[b].wj[j]);
    }
  }
  return hits;
}

// a4+a5 of a batch with shared target walks: warps take targets (the nodes
// with in-neighbours) from a counter; the 32 lanes walk the target's pairs
// j = j0, j0 + 1, ... with lane refill, one Philox2x32-10 block (counter
// (((i-1)>>1) << 24 | j, u) under the shared walk key) per odd and following
// even step; after
// every step the stepping lanes' nodes are tested against their pending
// sources (shared_meet), and lane b writes source b's count, weight sum and
// score at the end of the target.  A source's own row
// keeps its prefilled 1.
// 6 blocks of 256 threads per SM (40 registers): at 8 (32 registers) every
// form spilled.
template <int kLayout>
__global__ void __launch_bounds__(256, 6)
kb_shared_walks(const __grid_constant__ BatchArgs A, const int32_t *__restrict__ act,
                int32_t n_act, int32_t j0, unsigned long long *__restrict__ ctr) {
  __shared__ ShSrc src[64];
  __shared__ uint32_t cnt[8][64];
  __shared__ unsigned long long wsum[8][64];
  // per warp: the sources whose own row the target is, and the target's list
  // (read at refills only, so they hold no registers across the walk)
  __shared__ unsigned long long w_excl[8];
  __shared__ uint32_t w_deg[8];
  __shared__ int32_t w_base[8];
  __shared__ long long rowbase[SRK_MAX_LEN + 2];  // meeting-table rows (A.rowbase)
  for (int i = threadIdx.x; i <= SRK_MAX_LEN + 1; i += blockDim.x)
    rowbase[i] = (i <= A.Lmax) ? A.rowbase[i] : 0;
  for (int b = threadIdx.x; b < A.k; b += blockDim.x) {
    const BatchSrc &B = A.src[b];
    src[b] = ShSrc{B.wj, B.scores, B.counts, B.z, B.N_tot, B.s};
  }
  __syncthreads();
  const uint32_t key = A.shared_key;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const auto G = adj_view<kLayout>(A.adj, A.npos, A.pos_bits, A.row_ptr, A.col);
  const uint4 *M = A.M;
  const int32_t J = A.Jmax;
  const int tbits = A.tbits;
  unsigned long long warp_steps = 0;
  for (;;) {
    int32_t q = 0;
    if (lane == 0) q = (int32_t)atomicAdd(ctr, 1ull);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= n_act) break;
    const uint32_t u = (uint32_t)act[q];
    // sources whose own row this target is
    const unsigned long long excl =
        __ballot_sync(0xffffffffu, lane < A.k && src[lane].s == (int32_t)u) |
        ((unsigned long long)__ballot_sync(0xffffffffu, lane + 32 < A.k &&
                                                       src[lane + 32].s == (int32_t)u)
         << 32);
    cnt[wib][lane] = 0u;            // meetings of sources `lane`, `lane` + 32 at this target
    cnt[wib][lane + 32] = 0u;
    wsum[wib][lane] = 0ull;         // and their weight sums
    wsum[wib][lane + 32] = 0ull;
    if (lane == 0) {
      uint32_t deg_u = 0;
      w_base[wib] = node_start(G, A.row_ptr, (int32_t)u, deg_u);
      w_deg[wib] = deg_u;
      w_excl[wib] = excl;
    }
    __syncwarp();
    uint32_t st = 0;
    int32_t next = j0, j = 0, i = 1, b = 0;
    bool live = false;
    uint32_t deg = 0;
    unsigned long long pend = 0ull;
    uint2 sg = make_uint2(0u, 0u);  // the signature of the next test
    // pend &= the mask of row `row`; sg = its signature
    auto next_mask = [&](int64_t row) {
      const uint4 mn = M[row];
      pend &= ((unsigned long long)mn.y << 32) | mn.x;
      sg = make_uint2(mn.z, mn.w);
    };
    for (;;) {
      const uint32_t idle = __ballot_sync(0xffffffffu, !live);
      if (idle) {
        if (!live) {
          j = next + __popc(idle & lanes_below_mask());
          if (j < J) {
            const uint4 m1 = M[j];
            pend = (((unsigned long long)m1.y << 32) | m1.x) & ~w_excl[wib];
            sg = make_uint2(m1.z, m1.w);
            live = pend != 0ull;
            i = 1;
            b = w_base[wib];
            deg = w_deg[wib];
          }
        }
        next += __popc(idle);
      }
      if (!__any_sync(0xffffffffu, live)) {
        if (next >= J) break;
        continue;  // every pair of this round was dead: take the next ones
      }
      uint32_t x0 = 0, x1 = 0;
      int32_t x = 0;
      decltype(adj_entry(G, 0, 0u)) e{};
      // odd step i
      bool stepped = live;
      if (stepped) {
        philox2(key, walk_ctr0(i, (uint32_t)j), u, x0, x1);
        e = step_entry(G, b, x0, deg, key, i, (uint32_t)j, u);
        x = entry_pos(G, e);
        ++st;
      }
      pend &= ~shared_meet(src, A.T + ((rowbase[i] + j) << tbits), tbits, stepped, x, pend,
                           sg, j, cnt[wib], wsum[wib]);
      if (stepped) {
        next_mask((int64_t)i * J + j);  // still able to meet at step i + 1
        if (!pend) {
          live = false;
        } else {
          b = entry_next(G, e, x, deg);
          if (deg == 0) live = false;
        }
      }
      // even step i + 1
      stepped = live;
      if (stepped) {
        e = step_entry(G, b, x1, deg, key, i + 1, (uint32_t)j, u);
        x = entry_pos(G, e);
        ++st;
      }
      pend &= ~shared_meet(src, A.T + ((rowbase[i + 1] + j) << tbits), tbits, stepped, x,
                           pend, sg, j, cnt[wib], wsum[wib]);
      if (stepped) {
        next_mask((int64_t)(i + 1) * J + j);
        if (!pend) {
          live = false;
        } else {
          b = entry_next(G, e, x, deg);
          if (deg == 0) live = false;
          i += 2;
        }
      }
    }
    for (int off = 16; off > 0; off >>= 1) st += __shfl_xor_sync(0xffffffffu, st, off);
    warp_steps += st;
    __syncwarp();
    for (int bb = lane; bb < A.k; bb += 32) {
      if ((w_excl[wib] >> bb) & 1ull) continue;
      const ShSrc &S = src[bb];
      const unsigned long long W = wsum[wib][bb];
      S.scores[u] = (double)W * 2.3283064365386963e-10 / S.z;
      if (S.counts) S.counts[u] = cnt[wib][bb];
    }
    __syncwarp();
  }
  if (lane == 0 && warp_steps) atomicAdd(ctr + 1, warp_steps);
}

// The candidate launch shapes of the autotuner (block size, blocks per SM).
struct Shape {
  int block, per_sm;
};
static const Shape kShapes[] = {{256, 8}, {512, 4}, {128, 16}, {1024, 2}, {256, 6}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <int kLayout>
static void launch_targets_t(int shape, int grid, int block, size_t smem, cudaStream_t st,
                             const BatchArgs &A, const int32_t *act, int32_t n_act,
                             const int32_t *act_src, const int32_t *n_act_src,
                             unsigned long long *ctr, int64_t limit, int32_t rw) {
#define SRK_KB_LAUNCH(B, M)                                                                  \
  kb_target_walks<B, M, kLayout><<<grid, block, smem, st>>>(A, act, n_act, act_src, n_act_src, \
                                                            ctr, limit, rw)
  switch (shape) {
    case 0: SRK_KB_LAUNCH(256, 8); break;
    case 1: SRK_KB_LAUNCH(512, 4); break;
    case 2: SRK_KB_LAUNCH(128, 16); break;
    case 3: SRK_KB_LAUNCH(1024, 2); break;
    default: SRK_KB_LAUNCH(256, 6); break;
  }
#undef SRK_KB_LAUNCH
}

// Shared memory of the target kernel in launch shape `shape`: two rows of
// Lmax + 3 words per warp.
static size_t target_smem(int shape, int Lmax) {
  return sizeof(int32_t) * 2 * (size_t)(Lmax + 3) * (size_t)(kShapes[shape].block / 32);
}

// Lets every launch shape of layout kLayout take `bytes` of dynamic shared
// memory (above the default 48 KB a kernel must opt in).  Not a stream
// operation, so it runs before any capture.
template <int kLayout>
static cudaError_t allow_smem_t(size_t bytes) {
  const int b = (int)bytes;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  };
  set((const void *)kb_target_walks<256, 8, kLayout>);
  set((const void *)kb_target_walks<512, 4, kLayout>);
  set((const void *)kb_target_walks<128, 16, kLayout>);
  set((const void *)kb_target_walks<1024, 2, kLayout>);
  set((const void *)kb_target_walks<256, 6, kLayout>);
  return e;
}

static cudaError_t allow_smem(int layout, int Lmax) {
  size_t most = 0;
  for (int sh = 0; sh < kNumShapes; ++sh) most = std::max(most, target_smem(sh, Lmax));
  if (most <= 48 * 1024) return cudaSuccess;
  return layout == kWide ? allow_smem_t<kWide>(most)
         : layout == kCsr ? allow_smem_t<kCsr>(most)
                          : allow_smem_t<kNarrow>(most);
}

static void launch_targets(int layout, int shape, int sms, cudaStream_t st, const BatchArgs &A,
                           const int32_t *act, int32_t n_act, const int32_t *act_src,
                           const int32_t *n_act_src, unsigned long long *ctr,
                           int64_t limit, int Lmax) {
  const Shape sh = kShapes[shape];
  const int grid = sms * sh.per_sm;
  const int32_t rw = Lmax + 3;
  const size_t smem = target_smem(shape, Lmax);
  if (layout == kWide)
    launch_targets_t<kWide>(shape, grid, sh.block, smem, st, A, act, n_act, act_src,
                            n_act_src, ctr, limit, rw);
  else if (layout == kCsr)
    launch_targets_t<kCsr>(shape, grid, sh.block, smem, st, A, act, n_act, act_src, n_act_src,
                           ctr, limit, rw);
  else
    launch_targets_t<kNarrow>(shape, grid, sh.block, smem, st, A, act, n_act, act_src,
                              n_act_src, ctr, limit, rw);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The shared-walk kernel: a persistent grid of as many 256-thread blocks as
// fit at once (ctr[0]: the target counter, cleared here; ctr[1]: the steps).
// The first walk index of source table t whose length is at least i (walks
// are in stratum order): pairs below it cannot reach step i.
static int32_t first_reaching(const QueryTab &t, int i) {
  return i <= t.L ? t.P[i] : t.N_tot;
}

static void launch_shared(int layout, cudaStream_t st, const BatchArgs &A,
                          const int32_t *act, int32_t n_act, int32_t j0,
                          unsigned long long *ctr, int dev) {
  static int per_sm[3][64] = {};
  auto grid = [&](const void *f, int l) {
    int b = (dev >= 0 && dev < 64) ? per_sm[l][dev] : 0;
    if (!b) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, 256, 0) != cudaSuccess || b < 1)
        b = 1;
      if (dev >= 0 && dev < 64) per_sm[l][dev] = b;
    }
    return sm_count(dev) * b;
  };
#define SRK_SH_LAUNCH(L)                                                         \
  kb_shared_walks<L><<<grid((const void *)kb_shared_walks<L>, L), 256, 0, st>>>( \
      A, act, n_act, j0, ctr)
  cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), st);
  if (layout == kWide) SRK_SH_LAUNCH(kWide);
  else if (layout == kCsr) SRK_SH_LAUNCH(kCsr);
  else SRK_SH_LAUNCH(kNarrow);
#undef SRK_SH_LAUNCH
}

static std::mutex g_stream_mu;
static cudaStream_t g_cap_stream[64] = {};

// One lock per device around a batch's capture and graph launch: the capture
// stream and the handles' cached executables are shared.
static std::mutex g_capture_mu[64];
static std::mutex &capture_mutex(int dev) { return g_capture_mu[dev >= 0 && dev < 64 ? dev : 0]; }

// A library-owned non-blocking stream per device for graph capture (the
// caller's stream may be the legacy default stream, which cannot capture).
static cudaStream_t capture_stream(int dev) {
  std::lock_guard<std::mutex> lk(g_stream_mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!g_cap_stream[dev]) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    g_cap_stream[dev] = s;
  }
  return g_cap_stream[dev];
}

}  // namespace srk

using namespace srk;

namespace srk {

__global__ void k_source_degrees(const int32_t *__restrict__ row_ptr,
                                 int32_t *__restrict__ v, int32_t k) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) v[i] = row_ptr[v[i] + 1] - row_ptr[v[i]];
}

int source_in_degrees(const srk_graph *g, const int32_t *sources, int32_t k, cudaStream_t st,
                      std::vector<int32_t> *deg) {
  deg->assign((size_t)k, 0);
  if (k <= 0) return SRK_OK;
  cudaMemPool_t mp = pool(g->device);
  if (!mp) return fail(SRK_ECUDA, "cannot create the device memory pool");
  int32_t *d = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void **)&d, sizeof(int32_t) * (size_t)k, mp, st);
  if (e != cudaSuccess) return cuda_fail(e, "source degrees: allocation");
  e = cudaMemcpyAsync(d, sources, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_source_degrees<<<(k + 255) / 256, 256, 0, st>>>(g->row_ptr, d, k);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(deg->data(), d, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SRK_OK : cuda_fail(e, "source degrees");
}

}  // namespace srk

extern "C" int srk_multi_source(const srk_graph *g, const int32_t *sources,
                                int32_t k, double c, const double *eps,
                                uint64_t seed, const srk_opts *opt,
                                double *scores, uint32_t *meet_counts,
                                void *cuda_stream) {
  clear_error();
  if (!g) return fail(SRK_EINVAL, "null graph");
  if (k < 0) return fail(SRK_EINVAL, "k = %d is negative", k);
  if (k == 0) return SRK_OK;
  if (!sources || !eps || !scores) return fail(SRK_EINVAL, "null argument");
  if (opt && opt->step_counts)
    return fail(SRK_EINVAL, "step_counts is not supported by srk_multi_source");
  if (opt && (opt->flags & SRK_OPT_LITERAL_SHUFFLE))
    return fail(SRK_EINVAL, "the literal shuffle is not supported by srk_multi_source");
  if (opt && (opt->flags & ~(SRK_OPT_NO_GRAPH | SRK_OPT_WARMUP_RULE | SRK_OPT_SHARED_WALKS)))
    return fail(SRK_EINVAL, "unknown opts.flags 0x%x", opt->flags);
  if (opt && (opt->target_begin != 0 || opt->target_end != 0))
    return fail(SRK_EINVAL, "target ranges are not supported by srk_multi_source");
  const bool use_graph = !(opt && (opt->flags & SRK_OPT_NO_GRAPH));
  const bool shared = opt && (opt->flags & SRK_OPT_SHARED_WALKS);
  const size_t n = (size_t)g->n;
  // a1 for every source (host, FP64)
  std::vector<QueryTab> tabs((size_t)k);
  for (int32_t i = 0; i < k; ++i) {
    int rc = build_table(g->n, sources[i], c, eps[i], seed, opt, &tabs[i]);
    if (rc) return fail(rc, "source %d (index %d): %s", sources[i], i, srk_last_error());
  }
  // batch position -> the caller's row.  With shared target walks the
  // sources are grouped by walk budget (N_tot, then L), so that a batch's
  // sources share as many pairs as possible; a source's results do not
  // depend on its batch, since its target walks do not depend on it.
  std::vector<int32_t> row_of((size_t)k);
  for (int32_t i = 0; i < k; ++i) row_of[(size_t)i] = i;
  DeviceGuard guard(g->device);
  if (shared) {
    // sources without in-neighbours go last: their pairs meet nowhere, so they
    // would hold places in batches that share walks
    std::vector<int32_t> deg;
    const int rcd = source_in_degrees(g, sources, k, (cudaStream_t)cuda_stream, &deg);
    if (rcd) return rcd;
    std::stable_sort(row_of.begin(), row_of.end(), [&](int32_t a, int32_t b) {
      const QueryTab &ta = tabs[(size_t)a], &tb = tabs[(size_t)b];
      const bool za = deg[(size_t)a] == 0, zb = deg[(size_t)b] == 0;
      if (za != zb) return zb;
      return ta.N_tot != tb.N_tot ? ta.N_tot < tb.N_tot : ta.L < tb.L;
    });
    std::vector<QueryTab> sorted((size_t)k);
    for (int32_t p = 0; p < k; ++p) sorted[(size_t)p] = tabs[(size_t)row_of[(size_t)p]];
    tabs.swap(sorted);
  }
  const int dev = g->device;
  const int sms = sm_count(dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool d_scores = is_device_ptr(scores);
  const bool d_counts = !meet_counts || is_device_ptr(meet_counts);
  cudaMemPool_t mp = pool(dev);
  if (!mp) return fail(SRK_ECUDA, "cannot create the device memory pool");
  cudaStream_t cs = use_graph ? capture_stream(dev) : st;
  if (use_graph && !cs) return fail(SRK_ECUDA, "cannot create the capture stream");

  // batch shape: as many sources as fit a scratch budget
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  size_t budget = std::max<size_t>((size_t)256 << 20,
                                   std::min<size_t>((size_t)8 << 30, free_b / 4));
  if (const char *env = getenv("SRK_BATCH_BYTES")) {  // explicit scratch budget
    const unsigned long long v = strtoull(env, nullptr, 10);
    if (v > 0) budget = (size_t)v;
  }
  srk_stats total;
  memset(&total, 0, sizeof total);
  int32_t i0 = 0;
  int rc = SRK_OK;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  if (use_graph) {
    cudaError_t e = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      if (ev_in) cudaEventDestroy(ev_in);
      return cuda_fail(e, "srk_multi_source: creating the graph-launch events");
    }
  }
  while (i0 < k && rc == SRK_OK) {
    // sources [i0, i1) form this batch
    size_t need = 0;
    int32_t i1 = i0;
    std::vector<size_t> ws_off;
    int64_t sh_L = 1, sh_N = 0;  // shared walks: the tables' extent so far
    std::vector<int32_t> pmin((size_t)SRK_MAX_LEN + 2, INT32_MAX);
    while (i1 < k && !(shared && i1 - i0 >= 64)) {
      // shared walks: the batch's mask rows and meeting tables with this source
      int64_t L1 = sh_L, N1 = sh_N;
      size_t sb = 0;
      if (shared) {
        const QueryTab &t = tabs[(size_t)i1];
        L1 = std::max<int64_t>(sh_L, std::max(t.L, 1));
        N1 = std::max<int64_t>(sh_N, t.N_tot);
        int tb = 1;
        while ((1 << tb) < 2 * (i1 - i0 + 1)) ++tb;
        size_t tables = 0;
        for (int i = 1; i <= L1; ++i)
          tables += (size_t)(N1 - std::min<int64_t>(pmin[(size_t)i], first_reaching(t, i)));
        sb = 16 * (size_t)(L1 + 1) * (size_t)N1 + ((16 * tables) << tb);
      }
      Workspace w;
      const QueryTab &t1 = tabs[(size_t)i1];
      const size_t b = align256(plan(t1, &w, nullptr)) +
                       (d_scores ? 0 : align256(8 * n)) + (d_counts ? 0 : align256(4 * n)) +
                       (shared ? align256(8 * (size_t)t1.N_tot) : 0);
      if (i1 > i0 && need + b + sb > budget) break;
      sh_L = L1;
      sh_N = N1;
      if (shared)
        for (int i = 1; i <= SRK_MAX_LEN; ++i)
          pmin[(size_t)i] = std::min(pmin[(size_t)i], first_reaching(tabs[(size_t)i1], i));
      ws_off.push_back(need);
      need += b;
      ++i1;
    }
    const int32_t kb = i1 - i0;
    int Lmax = 0;
    int32_t Jmax = 0, j0 = INT32_MAX;
    for (int32_t b = i0; b < i1; ++b) {
      const QueryTab &t = tabs[(size_t)b];
      Lmax = std::max(Lmax, t.L);
      Jmax = std::max(Jmax, t.N_tot);
      j0 = std::min(j0, t.L >= 1 ? t.P[1] : t.N_tot);  // below, every pair has length 0
    }
    // shared walks: meeting tables of 2^tbits >= 2 kb slots, one per (step i,
    // pair j >= pmin[i]), in rows by step: rowbase[i] + j is the table's index
    int tbits = 1;
    while ((1 << tbits) < 2 * kb) ++tbits;
    std::vector<int64_t> rowbase((size_t)std::max(Lmax, 1) + 1, 0);
    int64_t n_tables = 0;
    for (int i = 1; i <= std::max(Lmax, 1); ++i) {
      const int64_t pm = std::min<int64_t>(pmin[(size_t)i], Jmax);
      rowbase[(size_t)i] = n_tables - pm;
      n_tables += Jmax - pm;
    }
    // shared walks: the step masks and signatures, Lmax + 1 rows of Jmax
    // 16-byte cells, the table rows and the tables
    const size_t m_bytes = shared ? 16 * (size_t)(Lmax + 1) * (size_t)Jmax : 0;
    const size_t r_bytes = shared ? sizeof(int64_t) * rowbase.size() : 0;
    const size_t h_bytes = shared ? (16 * (size_t)n_tables) << tbits : 0;
    const size_t head = align256(sizeof(BatchSrc) * kb) + align256(sizeof(QueryTab) * kb) +
                        align256(sizeof(int64_t) * (kb + 1)) +
                        align256(sizeof(int32_t) * (kb + 1)) +
                        align256(sizeof(unsigned long long) * (kb + 2)) + align256(m_bytes) +
                        align256(r_bytes) + align256(h_bytes);
    char *base = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&base, head + need, mp, st);
    if (e != cudaSuccess) { rc = cuda_fail(e, "batch workspace allocation"); break; }
    BatchSrc *d_src = (BatchSrc *)base;
    QueryTab *d_tab = (QueryTab *)(base + align256(sizeof(BatchSrc) * kb));
    int64_t *d_off = (int64_t *)((char *)d_tab + align256(sizeof(QueryTab) * kb));
    int32_t *d_act_src = (int32_t *)((char *)d_off + align256(sizeof(int64_t) * (kb + 1)));
    unsigned long long *d_ctr = (unsigned long long *)((char *)d_act_src +
                                                         align256(sizeof(int32_t) * (kb + 1)));
    uint4 *d_M = (uint4 *)((char *)d_ctr + align256(sizeof(unsigned long long) * (kb + 2)));
    int64_t *d_rowbase = (int64_t *)((char *)d_M + align256(m_bytes));
    uint4 *d_T = (uint4 *)((char *)d_rowbase + align256(r_bytes));
    // d_ctr[0] = item counter, d_ctr[1 + i] = steps of source i; n_act_src in d_act_src[kb]
    char *ws_base = base + head;
    std::vector<BatchSrc> hsrc((size_t)kb);
    std::vector<int64_t> hoff((size_t)kb + 1);
    hoff[0] = 0;
    for (int32_t b = 0; b < kb; ++b) {
      const QueryTab &t = tabs[(size_t)(i0 + b)];
      BatchSrc &S = hsrc[(size_t)b];
      char *wb = ws_base + ws_off[(size_t)b];
      const size_t core = align256(plan(t, &S.w, wb));
      char *extra = wb + core;
      S.tab = d_tab + b;
      const size_t row = (size_t)row_of[(size_t)(i0 + b)];
      S.scores = d_scores ? scores + row * n : (double *)extra;
      if (!d_scores) extra += align256(8 * n);
      S.counts = !meet_counts ? nullptr
                 : (d_counts ? meet_counts + row * n : (uint32_t *)extra);
      if (meet_counts && !d_counts) extra += align256(4 * n);
      S.wj = nullptr;
      if (shared) {
        S.wj = (unsigned long long *)extra;
        extra += align256(8 * (size_t)t.N_tot);
      }
      S.steps = d_ctr + 1 + b;
      S.s = t.s;
      S.L = t.L;
      S.N_tot = t.N_tot;
      S.z = t.z;
      hoff[(size_t)b + 1] = hoff[(size_t)b] + t.N_tot;
    }
    // tables and source descriptors (synchronous staging of pageable memory)
    if ((e = cudaMemcpyAsync(d_tab, tabs.data() + i0, sizeof(QueryTab) * kb,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_src, hsrc.data(), sizeof(BatchSrc) * kb,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_off, hoff.data(), sizeof(int64_t) * (kb + 1),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (shared && (e = cudaMemcpyAsync(d_rowbase, rowbase.data(), r_bytes,
                                        cudaMemcpyHostToDevice, st)) != cudaSuccess)) {
      rc = cuda_fail(e, "batch descriptors");
      cudaFreeAsync(base, st);
      break;
    }
    BatchArgs A;
    A.src = d_src;
    A.walk_off = d_off;
    A.k = kb;
    A.total_walks = hoff[(size_t)kb];
    A.row_ptr = g->row_ptr;
    A.col = g->col;
    A.adj = g->adj;
    A.npos = g->npos;
    A.pos_bits = g->pos_bits;
    A.key0 = (uint32_t)seed;
    A.key1 = (uint32_t)(seed >> 32);
    A.shared_key = walk_key(seed, kSharedWalkKey);
    A.M = d_M;
    A.T = d_T;
    A.rowbase = d_rowbase;
    A.tbits = tbits;
    A.Lmax = Lmax;
    A.Jmax = Jmax;
    const int gw = (int)std::max<int64_t>(1, std::min<int64_t>((A.total_walks + 255) / 256,
                                                                (int64_t)sms * 8));
    auto enqueue_source_side = [&](cudaStream_t s2) {
      for (int32_t b = 0; b < kb; ++b)
        cudaMemsetAsync(hsrc[(size_t)b].w.small, 0, kSmallBytes, s2);
      cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long) * (kb + 1), s2);
      if (g->layout == kWide)
        kb_source_walks<kWide><<<gw, 256, 0, s2>>>(A);
      else if (g->layout == kCsr)
        kb_source_walks<kCsr><<<gw, 256, 0, s2>>>(A);
      else
        kb_source_walks<kNarrow><<<gw, 256, 0, s2>>>(A);
      kb_fy_rank<<<gw, 256, 0, s2>>>(A);
      kb_scan<<<kb, 1024, 0, s2>>>(A);
      kb_fy_scatter<<<gw, 256, 0, s2>>>(A);
      kb_fy_groups<<<gw, 256, 0, s2>>>(A);
      kb_pairs<<<gw, 256, 0, s2>>>(A);
      if (shared) {
        cudaMemsetAsync(d_M, 0, m_bytes, s2);
        cudaMemsetAsync(d_T, 0, h_bytes, s2);
        kb_hitj<<<gw, 256, 0, s2>>>(A);
      } else {
        kb_rows<<<1, 256, 0, s2>>>(A, d_act_src, d_act_src + kb);
        kb_hit_table<<<gw, 256, 0, s2>>>(A);
      }
      const int gp = (int)std::min<int64_t>(((int64_t)kb * (int64_t)n + 255) / 256,
                                            (int64_t)sms * 16);
      kb_prefill<<<gp, 256, 0, s2>>>(d_src, kb, (int32_t)n);
    };
    if ((e = allow_smem(g->layout, Lmax)) != cudaSuccess) {
      rc = cuda_fail(e, "batched query: shared memory of the target kernel");
      cudaFreeAsync(base, st);
      break;
    }
    // autotune the persistent kernel's launch shape on the first batch
    int shape = g->batch_cfg;
    if (!shared && (shape < 0 || shape >= kNumShapes)) {
      enqueue_source_side(st);
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      e = cudaEventCreate(&t0);
      if (e == cudaSuccess) e = cudaEventCreate(&t1);
      if (e != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        rc = cuda_fail(e, "batched query: creating the autotuner's events");
        cudaFreeAsync(base, st);
        break;
      }
      const int64_t trial = (int64_t)sms * 64 * 3;  // about three items per warp
      float best = 1e30f;
      shape = 0;
      for (int sh = 0; sh < kNumShapes; ++sh) {
        cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long), st);
        cudaEventRecord(t0, st);
        launch_targets(g->layout, sh, sms, st, A, g->act, g->n_act, d_act_src, d_act_src + kb,
                       d_ctr, trial, Lmax);
        const bool launched = cudaGetLastError() == cudaSuccess;  // a shape that cannot run
        cudaEventRecord(t1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(t1) == cudaSuccess && launched &&
            cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && ms < best) {
          best = ms;
          shape = sh;
        }
      }
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      const_cast<srk_graph *>(g)->batch_cfg = shape;
    }
    auto enqueue_all = [&](cudaStream_t s2) {
      enqueue_source_side(s2);
      if (shared)
        launch_shared(g->layout, s2, A, g->act, g->n_act, j0, d_ctr, dev);
      else
        launch_targets(g->layout, shape, sms, s2, A, g->act, g->n_act, d_act_src, d_act_src + kb,
                       d_ctr, INT64_MAX, Lmax);
    };
    if (use_graph) {
      // The batch is captured every time (its buffers move), but the graph's
      // executable is kept in the handle and only updated with the new
      // parameters while the launch sequence keeps its shape (same kernels,
      // same order); otherwise it is instantiated anew.
      std::lock_guard<std::mutex> lk(capture_mutex(dev));
      srk_graph *gm = const_cast<srk_graph *>(g);
      cudaGraph_t graph = nullptr;
      e = cudaEventRecord(ev_in, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in, 0);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        enqueue_all(cs);
        e = cudaStreamEndCapture(cs, &graph);
      }
      if (e == cudaSuccess && gm->batch_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(gm->batch_exec, graph, &info) != cudaSuccess) {
          cudaGetLastError();  // a different shape: instantiate below
          cudaGraphExecDestroy(gm->batch_exec);
          gm->batch_exec = nullptr;
        } else {
          ++total.graph_updates;
        }
      }
      if (e == cudaSuccess && !gm->batch_exec) e = cudaGraphInstantiate(&gm->batch_exec, graph, 0);
      if (e == cudaSuccess) e = cudaGraphLaunch(gm->batch_exec, cs);
      if (e == cudaSuccess) e = cudaEventRecord(ev_out, cs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_out, 0);
      if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
      if (graph) cudaGraphDestroy(graph);
    } else {
      enqueue_all(st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "batched query launch");
      cudaFreeAsync(base, st);
      break;
    }
    // results of host callers
    for (int32_t b = 0; b < kb && e == cudaSuccess; ++b) {
      const BatchSrc &S = hsrc[(size_t)b];
      if (!d_scores)
        e = cudaMemcpyAsync(scores + (size_t)row_of[(size_t)(i0 + b)] * n, S.scores, 8 * n,
                            cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && meet_counts && !d_counts)
        e = cudaMemcpyAsync(meet_counts + (size_t)row_of[(size_t)(i0 + b)] * n, S.counts, 4 * n,
                            cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess && opt && opt->stats) {
      std::vector<unsigned long long> steps((size_t)kb + 1);
      e = cudaMemcpyAsync(steps.data(), d_ctr, sizeof(unsigned long long) * (kb + 1),
                          cudaMemcpyDeviceToHost, st);
      for (int32_t b = 0; b < kb && e == cudaSuccess; ++b) {
        unsigned long long sc[2];
        int32_t act = 0;
        const Small sm = small_view(hsrc[(size_t)b].w.small);
        e = cudaMemcpyAsync(sc, sm.ctr, sizeof sc, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(&act, sm.cnt + 1, sizeof act, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        total.source_steps += sc[1];
        total.n_active_pairs += act;
        total.n_walks += tabs[(size_t)(i0 + b)].N_tot;
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      for (int32_t b = 0; b < kb; ++b) total.target_steps += steps[(size_t)b + 1];
      total.z = tabs[(size_t)(i1 - 1)].z;
      total.L = tabs[(size_t)(i1 - 1)].L;
    }
    cudaFreeAsync(base, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "batched query results");
    i0 = i1;
  }
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (rc == SRK_OK && (!d_scores || !d_counts)) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "srk_multi_source");
  }
  total.batch_shape = g->batch_cfg;
  if (rc == SRK_OK && opt && opt->stats) *opt->stats = total;
  return rc;
}
