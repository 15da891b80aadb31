// Device-side building blocks of the walk kernels (sm_103a).
//
// Two generators of Salmon, Moraes, Dror, Shaw ("Parallel random numbers: as
// easy as 1, 2, 3", SC'11) are restated from that paper's definitions:
//   Philox4x32-10 (the Fisher-Yates draws): ten rounds, each multiplying
//     counter words 0 and 2 by 0xD2511F53 and 0xCD9E8D57 into 64-bit
//     products, then x0' = hi(M1 x2) ^ x1 ^ k0, x1' = lo(M1 x2),
//     x2' = hi(M0 x0) ^ x3 ^ k1, x3' = lo(M0 x0), the key advanced by the
//     Weyl constants 0x9E3779B9 and 0xBB67AE85 after every round;
//   Philox2x32-10 (the walk steps): ten rounds of x0' = hi(M x0) ^ x1 ^ k,
//     x1' = lo(M x0) with M = 0xD256D193, the 32-bit key advanced by
//     0x9E3779B9 after every round.
// Keys are launch- or warp-uniform, so the round keys are computed once.
#pragma once
#include <stdint.h>

#include "srk_internal.h"

namespace srk {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kPhilox2M = 0xD256D193u;

struct RoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

__device__ __forceinline__ RoundKeys round_keys(uint32_t key0, uint32_t key1) {
  RoundKeys rk;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = key0 + (uint32_t)r * kPhiloxW0;
    rk.k1[r] = key1 + (uint32_t)r * kPhiloxW1;
  }
  return rk;
}

// One Philox4x32-10 block: counter (c0..c3) -> 128 random bits in (x0..x3).
__device__ __forceinline__ void philox(const RoundKeys &rk, uint32_t c0,
                                       uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t &x0, uint32_t &x1,
                                       uint32_t &x2, uint32_t &x3) {
  x0 = c0; x1 = c1; x2 = c2; x3 = c3;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, x0), lo0 = kPhiloxM0 * x0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, x2), lo1 = kPhiloxM1 * x2;
    const uint32_t y0 = hi1 ^ x1 ^ rk.k0[r];
    const uint32_t y2 = hi0 ^ x3 ^ rk.k1[r];
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
  }
}

// One Philox2x32-10 block: counter (c0, c1), key k -> 64 random bits (x0, x1).
__device__ __forceinline__ void philox2(uint32_t k, uint32_t c0, uint32_t c1,
                                        uint32_t &x0, uint32_t &x1) {
  x0 = c0; x1 = c1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi = __umulhi(kPhilox2M, x0), lo = kPhilox2M * x0;
    x0 = hi ^ x1 ^ (k + (uint32_t)r * kPhiloxW0);
    x1 = lo;
  }
}

// floor(R * d / 2^64) for a 64-bit draw R = (hi:lo) and 0 < d < 2^32: a
// uniform index in [0, d).  R*d = hi*d*2^32 + lo*d, and adding the fraction
// of lo*d/2^32 cannot carry past a multiple of 2^32, so
// floor(R*d/2^64) = (hi*d + floor(lo*d/2^32)) >> 32.
__device__ __forceinline__ uint32_t draw_index(uint32_t hi, uint32_t lo,
                                               uint32_t d) {
  const uint64_t t = (uint64_t)hi * d + __umulhi(lo, d);
  return (uint32_t)(t >> 32);
}

// Walk steps.  Step i of walk replica r from node v, under the query's walk
// key k (walk_key): the Philox2x32-10 block of counter
// (((i-1)>>1) << 24 | r, v) serves
// the odd step i = 2t+1 (word x0) and the even step 2t+2 (word x1)
// (r < 2^24, t < 2^7, v < 2^31: the top bits of both counter words stay
// clear).  The in-neighbour index below d is Lemire's bounded draw ("Fast
// random integer generation in an interval", ACM TOMACS 2019) of the 32-bit
// word w: floor(w d / 2^32), accepted when (w d mod 2^32) >= 2^32 mod d, which
// leaves exactly floor(2^32 / d) words per index; a rejected word (probability
// below d / 2^32) is replaced by the 64-bit draw floor(R d / 2^64) from the
// block whose counter has the top bit of word 0 (odd step) or word 1 (even
// step) set, R = (x0:x1).  The index is uniform up to d / 2^64.
__device__ __forceinline__ uint32_t walk_ctr0(int i, uint32_t r) {
  return ((uint32_t)(i - 1) << 23 & 0x7F000000u) | r;
}

// The index of a step whose word was rejected (kept out of line: it runs on
// fewer than d / 2^32 of the steps).
static __device__ __noinline__ uint32_t step_index_redraw(uint32_t k, int i, uint32_t r,
                                                          uint32_t v, uint32_t d) {
  const uint32_t even = (uint32_t)(i - 1) & 1u;
  uint32_t y0, y1;
  philox2(k, walk_ctr0(i, r) | (even ? 0u : 0x80000000u), v | (even ? 0x80000000u : 0u),
          y0, y1);
  return draw_index(y0, y1, d);
}

// The mask of the warp's lanes below this one, read from the special
// register rather than kept live across the walk loop.
__device__ __forceinline__ uint32_t lanes_below_mask() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Stratum (walk length) of walk index r: the l with P[l] <= r < P[l+1],
// for a prefix array P[0..L+1] held in shared memory.
__device__ __forceinline__ int stratum_of(const int32_t *P, int L, int32_t r) {
  int lo = 0, hi = L;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace srk

// ------------------------------------------------------------------------
// Shared pieces of the query kernels (single-source and batched paths).
// ------------------------------------------------------------------------
#include "srk.h"

namespace srk {

// Control block of one query (int32 words): cap histogram, row sizes cnt[i]
// (pairs with cap >= i), hit-table row offsets R[i], per-cap cursors, then
// four uint64 slots: [0] target steps, [1] source steps, [2] the target
// kernel's work counter (low word; the batched path's item counter uses the
// whole slot) and the end of its active-target range (high word), [3] spare.
constexpr int kRowWords = SRK_MAX_LEN + 2;
constexpr int kSmallWords = 4 * kRowWords;
constexpr int kSmallBytes = 4 * kSmallWords + 32;

struct Small {
  int32_t *cap_hist;
  int32_t *cnt;
  int32_t *R;
  int32_t *cursor;
  unsigned long long *ctr;
};

__host__ __device__ __forceinline__ Small small_view(int32_t *base) {
  Small s;
  s.cap_hist = base;
  s.cnt = base + kRowWords;
  s.R = base + 2 * kRowWords;
  s.cursor = base + 3 * kRowWords;
  s.ctr = reinterpret_cast<unsigned long long *>(base + kSmallWords);
  return s;
}

// The walks hold the node they are at as (base, deg): the index of its
// list's first entry and its in-degree.  Each layout supplies
//   adj_entry(G, base, k): entry k of the list, the in-neighbour a step
//       reads with the index k drawn below deg (step_entry);
//   entry_pos(G, e): the identity of the node that entry names (what the hit
//       table holds);
//   entry_next(G, e, x, deg): base (returned) and degree of that node x;
//   node_start(G, row_ptr, v, deg): base and degree of node v, by id.

// The packed adjacency with 4-byte entries: node v's identity is its position
// pos[v]; a node of degree d < dmax has the word d there and its list right
// after it; a hub (d >= dmax) has {d, list offset} at an even position of the
// hub region; entry k of a list is (min(|I(y)|, dmax) << pb) | pos[y].
struct Adj {
  const uint32_t *adj;
  const int32_t *pos;
  int pb;
  uint32_t pmask, dmax;
};

__host__ __device__ __forceinline__ Adj make_adj(const uint32_t *adj, const int32_t *pos,
                                                 int pb) {
  Adj a;
  a.adj = adj;
  a.pos = pos;
  a.pb = pb;
  a.pmask = (uint32_t)((1ull << pb) - 1ull);
  a.dmax = (uint32_t)((1ull << (32 - pb)) - 1ull);
  return a;
}

__device__ __forceinline__ uint32_t adj_entry(const Adj &G, int32_t base, uint32_t k) {
  return G.adj[base + (int32_t)k];
}
__device__ __forceinline__ int32_t entry_pos(const Adj &G, uint32_t e) {
  return (int32_t)(e & G.pmask);
}
// The degree comes with the entry unless x is a hub; a hub's two header
// words are read together (its position is even).
__device__ __forceinline__ int32_t entry_next(const Adj &G, uint32_t e, int32_t x,
                                              uint32_t &deg) {
  const uint32_t code = e >> G.pb;
  if (code < G.dmax) {
    deg = code;
    return x + 1;
  }
  const uint2 h = *reinterpret_cast<const uint2 *>(G.adj + x);
  deg = h.x;
  return (int32_t)h.y;
}
__device__ __forceinline__ int32_t node_start(const Adj &G, const int32_t *, int32_t v,
                                              uint32_t &deg) {
  const int32_t x = G.pos[v];
  deg = G.adj[x];
  return deg < G.dmax ? x + 1 : (int32_t)G.adj[x + 1];
}

// The wide packed adjacency, for graphs whose positions need more than 28
// bits (the degree code of a 32-bit entry would then be too small to spare
// most steps a second random read): 8-byte words at positions
// pos(v) = v + row_ptr[v], adj[pos(v)] = {0, |I(v)|}; entry k of v's list,
// adj[pos(v) + 1 + k], is {position of the k-th in-neighbour y, |I(y)|}.
struct AdjW {
  const uint2 *adj;
};

__host__ __device__ __forceinline__ AdjW make_adjw(const uint32_t *words) {
  AdjW a;
  a.adj = reinterpret_cast<const uint2 *>(words);
  return a;
}
__device__ __forceinline__ uint2 adj_entry(const AdjW &G, int32_t base, uint32_t k) {
  return G.adj[base + (int32_t)k];
}
__device__ __forceinline__ int32_t entry_pos(const AdjW &, uint2 e) { return (int32_t)e.x; }
__device__ __forceinline__ int32_t entry_next(const AdjW &, uint2 e, int32_t x,
                                              uint32_t &deg) {
  deg = e.y;
  return x + 1;
}
__device__ __forceinline__ int32_t node_start(const AdjW &G, const int32_t *row_ptr,
                                              int32_t v, uint32_t &deg) {
  const int32_t x = v + row_ptr[v];
  deg = G.adj[x].y;
  return x + 1;
}

// The CSR layout: nodes are their own ids; landing on x reads row_ptr[x] and
// row_ptr[x+1] (the list and its degree), a step one col entry.
struct AdjC {
  const int32_t *row_ptr;
  const int32_t *col;
};
__device__ __forceinline__ int32_t adj_entry(const AdjC &G, int32_t base, uint32_t k) {
  return G.col[base + (int32_t)k];
}
__device__ __forceinline__ int32_t entry_pos(const AdjC &, int32_t e) { return e; }
__device__ __forceinline__ int32_t entry_next(const AdjC &G, int32_t, int32_t x,
                                              uint32_t &deg) {
  const int32_t b = G.row_ptr[x];
  deg = (uint32_t)(G.row_ptr[x + 1] - b);
  return b;
}
__device__ __forceinline__ int32_t node_start(const AdjC &G, const int32_t *, int32_t v,
                                              uint32_t &deg) {
  const int32_t b = G.row_ptr[v];
  deg = (uint32_t)(G.row_ptr[v + 1] - b);
  return b;
}

// Adjacency layouts (srk_graph::layout).
constexpr int kNarrow = 0, kWide = 1, kCsr = 2;

// The view of a graph's adjacency in layout kLayout.
template <int kLayout>
__device__ __forceinline__ auto adj_view(const uint32_t *words, const int32_t *pos, int pb,
                                         const int32_t *row_ptr, const int32_t *col) {
  if constexpr (kLayout == kWide) return make_adjw(words);
  else if constexpr (kLayout == kCsr) return AdjC{row_ptr, col};
  else return make_adj(words, pos, pb);
}

// The entry step i of walk replica r from node v reads (list base b, degree
// d), from the step's word w of block (walk_ctr0(i, r), v) under key k.  The
// load of floor(w d / 2^32) is issued before the acceptance test, which only
// replaces it when the word was rejected, so the test is off the chain of
// dependent loads.
template <class GA>
__device__ __forceinline__ auto step_entry(const GA &G, int32_t b, uint32_t w, uint32_t d,
                                           uint32_t k, int i, uint32_t r, uint32_t v) {
  auto e = adj_entry(G, b, __umulhi(w, d));
  const uint32_t lo = w * d;
  if (lo < d && lo < (0u - d) % d) e = adj_entry(G, b, step_index_redraw(k, i, r, v, d));
  return e;
}

// Source walk r of length len from s (list base b_s, degree deg_s) under the
// source's walk key k: writes the identity of the node at step i to out[i-1];
// returns the steps taken.
template <class GA>
__device__ __forceinline__ int source_walk(uint32_t k, const GA &G,
                                           uint32_t s, int32_t b_s, uint32_t deg_s,
                                           int32_t r, int len, int32_t *out) {
  int32_t b = b_s;
  uint32_t deg = deg_s;
  uint32_t x0 = 0, x1 = 0;
  for (int i = 1; i <= len; ++i) {
    if (deg == 0) return i - 1;
    if (i & 1) {
      philox2(k, walk_ctr0(i, (uint32_t)r), s, x0, x1);
    }
    const auto e = step_entry(G, b, (i & 1) ? x0 : x1, deg, k, i, (uint32_t)r, s);
    const int32_t x = entry_pos(G, e);
    out[i - 1] = x;
    b = entry_next(G, e, x, deg);
  }
  return len;
}

// Fisher-Yates draw t >= 1 of source s: k_t = floor(R (t+1) / 2^64), R from
// counter (t>>1, ~0, ~0, s), words 2(t&1), +1.
__device__ __forceinline__ int32_t fy_draw(const RoundKeys &rk, uint32_t s, int32_t t) {
  uint32_t x0, x1, x2, x3;
  philox(rk, (uint32_t)t >> 1, 0xFFFFFFFFu, 0xFFFFFFFFu, s, x0, x1, x2, x3);
  return (int32_t)draw_index((t & 1) ? x2 : x0, (t & 1) ? x3 : x1, (uint32_t)t + 1u);
}

// sigma[j] of the sequential Fisher-Yates loop, from the draws and the
// "next write of a position" links (see k_pairs in srk_query.cu).
__device__ __forceinline__ int32_t resolve_sigma(int32_t j, const int32_t *kdraw,
                                                 const int32_t *first,
                                                 const int32_t *succ, int32_t N) {
  int32_t p, h;
  if (j == 0) {
    p = 0;
    h = first[0];
  } else {
    p = kdraw[j];
    h = succ[j];
  }
  for (int32_t guard = 0; h >= 0 && guard < N; ++guard) {
    p = h;
    const int32_t f = first[p];
    h = (f == p) ? succ[p] : f;
  }
  return p;
}

// One source's pairs as the target walks see them.
struct PairSet {
  const int2 *rc;      // rc[i] = {R[i], cnt[i+1]}: hit-table row i's offset and the
                       // pairs with cap >= i+1 (cnt[L+1] = cnt[L+2] = 0)
  const int32_t *pair_j;
  const unsigned long long *pair_w;
  const int32_t *Hc;
  int32_t n_pairs;     // cnt[1]
  uint32_t key;        // walk key of the target walks (walk_key)
};

// All pairs of target u (list base b_u, degree deg_u > 0) walked by one
// warp with lane refill; per-lane totals of meetings c, weight W and steps st
// are added to the arguments (not reduced across the warp).
template <class GA>
__device__ __forceinline__ void walk_target(const GA &G,
                                            const PairSet &S, uint32_t u,
                                            int32_t b_u, uint32_t deg_u, uint32_t &c,
                                            unsigned long long &W, uint32_t &st) {
  int32_t next = 0;  // first unassigned pair (warp-uniform)
  bool live = false;
  int32_t a = 0, i = 1, b = 0;
  uint32_t deg = 0, j = 0;
  for (;;) {
    const uint32_t idle = __ballot_sync(0xffffffffu, !live);
    if (idle) {
      if (!live) {
        a = next + __popc(idle & lanes_below_mask());
        if (a < S.n_pairs) {
          live = true;
          j = (uint32_t)S.pair_j[a];
          i = 1;
          b = b_u;
          deg = deg_u;
        }
      }
      next += __popc(idle);
    }
    if (!__any_sync(0xffffffffu, live)) break;
    if (live) {
      uint32_t x0, x1;
      philox2(S.key, walk_ctr0(i, j), u, x0, x1);
      // odd step i
      auto e = step_entry(G, b, x0, deg, S.key, i, j, u);
      int32_t x = entry_pos(G, e);
      ++st;
      const int2 r1 = S.rc[i];
      if (x == S.Hc[r1.x + a]) {
        ++c;
        W += S.pair_w[a];
        live = false;
      } else if (a >= r1.y) {
        live = false;  // cap reached
      } else {
        b = entry_next(G, e, x, deg);
        if (deg == 0) {
          live = false;  // no in-neighbours: the walk ends
        } else {
          // even step i+1
          e = step_entry(G, b, x1, deg, S.key, i + 1, j, u);
          x = entry_pos(G, e);
          ++st;
          const int2 r2 = S.rc[i + 1];
          if (x == S.Hc[r2.x + a]) {
            ++c;
            W += S.pair_w[a];
            live = false;
          } else if (a >= r2.y) {
            live = false;
          } else {
            b = entry_next(G, e, x, deg);
            if (deg == 0) live = false;
            i += 2;
          }
        }
      }
    }
  }
}

}  // namespace srk

namespace srk {

// ---------------------------------------------------------------------------
// Literal target shuffle: target u pairs its walk pi_u(j) with source walk
// sigma[j].  pi_u is the identity when N = 1 and otherwise an unbalanced
// 4-round Feistel network on b bits, b the smallest integer with 2^b >= N:
// the value splits into A (high floor(b/2) bits) and B (low ceil(b/2) bits),
// a round maps (A, B) to (B, A ^ (F_r(B) mod 2^|A|)) so the widths swap and
// are back after four rounds, and the network is applied again until the
// value is below N (cycle walking; fewer than two passes on average).  The
// round function of target u is F_r(B) = h32(B ^ K_r(u)), h32 the 32-bit
// finalizer "lowbias32" of C. Wellons (2018), with 32-bit round keys
// K_r(u) = low half of mix64(k_r ^ u) and k_r = mix64(seed + (4 s + r + 1)
// 0x9E3779B97F4A7C15), mix64 the output function of SplitMix64 (Steele, Lea,
// Flood, OOPSLA 2014).
struct FeistelShape {
  int lo_bits, hi_bits;  // widths of B and A at the start
  int32_t N;
  uint64_t k[4];         // round keys
};

__host__ __device__ __forceinline__ FeistelShape feistel_shape(int32_t N, uint64_t seed,
                                                              uint32_t s) {
  int b = 1;
  while (((int64_t)1 << b) < (int64_t)N) ++b;
  FeistelShape f;
  f.hi_bits = b / 2;
  f.lo_bits = b - f.hi_bits;
  f.N = N;
  for (int r = 0; r < 4; ++r)
    f.k[r] = mix64(seed + (4 * (uint64_t)s + (uint64_t)r + 1) * 0x9E3779B97F4A7C15ull);
  return f;
}

// The round keys K_r(u) of target u.
struct FeistelKeys {
  uint32_t K[4];
};
__device__ __forceinline__ FeistelKeys feistel_keys(const FeistelShape &f, uint32_t u) {
  FeistelKeys k;
#pragma unroll
  for (int r = 0; r < 4; ++r) k.K[r] = (uint32_t)mix64(f.k[r] ^ (uint64_t)u);
  return k;
}

__device__ __forceinline__ int32_t feistel_pi(const FeistelShape &f, const FeistelKeys &K,
                                              int32_t j) {
  if (f.N <= 1) return 0;
  uint32_t v = (uint32_t)j;
  const uint32_t limit = 1u << (f.lo_bits + f.hi_bits);  // an orbit is no longer
  for (uint32_t guard = 0; guard < limit; ++guard) {
    int na = f.hi_bits, nb = f.lo_bits;
    uint32_t A = v >> f.lo_bits, B = v & ((1u << f.lo_bits) - 1u);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t fr = h32(B ^ K.K[r]);
      const uint32_t C = A ^ (fr & ((1u << na) - 1u));
      A = B;
      B = C;
      const int t = na;
      na = nb;
      nb = t;
    }
    v = (A << nb) | B;
    if (v < (uint32_t)f.N) break;
  }
  return (int32_t)v;
}

// walk_target in the literal mode: pair a (index j, source length l1 stored
// in pair_w[a]) walks target walk t = pi_u(j) of length l2 = stratum(t),
// walk replica t; it ends after min(l2, source cap) steps; a meeting adds
// round(a(l1) a(l2) 2^32).  P (stratum prefix, shared memory) and a (Lemma 7
// weights) come from the query table.
template <class GA>
__device__ __forceinline__ void walk_target_literal(
    const GA &G, const PairSet &S, const FeistelShape &f,
    const int32_t *P, int L, const double *aw, uint32_t u,
    int32_t b_u, uint32_t deg_u, uint32_t lanes_below, uint32_t &c,
    unsigned long long &W, uint32_t &st) {
  int32_t next = 0;
  bool live = false;
  int32_t a = 0, i = 1, b = 0, l2 = 0;
  uint32_t deg = 0, t = 0;
  // The target walks of pairs [base, base + 64), computed by the whole warp
  // (lane k: pair base + k in tw0, base + 32 + k in tw1) so that no lane
  // evaluates the permutation alone while the others wait; packed as
  // walk | (length << 24) (N_tot <= 2^24, L <= 255).
  const int32_t lane = __popc(lanes_below);
  const FeistelKeys K = feistel_keys(f, u);
  auto batch = [&](int32_t first) -> uint32_t {
    const int32_t q = first + lane;
    if (q >= S.n_pairs) return 0u;
    const uint32_t tw = (uint32_t)feistel_pi(f, K, S.pair_j[q]);
    return tw | ((uint32_t)stratum_of(P, L, (int32_t)tw) << 24);
  };
  int32_t base = 0;
  uint32_t tw0 = batch(0), tw1 = batch(32);
  for (;;) {
    const uint32_t idle = __ballot_sync(0xffffffffu, !live);
    if (idle) {
      if (next >= base + 32) {  // warp-uniform: advance the batches
        base += 32;
        tw0 = tw1;
        tw1 = batch(base + 32);
      }
      const int32_t an = next + __popc(idle & lanes_below);  // < base + 64
      const int32_t k = an - base;
      const uint32_t g0 = __shfl_sync(0xffffffffu, tw0, k & 31);
      const uint32_t g1 = __shfl_sync(0xffffffffu, tw1, k & 31);
      if (!live && an < S.n_pairs) {
        a = an;
        const uint32_t g = k < 32 ? g0 : g1;
        t = g & 0xFFFFFFu;
        l2 = (int32_t)(g >> 24);
        live = l2 >= 1;  // a length-0 target walk takes no step
        i = 1;
        b = b_u;
        deg = deg_u;
      }
      next += __popc(idle);
    }
    if (!__any_sync(0xffffffffu, live)) break;
    if (live) {
      uint32_t x0, x1;
      philox2(S.key, walk_ctr0(i, t), u, x0, x1);
      auto e = step_entry(G, b, x0, deg, S.key, i, t, u);
      int32_t x = entry_pos(G, e);
      ++st;
      const int2 r1 = S.rc[i];
      if (x == S.Hc[r1.x + a]) {
        ++c;
        W += __double2ull_rn(aw[(int)S.pair_w[a]] * aw[l2] * 4294967296.0);
        live = false;
      } else if (a >= r1.y || i >= l2) {
        live = false;
      } else {
        b = entry_next(G, e, x, deg);
        if (deg == 0) {
          live = false;
        } else {
          e = step_entry(G, b, x1, deg, S.key, i + 1, t, u);
          x = entry_pos(G, e);
          ++st;
          const int2 r2 = S.rc[i + 1];
          if (x == S.Hc[r2.x + a]) {
            ++c;
            W += __double2ull_rn(aw[(int)S.pair_w[a]] * aw[l2] * 4294967296.0);
            live = false;
          } else if (a >= r2.y || i + 1 >= l2) {
            live = false;
          } else {
            b = entry_next(G, e, x, deg);
            if (deg == 0) live = false;
            i += 2;
          }
        }
      }
    }
  }
}

}  // namespace srk
