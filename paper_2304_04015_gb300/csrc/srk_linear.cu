// Truncated linearised single-source SimRank and its adjoint (FP32).
//
// The linearised form of SimRank (Appendix A: S = c P^T S P + D, truncated to
// L + 1 terms) gives for one source s
//     s_vec = sum_{t=0}^{L} c^t (P^T)^t D P^t e_s,   D = (1 - c) I,
// with P[u][a] = w_e / W_a for the edge e = (u -> a) of a's in-list and
// W_a = sum of a's in-weights.  Forward, with y_t = P^t e_s:
//     y_0 = e_s,  y_t = P y_{t-1};   h_L = D y_L,  h_t = D y_t + c P^T h_{t+1};
//     s_vec = h_0.
// Backward for a loss with gradient g = dLoss/ds_vec (adjoint of the two
// recursions):
//     gb_0 = g,  gb_t = c P gb_{t-1};   yb_L = D gb_L,  yb_t = D gb_t + P^T yb_{t+1};
//     G_e = sum_{t=0}^{L-1} ( c gb_t[a] h_{t+1}[u] + yb_{t+1}[u] y_t[a] )
// (the gradient w.r.t. the entry P[u][a]), and through the normalisation
//     dLoss/dw_e = ( G_e - sum_{e' in I(a)} G_e' P_e' ) / W_a.
//
// Every product with P or P^T is a gather: P^T v along the in-lists, P v along
// the out-lists of a transpose of the graph that is built once per graph (a
// stable radix sort of the edges by source node, so each out-list keeps edge
// order) and cached in the handle.  Each list is reduced in a fixed order by
// one thread (up to 4 entries), a group of 8 lanes (up to 32), a warp (up to
// 512), or warps over chunks of 512 entries whose partial sums are added in
// chunk order by the warp that finishes the list's last chunk, so no result
// depends on timing.  The vectors are stored term-major, (L+1) x n: a gather
// reads one contiguous term, whose most referenced entries (R-MAT's low ids)
// share sectors and stay in L1.  The per-edge gradient pass reads, for each
// source node, one node-major row of the pairs (h_{t+1}, yb_{t+1}) made by
// one transpose, so each node's 2L values come together.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "srk_internal.h"

namespace srk {

// List size classes of the segmented reductions.
constexpr int32_t kTiny = 4;      // up to this many entries: one thread
constexpr int32_t kShort = 32;    // up to this many: 8-lane groups
constexpr int32_t kMid = 512;     // up to this many: one warp
constexpr int32_t kChunk = 512;   // longer lists: chunks of this many entries, one warp each
constexpr int kGroup = 8;
constexpr int kSegBlock = 256;    // threads per block of the reduction kernel
// Radix sort of the transpose: 8-bit digits, tiles of 256 threads x 16 keys.
constexpr int kSortBlock = 256, kSortItems = 16, kSortTile = kSortBlock * kSortItems;

// Size-class lists of one direction (in-lists or out-lists) of the graph.
struct Classes {
  int4 *small = nullptr;          // {node, beg, end, 0} of the lists with kTiny < len <= kShort
  int4 *mid = nullptr;            // {node, beg, end, 0} of the lists with kShort < len <= kMid
  int32_t *item_node = nullptr;   // chunk items of the longer lists: the node,
  int32_t *item_beg = nullptr;    //   the entry range [beg, end),
  int32_t *item_end = nullptr;
  int32_t *item_long = nullptr;   //   the node's index among the long lists
  int32_t *long_first = nullptr;  // first item and item count of each long list
  int32_t *long_count = nullptr;
  int32_t *order = nullptr;       // the work units, heaviest first (see k_seg)
  int32_t n_small = 0, n_mid = 0, n_long = 0, n_items = 0;
};

}  // namespace srk

// Per-graph topology of the linearised form (built on first use, freed with
// the graph).
struct srk_lin_topo {
  int32_t *erow = nullptr;     // m: the node whose in-list holds edge e
  int32_t *out_ptr = nullptr;  // n + 1: out-list offsets of the transpose
  int32_t *t_a = nullptr;      // m: out-list entry k is the edge (u -> t_a[k]) ...
  int32_t *t_e = nullptr;      // m: ... of edge index t_e[k] (ascending per list)
  srk::Classes in, out;
  void *block = nullptr;
};

struct srk_linear_ctx {
  const srk_graph *g = nullptr;
  const srk_lin_topo *topo = nullptr;
  int device = 0;
  int32_t n = 0, L = 0, s = 0;
  int64_t m = 0;
  double c = 0.0;
  float *Pe = nullptr;      // m: w_e / W_a, in-list order
  float *PeT = nullptr;     // m: the same values in out-list order
  float *Wa = nullptr;      // n: in-weight sums
  float *y = nullptr;       // (L+1) x n, term-major: y[t n + a] = (P^t e_s)[a]
  float *h = nullptr;       // (L+1) x n, term-major partial sums, h_0 = s_vec
  double *part = nullptr;   // partial sums of the chunk items (either direction)
  int32_t *done = nullptr;  // finished chunks per long list (zero between uses)
  int *bad = nullptr;       // weight check flag
  void *block = nullptr;    // the device block all arrays above live in
};

namespace srk {

// ------------------------------------------------------------ reductions --

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
template <class T>
__device__ __forceinline__ T group_sum(T v) {  // over aligned groups of kGroup lanes
  for (int off = kGroup / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
// Sum of val(k) over k in [b, e) taken by thread tid of nthr: four strided
// entries per round, all loaded before any is added, in a fixed order.
template <class T, class V>
__device__ __forceinline__ T list_partial(const V &val, int64_t b, int64_t e, int tid,
                                          int nthr) {
  T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int64_t k = b + tid; k < e; k += 4 * (int64_t)nthr) {
    const int64_t k1 = k + nthr, k2 = k + 2 * nthr, k3 = k + 3 * nthr;
    const T v0 = val(k);
    const T v1 = (k1 < e) ? val(k1) : (T)0;
    const T v2 = (k2 < e) ? val(k2) : (T)0;
    const T v3 = (k3 < e) ? val(k3) : (T)0;
    s0 += v0;
    s1 += v1;
    s2 += v2;
    s3 += v3;
  }
  return (s0 + s1) + (s2 + s3);
}

// Entry values and result writers of the segmented reductions.
struct GatherVal {  // w[k] in[idx[k]]
  const int32_t *idx;
  const float *w;
  const float *in;
  __device__ __forceinline__ float operator()(int64_t k) const { return w[k] * in[idx[k]]; }
};
struct DotVal {  // x[k] w[k]
  const float *x;
  const float *w;
  __device__ __forceinline__ float operator()(int64_t k) const { return x[k] * w[k]; }
};
struct WeightVal {  // w[k]
  const float *w;
  __device__ __forceinline__ float operator()(int64_t k) const { return w[k]; }
};
struct WriteAxpy {  // out[a] = alpha add[a] + beta sum (add may be null)
  float *out;
  const float *add;
  float alpha, beta;
  __device__ __forceinline__ void operator()(int32_t a, float sum) const {
    out[a] = (add ? alpha * add[a] : 0.0f) + beta * sum;
  }
};
struct WriteVec {  // out[a] = sum
  float *out;
  __device__ __forceinline__ void operator()(int32_t a, float sum) const { out[a] = sum; }
};

// One segmented reduction over the work units: the chunks of the lists
// longer than kMid (one warp each), the lists of kShort < len <= kMid (one
// warp each), groups of 8 lists of kTiny < len <= kShort (two per 8 lanes)
// and runs of 64 consecutive nodes, of which each lane reduces the lists of
// two nodes that have at most kTiny entries (empty lists included), numbered
// in that order.  C.order lists them by rounds of loads, heaviest first.  With
// a warp per unit (the launch in segmented()) warp w takes rank w; a smaller
// grid of W warps deals the ranks out in snake order (warp w takes w,
// 2W - 1 - w, 2W + w, ...).  A long list's chunk sums are added in chunk
// order by the warp that finishes its last chunk, which then re-arms the
// list's counter for the next launch.
template <class T, class V, class W>
__global__ void __launch_bounds__(kSegBlock)
k_seg(const int32_t *__restrict__ ptr, int32_t n, Classes C, V val, W write,
      T *__restrict__ part, int32_t *__restrict__ done) {
  const int lane = threadIdx.x & 31;
  const int64_t e1 = C.n_items, e2 = e1 + C.n_mid, e3 = e2 + ((int64_t)C.n_small + 7) / 8,
                e4 = e3 + ((int64_t)n + 63) / 64;
  const int64_t W_all = ((int64_t)gridDim.x * blockDim.x) / 32;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  for (int64_t k = 0;; ++k) {
    const int64_t r = k * W_all + ((k & 1) ? W_all - 1 - w : w);
    if (r >= e4) break;  // every later rank is larger
    const int64_t u = C.order[r];
    if (u < e1) {
      const T s = warp_sum(list_partial<T>(val, C.item_beg[u], C.item_end[u], lane, 32));
      if (lane == 0) {
        const int32_t l = C.item_long[u];
        part[u] = s;
        __threadfence();
        if (atomicAdd(&done[l], 1) == C.long_count[l] - 1) {
          __threadfence();
          const int32_t f = C.long_first[l], cnt = C.long_count[l];
          const volatile T *p = part;
          T t = 0;
          for (int32_t i = 0; i < cnt; ++i) t += p[f + i];
          write(C.item_node[u], t);
          done[l] = 0;
        }
      }
    } else if (u < e2) {
      const int4 r = C.mid[u - e1];
      const T sum = warp_sum(list_partial<T>(val, r.y, r.z, lane, 32));
      if (lane == 0) write(r.x, sum);
    } else if (u < e3) {
      // two lists per 8-lane group, each at most 4 entries per lane, loaded
      // together
      const int gl = lane & (kGroup - 1);
      const int64_t q0 = (u - e2) * 8 + lane / kGroup, q1 = q0 + 4;
      const int4 r0 = q0 < C.n_small ? C.small[q0] : make_int4(-1, 0, 0, 0);
      const int4 r1 = q1 < C.n_small ? C.small[q1] : make_int4(-1, 0, 0, 0);
      T v0[4], v1[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int32_t k0 = r0.y + gl + j * kGroup, k1 = r1.y + gl + j * kGroup;
        v0[j] = k0 < r0.z ? val(k0) : (T)0;
        v1[j] = k1 < r1.z ? val(k1) : (T)0;
      }
      const T s0 = group_sum((v0[0] + v0[1]) + (v0[2] + v0[3]));
      const T s1 = group_sum((v1[0] + v1[1]) + (v1[2] + v1[3]));
      if (gl == 0 && r0.x >= 0) write(r0.x, s0);
      if (gl == 0 && r1.x >= 0) write(r1.x, s1);
    } else {
      // two nodes per lane: a and a + 32 of a run of 64
      const int64_t a0 = (u - e3) * 64 + lane, a1 = a0 + 32;
      int32_t b0 = 0, f0 = 0, b1 = 0, f1 = 0;  // f: end, or the start when not tiny
      if (a0 < n) {
        b0 = ptr[a0];
        f0 = ptr[a0 + 1];
      }
      if (a1 < n) {
        b1 = ptr[a1];
        f1 = ptr[a1 + 1];
      }
      const bool t0 = a0 < n && f0 - b0 <= kTiny, t1 = a1 < n && f1 - b1 <= kTiny;
      if (!t0) f0 = b0;
      if (!t1) f1 = b1;
      T v0[kTiny], v1[kTiny];
#pragma unroll
      for (int j = 0; j < kTiny; ++j) {
        v0[j] = (b0 + j < f0) ? val(b0 + j) : (T)0;
        v1[j] = (b1 + j < f1) ? val(b1 + j) : (T)0;
      }
      if (t0) write((int32_t)a0, (v0[0] + v0[1]) + (v0[2] + v0[3]));
      if (t1) write((int32_t)a1, (v1[0] + v1[1]) + (v1[2] + v1[3]));
    }
  }
}

// ------------------------------------------------------ topology kernels --

// erow[k] = the node a with row_ptr[a] <= k < row_ptr[a+1] (binary search).
__global__ void k_erow(const int32_t *__restrict__ row_ptr, int32_t n, int64_t m,
                       int32_t *__restrict__ erow) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = n - 1;  // the largest a with row_ptr[a] <= k
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo + 1) / 2;
      if (row_ptr[mid] <= k) lo = mid;
      else hi = mid - 1;
    }
    erow[k] = lo;
  }
}

__global__ void k_out_degree(const int32_t *__restrict__ col, int64_t m,
                             int32_t *__restrict__ odeg) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&odeg[col[k]], 1);
}

__global__ void k_iota(int32_t *__restrict__ v, int64_t m) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x)
    v[k] = (int32_t)k;
}

// Radix sort pass, step 1: digit histogram of each tile, stored digit-major
// (hist[d * tiles + tile]) so that its exclusive scan gives each
// (digit, tile) its first output position.
__global__ void __launch_bounds__(kSortBlock)
k_sort_hist(const int32_t *__restrict__ keys, int64_t m, int shift, int32_t tiles,
            int32_t *__restrict__ hist) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = base + (int64_t)r * kSortBlock + threadIdx.x;
    if (i < m) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Radix sort pass, step 2: stable scatter.  Round r of a tile covers 256
// consecutive keys; a key goes to its (digit, tile) offset plus the number of
// keys of its digit in earlier rounds, earlier warps and lower lanes.
__global__ void __launch_bounds__(kSortBlock)
k_sort_scatter(const int32_t *__restrict__ keys, const int32_t *__restrict__ vals, int64_t m,
               int shift, int32_t tiles, const int32_t *__restrict__ off,
               int32_t *__restrict__ keys_out, int32_t *__restrict__ vals_out) {
  constexpr int kWarps = kSortBlock / 32;
  __shared__ int32_t base[256];
  __shared__ int32_t wcnt[kWarps][256];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  base[t] = off[(int64_t)t * tiles + blockIdx.x];
  for (int i = 0; i < kWarps; ++i) wcnt[i][t] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = tile0 + (int64_t)r * kSortBlock + t;
    const bool valid = i < m;
    int32_t key = 0, val = 0, d = 256;  // 256: no key in this slot
    if (valid) {
      key = keys[i];
      val = vals[i];
      d = (key >> shift) & 255;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    int32_t run = 0;  // thread t: digit t's counts over the warps, made exclusive
    for (int k = 0; k < kWarps; ++k) {
      const int32_t c = wcnt[k][t];
      wcnt[k][t] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      const int64_t pos = (int64_t)base[d] + wcnt[w][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    base[t] += run;
    for (int k = 0; k < kWarps; ++k) wcnt[k][t] = 0;
    __syncthreads();
  }
}

__global__ void k_gather_i32(const int32_t *__restrict__ src, const int32_t *__restrict__ idx,
                             int64_t m, int32_t *__restrict__ dst) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[idx[k]];
}

// Size classes of the lists of ptr: cnt[0] mid lists, cnt[1] long lists,
// cnt[2] chunk items, cnt[3] small lists.  Where a node lands in these lists
// depends on timing; what is computed for the node does not.
__global__ void k_classify(const int32_t *__restrict__ ptr, int32_t n, Classes C,
                           int32_t *__restrict__ cnt) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = ptr[a], e = ptr[a + 1], len = e - b;
    if (len > kTiny && len <= kShort) {
      C.small[atomicAdd(&cnt[3], 1)] = make_int4((int32_t)a, b, e, 0);
    } else if (len > kShort && len <= kMid) {
      C.mid[atomicAdd(&cnt[0], 1)] = make_int4((int32_t)a, b, e, 0);
    } else if (len > kMid) {
      const int32_t l = atomicAdd(&cnt[1], 1);
      const int32_t c = (len + kChunk - 1) / kChunk;
      const int32_t f = atomicAdd(&cnt[2], c);
      C.long_first[l] = f;
      C.long_count[l] = c;
      for (int32_t i = 0; i < c; ++i) {
        C.item_node[f + i] = (int32_t)a;
        C.item_beg[f + i] = b + i * kChunk;
        C.item_end[f + i] = min(e, b + (i + 1) * kChunk);
        C.item_long[f + i] = l;
      }
    }
  }
}

// ------------------------------------------------------- prep and vectors --

// P_e = w_e / W_a (IEEE FP32 division); flags weights that are not positive
// and finite.
__global__ void k_lin_pe(const float *__restrict__ w, const int32_t *__restrict__ erow,
                         const float *__restrict__ Wa, int64_t m, float *__restrict__ Pe,
                         int *bad) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[k];
    if (!(x > 0.0f) || !isfinite(x)) *bad = 1;
    Pe[k] = x / Wa[erow[k]];
  }
}

__global__ void k_gather_f32(const float *__restrict__ src, const int32_t *__restrict__ idx,
                             int64_t m, float *__restrict__ dst) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[idx[k]];
}

// v[a] = (a == s).
__global__ void k_lin_unit(float *__restrict__ v, int32_t n, int32_t s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (i == s) ? 1.0f : 0.0f;
}

// out[a] = d in[a].
__global__ void k_lin_scale(const float *__restrict__ in, float d, int32_t n,
                            float *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = d * in[i];
}

// The node-major rows of the pairs (h_{t+1}[u], yb_{t+1}[u]), t < L, from the
// term-major h and yb: hy[u][t] = {h[(t+1) n + u], yb[(t+1) n + u]}.  Block b
// moves nodes [32 b, 32 b + 32) through shared memory (2 L x 33 floats),
// reading 32 consecutive nodes of a term and writing the 32 L consecutive
// pairs.
__global__ void __launch_bounds__(256) k_lin_pairs(const float *__restrict__ h,
                                                   const float *__restrict__ yb, int32_t L,
                                                   int32_t n, float2 *__restrict__ hy) {
  extern __shared__ float tile[];  // [0, 33 L): h terms 1..L; [33 L, 66 L): yb terms
  const int64_t a0 = (int64_t)blockIdx.x * 32;
  const int na = (int)((int64_t)n - a0 < 32 ? (int64_t)n - a0 : 32);
  for (int q = threadIdx.x; q < L * 32; q += blockDim.x) {
    const int t = q >> 5, j = q & 31;
    if (j < na) {
      tile[t * 33 + j] = h[(int64_t)(t + 1) * n + a0 + j];
      tile[(L + t) * 33 + j] = yb[(int64_t)(t + 1) * n + a0 + j];
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < na * L; q += blockDim.x) {
    const int j = q / L, t = q - j * L;
    hy[(a0 + j) * L + t] = make_float2(tile[t * 33 + j], tile[(L + t) * 33 + j]);
  }
}

// G_e for every edge e = (u -> a), edge-parallel.  gb and y are term-major
// (consecutive edges mostly share a, so a warp reads one word per term); h
// and yb come as u's row of pairs in hy (u is scattered, so a thread reads
// its 2 L values from one row).
__global__ void k_lin_edge_G(const int32_t *__restrict__ erow, const int32_t *__restrict__ col,
                             int64_t m, int32_t n, const float *__restrict__ y,
                             const float2 *__restrict__ hy, const float *__restrict__ gb,
                             int32_t L, float c, float *__restrict__ G) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = erow[k], u = col[k];
    const float2 *hyu = hy + u * L;
    float g = 0.0f;
    for (int t0 = 0; t0 < L; t0 += 4) {  // four terms' loads in flight
      float gv[4], yv[4], hv[4], bv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int t = t0 + j;
        const bool ok = t < L;
        const float2 p = ok ? hyu[t] : make_float2(0.0f, 0.0f);
        gv[j] = ok ? gb[(int64_t)t * n + a] : 0.0f;
        yv[j] = ok ? y[(int64_t)t * n + a] : 0.0f;
        hv[j] = p.x;
        bv[j] = p.y;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // t ascending; the padding terms add exact zeros
        g = fmaf(c * gv[j], hv[j], g);
        g = fmaf(bv[j], yv[j], g);
      }
    }
    G[k] = g;
  }
}

// grad_e = (G_e - T_a) / W_a with T_a = sum_{e' in I(a)} G_e' P_e'.
__global__ void k_lin_edge_fin(const int32_t *__restrict__ erow, int64_t m,
                               const float *__restrict__ T, const float *__restrict__ Wa,
                               float *__restrict__ grad) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = erow[k];
    grad[k] = (grad[k] - T[a]) * (1.0f / Wa[a]);
  }
}

// ------------------------------------------------------------- host side --

static int grid_of(int64_t work, int per_block, int dev, int per_sm = 8) {
  const int64_t want = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)sm_count(dev) * per_sm;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

// Segmented reduction over the lists of ptr (size classes C): one launch
// with a warp per work unit.  Blocks take the units heaviest first (C.order)
// and the block scheduler starts each next block on the first SM with room,
// which makes a greedy longest-first schedule (measured faster than a grid of
// resident blocks dealing the units among themselves).
template <class T, class V, class W>
static void segmented(srk_linear_ctx *x, const int32_t *ptr, const Classes &C, V val, W write,
                      cudaStream_t st) {
  const int64_t units = (int64_t)C.n_items + C.n_mid + ((int64_t)C.n_small + 7) / 8 +
                        ((int64_t)x->n + 63) / 64;
  const int warps = kSegBlock / 32;
  int64_t blocks = (units + warps - 1) / warps;
  if (blocks < 1) blocks = 1;
  k_seg<T><<<(int)blocks, kSegBlock, 0, st>>>(ptr, x->n, C, val, write,
                                              reinterpret_cast<T *>(x->part), x->done);
}

// out = alpha add + beta P^T in (n-vectors; gather along in-lists).
static void gather_t(srk_linear_ctx *x, const float *in, const float *add, float alpha,
                     float beta, float *out, cudaStream_t st) {
  segmented<float>(x, x->g->row_ptr, x->topo->in, GatherVal{x->g->col, x->Pe, in},
                   WriteAxpy{out, add, alpha, beta}, st);
}

// out = scale P in (n-vectors; gather along the transpose's out-lists).
static void gather_p(srk_linear_ctx *x, const float *in, float scale, float *out,
                     cudaStream_t st) {
  segmented<float>(x, x->topo->out_ptr, x->topo->out, GatherVal{x->topo->t_a, x->PeT, in},
                   WriteAxpy{out, nullptr, 0.0f, scale}, st);
}

// Capacities of the class arrays of one direction.
static size_t long_lists_max(int64_t m) { return (size_t)(m / (kMid + 1)) + 1; }
static size_t items_max(int64_t m) { return (size_t)(m / kChunk) + long_lists_max(m) + 1; }
static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Carves the class arrays of one direction from p (sizes only when p is
// null); returns the bytes used.
static size_t class_layout(Classes *C, char *p, int32_t n, int64_t m) {
  size_t off = 0;
  for (int4 **rec : {&C->small, &C->mid}) {  // at most n lists each
    if (p) *rec = reinterpret_cast<int4 *>(p + off);
    off += up256(sizeof(int4) * (size_t)n);
  }
  const size_t sizes[6] = {items_max(m), items_max(m),      items_max(m),
                           items_max(m), long_lists_max(m), long_lists_max(m)};
  int32_t **dst[6] = {&C->item_node, &C->item_beg,   &C->item_end,
                      &C->item_long, &C->long_first, &C->long_count};
  for (int i = 0; i < 6; ++i) {
    if (p) *dst[i] = reinterpret_cast<int32_t *>(p + off);
    off += up256(sizeof(int32_t) * sizes[i]);
  }
  return off;
}

static std::mutex topo_mu;

// Builds g's linear topology on stream st and waits for it.
// The static schedule of one direction's work units (k_seg): units sorted by
// their rounds of 128 loads (4 per lane), ceil(len / 128) for chunks and mid
// lists and 1 for the rest, descending; equal costs keep unit order.
static cudaError_t build_order(Classes &C, int32_t n, cudaStream_t st) {
  const int64_t e1 = C.n_items, e2 = e1 + C.n_mid, e3 = e2 + ((int64_t)C.n_small + 7) / 8,
                e4 = e3 + ((int64_t)n + 63) / 64;
  std::vector<int32_t> beg((size_t)C.n_items), end((size_t)C.n_items);
  std::vector<int4> mid((size_t)C.n_mid);
  cudaError_t e = cudaSuccess;
  if (C.n_items > 0) {
    e = cudaMemcpyAsync(beg.data(), C.item_beg, sizeof(int32_t) * beg.size(),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(end.data(), C.item_end, sizeof(int32_t) * end.size(),
                          cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && C.n_mid > 0)
    e = cudaMemcpyAsync(mid.data(), C.mid, sizeof(int4) * mid.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  constexpr int kRound = 128, kMaxCost = (kChunk > kMid ? kChunk : kMid) / kRound;
  std::vector<uint8_t> cost((size_t)e4, 1);
  for (int64_t u = 0; u < e2; ++u) {
    const int64_t len = u < e1 ? (int64_t)end[(size_t)u] - beg[(size_t)u]
                               : (int64_t)mid[(size_t)(u - e1)].z - mid[(size_t)(u - e1)].y;
    const int64_t c = (len + kRound - 1) / kRound;
    cost[(size_t)u] = (uint8_t)(c < 1 ? 1 : (c > kMaxCost ? kMaxCost : c));
  }
  std::vector<int32_t> order;
  order.reserve((size_t)e4);
  for (int c = kMaxCost; c >= 1; --c)
    for (int64_t u = 0; u < e4; ++u)
      if (cost[(size_t)u] == c) order.push_back((int32_t)u);
  e = cudaMalloc(&C.order, sizeof(int32_t) * (size_t)(e4 > 0 ? e4 : 1));
  if (e == cudaSuccess && e4 > 0)
    e = cudaMemcpy(C.order, order.data(), sizeof(int32_t) * (size_t)e4, cudaMemcpyHostToDevice);
  return e;
}

static int build_topo(const srk_graph *g, cudaStream_t st, srk_lin_topo **out) {
  const int dev = g->device;
  const int32_t n = g->n;
  const int64_t m = g->m;
  const size_t mm = (size_t)(m > 0 ? m : 1);
  const size_t words_m = up256(sizeof(int32_t) * mm);
  Classes sizing;
  const size_t cls = class_layout(&sizing, nullptr, n, m);
  const size_t keep = 3 * words_m + up256(sizeof(int32_t) * ((size_t)n + 1)) + 2 * cls;
  srk_lin_topo *T = new srk_lin_topo;
  cudaError_t e = cudaMalloc(&T->block, keep);
  if (e != cudaSuccess) {
    delete T;
    return cuda_fail(e, "linear topology: allocation");
  }
  char *p = (char *)T->block;
  T->erow = (int32_t *)p;
  T->t_a = (int32_t *)(p + words_m);
  T->t_e = (int32_t *)(p + 2 * words_m);
  T->out_ptr = (int32_t *)(p + 3 * words_m);
  p += 3 * words_m + up256(sizeof(int32_t) * ((size_t)n + 1));
  p += class_layout(&T->in, p, n, m);
  class_layout(&T->out, p, n, m);

  // scratch: out-degrees, two key/value buffers, histogram and its scan, counters
  const int32_t tiles = (int32_t)((m + kSortTile - 1) / kSortTile);
  const size_t H = (size_t)256 * (size_t)(tiles > 0 ? tiles : 1);
  const size_t scratch = up256(sizeof(int32_t) * (size_t)n) + 4 * words_m +
                         up256(sizeof(int32_t) * H) + up256(sizeof(int32_t) * (H + 1)) +
                         up256(sizeof(int32_t) * 8);
  cudaMemPool_t mp = pool(dev);
  void *sb = nullptr;
  e = mp ? cudaMallocFromPoolAsync(&sb, scratch, mp, st) : cudaErrorMemoryAllocation;
  if (e != cudaSuccess) {
    cudaFree(T->block);
    delete T;
    return cuda_fail(e, "linear topology: scratch");
  }
  char *q = (char *)sb;
  int32_t *odeg = (int32_t *)q;
  q += up256(sizeof(int32_t) * (size_t)n);
  int32_t *kA = (int32_t *)q, *vA = (int32_t *)(q + words_m);
  int32_t *kB = (int32_t *)(q + 2 * words_m), *vB = (int32_t *)(q + 3 * words_m);
  q += 4 * words_m;
  int32_t *hist = (int32_t *)q;
  q += up256(sizeof(int32_t) * H);
  int32_t *hoff = (int32_t *)q;
  q += up256(sizeof(int32_t) * (H + 1));
  int32_t *cnt = (int32_t *)q;

  const int gm = grid_of(m, 256, dev), gn = grid_of(n, 256, dev);
  cudaMemsetAsync(odeg, 0, sizeof(int32_t) * (size_t)n, st);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 8, st);
  if (m > 0) {
    k_erow<<<gm, 256, 0, st>>>(g->row_ptr, n, m, T->erow);
    k_out_degree<<<gm, 256, 0, st>>>(g->col, m, odeg);
  }
  k_scan<<<1, 1024, 0, st>>>(odeg, T->out_ptr, n);
  if (m > 0) {
    // stable LSD radix sort of the edge indices by their source node col[e]
    cudaMemcpyAsync(kA, g->col, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToDevice, st);
    k_iota<<<gm, 256, 0, st>>>(vA, m);
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) ++bits;  // keys < n <= 2^bits
    for (int shift = 0; shift < bits; shift += 8) {
      k_sort_hist<<<tiles, kSortBlock, 0, st>>>(kA, m, shift, tiles, hist);
      k_scan<<<1, 1024, 0, st>>>(hist, hoff, (int32_t)H);
      k_sort_scatter<<<tiles, kSortBlock, 0, st>>>(kA, vA, m, shift, tiles, hoff, kB, vB);
      int32_t *tk = kA, *tv = vA;
      kA = kB;
      vA = vB;
      kB = tk;
      vB = tv;
    }
    cudaMemcpyAsync(T->t_e, vA, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToDevice, st);
    k_gather_i32<<<gm, 256, 0, st>>>(T->erow, T->t_e, m, T->t_a);
  }
  k_classify<<<gn, 256, 0, st>>>(g->row_ptr, n, T->in, cnt);
  k_classify<<<gn, 256, 0, st>>>(T->out_ptr, n, T->out, cnt + 4);
  int32_t hc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(sb, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    cudaFree(T->block);
    delete T;
    return cuda_fail(e, "linear topology: build");
  }
  T->in.n_mid = hc[0];
  T->in.n_long = hc[1];
  T->in.n_items = hc[2];
  T->in.n_small = hc[3];
  T->out.n_mid = hc[4];
  T->out.n_long = hc[5];
  T->out.n_items = hc[6];
  T->out.n_small = hc[7];
  if ((e = build_order(T->in, n, st)) != cudaSuccess ||
      (e = build_order(T->out, n, st)) != cudaSuccess) {
    if (T->in.order) cudaFree(T->in.order);
    if (T->out.order) cudaFree(T->out.order);
    cudaFree(T->block);
    delete T;
    return cuda_fail(e, "linear topology: unit order");
  }
  *out = T;
  return SRK_OK;
}

static int get_topo(const srk_graph *g, cudaStream_t st, const srk_lin_topo **out) {
  std::lock_guard<std::mutex> lock(topo_mu);
  if (!g->lin) {
    srk_lin_topo *T = nullptr;
    const int rc = build_topo(g, st, &T);
    if (rc != SRK_OK) return rc;
    const_cast<srk_graph *>(g)->lin = T;
  }
  *out = g->lin;
  return SRK_OK;
}

void free_lin_topo(srk_graph *g) {
  if (!g || !g->lin) return;
  if (g->lin->in.order) cudaFree(g->lin->in.order);
  if (g->lin->out.order) cudaFree(g->lin->out.order);
  if (g->lin->block) cudaFree(g->lin->block);
  delete g->lin;
  g->lin = nullptr;
}

// The context's device memory is one block from the library's stream-ordered
// pool, carved into its arrays.
static void free_ctx(srk_linear_ctx *x, cudaStream_t st = nullptr) {
  if (!x) return;
  DeviceGuard guard(x->device);
  if (x->block) cudaFreeAsync(x->block, st);
  delete x;
}

}  // namespace srk

using namespace srk;

extern "C" int srk_linear_ctx_free(srk_linear_ctx *ctx) {
  if (!ctx) return SRK_OK;
  {
    DeviceGuard guard(ctx->device);
    cudaDeviceSynchronize();
  }
  free_ctx(ctx);
  return SRK_OK;
}

extern "C" int srk_linear_fwd(const srk_graph *g, const float *edge_w, int32_t s,
                              double c, int32_t L, float *s_out,
                              srk_linear_ctx **ctx_out, void *cuda_stream) {
  clear_error();
  if (ctx_out) *ctx_out = nullptr;
  if (!g) return fail(SRK_EINVAL, "null graph");
  if (!edge_w) edge_w = g->edge_w;
  if (!edge_w && g->m > 0)
    return fail(SRK_EINVAL, "no edge weights: pass edge_w or load the graph with them");
  if (s < 0 || s >= g->n) return fail(SRK_EINVAL, "source %d outside [0, %d)", s, g->n);
  if (!(c > 0.0 && c < 1.0)) return fail(SRK_EINVAL, "c = %g outside (0, 1)", c);
  if (L < 0 || L > SRK_MAX_LEN) return fail(SRK_EINVAL, "L = %d outside [0, %d]", L, SRK_MAX_LEN);
  if (!s_out) return fail(SRK_EINVAL, "s_out is null");
  DeviceGuard guard(g->device);
  if ((g->m > 0 && !is_device_ptr(edge_w)) || !is_device_ptr(s_out))
    return fail(SRK_EINVAL, "srk_linear_fwd takes device pointers for edge_w and s_out");
  const int dev = g->device;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const srk_lin_topo *topo = nullptr;
  const int rc = get_topo(g, st, &topo);
  if (rc != SRK_OK) return rc;
  srk_linear_ctx *x = new srk_linear_ctx;
  x->g = g;
  x->topo = topo;
  x->device = dev;
  x->n = g->n;
  x->m = g->m;
  x->L = L;
  x->s = s;
  x->c = c;
  const size_t n = (size_t)g->n, m = (size_t)(g->m > 0 ? g->m : 1);
  const int32_t S = L + 1;
  const size_t vec = (size_t)S * n;
  const size_t cap = items_max(g->m) + long_lists_max(g->m);
  const size_t sizes[8] = {sizeof(float) * m,   sizeof(float) * m,     sizeof(float) * n,
                           sizeof(float) * vec, sizeof(float) * vec,   sizeof(double) * cap,
                           sizeof(int32_t) * cap, sizeof(int)};
  size_t total = 0;
  for (size_t b : sizes) total += up256(b);
  cudaMemPool_t mp = pool(dev);
  if (!mp) {
    delete x;
    return fail(SRK_ECUDA, "cannot create the device memory pool");
  }
  cudaError_t e = cudaMallocFromPoolAsync(&x->block, total, mp, st);
  if (e != cudaSuccess) {
    x->block = nullptr;
    free_ctx(x, st);
    return cuda_fail(e, "srk_linear_fwd: allocation");
  }
  {
    char *p = (char *)x->block;
    void **dst[8] = {(void **)&x->Pe,   (void **)&x->PeT,  (void **)&x->Wa,
                     (void **)&x->y,    (void **)&x->h,    (void **)&x->part,
                     (void **)&x->done, (void **)&x->bad};
    for (int i = 0; i < 8; ++i) {
      *dst[i] = p;
      p += up256(sizes[i]);
    }
  }
  const int gn = grid_of((int64_t)n, 256, dev), gm = grid_of(g->m, 256, dev);
  const float fc = (float)c, d = (float)(1.0 - c);
  cudaMemsetAsync(x->done, 0, sizeof(int32_t) * cap, st);
  cudaMemsetAsync(x->bad, 0, sizeof(int), st);
  // W_a (FP32 sums in a fixed order), then P in in-list and in out-list order
  segmented<float>(x, g->row_ptr, topo->in, WeightVal{edge_w}, WriteVec{x->Wa}, st);
  if (g->m > 0) {
    k_lin_pe<<<gm, 256, 0, st>>>(edge_w, topo->erow, x->Wa, g->m, x->Pe, x->bad);
    k_gather_f32<<<gm, 256, 0, st>>>(x->Pe, topo->t_e, g->m, x->PeT);
  }
  float *const y = x->y, *const h = x->h;
  k_lin_unit<<<gn, 256, 0, st>>>(y, g->n, s);
  for (int t = 1; t <= L; ++t) gather_p(x, y + (t - 1) * n, 1.0f, y + t * n, st);  // y_t = P y_{t-1}
  // h_L = D y_L, then h_t = D y_t + c P^T h_{t+1}
  k_lin_scale<<<gn, 256, 0, st>>>(y + L * n, d, g->n, h + L * n);
  for (int t = L - 1; t >= 0; --t) gather_t(x, h + (t + 1) * n, y + t * n, d, fc, h + t * n, st);
  // s_out = h_0
  e = cudaMemcpyAsync(s_out, h, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
  int hbad = 0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, x->bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_ctx(x, st);
    return cuda_fail(e, "srk_linear_fwd");
  }
  if (hbad) {
    free_ctx(x, st);
    return fail(SRK_EINVAL, "edge weights must be positive and finite");
  }
  if (ctx_out) *ctx_out = x;
  else free_ctx(x, st);
  return SRK_OK;
}

extern "C" int srk_linear_bwd(srk_linear_ctx *x, const float *grad_s, float *grad_w,
                              void *cuda_stream) {
  clear_error();
  if (!x) return fail(SRK_EINVAL, "null context");
  if (!grad_s || (!grad_w && x->m > 0)) return fail(SRK_EINVAL, "null gradient pointer");
  DeviceGuard guard(x->device);
  if (!is_device_ptr(grad_s) || (x->m > 0 && !is_device_ptr(grad_w)))
    return fail(SRK_EINVAL, "srk_linear_bwd takes device pointers");
  const srk_graph *g = x->g;
  const srk_lin_topo *topo = x->topo;
  const int dev = x->device;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)x->n;
  const int L = x->L;
  const int32_t S = L + 1;
  const size_t vec = (size_t)S * n;
  cudaMemPool_t mp = pool(dev);
  if (!mp) return fail(SRK_ECUDA, "cannot create the device memory pool");
  float *gb = nullptr;
  // gb, yb (term-major), the rows of pairs (2 L n floats) and T_a
  cudaError_t e = cudaMallocFromPoolAsync((void **)&gb, sizeof(float) * (4 * vec + n), mp, st);
  if (e != cudaSuccess) return cuda_fail(e, "srk_linear_bwd: allocation");
  float *yb = gb + vec, *T = gb + 2 * vec;
  float2 *hy = reinterpret_cast<float2 *>(gb + 2 * vec + n + (n & 1));
  const int gn = grid_of((int64_t)n, 256, dev), gm = grid_of(x->m, 256, dev);
  const float fc = (float)x->c, d = (float)(1.0 - x->c);
  // gb_0 = g
  cudaMemcpyAsync(gb, grad_s, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
  for (int t = 1; t <= L; ++t) gather_p(x, gb + (t - 1) * n, fc, gb + t * n, st);  // gb_t = c P gb_{t-1}
  if (L >= 1) {
    // yb_L = D gb_L, yb_t = D gb_t + P^T yb_{t+1} for t = L-1 .. 1 (yb_0 is not used)
    cudaMemsetAsync(yb, 0, sizeof(float) * n, st);
    k_lin_scale<<<gn, 256, 0, st>>>(gb + L * n, d, x->n, yb + L * n);
    for (int t = L - 1; t >= 1; --t)
      gather_t(x, yb + (t + 1) * n, gb + t * n, d, 1.0f, yb + t * n, st);
  }
  if (x->m > 0) {
    if (L >= 1) {
      // the rows of pairs (h_{t+1}, yb_{t+1}), G_e into grad_w, T_a = sum
      // G_e P_e per in-list, then the normalisation
      const size_t tile = sizeof(float) * 66 * (size_t)L;
      if (tile > 48 * 1024)
        cudaFuncSetAttribute(k_lin_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile);
      k_lin_pairs<<<(int)((n + 31) / 32), 256, tile, st>>>(x->h, yb, L, x->n, hy);
      k_lin_edge_G<<<gm, 256, 0, st>>>(topo->erow, g->col, x->m, x->n, x->y, hy, gb, L, fc,
                                       grad_w);
      segmented<float>(x, g->row_ptr, topo->in, DotVal{grad_w, x->Pe}, WriteVec{T}, st);
      k_lin_edge_fin<<<gm, 256, 0, st>>>(topo->erow, x->m, T, x->Wa, grad_w);
    } else {
      cudaMemsetAsync(grad_w, 0, sizeof(float) * (size_t)x->m, st);  // s_vec = D e_s
    }
  }
  e = cudaGetLastError();
  cudaFreeAsync(gb, st);
  if (e != cudaSuccess) return cuda_fail(e, "srk_linear_bwd");
  return SRK_OK;
}
