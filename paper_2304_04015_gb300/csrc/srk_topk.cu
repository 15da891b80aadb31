// srk_multi_source_topk: many single-source queries with a sparse output --
// per source, the `top` targets of largest score (the source itself left
// out), ties broken by the smaller node id, and the number of targets with a
// nonzero score.  A dense k x n score matrix (550 GB for 4,096 sources on a
// graph of 16.8M nodes) is never formed: the sources run in chunks whose rows
// fit a scratch budget, srk_multi_source fills the chunk's rows on the
// device, and the selection runs on those rows.
//
// Selection of one row (scores are non-negative doubles, whose IEEE bit
// patterns order like unsigned integers): eight radix-select passes over the
// 64-bit key, one byte per pass from the top, find the key T of the top-th
// largest entry and how many entries equal to T are still needed; then every
// entry above T is taken, and of the entries equal to T the ones with the
// smallest ids (a chunked scan keeps id order); a block sorts the selection by
// (score descending, id ascending).
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "srk_internal.h"

namespace srk {
namespace {

constexpr int kChunk = 65536;     // targets per block of the tie scan
constexpr int kMaxTop = 4096;     // largest `top` (the final sort is one block)

struct RowSel {
  unsigned long long prefix, mask;  // key bits fixed so far
  int64_t need;                     // entries still to take at or below the prefix
  int64_t nnz;                      // nonzero scores of the row (the source excluded)
  unsigned long long thr;           // final threshold key T
  int64_t take_eq;                  // entries equal to T to take
  int32_t n_gt;                     // entries above T (taken, in any order)
  int32_t pad;
};

__device__ __forceinline__ unsigned long long key_of(const double *row, int32_t u) {
  return (unsigned long long)__double_as_longlong(row[u]);
}

// Nonzero scores per row, the source excluded.
__global__ void k_topk_count(const double *__restrict__ rows, int64_t n, int32_t R,
                             const int32_t *__restrict__ src, RowSel *__restrict__ sel) {
  const int r = blockIdx.y;
  const double *row = rows + (int64_t)r * n;
  int64_t c = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    c += (u != src[r] && key_of(row, (int32_t)u) != 0ull) ? 1 : 0;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long *)&sel[r].nnz,
                                              (unsigned long long)c);
}

// Histogram of key byte `shift` over the row's candidates (nonzero keys
// matching the prefix so far).
__global__ void k_topk_hist(const double *__restrict__ rows, int64_t n,
                            const int32_t *__restrict__ src, const RowSel *__restrict__ sel,
                            int shift, unsigned int *__restrict__ hist) {
  __shared__ unsigned int h[256];
  const int r = blockIdx.y;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const RowSel S = sel[r];
  if (S.nnz > S.need || S.mask != 0ull) {  // rows with nnz <= top take every nonzero key
    const double *row = rows + (int64_t)r * n;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
      const unsigned long long k = key_of(row, (int32_t)u);
      if (k != 0ull && u != src[r] && (k & S.mask) == S.prefix)
        atomicAdd(&h[(k >> shift) & 255ull], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[r * 256 + i], h[i]);
}

// One thread per row: the byte at `shift` of the need-th largest candidate.
__global__ void k_topk_pick(int32_t R, int shift, unsigned int *__restrict__ hist,
                            RowSel *__restrict__ sel) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  RowSel &S = sel[r];
  unsigned int *h = hist + r * 256;
  if (S.nnz > S.need || S.mask != 0ull) {
    int64_t above = 0;
    int b = 255;
    for (; b > 0; --b) {
      if (above + (int64_t)h[b] >= S.need) break;
      above += h[b];
    }
    S.prefix |= (unsigned long long)b << shift;
    S.mask |= 255ull << shift;
    S.need -= above;
  }
  for (int i = 0; i < 256; ++i) h[i] = 0;
  if (shift == 0) {  // done: entries above T, then `need` entries equal to T
    if (S.mask == 0ull) {  // nnz <= top: every nonzero key, none by tie rank
      S.thr = 0ull;
      S.take_eq = 0;
    } else {
      S.thr = S.prefix;
      S.take_eq = S.need;
    }
  }
}

// Entries equal to T per chunk of the row (the tie scan's first half).
__global__ void k_topk_ties(const double *__restrict__ rows, int64_t n,
                            const int32_t *__restrict__ src, const RowSel *__restrict__ sel,
                            int32_t n_chunks, int32_t *__restrict__ ties) {
  const int r = blockIdx.y, ch = blockIdx.x;
  const RowSel S = sel[r];
  const double *row = rows + (int64_t)r * n;
  int c = 0;
  if (S.take_eq > 0) {
    const int64_t b = (int64_t)ch * kChunk, e = std::min<int64_t>(n, b + kChunk);
    for (int64_t u = b + threadIdx.x; u < e; u += blockDim.x)
      c += (u != src[r] && key_of(row, (int32_t)u) == S.thr) ? 1 : 0;
  }
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  __shared__ int ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    ties[r * n_chunks + ch] = t;
  }
}

// The selection: every entry above T (slots by atomics), then the entries
// equal to T in id order until take_eq are taken (each chunk knows how many
// ties precede it; inside the chunk a block-wide ordered scan ranks them).
__global__ void __launch_bounds__(256)
k_topk_collect(const double *__restrict__ rows, int64_t n, const int32_t *__restrict__ src,
               RowSel *__restrict__ sel, int32_t n_chunks, const int32_t *__restrict__ ties,
               int32_t top, unsigned long long *__restrict__ out_key,
               int32_t *__restrict__ out_id) {
  const int r = blockIdx.y, ch = blockIdx.x;
  const RowSel S = sel[r];
  const double *row = rows + (int64_t)r * n;
  __shared__ int64_t before;
  __shared__ int wsum[8];
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int c = 0; c < ch; ++c) t += ties[r * n_chunks + c];
    before = t;
  }
  __syncthreads();
  const int64_t n_gt_total = S.mask == 0ull ? S.nnz : (int64_t)top - S.take_eq;
  unsigned long long *ok = out_key + (int64_t)r * top;
  int32_t *oi = out_id + (int64_t)r * top;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t run = before;  // ties before this tile (same in every thread)
  const int64_t b = (int64_t)ch * kChunk, e = std::min<int64_t>(n, b + kChunk);
  for (int64_t t0 = b; t0 < e; t0 += blockDim.x) {
    const int64_t u = t0 + threadIdx.x;
    unsigned long long k = 0ull;
    bool valid = u < e && u != src[r];
    if (valid) k = key_of(row, (int32_t)u);
    if (valid && k > S.thr) {
      const int slot = atomicAdd(&sel[r].n_gt, 1);
      if (slot < n_gt_total && slot < top) {
        ok[slot] = k;
        oi[slot] = (int32_t)u;
      }
    }
    const bool tie = valid && S.take_eq > 0 && k == S.thr;
    const unsigned int bal = __ballot_sync(0xffffffffu, tie);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int64_t rank = run + __popc(bal & ((1u << lane) - 1u));
    int64_t tile = 0;
    for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
      if (x < w) rank += wsum[x];
      tile += wsum[x];
    }
    if (tie && rank < S.take_eq) {
      const int64_t slot = n_gt_total + rank;
      ok[slot] = k;
      oi[slot] = (int32_t)u;
    }
    run += tile;
    __syncthreads();
  }
}

// One block per row: sorts the row's selected entries by (key descending, id
// ascending) with a bitonic network in shared memory and writes the outputs
// (padding: node -1, score 0).
__global__ void __launch_bounds__(1024)
k_topk_sort(const RowSel *__restrict__ sel, int32_t top, int32_t P,
            const unsigned long long *__restrict__ in_key, const int32_t *__restrict__ in_id,
            const int32_t *__restrict__ dst_row, int32_t *__restrict__ top_nodes,
            double *__restrict__ top_scores, int32_t *__restrict__ top_count,
            int64_t *__restrict__ nnz_out) {
  extern __shared__ unsigned long long smk[];
  int32_t *smi = reinterpret_cast<int32_t *>(smk + P);
  const int r = blockIdx.x;
  const int64_t d = dst_row[r];  // the caller's row of this chunk row
  const RowSel S = sel[r];
  const int cnt = (int)std::min<int64_t>(S.nnz, (int64_t)top);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < cnt) {
      smk[i] = in_key[(int64_t)r * top + i];
      smi[i] = in_id[(int64_t)r * top + i];
    } else {
      smk[i] = 0ull;
      smi[i] = 0x7FFFFFFF;
    }
  }
  __syncthreads();
  // "a before b" when key_a > key_b, or equal keys and id_a < id_b
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool asc = (i & size) == 0;  // this run sorts into "before" order
          const unsigned long long ki = smk[i], kj = smk[j];
          const int32_t ii = smi[i], ij = smi[j];
          const bool j_first = kj > ki || (kj == ki && ij < ii);
          if (j_first == asc) {
            smk[i] = kj;
            smk[j] = ki;
            smi[i] = ij;
            smi[j] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < top; i += blockDim.x) {
    top_nodes[d * top + i] = i < cnt ? smi[i] : -1;
    top_scores[d * top + i] = i < cnt ? __longlong_as_double((long long)smk[i]) : 0.0;
  }
  if (threadIdx.x == 0) {
    if (top_count) top_count[d] = cnt;
    if (nnz_out) nnz_out[d] = S.nnz;
  }
}

}  // namespace
}  // namespace srk

using namespace srk;

extern "C" int srk_multi_source_topk(const srk_graph *g, const int32_t *sources, int32_t k,
                                     double c, const double *eps, uint64_t seed,
                                     const srk_opts *opt, int32_t top, int32_t *top_nodes,
                                     double *top_scores, int32_t *top_count, int64_t *nnz,
                                     void *cuda_stream) {
  clear_error();
  if (!g) return fail(SRK_EINVAL, "null graph");
  if (k < 0) return fail(SRK_EINVAL, "k = %d is negative", k);
  if (top < 1 || top > kMaxTop) return fail(SRK_EINVAL, "top = %d outside [1, %d]", top, kMaxTop);
  if (k == 0) return SRK_OK;
  if (!sources || !eps || !top_nodes || !top_scores)
    return fail(SRK_EINVAL, "null argument");
  DeviceGuard guard(g->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!is_device_ptr(top_nodes) || !is_device_ptr(top_scores) ||
      (top_count && !is_device_ptr(top_count)) || (nnz && !is_device_ptr(nnz)))
    return fail(SRK_EINVAL, "srk_multi_source_topk takes device output pointers");
  const int64_t n = g->n;
  // chunk of sources whose dense rows fit the scratch budget
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  size_t budget = std::max<size_t>((size_t)64 << 20, std::min<size_t>((size_t)16 << 30, free_b / 8));
  if (const char *env = getenv("SRK_TOPK_ROWS_BYTES")) {
    const unsigned long long v = strtoull(env, nullptr, 10);
    if (v > 0) budget = (size_t)v;
  }
  int32_t R = (int32_t)std::max<int64_t>(1, std::min<int64_t>(k, (int64_t)(budget / (8 * (size_t)n))));
  if (R >= 64 && R < k) R -= R % 64;  // whole batches of shared target walks
  const int32_t n_chunks = (int32_t)((n + kChunk - 1) / kChunk);
  int P = 1;
  while (P < top) P <<= 1;
  // scratch: rows, per-row state, histograms, tie counts, selection, sources
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t b_rows = al(8 * (size_t)R * n), b_sel = al(sizeof(RowSel) * R),
               b_hist = al(4 * 256 * (size_t)R), b_ties = al(4 * (size_t)R * n_chunks),
               b_key = al(8 * (size_t)R * top), b_id = al(4 * (size_t)R * top),
               b_src = al(4 * (size_t)R), b_dst = al(4 * (size_t)R);
  cudaMemPool_t mp = pool(g->device);
  if (!mp) return fail(SRK_ECUDA, "cannot create the device memory pool");
  char *base = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(
      (void **)&base, b_rows + b_sel + b_hist + b_ties + b_key + b_id + b_src + b_dst, mp, st);
  if (e != cudaSuccess) return cuda_fail(e, "srk_multi_source_topk: scratch");
  double *rows = (double *)base;
  RowSel *sel = (RowSel *)(base + b_rows);
  unsigned int *hist = (unsigned int *)((char *)sel + b_sel);
  int32_t *ties = (int32_t *)((char *)hist + b_hist);
  unsigned long long *skey = (unsigned long long *)((char *)ties + b_ties);
  int32_t *sid = (int32_t *)((char *)skey + b_key);
  int32_t *dsrc = (int32_t *)((char *)sid + b_id);
  int32_t *ddst = (int32_t *)((char *)dsrc + b_src);
  // the order the sources run in: as given, or, when they share target walks,
  // the sources with in-neighbours grouped by eps (descending, so by walk
  // budget) and the others last, so that a chunk's batches share as many
  // pairs as possible
  std::vector<int32_t> order((size_t)k);
  for (int32_t i = 0; i < k; ++i) order[(size_t)i] = i;
  if (opt && (opt->flags & SRK_OPT_SHARED_WALKS)) {
    for (int32_t i = 0; i < k; ++i)
      if (sources[i] < 0 || sources[i] >= g->n)
        return fail(SRK_EINVAL, "source %d (index %d) outside [0, %d)", sources[i], i, g->n);
    std::vector<int32_t> deg;
    const int rcd = source_in_degrees(g, sources, k, st, &deg);
    if (rcd) return rcd;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      const bool za = deg[(size_t)a] == 0, zb = deg[(size_t)b] == 0;
      if (za != zb) return zb;
      return eps[a] > eps[b];
    });
  }
  std::vector<int32_t> src_o((size_t)k);
  std::vector<double> eps_o((size_t)k);
  for (int32_t i = 0; i < k; ++i) {
    src_o[(size_t)i] = sources[order[(size_t)i]];
    eps_o[(size_t)i] = eps[order[(size_t)i]];
  }
  int rc = SRK_OK;
  srk_stats total;
  memset(&total, 0, sizeof total);
  srk_opts o;
  if (opt) o = *opt;
  else {
    memset(&o, 0, sizeof o);
    o.L_override = -1;
  }
  srk_stats part;
  const int sms = sm_count(g->device);
  for (int32_t i0 = 0; i0 < k && rc == SRK_OK; i0 += R) {
    const int32_t r = std::min(R, k - i0);
    o.stats = (opt && opt->stats) ? &part : nullptr;
    rc = srk_multi_source(g, src_o.data() + i0, r, c, eps_o.data() + i0, seed, &o, rows, nullptr,
                          st);
    if (rc) break;
    if (opt && opt->stats) {
      total.source_steps += part.source_steps;
      total.target_steps += part.target_steps;
      total.n_walks += part.n_walks;
      total.n_active_pairs += part.n_active_pairs;
      total.graph_updates += part.graph_updates;
      total.z = part.z;
      total.L = part.L;
      total.batch_shape = part.batch_shape;
    }
    std::vector<RowSel> h((size_t)r);
    for (auto &x : h) {
      memset(&x, 0, sizeof x);
      x.need = top;
    }
    if ((e = cudaMemcpyAsync(sel, h.data(), sizeof(RowSel) * r, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(dsrc, src_o.data() + i0, 4 * (size_t)r, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(ddst, order.data() + i0, 4 * (size_t)r, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemsetAsync(hist, 0, 4 * 256 * (size_t)r, st)) != cudaSuccess) {
      rc = cuda_fail(e, "srk_multi_source_topk: row state");
      break;
    }
    const dim3 grid_rows((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (int64_t)sms * 4)),
                         (unsigned)r);
    k_topk_count<<<grid_rows, 256, 0, st>>>(rows, n, r, dsrc, sel);
    for (int shift = 56; shift >= 0; shift -= 8) {
      k_topk_hist<<<grid_rows, 256, 0, st>>>(rows, n, dsrc, sel, shift, hist);
      k_topk_pick<<<(r + 127) / 128, 128, 0, st>>>(r, shift, hist, sel);
    }
    const dim3 grid_chunks((unsigned)n_chunks, (unsigned)r);
    k_topk_ties<<<grid_chunks, 256, 0, st>>>(rows, n, dsrc, sel, n_chunks, ties);
    k_topk_collect<<<grid_chunks, 256, 0, st>>>(rows, n, dsrc, sel, n_chunks, ties, top, skey, sid);
    const size_t smem = (size_t)P * (8 + 4);
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_topk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess) {
      rc = cuda_fail(e, "srk_multi_source_topk: sort shared memory");
      break;
    }
    k_topk_sort<<<r, 1024, smem, st>>>(sel, top, P, skey, sid, ddst, top_nodes, top_scores,
                                        top_count, nnz);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "srk_multi_source_topk: selection");
  }
  cudaFreeAsync(base, st);
  if (rc == SRK_OK && opt && opt->stats) *opt->stats = total;
  return rc;
}
