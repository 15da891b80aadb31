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
// P v (a scatter along in-lists) accumulates in FP64 with atomics, so its
// result does not depend on the order of the additions beyond FP64 rounding;
// P^T v (a gather along in-lists: one warp per node, one block per node whose
// in-list is long) is deterministic.  The vectors are stored node-major,
// n x (L+1), so the per-edge gradient pass reads each node's L values
// together.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "srk_internal.h"

struct srk_linear_ctx {
  const srk_graph *g = nullptr;
  int device = 0;
  int32_t n = 0, L = 0, s = 0;
  int64_t m = 0;
  double c = 0.0;
  float *Pe = nullptr;     // m: w_e / W_a
  float *Wa = nullptr;     // n: in-weight sums
  int32_t *erow = nullptr; // m: the node whose in-list holds edge e
  float *y = nullptr;      // n x (L+1), node-major: y[a (L+1) + t] = (P^t e_s)[a]
  float *h = nullptr;      // n x (L+1), node-major partial sums, h_0 = s_vec
  double *acc = nullptr;   // n: scatter accumulator (zero between uses)
  int32_t *longs = nullptr;  // nodes whose in-list is longer than kLongRow
  int32_t *n_long = nullptr; // their count (device)
  int *bad = nullptr;      // weight check flag
  void *block = nullptr;   // the device block all arrays above live in
};

namespace srk {

// In-lists longer than this are reduced by a whole block instead of a warp,
// so the hubs of a power-law graph do not serialise on one warp.
constexpr int32_t kLongRow = 256;
constexpr int kLongBlock = 1024;
// Short in-lists are handled by groups of kGroup lanes (4 lists per warp):
// in-lists average ~16 entries, so a whole warp per list would idle most
// lanes and serialise the lists' load latencies.
constexpr int kGroup = 8;

// Fixed-order reductions (the result does not depend on timing).
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
template <class T>
__device__ __forceinline__ T block_sum(T v, T *sh) {  // blockDim.x == kLongBlock
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = 0;
  if (wid == 0) {
    t = (lane < kLongBlock / 32) ? sh[lane] : (T)0;
    t = warp_sum(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  return sh[0];
}

// Nodes with long in-lists (order of the list does not matter: each node's
// result is computed independently).
__global__ void k_lin_classify(const int32_t *__restrict__ row_ptr, int32_t n,
                               int32_t *__restrict__ longs, int32_t *n_long) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x)
    if (row_ptr[a + 1] - row_ptr[a] > kLongRow) longs[atomicAdd(n_long, 1)] = (int32_t)a;
}

// W_a, P_e = w_e / W_a and erow for one node; flags weights that are not
// positive and finite.  Warp version (short lists) and block version.
__device__ __forceinline__ double prep_partial(const float *w, int32_t b, int32_t e, int32_t a,
                                               int32_t *erow, int *bad, int tid, int nthr) {
  double sum = 0.0;
  for (int32_t k = b + tid; k < e; k += nthr) {
    const float x = w[k];
    if (!(x > 0.0f) || !isfinite(x)) *bad = 1;
    sum += (double)x;
    erow[k] = a;
  }
  return sum;
}

// Group loops: every lane of the warp runs the same number of iterations, so
// the group shuffles see all 32 lanes; nodes past n and long lists are empty.
#define SRK_GROUP_LOOP(n)                                                         \
  const int gl = threadIdx.x & (kGroup - 1);                                      \
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / kGroup;              \
  const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kGroup; \
  const int64_t warp_first = first - ((threadIdx.x & 31) / kGroup);               \
  for (int64_t base = warp_first; base < (n); base += groups)

__global__ void k_lin_prep(const int32_t *__restrict__ row_ptr, const float *__restrict__ w,
                           int32_t n, float *__restrict__ Pe, float *__restrict__ Wa,
                           int32_t *__restrict__ erow, int *bad) {
  SRK_GROUP_LOOP(n) {
    const int64_t a = base + ((threadIdx.x & 31) / kGroup);
    int32_t b = 0, e = 0;
    if (a < n) {
      b = row_ptr[a];
      e = row_ptr[a + 1];
      if (e - b > kLongRow) e = b;
    }
    const double sum = group_sum(prep_partial(w, b, e, (int32_t)a, erow, bad, gl, kGroup));
    for (int32_t k = b + gl; k < e; k += kGroup) Pe[k] = (float)((double)w[k] / sum);
    if (gl == 0 && e > b) Wa[a] = (float)sum;
  }
}

__global__ void __launch_bounds__(kLongBlock)
k_lin_prep_long(const int32_t *__restrict__ row_ptr, const float *__restrict__ w,
                const int32_t *__restrict__ longs, const int32_t *n_long,
                float *__restrict__ Pe, float *__restrict__ Wa,
                int32_t *__restrict__ erow, int *bad) {
  __shared__ double sh[kLongBlock / 32];
  const int32_t nl = *n_long;
  for (int32_t q = blockIdx.x; q < nl; q += gridDim.x) {
    const int32_t a = longs[q];
    const int32_t b = row_ptr[a], e = row_ptr[a + 1];
    const double sum =
        block_sum(prep_partial(w, b, e, a, erow, bad, threadIdx.x, kLongBlock), sh);
    for (int32_t k = b + threadIdx.x; k < e; k += kLongBlock) Pe[k] = (float)((double)w[k] / sum);
    if (threadIdx.x == 0) Wa[a] = (float)sum;
  }
}

// v[a] = (a == s) for a node-major vector column (stride S).
__global__ void k_lin_unit(float *__restrict__ v, int32_t S, int32_t n, int32_t s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i * S] = (i == s) ? 1.0f : 0.0f;
}

// acc[u] += P_e v[a] for every edge e = (u -> a); v is a column of stride S.
__global__ void k_lin_scatter(const float *__restrict__ v, int32_t S,
                              const float *__restrict__ Pe, const int32_t *__restrict__ col,
                              const int32_t *__restrict__ erow, int64_t m,
                              double *__restrict__ acc) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float va = v[(int64_t)erow[e] * S];
    if (va != 0.0f) atomicAdd(&acc[col[e]], (double)(Pe[e] * va));
  }
}

// out[u] = scale * acc[u] (column of stride S); acc[u] = 0.
__global__ void k_lin_finish(double *__restrict__ acc, float scale, int32_t n, int32_t S,
                             float *__restrict__ out) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    out[u * S] = (float)(acc[u] * (double)scale);
    acc[u] = 0.0;
  }
}

// out[a] = alpha add[a] + beta sum_{e in I(a)} P_e in[u_e], all three columns
// of stride S: one warp per short in-list, one block per long in-list.
__device__ __forceinline__ float gather_partial(const int32_t *col, const float *Pe,
                                                const float *in, int32_t S, int32_t b,
                                                int32_t e, int tid, int nthr) {
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
  int32_t k = b + tid;
  for (; k + 3 * nthr < e; k += 4 * nthr) {  // four independent loads in flight
    s0 = fmaf(Pe[k], in[(int64_t)col[k] * S], s0);
    s1 = fmaf(Pe[k + nthr], in[(int64_t)col[k + nthr] * S], s1);
    s2 = fmaf(Pe[k + 2 * nthr], in[(int64_t)col[k + 2 * nthr] * S], s2);
    s3 = fmaf(Pe[k + 3 * nthr], in[(int64_t)col[k + 3 * nthr] * S], s3);
  }
  for (; k < e; k += nthr) s0 = fmaf(Pe[k], in[(int64_t)col[k] * S], s0);
  return (s0 + s1) + (s2 + s3);
}

__global__ void k_lin_gather(const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col,
                             const float *__restrict__ Pe, const float *__restrict__ in,
                             const float *__restrict__ add, float alpha, float beta,
                             int32_t n, int32_t S, float *__restrict__ out) {
  SRK_GROUP_LOOP(n) {
    const int64_t a = base + ((threadIdx.x & 31) / kGroup);
    int32_t b = 0, e = 0;
    if (a < n) {
      b = row_ptr[a];
      e = row_ptr[a + 1];
      if (e - b > kLongRow) e = b - 1;  // handled by the long-list kernel
    }
    const float sum = group_sum(gather_partial(col, Pe, in, S, b, e > b ? e : b, gl, kGroup));
    if (gl == 0 && a < n && e >= b) out[a * S] = alpha * add[a * S] + beta * sum;
  }
}

__global__ void __launch_bounds__(kLongBlock)
k_lin_gather_long(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                  const float *__restrict__ Pe, const float *__restrict__ in,
                  const float *__restrict__ add, float alpha, float beta, int32_t S,
                  const int32_t *__restrict__ longs, const int32_t *n_long,
                  float *__restrict__ out) {
  __shared__ float sh[kLongBlock / 32];
  const int32_t nl = *n_long;
  for (int32_t q = blockIdx.x; q < nl; q += gridDim.x) {
    const int32_t a = longs[q];
    const float sum = block_sum(
        gather_partial(col, Pe, in, S, row_ptr[a], row_ptr[a + 1], threadIdx.x, kLongBlock), sh);
    if (threadIdx.x == 0) out[(int64_t)a * S] = alpha * add[(int64_t)a * S] + beta * sum;
  }
}

// Edge gradients of node a's in-list: G_e, then the normalisation term.
// Node-major vectors: the L values of h and yb a source node needs are
// contiguous, and so are the values of gb and y the node a needs.
__device__ __forceinline__ float edge_G(const float *y, const float *h, const float *gb,
                                        const float *yb, int32_t S, int32_t L, float c,
                                        int64_t a, int64_t u) {
  const float *ga = gb + a * S, *ya = y + a * S, *hu = h + u * S, *ybu = yb + u * S;
  float G = 0.0f;
  for (int t = 0; t < L; ++t) {
    G = fmaf(c * ga[t], hu[t + 1], G);
    G = fmaf(ybu[t + 1], ya[t], G);
  }
  return G;
}

__global__ void k_lin_edge_grad(const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col,
                                const float *__restrict__ Pe, const float *__restrict__ Wa,
                                const float *__restrict__ y, const float *__restrict__ h,
                                const float *__restrict__ gb, const float *__restrict__ yb,
                                int32_t L, int32_t n, float c, float *__restrict__ grad) {
  const int32_t S = L + 1;
  SRK_GROUP_LOOP(n) {
    const int64_t a = base + ((threadIdx.x & 31) / kGroup);
    int32_t b = 0, e = 0;
    if (a < n) {
      b = row_ptr[a];
      e = row_ptr[a + 1];
      if (e - b > kLongRow) e = b;
    }
    float T = 0.0f;
    for (int32_t k = b + gl; k < e; k += kGroup) {
      const float G = edge_G(y, h, gb, yb, S, L, c, a, col[k]);
      grad[k] = G;
      T = fmaf(G, Pe[k], T);
    }
    T = group_sum(T);
    if (e > b) {
      const float inv = 1.0f / Wa[a];
      for (int32_t k = b + gl; k < e; k += kGroup) grad[k] = (grad[k] - T) * inv;
    }
  }
}

__global__ void __launch_bounds__(kLongBlock)
k_lin_edge_grad_long(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                     const float *__restrict__ Pe, const float *__restrict__ Wa,
                     const float *__restrict__ y, const float *__restrict__ h,
                     const float *__restrict__ gb, const float *__restrict__ yb, int32_t L,
                     float c, const int32_t *__restrict__ longs, const int32_t *n_long,
                     float *__restrict__ grad) {
  __shared__ float sh[kLongBlock / 32];
  const int32_t S = L + 1;
  const int32_t nl = *n_long;
  for (int32_t q = blockIdx.x; q < nl; q += gridDim.x) {
    const int32_t a = longs[q];
    const int32_t b = row_ptr[a], e = row_ptr[a + 1];
    float T = 0.0f;
    for (int32_t k = b + threadIdx.x; k < e; k += kLongBlock) {
      const float G = edge_G(y, h, gb, yb, S, L, c, a, col[k]);
      grad[k] = G;
      T = fmaf(G, Pe[k], T);
    }
    T = block_sum(T, sh);
    const float inv = 1.0f / Wa[a];
    for (int32_t k = b + threadIdx.x; k < e; k += kLongBlock) grad[k] = (grad[k] - T) * inv;
  }
}

static int grid_of(int64_t work, int per_block, int dev) {
  const int64_t want = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)sm_count(dev) * 16;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

// The context's device memory is one block from the library's stream-ordered
// pool, carved into its arrays.
static void free_ctx(srk_linear_ctx *x, cudaStream_t st = nullptr) {
  if (!x) return;
  DeviceGuard guard(x->device);
  if (x->block) cudaFreeAsync(x->block, st);
  delete x;
}

// out = alpha add + beta P^T in (columns of stride S): short and long lists.
static void gather(const srk_linear_ctx *x, const float *in, const float *add, float alpha,
                   float beta, float *out, cudaStream_t st) {
  const srk_graph *g = x->g;
  const int32_t S = x->L + 1;
  const int gw = grid_of((int64_t)x->n * kGroup, 256, x->device);
  k_lin_gather<<<gw, 256, 0, st>>>(g->row_ptr, g->col, x->Pe, in, add, alpha, beta, x->n, S,
                                   out);
  k_lin_gather_long<<<sm_count(x->device) * 2, kLongBlock, 0, st>>>(
      g->row_ptr, g->col, x->Pe, in, add, alpha, beta, S, x->longs, x->n_long, out);
}

// out = scale P in (columns of stride S), through the FP64 accumulator.
static void scatter(const srk_linear_ctx *x, const float *in, float scale, float *out,
                    cudaStream_t st) {
  const srk_graph *g = x->g;
  const int32_t S = x->L + 1;
  const int gm = grid_of(x->m, 256, x->device), gn = grid_of(x->n, 256, x->device);
  k_lin_scatter<<<gm, 256, 0, st>>>(in, S, x->Pe, g->col, x->erow, x->m, x->acc);
  k_lin_finish<<<gn, 256, 0, st>>>(x->acc, scale, x->n, S, out);
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
  if (!edge_w) return fail(SRK_EINVAL, "no edge weights: pass edge_w or load the graph with them");
  if (s < 0 || s >= g->n) return fail(SRK_EINVAL, "source %d outside [0, %d)", s, g->n);
  if (!(c > 0.0 && c < 1.0)) return fail(SRK_EINVAL, "c = %g outside (0, 1)", c);
  if (L < 0 || L > SRK_MAX_LEN) return fail(SRK_EINVAL, "L = %d outside [0, %d]", L, SRK_MAX_LEN);
  if (!s_out) return fail(SRK_EINVAL, "s_out is null");
  DeviceGuard guard(g->device);
  if ((g->m > 0 && !is_device_ptr(edge_w)) || !is_device_ptr(s_out))
    return fail(SRK_EINVAL, "srk_linear_fwd takes device pointers for edge_w and s_out");
  const int dev = g->device;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  srk_linear_ctx *x = new srk_linear_ctx;
  x->g = g;
  x->device = dev;
  x->n = g->n;
  x->m = g->m;
  x->L = L;
  x->s = s;
  x->c = c;
  const size_t n = (size_t)g->n, m = (size_t)(g->m > 0 ? g->m : 1);
  const int32_t S = L + 1;
  const size_t vec = (size_t)S * n;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t sizes[9] = {sizeof(float) * m, sizeof(float) * n, sizeof(int32_t) * m,
                           sizeof(float) * vec, sizeof(float) * vec, sizeof(double) * n,
                           sizeof(int32_t) * n, sizeof(int32_t), sizeof(int)};
  size_t total = 0;
  for (size_t b : sizes) total += up(b);
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
    void **dst[9] = {(void **)&x->Pe, (void **)&x->Wa, (void **)&x->erow, (void **)&x->y,
                     (void **)&x->h, (void **)&x->acc, (void **)&x->longs,
                     (void **)&x->n_long, (void **)&x->bad};
    for (int i = 0; i < 9; ++i) {
      *dst[i] = p;
      p += up(sizes[i]);
    }
  }
  const int gn = grid_of((int64_t)n, 256, dev), gw = grid_of((int64_t)n * kGroup, 256, dev);
  const float fc = (float)c, d = (float)(1.0 - c);
  e = cudaSuccess;
  cudaMemsetAsync(x->acc, 0, sizeof(double) * n, st);
  cudaMemsetAsync(x->bad, 0, sizeof(int), st);
  cudaMemsetAsync(x->n_long, 0, sizeof(int32_t), st);
  k_lin_classify<<<gn, 256, 0, st>>>(g->row_ptr, g->n, x->longs, x->n_long);
  k_lin_prep<<<gw, 256, 0, st>>>(g->row_ptr, edge_w, g->n, x->Pe, x->Wa, x->erow, x->bad);
  k_lin_prep_long<<<sm_count(dev) * 2, kLongBlock, 0, st>>>(g->row_ptr, edge_w, x->longs,
                                                            x->n_long, x->Pe, x->Wa, x->erow,
                                                            x->bad);
  k_lin_unit<<<gn, 256, 0, st>>>(x->y, S, g->n, s);
  for (int t = 1; t <= L; ++t) scatter(x, x->y + (t - 1), 1.0f, x->y + t, st);  // y_t = P y_{t-1}
  // h_L = D y_L (a gather with beta = 0), then h_t = D y_t + c P^T h_{t+1}
  gather(x, x->y + L, x->y + L, d, 0.0f, x->h + L, st);
  for (int t = L - 1; t >= 0; --t) gather(x, x->h + (t + 1), x->y + t, d, fc, x->h + t, st);
  // s_out = column 0 of h (stride S)
  e = cudaMemcpy2DAsync(s_out, sizeof(float), x->h, sizeof(float) * S, sizeof(float), n,
                        cudaMemcpyDeviceToDevice, st);
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
  if (!grad_s || !grad_w) return fail(SRK_EINVAL, "null gradient pointer");
  DeviceGuard guard(x->device);
  if (!is_device_ptr(grad_s) || (x->m > 0 && !is_device_ptr(grad_w)))
    return fail(SRK_EINVAL, "srk_linear_bwd takes device pointers");
  const srk_graph *g = x->g;
  const int dev = x->device;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)x->n;
  const int L = x->L;
  const int32_t S = L + 1;
  const size_t vec = (size_t)S * n;
  cudaMemPool_t mp = pool(dev);
  if (!mp) return fail(SRK_ECUDA, "cannot create the device memory pool");
  float *gb = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void **)&gb, sizeof(float) * 2 * vec, mp, st);
  if (e != cudaSuccess) return cuda_fail(e, "srk_linear_bwd: allocation");
  float *yb = gb + vec;
  const int gw = grid_of((int64_t)n * kGroup, 256, dev);
  const float fc = (float)x->c, d = (float)(1.0 - x->c);
  // gb column 0 = g (stride S)
  cudaMemcpy2DAsync(gb, sizeof(float) * S, grad_s, sizeof(float), sizeof(float), n,
                    cudaMemcpyDeviceToDevice, st);
  for (int t = 1; t <= L; ++t) scatter(x, gb + (t - 1), fc, gb + t, st);  // gb_t = c P gb_{t-1}
  if (L >= 1) {
    // yb_L = D gb_L, yb_t = D gb_t + P^T yb_{t+1} for t = L-1 .. 1
    gather(x, gb + L, gb + L, d, 0.0f, yb + L, st);
    for (int t = L - 1; t >= 1; --t) gather(x, yb + (t + 1), gb + t, d, 1.0f, yb + t, st);
  }
  if (x->m > 0) {
    if (L >= 1) {
      k_lin_edge_grad<<<gw, 256, 0, st>>>(g->row_ptr, g->col, x->Pe, x->Wa, x->y, x->h, gb, yb,
                                          L, x->n, fc, grad_w);
      k_lin_edge_grad_long<<<sm_count(dev) * 2, kLongBlock, 0, st>>>(
          g->row_ptr, g->col, x->Pe, x->Wa, x->y, x->h, gb, yb, L, fc, x->longs, x->n_long,
          grad_w);
    } else {
      cudaMemsetAsync(grad_w, 0, sizeof(float) * (size_t)x->m, st);  // s_vec = D e_s
    }
  }
  e = cudaGetLastError();
  cudaFreeAsync(gb, st);
  if (e != cudaSuccess) return cuda_fail(e, "srk_linear_bwd");
  return SRK_OK;
}
