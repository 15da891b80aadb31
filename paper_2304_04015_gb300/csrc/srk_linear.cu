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
// P^T v (a gather along in-lists, one warp per node) is deterministic.
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
  float *y = nullptr;      // (L+1) x n: P^t e_s
  float *h = nullptr;      // (L+1) x n: partial sums, h_0 = s_vec
  double *acc = nullptr;   // n: scatter accumulator (zero between uses)
  int *bad = nullptr;      // weight check flag
};

namespace srk {

// Per node a (one warp): W_a, P_e = w_e / W_a and erow; flags weights that are
// not positive and finite.
__global__ void k_lin_prep(const int32_t *__restrict__ row_ptr, const float *__restrict__ w,
                           int32_t n, float *__restrict__ Pe, float *__restrict__ Wa,
                           int32_t *__restrict__ erow, int *bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
    const int32_t b = row_ptr[a], e = row_ptr[a + 1];
    double sum = 0.0;
    for (int32_t k = b + lane; k < e; k += 32) {
      const float x = w[k];
      if (!(x > 0.0f) || !isfinite(x)) *bad = 1;
      sum += (double)x;
      erow[k] = (int32_t)a;
    }
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    for (int32_t k = b + lane; k < e; k += 32) Pe[k] = (float)((double)w[k] / sum);
    if (lane == 0) Wa[a] = (float)sum;
  }
}

__global__ void k_lin_unit(float *__restrict__ v, int32_t n, int32_t s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (i == s) ? 1.0f : 0.0f;
}

// acc[u] += P_e v[a] for every edge e = (u -> a).
__global__ void k_lin_scatter(const float *__restrict__ v, const float *__restrict__ Pe,
                              const int32_t *__restrict__ col,
                              const int32_t *__restrict__ erow, int64_t m,
                              double *__restrict__ acc) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float va = v[erow[e]];
    if (va != 0.0f) atomicAdd(&acc[col[e]], (double)(Pe[e] * va));
  }
}

// out[u] = scale * acc[u]; acc[u] = 0.
__global__ void k_lin_finish(double *__restrict__ acc, float scale, int32_t n,
                             float *__restrict__ out) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    out[u] = (float)(acc[u] * (double)scale);
    acc[u] = 0.0;
  }
}

// out[a] = alpha add[a] + beta sum_{e in I(a)} P_e in[u_e] (one warp per node).
__global__ void k_lin_gather(const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col,
                             const float *__restrict__ Pe, const float *__restrict__ in,
                             const float *__restrict__ add, float alpha, float beta,
                             int32_t n, float *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
    const int32_t b = row_ptr[a], e = row_ptr[a + 1];
    float sum = 0.0f;
    for (int32_t k = b + lane; k < e; k += 32) sum = fmaf(Pe[k], in[col[k]], sum);
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) out[a] = alpha * add[a] + beta * sum;
  }
}

// Edge gradients (one warp per node a): G_e, then the normalisation term.
__global__ void k_lin_edge_grad(const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col,
                                const float *__restrict__ Pe, const float *__restrict__ Wa,
                                const float *__restrict__ y, const float *__restrict__ h,
                                const float *__restrict__ gb, const float *__restrict__ yb,
                                int32_t L, int32_t n, float c, float *__restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
    const int32_t b = row_ptr[a], e = row_ptr[a + 1];
    if (e == b) continue;
    float T = 0.0f;
    for (int32_t k = b + lane; k < e; k += 32) {
      const int32_t u = col[k];
      float G = 0.0f;
      for (int t = 0; t < L; ++t) {
        const size_t ot = (size_t)t * n, o1 = (size_t)(t + 1) * n;
        G = fmaf(c * gb[ot + a], h[o1 + u], G);
        G = fmaf(yb[o1 + u], y[ot + a], G);
      }
      grad[k] = G;
      T = fmaf(G, Pe[k], T);
    }
    for (int off = 16; off > 0; off >>= 1) T += __shfl_xor_sync(0xffffffffu, T, off);
    const float inv = 1.0f / Wa[a];
    for (int32_t k = b + lane; k < e; k += 32) grad[k] = (grad[k] - T) * inv;
  }
}

static int grid_of(int64_t work, int per_block, int dev) {
  const int64_t want = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)sm_count(dev) * 16;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

static void free_ctx(srk_linear_ctx *x) {
  if (!x) return;
  DeviceGuard guard(x->device);
  cudaFree(x->Pe);
  cudaFree(x->Wa);
  cudaFree(x->erow);
  cudaFree(x->y);
  cudaFree(x->h);
  cudaFree(x->acc);
  cudaFree(x->bad);
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
  const size_t vec = (size_t)(L + 1) * n;
  cudaError_t e;
  if ((e = cudaMalloc(&x->Pe, sizeof(float) * m)) != cudaSuccess ||
      (e = cudaMalloc(&x->Wa, sizeof(float) * n)) != cudaSuccess ||
      (e = cudaMalloc(&x->erow, sizeof(int32_t) * m)) != cudaSuccess ||
      (e = cudaMalloc(&x->y, sizeof(float) * vec)) != cudaSuccess ||
      (e = cudaMalloc(&x->h, sizeof(float) * vec)) != cudaSuccess ||
      (e = cudaMalloc(&x->acc, sizeof(double) * n)) != cudaSuccess ||
      (e = cudaMalloc(&x->bad, sizeof(int))) != cudaSuccess) {
    free_ctx(x);
    return cuda_fail(e, "srk_linear_fwd: allocation");
  }
  const int gn = grid_of((int64_t)n, 256, dev), gw = grid_of((int64_t)n * 32, 256, dev),
            gm = grid_of((int64_t)g->m, 256, dev);
  const float fc = (float)c, d = (float)(1.0 - c);
  cudaMemsetAsync(x->acc, 0, sizeof(double) * n, st);
  cudaMemsetAsync(x->bad, 0, sizeof(int), st);
  k_lin_prep<<<gw, 256, 0, st>>>(g->row_ptr, edge_w, g->n, x->Pe, x->Wa, x->erow, x->bad);
  k_lin_unit<<<gn, 256, 0, st>>>(x->y, g->n, s);
  for (int t = 1; t <= L; ++t) {  // y_t = P y_{t-1}
    k_lin_scatter<<<gm, 256, 0, st>>>(x->y + (size_t)(t - 1) * n, x->Pe, g->col, x->erow,
                                      g->m, x->acc);
    k_lin_finish<<<gn, 256, 0, st>>>(x->acc, 1.0f, g->n, x->y + (size_t)t * n);
  }
  // h_L = D y_L (a gather with beta = 0), then h_t = D y_t + c P^T h_{t+1}
  k_lin_gather<<<gw, 256, 0, st>>>(g->row_ptr, g->col, x->Pe, x->y + (size_t)L * n,
                                   x->y + (size_t)L * n, d, 0.0f, g->n, x->h + (size_t)L * n);
  for (int t = L - 1; t >= 0; --t)
    k_lin_gather<<<gw, 256, 0, st>>>(g->row_ptr, g->col, x->Pe, x->h + (size_t)(t + 1) * n,
                                     x->y + (size_t)t * n, d, fc, g->n, x->h + (size_t)t * n);
  e = cudaMemcpyAsync(s_out, x->h, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
  int hbad = 0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, x->bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_ctx(x);
    return cuda_fail(e, "srk_linear_fwd");
  }
  if (hbad) {
    free_ctx(x);
    return fail(SRK_EINVAL, "edge weights must be positive and finite");
  }
  if (ctx_out) *ctx_out = x;
  else free_ctx(x);
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
  const size_t vec = (size_t)(L + 1) * n;
  cudaMemPool_t mp = pool(dev);
  if (!mp) return fail(SRK_ECUDA, "cannot create the device memory pool");
  float *gb = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void **)&gb, sizeof(float) * 2 * vec, mp, st);
  if (e != cudaSuccess) return cuda_fail(e, "srk_linear_bwd: allocation");
  float *yb = gb + vec;
  const int gn = grid_of((int64_t)n, 256, dev), gw = grid_of((int64_t)n * 32, 256, dev),
            gm = grid_of(x->m, 256, dev);
  const float fc = (float)x->c, d = (float)(1.0 - x->c);
  cudaMemcpyAsync(gb, grad_s, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
  for (int t = 1; t <= L; ++t) {  // gb_t = c P gb_{t-1}
    k_lin_scatter<<<gm, 256, 0, st>>>(gb + (size_t)(t - 1) * n, x->Pe, g->col, x->erow, x->m,
                                      x->acc);
    k_lin_finish<<<gn, 256, 0, st>>>(x->acc, fc, x->n, gb + (size_t)t * n);
  }
  if (L >= 1) {
    // yb_L = D gb_L, yb_t = D gb_t + P^T yb_{t+1} for t = L-1 .. 1
    k_lin_gather<<<gw, 256, 0, st>>>(g->row_ptr, g->col, x->Pe, gb + (size_t)L * n,
                                     gb + (size_t)L * n, d, 0.0f, x->n, yb + (size_t)L * n);
    for (int t = L - 1; t >= 1; --t)
      k_lin_gather<<<gw, 256, 0, st>>>(g->row_ptr, g->col, x->Pe, yb + (size_t)(t + 1) * n,
                                       gb + (size_t)t * n, d, 1.0f, x->n, yb + (size_t)t * n);
  }
  if (x->m > 0) {
    if (L >= 1)
      k_lin_edge_grad<<<gw, 256, 0, st>>>(g->row_ptr, g->col, x->Pe, x->Wa, x->y, x->h, gb, yb,
                                          L, x->n, fc, grad_w);
    else
      cudaMemsetAsync(grad_w, 0, sizeof(float) * (size_t)x->m, st);  // s_vec = D e_s
  }
  e = cudaGetLastError();
  cudaFreeAsync(gb, st);
  if (e != cudaSuccess) return cuda_fail(e, "srk_linear_bwd");
  return SRK_OK;
}
