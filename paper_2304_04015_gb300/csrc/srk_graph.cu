// Graph residency, error reporting, memory pools and the sample-count table.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "srk_internal.h"

namespace srk {

static thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  const int code = (e == cudaErrorMemoryAllocation) ? SRK_ENOMEM : SRK_ECUDA;
  return fail(code, "%s: %s (%s)", what, cudaGetErrorString(e),
              cudaGetErrorName(e));
}

void clear_error() { g_last_error.clear(); }

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};
static int g_sms[64] = {};

cudaMemPool_t pool(int device) {
  if (device < 0 || device >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[device]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    // keep freed blocks cached for the next query
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[device] = p;
  }
  return g_pools[device];
}

int sm_count(int device) {
  if (device < 0 || device >= 64) return 1;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_sms[device]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess || v <= 0)
      v = 1;
    g_sms[device] = v;
  }
  return g_sms[device];
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Algorithm 1 line 3 (truncation), line 5 (N_i), Algorithm 2 line 2 (z, Z, Z^),
// Lemma 7 (a(l) = |Z_l| / |Z^_l|), Appendix B.5 (p, q).  FP64, evaluated in a
// fixed order (host code is built without floating-point contraction):
//   z   = ln(2 n^q) / (2 lambda^2),  lambda = eps - 3 / n^p
//   L   = floor(p ln n / (-ln sqrt(c)))
//   Z_l = z * (sqrt(c)^l * (1 - sqrt(c))),  N_l = ceil(Z_l),  a(l) = Z_l / N_l
int build_table(int32_t n, int32_t s, double c, double eps, uint64_t seed,
                const srk_opts *opt, QueryTab *t) {
  if (n < 1) return fail(SRK_EINVAL, "graph has no nodes");
  if (s < 0 || s >= n) return fail(SRK_EINVAL, "source %d outside [0, %d)", s, n);
  if (!(c > 0.0 && c < 1.0)) return fail(SRK_EINVAL, "c = %g outside (0, 1)", c);
  double p = 1.0, q = 1.0, z_ovr = 0.0;
  int32_t L_ovr = -1;
  const bool warmup = opt && (opt->flags & SRK_OPT_WARMUP_RULE);
  if (opt) {
    if (opt->p != 0.0) p = opt->p;
    if (opt->q != 0.0) q = opt->q;
    z_ovr = opt->z_override;
    L_ovr = opt->L_override;
  }
  if (!(p >= 1.0) || !(q >= 1.0) || !isfinite(p) || !isfinite(q))
    return fail(SRK_EINVAL, "p = %g and q = %g must be >= 1", p, q);
  if (z_ovr != 0.0 && !(z_ovr > 0.0 && isfinite(z_ovr)))
    return fail(SRK_EINVAL, "z_override = %g must be 0 (none) or positive and finite", z_ovr);
  const double rc = sqrt(c);
  double z;
  if (z_ovr > 0.0) {
    if (!isfinite(z_ovr)) return fail(SRK_EINVAL, "z_override is not finite");
    z = z_ovr;
  } else if (warmup) {  // Section 3: N = ln(2 n^2) / (2 eps^2)
    if (!(eps > 0.0 && eps < 1.0)) return fail(SRK_EINVAL, "eps = %g outside (0, 1)", eps);
    z = log(2.0 * (double)n * (double)n) / (2.0 * eps * eps);
  } else {
    const double thr = 3.0 / pow((double)n, p);
    if (!(eps > thr && eps < 1.0))
      return fail(SRK_EINVAL, "eps = %g must satisfy 3/n^p = %g < eps < 1", eps, thr);
    const double lam = eps - thr;
    z = log(2.0 * pow((double)n, q)) / (2.0 * lam * lam);
  }
  int L;
  if (L_ovr >= 0) {
    L = L_ovr;
  } else if (warmup) {  // Section 3: walks of length >= 3 log_{1/sqrt c}(n/eps) are dropped
    if (!(eps > 0.0 && eps < 1.0)) return fail(SRK_EINVAL, "eps = %g outside (0, 1)", eps);
    const double Lf = floor(3.0 * log((double)n / eps) / (-log(rc)));
    if (!(Lf <= (double)SRK_MAX_LEN))
      return fail(SRK_EINVAL, "truncation length %g exceeds %d", Lf, SRK_MAX_LEN);
    L = (int)Lf;
  } else {
    const double Lf = floor(p * log((double)n) / (-log(rc)));
    if (!(Lf <= (double)SRK_MAX_LEN))
      return fail(SRK_EINVAL, "truncation length %g exceeds %d", Lf, SRK_MAX_LEN);
    L = (int)Lf;
  }
  if (L > SRK_MAX_LEN)
    return fail(SRK_EINVAL, "truncation length %d exceeds %d", L, SRK_MAX_LEN);
  t->s = s;
  t->n = n;
  t->L = L;
  t->key0 = (uint32_t)seed;
  t->key1 = (uint32_t)(seed >> 32);
  t->literal = (opt && (opt->flags & SRK_OPT_LITERAL_SHUFFLE)) ? 1 : 0;
  t->shared = (opt && (opt->flags & SRK_OPT_SHARED_WALKS)) ? 1 : 0;
  t->skey = walk_key(seed, (uint32_t)s);
  t->tkey = t->shared ? walk_key(seed, kSharedWalkKey) : t->skey;
  t->z = z;
  int64_t acc = 0;
  t->P[0] = 0;
  for (int l = 0; l <= L; ++l) {
    const double Zl = z * (pow(rc, (double)l) * (1.0 - rc));
    const double Nl = ceil(Zl);
    if (!(Nl >= 1.0) || Nl > (double)SRK_MAX_WALKS)
      return fail(SRK_EINVAL, "walk count %g for length %d out of range", Nl, l);
    acc += (int64_t)Nl;
    if (acc > SRK_MAX_WALKS)
      return fail(SRK_EINVAL, "N_tot exceeds %d walks", SRK_MAX_WALKS);
    t->a[l] = Zl / Nl;
    t->P[l + 1] = (int32_t)acc;
  }
  t->N_tot = (int32_t)acc;
  // the hit table holds at most sum_l l N_l entries, indexed with int32
  int64_t cells = 0;
  for (int l = 1; l <= L; ++l) cells += (int64_t)l * (t->P[l + 1] - t->P[l]);
  if (cells > INT32_MAX)
    return fail(SRK_EINVAL, "walk budget too large: sum_l l N_l = %lld exceeds 2^31",
                (long long)cells);
  return SRK_OK;
}

// Checks row_ptr[0] = 0, row_ptr[n] = m, row_ptr non-decreasing and
// 0 <= col < n; sets *bad to 1 on any violation.
__global__ void k_validate_csr(const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, int32_t n,
                               int64_t m, int *bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[n] != m)) *bad = 1;
  for (int64_t v = t0; v < n; v += stride)
    if (row_ptr[v + 1] < row_ptr[v]) *bad = 1;
  for (int64_t e = t0; e < m; e += stride) {
    const int32_t x = col[e];
    if (x < 0 || x >= n) *bad = 1;
  }
}

// Packed adjacency with 4-byte entries (layout in srk_internal.h).  A walk
// step reads one entry, which names the next node and, unless that node is a
// hub, its degree too, instead of a row_ptr pair and a col entry.

// Last v with row_ptr[v] <= e: the owner of edge e.
__device__ __forceinline__ int32_t edge_owner(const int32_t *row_ptr, int32_t n, int64_t e) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int32_t mid = lo + (hi - lo + 1) / 2;
    if ((int64_t)row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Expected visits of the walks, used to order the packed adjacency: a walk
// starts at a uniformly drawn node with in-neighbours and moves to a
// uniformly drawn in-neighbour.  In 2^-40 fixed point, p_0 = 2^40 / n_act on
// those nodes and p_{k+1}(y) = sum over the lists I(v) that hold y of
// floor(p_k(v) / |I(v)|); the additions are integer, so their order does not
// change the result.
__global__ void k_visit_init(const int32_t *__restrict__ row_ptr, int32_t n, int32_t n_act,
                             unsigned long long *__restrict__ p) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned long long unit = (1ull << 40) / (unsigned long long)(n_act > 0 ? n_act : 1);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    p[v] = row_ptr[v + 1] > row_ptr[v] ? unit : 0ull;
}

__global__ void k_visit_step(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                             int32_t n, int64_t m, const unsigned long long *__restrict__ p,
                             unsigned long long *__restrict__ q) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int32_t v = edge_owner(row_ptr, n, e);
    const unsigned long long share =
        p[v] / (unsigned long long)(row_ptr[v + 1] - row_ptr[v]);
    if (share) atomicAdd(&q[col[e]], share);
  }
}

// acc += w * p (the visit weights of one step).
__global__ void k_visit_acc(const unsigned long long *__restrict__ p, int32_t n, unsigned int w,
                            unsigned long long *__restrict__ acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    acc[v] += (unsigned long long)w * p[v];
}

// Header word of every node that is not a hub: its degree, at its position.
__global__ void k_narrow_heads(const int32_t *__restrict__ row_ptr, int32_t n, uint32_t dmax,
                               const int32_t *__restrict__ npos, uint32_t *__restrict__ adj) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint32_t d = (uint32_t)(row_ptr[v + 1] - row_ptr[v]);
    if (d < dmax) adj[npos[v]] = d;
  }
}

// Edge e of list v lands at base(v) + (e - row_ptr[v]), base(v) = npos[v] + 1
// or, for a hub, the list offset in its header.
__global__ void k_narrow_lists(const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, int32_t n, int64_t m,
                               int pos_bits, const int32_t *__restrict__ npos,
                               uint32_t *__restrict__ adj) {
  const uint32_t dmax = (uint32_t)((1ull << (32 - pos_bits)) - 1ull);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int32_t v = edge_owner(row_ptr, n, e);
    const uint32_t dv = (uint32_t)(row_ptr[v + 1] - row_ptr[v]);
    const int64_t base = dv < dmax ? (int64_t)npos[v] + 1 : (int64_t)adj[npos[v] + 1];
    const int32_t y = col[e];
    const uint32_t dy = (uint32_t)(row_ptr[y + 1] - row_ptr[y]);
    const uint32_t code = dy < dmax ? dy : dmax;
    adj[base + (e - row_ptr[v])] = (code << pos_bits) | (uint32_t)npos[y];
  }
}

// The wide layout (srk_internal.h): adj2[pos(v)] = {0, |I(v)|} and entry e
// of list v = {pos(y), |I(y)|} for y = col[e], at the same positions.
__global__ void k_build_adjw_heads(const int32_t *__restrict__ row_ptr, int32_t n,
                                   uint2 *__restrict__ adj2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    adj2[v + row_ptr[v]] = make_uint2(0u, (uint32_t)(row_ptr[v + 1] - row_ptr[v]));
}

__global__ void k_build_adjw_lists(const int32_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col, int32_t n, int64_t m,
                                   uint2 *__restrict__ adj2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int32_t lo = edge_owner(row_ptr, n, e);
    const int32_t y = col[e];
    adj2[(int64_t)lo + 1 + e] =
        make_uint2((uint32_t)(y + row_ptr[y]), (uint32_t)(row_ptr[y + 1] - row_ptr[y]));
  }
}

__global__ void k_active_flags(const int32_t *__restrict__ row_ptr, int32_t n,
                               int32_t *__restrict__ flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    flag[v] = row_ptr[v + 1] > row_ptr[v] ? 1 : 0;
}

__global__ void k_active_scatter(const int32_t *__restrict__ flag,
                                 const int32_t *__restrict__ off, int32_t n,
                                 int32_t *__restrict__ act) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    if (flag[v]) act[off[v]] = (int32_t)v;
}

}  // namespace srk

using namespace srk;

extern "C" const char *srk_last_error(void) { return g_last_error.c_str(); }

extern "C" int srk_pool_stats(int32_t device, uint64_t *reserved, uint64_t *used,
                              uint64_t *used_high, int reset_high) {
  clear_error();
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "srk_pool_stats: device count");
  if (device < 0 || device >= count || device >= 64)
    return fail(SRK_EINVAL, "device %d outside [0, %d)", device, count);
  DeviceGuard guard(device);
  cudaMemPool_t p = pool(device);
  if (!p) return fail(SRK_ECUDA, "srk_pool_stats: cannot create the memory pool");
  uint64_t r = 0, u = 0, h = 0;  // the attributes are 64-bit values
  e = cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &r);
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &u);
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemHigh, &h);
  if (e == cudaSuccess && reset_high) {
    uint64_t zero = 0;  // resets the high-water mark to the current use
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrUsedMemHigh, &zero);
  }
  if (e != cudaSuccess) return cuda_fail(e, "srk_pool_stats");
  if (reserved) *reserved = r;
  if (used) *used = u;
  if (used_high) *used_high = h;
  return SRK_OK;
}

extern "C" int srk_graph_layout(const srk_graph *g, int32_t *layout) {
  if (!g || !layout) return fail(SRK_EINVAL, "null argument");
  *layout = g->layout == 1 ? SRK_ADJ_WIDE : g->layout == 2 ? SRK_ADJ_CSR : SRK_ADJ_NARROW;
  return SRK_OK;
}

extern "C" int srk_graph_info(const srk_graph *g, int32_t *n, int64_t *m) {
  if (!g) return fail(SRK_EINVAL, "null graph");
  if (n) *n = g->n;
  if (m) *m = g->m;
  return SRK_OK;
}

extern "C" int srk_graph_free(srk_graph *g) {
  if (!g) return SRK_OK;
  int rc = SRK_OK;
  {
    DeviceGuard guard(g->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "srk_graph_free: synchronize");
    if (g->own_row_ptr) cudaFree(g->own_row_ptr);
    if (g->own_col) cudaFree(g->own_col);
    if (g->own_w) cudaFree(g->own_w);
    if (g->adj) cudaFree(g->adj);
    if (g->npos) cudaFree(g->npos);
    if (g->act) cudaFree(g->act);
    if (g->batch_exec) cudaGraphExecDestroy(g->batch_exec);
    free_lin_topo(g);
  }
  delete g;
  return rc;
}

// Smallest b with 2^b >= x (x >= 1), at most 31.
static int bits_for(int64_t x) {
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < x) ++b;
  return b;
}

// Expected visits of every node (k_visit_*): 25 p_1 + 15 p_2 + 9 p_3, the
// landing mass of the first three steps weighted by survival at c = 0.6
// (the layout does not depend on a query's c).  Read back to the host.
static int visit_mass(const srk_graph *g, int dev, int32_t n_act, std::vector<uint64_t> *out) {
  const int32_t n = g->n;
  const int64_t m = g->m;
  unsigned long long *buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(unsigned long long) * 3 * (size_t)n);
  if (e != cudaSuccess) return cuda_fail(e, "srk_graph_load: visit mass");
  unsigned long long *p = buf, *q = buf + n, *acc = buf + 2 * (size_t)n;
  const int blocks = sm_count(dev) * 4;
  cudaMemset(acc, 0, sizeof(unsigned long long) * (size_t)n);
  k_visit_init<<<blocks, 256>>>(g->row_ptr, n, n_act, p);
  const unsigned int w[3] = {25u, 15u, 9u};
  for (int k = 0; k < 3; ++k) {
    cudaMemset(q, 0, sizeof(unsigned long long) * (size_t)n);
    if (m > 0) k_visit_step<<<sm_count(dev) * 8, 256>>>(g->row_ptr, g->col, n, m, p, q);
    k_visit_acc<<<blocks, 256>>>(q, n, w[k], acc);
    std::swap(p, q);
  }
  out->resize((size_t)n);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpy(out->data(), acc, sizeof(unsigned long long) * (size_t)n,
                   cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "srk_graph_load: visit mass");
  return SRK_OK;
}

// Builds the 4-byte-entry adjacency of g (sets adj, npos, n_hubs, pos_bits).
// The hub count H and the position width pb depend on each other (a hub has
// degree 2^(32-pb) - 1 or more, and positions run to n + m + H): pb grows
// from ceil(log2(n + m)) until it holds.  Order: the hubs' headers first, by
// expected visits (the header of the node a walk lands on is read at the
// landing), then every node's list (a non-hub's after its header word) by
// expected visits per list entry, descending, so that the lists read most
// per byte share sectors and the front of the array; ties by id, nodes
// without in-neighbours
// last.  (Measured: on R-MAT 20 this order gives 37.1 queries/s against 37.0
// for id order; on R-MAT 22-24, where the graph exceeds the L2, it changes
// nothing measurable, nor did L2 eviction-priority hints that kept its front
// part resident.)  The layout is a function of the graph alone.
static int build_narrow(srk_graph *g, int dev) {
  const int32_t n = g->n;
  const int64_t m = g->m;
  std::vector<int32_t> rp((size_t)n + 1);
  cudaError_t e = cudaMemcpy(rp.data(), g->row_ptr, sizeof(int32_t) * ((size_t)n + 1),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "srk_graph_load: reading row_ptr");
  auto deg = [&](int32_t v) { return (uint32_t)(rp[(size_t)v + 1] - rp[(size_t)v]); };
  int32_t n_act = 0;
  for (int32_t v = 0; v < n; ++v) n_act += deg(v) > 0;
  int pb = bits_for((int64_t)n + m);
  int64_t H = 0;
  for (int it = 0;; ++it) {
    const uint32_t dmax = (uint32_t)((1ull << (32 - pb)) - 1ull);
    H = 0;
    for (int32_t v = 0; v < n; ++v) H += deg(v) >= dmax;
    const int64_t total = (int64_t)n + m + H;
    if (total > INT32_MAX || it >= 32)
      return fail(SRK_EINVAL, "graph too large for 4-byte adjacency entries (n + m + hubs = %lld)",
                  (long long)total);
    const int pb2 = bits_for(total);
    if (pb2 <= pb) break;
    pb = pb2;
  }
  const uint32_t dmax = (uint32_t)((1ull << (32 - pb)) - 1ull);
  std::vector<uint64_t> vis;
  int rc = visit_mass(g, dev, n_act, &vis);
  if (rc) return rc;
  // hubs by visits; every node by visits per entry
  std::vector<int32_t> hubs, order((size_t)n);
  for (int32_t v = 0; v < n; ++v) {
    order[(size_t)v] = v;
    if (deg(v) >= dmax) hubs.push_back(v);
  }
  std::stable_sort(hubs.begin(), hubs.end(), [&](int32_t a, int32_t b) {
    return vis[(size_t)a] > vis[(size_t)b];
  });
  std::vector<double> key((size_t)n);
  for (int32_t v = 0; v < n; ++v)
    key[(size_t)v] = deg(v) > 0 ? (double)vis[(size_t)v] / (double)deg(v) : -1.0;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return key[(size_t)a] > key[(size_t)b];
  });
  std::vector<int32_t> npos((size_t)n), hub_rank((size_t)n, -1);
  std::vector<uint32_t> head(2 * (size_t)std::max<int64_t>(H, 1));
  for (int64_t r = 0; r < H; ++r) hub_rank[(size_t)hubs[(size_t)r]] = (int32_t)r;
  int64_t at = 2 * H;
  for (int32_t v : order) {
    const uint32_t d = deg(v);
    if (d < dmax) {
      npos[(size_t)v] = (int32_t)at;
      at += 1 + (int64_t)d;
    } else {
      const int32_t r = hub_rank[(size_t)v];
      npos[(size_t)v] = 2 * r;
      head[2 * (size_t)r] = d;
      head[2 * (size_t)r + 1] = (uint32_t)at;
      at += d;
    }
  }
  const size_t words = (size_t)n + (size_t)m + (size_t)H;
  if ((size_t)at != words) return fail(SRK_ECUDA, "srk_graph_load: inconsistent layout size");
  if ((e = cudaMalloc(&g->adj, sizeof(uint32_t) * (words > 0 ? words : 1))) != cudaSuccess ||
      (e = cudaMalloc(&g->npos, sizeof(int32_t) * (size_t)n)) != cudaSuccess)
    return cuda_fail(e, "srk_graph_load: packed adjacency");
  if ((e = cudaMemcpy(g->npos, npos.data(), sizeof(int32_t) * (size_t)n,
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (H > 0 && (e = cudaMemcpy(g->adj, head.data(), sizeof(uint32_t) * 2 * (size_t)H,
                                cudaMemcpyHostToDevice)) != cudaSuccess))
    return cuda_fail(e, "srk_graph_load: positions and hub headers");
  k_narrow_heads<<<sm_count(dev) * 4, 256>>>(g->row_ptr, n, dmax, g->npos, g->adj);
  if (m > 0)
    k_narrow_lists<<<sm_count(dev) * 8, 256>>>(g->row_ptr, g->col, n, m, pb, g->npos, g->adj);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "srk_graph_load: building the packed adjacency");
  g->pos_bits = pb;
  g->n_hubs = (int32_t)H;
  return SRK_OK;
}

extern "C" int srk_graph_load(const int32_t *row_ptr, const int32_t *col,
                              int32_t n, int64_t m, int flags,
                              const float *edge_w, srk_graph **out) {
  clear_error();
  if (!out) return fail(SRK_EINVAL, "out is null");
  *out = nullptr;
  if (n < 1) return fail(SRK_EINVAL, "n = %d must be >= 1", n);
  if (m < 0 || m > INT32_MAX) return fail(SRK_EINVAL, "m = %lld outside [0, 2^31)", (long long)m);
  if ((int64_t)n + m > INT32_MAX)
    return fail(SRK_EINVAL, "n + m = %lld must stay below 2^31", (long long)n + (long long)m);
  if (!row_ptr || (m > 0 && !col)) return fail(SRK_EINVAL, "null CSR array");
  if (flags & ~(SRK_DEVICE_PTRS | SRK_VALIDATE | SRK_ADJ_NARROW | SRK_ADJ_WIDE | SRK_ADJ_CSR))
    return fail(SRK_EINVAL, "unknown flags 0x%x", flags);
  {
    const int layouts = !!(flags & SRK_ADJ_NARROW) + !!(flags & SRK_ADJ_WIDE) +
                        !!(flags & SRK_ADJ_CSR);
    if (layouts > 1)
      return fail(SRK_EINVAL, "SRK_ADJ_NARROW, SRK_ADJ_WIDE and SRK_ADJ_CSR exclude each other");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "srk_graph_load: no CUDA device");
  srk_graph *g = new srk_graph;
  g->n = n;
  g->m = m;
  g->device = dev;
  if (flags & SRK_DEVICE_PTRS) {
    if (!is_device_ptr(row_ptr) || (m > 0 && !is_device_ptr(col)) ||
        (edge_w && m > 0 && !is_device_ptr(edge_w))) {
      delete g;
      return fail(SRK_EINVAL, "SRK_DEVICE_PTRS given but an array is not device memory");
    }
    g->row_ptr = row_ptr;
    g->col = col;
    g->edge_w = edge_w;
  } else {
    const size_t rb = sizeof(int32_t) * ((size_t)n + 1);
    const size_t cb = sizeof(int32_t) * (size_t)(m > 0 ? m : 1);
    if ((e = cudaMalloc(&g->own_row_ptr, rb)) != cudaSuccess ||
        (e = cudaMalloc(&g->own_col, cb)) != cudaSuccess ||
        (edge_w && (e = cudaMalloc(&g->own_w, sizeof(float) * (size_t)(m > 0 ? m : 1))) !=
                       cudaSuccess)) {
      int rc = cuda_fail(e, "srk_graph_load: device allocation");
      srk_graph_free(g);
      return rc;
    }
    if ((e = cudaMemcpy(g->own_row_ptr, row_ptr, rb, cudaMemcpyDefault)) != cudaSuccess ||
        (m > 0 && (e = cudaMemcpy(g->own_col, col, sizeof(int32_t) * (size_t)m,
                                  cudaMemcpyDefault)) != cudaSuccess) ||
        (edge_w && m > 0 && (e = cudaMemcpy(g->own_w, edge_w, sizeof(float) * (size_t)m,
                                            cudaMemcpyDefault)) != cudaSuccess)) {
      int rc = cuda_fail(e, "srk_graph_load: copy to device");
      srk_graph_free(g);
      return rc;
    }
    g->row_ptr = g->own_row_ptr;
    g->col = g->own_col;
    g->edge_w = g->own_w;
  }
  {  // always validate: the walk kernels index with these values
    int *bad = nullptr;
    int hbad = 0;
    if ((e = cudaMalloc(&bad, sizeof(int))) != cudaSuccess) {
      int rc = cuda_fail(e, "srk_graph_load: validation flag");
      srk_graph_free(g);
      return rc;
    }
    cudaMemset(bad, 0, sizeof(int));
    const int blocks = sm_count(dev) * 4;
    k_validate_csr<<<blocks, 256>>>(g->row_ptr, g->col, n, m, bad);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    if (e != cudaSuccess) {
      int rc = cuda_fail(e, "srk_graph_load: validation");
      srk_graph_free(g);
      return rc;
    }
    if (hbad) {
      srk_graph_free(g);
      return fail(SRK_EINVAL, "malformed CSR: row_ptr must start at 0, end at m and "
                              "not decrease; col entries must lie in [0, n)");
    }
  }
  {
    const int pb = bits_for((int64_t)n + m);  // positions < n + m (wide layout)
    g->pos_bits = pb;
    // Layout by size (measured on R-MAT graphs 20-24): 4-byte entries up to
    // 28 position bits (degree codes down to 15; the hubs' headers, packed
    // at the front in landing order, stay cached while the entries are half
    // the size of 8-byte ones); beyond, 8-byte entries, which need no header
    // read.  The CSR layout is only taken when asked for.
    g->layout = (flags & SRK_ADJ_WIDE)     ? 1
                : (flags & SRK_ADJ_CSR)    ? 2
                : (flags & SRK_ADJ_NARROW) ? 0
                : pb <= 28                 ? 0
                                           : 1;
    int rc = SRK_OK;
    if (g->layout == 0) {
      rc = build_narrow(g, dev);
    } else if ((e = cudaMalloc(&g->adj, sizeof(uint32_t) *
                                            (g->layout == 2 ? 1 : 2 * ((size_t)n + (size_t)m)))) !=
               cudaSuccess) {
      rc = cuda_fail(e, "srk_graph_load: packed adjacency");
    } else if (g->layout == 1) {
      uint2 *adj2 = reinterpret_cast<uint2 *>(g->adj);
      k_build_adjw_heads<<<sm_count(dev) * 4, 256>>>(g->row_ptr, n, adj2);
      if (m > 0) k_build_adjw_lists<<<sm_count(dev) * 8, 256>>>(g->row_ptr, g->col, n, m, adj2);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e != cudaSuccess) rc = cuda_fail(e, "srk_graph_load: building the packed adjacency");
    }  // CSR: the walks read row_ptr and col directly
    if (rc != SRK_OK) {
      srk_graph_free(g);
      return rc;
    }
  }
  {  // ascending list of the nodes with in-neighbours
    int32_t *flag = nullptr, *off = nullptr;
    if ((e = cudaMalloc(&flag, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
        (e = cudaMalloc(&off, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess) {
      if (flag) cudaFree(flag);
      int rc = cuda_fail(e, "srk_graph_load: active-node list");
      srk_graph_free(g);
      return rc;
    }
    k_active_flags<<<sm_count(dev) * 4, 256>>>(g->row_ptr, n, flag);
    k_scan<<<1, 1024>>>(flag, off, n);
    int32_t n_act = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpy(&n_act, off + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess &&
        (e = cudaMalloc(&g->act, sizeof(int32_t) * (size_t)(n_act > 0 ? n_act : 1))) ==
            cudaSuccess) {
      k_active_scatter<<<sm_count(dev) * 4, 256>>>(flag, off, n, g->act);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(flag);
    cudaFree(off);
    if (e != cudaSuccess) {
      int rc = cuda_fail(e, "srk_graph_load: active-node list");
      srk_graph_free(g);
      return rc;
    }
    g->n_act = n_act;
  }
  *out = g;
  return SRK_OK;
}
