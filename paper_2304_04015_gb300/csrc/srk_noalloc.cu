// srk_single_source_noalloc: the single-source query with its scratch taken
// from a fixed, statically allocated device array instead of a memory pool.
//
// Who needs it: callers that must not allocate device memory while they issue
// queries -- an application whose own caching allocator owns the whole device
// budget, a serving thread that must not block on (or fail in) the driver's
// allocator, or code running where allocation calls are off limits.  The graph
// handle is created beforehand (srk_graph_load with SRK_DEVICE_PTRS borrows the
// caller's arrays); after that this entry point calls no cudaMalloc, cudaFree,
// cudaMallocAsync or any other allocating routine.
//
// The scratch is one file-scope __device__ array of SRK_NOALLOC_SCRATCH_BYTES.
// It exists on every device on which this module is loaded, until the process
// exits.  Its device address is looked up with cudaGetSymbolAddress by the
// first call in each CUDA context (so that first call should come before any
// stream capture); the address is kept per device together with the unique id
// of the context it was taken in, and taken again when that context has been
// replaced (after cudaDeviceReset, for instance).  All calls share the array
// and it keeps the previous call's contents: every part a query needs zeroed
// is cleared by the query itself, and calls whose work overlaps on the GPU
// (for instance on two streams) race on it.
#include <cuda.h>

#include <mutex>

#include "srk_internal.h"

// The scratch of every srk_single_source_noalloc call (see above).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SRK_NOALLOC_SCRATCH_BYTES];

namespace srk {
namespace {

std::mutex g_addr_mu;
struct ScratchAddr {
  unsigned long long ctx_id;  // the context the address belongs to (0: none yet)
  void *addr;
};
ScratchAddr g_addr[64] = {};

// Unique id of the calling thread's current CUDA context (0 when there is
// none), through the driver's cuCtxGetCurrent and cuCtxGetId, reached via the
// runtime so that the library links no driver stub.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(f1);
      get_id = reinterpret_cast<GetId>(f2);
    }
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array on `device` (the current device), in
// the current context.
int scratch_address(int device, char **out) {
  if (device < 0 || device >= 64) return fail(SRK_EINVAL, "device %d out of range", device);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  unsigned long long ctx = current_context_id();
  ScratchAddr &a = g_addr[device];
  if (!a.addr || ctx == 0 || ctx != a.ctx_id) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                       "srk_single_source_noalloc: scratch address");
    a.addr = p;
    a.ctx_id = ctx ? ctx : current_context_id();  // the lookup made the context current
  }
  *out = static_cast<char *>(a.addr);
  return SRK_OK;
}

}  // namespace
}  // namespace srk

using namespace srk;

extern "C" int srk_single_source_noalloc(const srk_graph *g, int32_t s, double c,
                                         double eps, uint64_t seed,
                                         const srk_opts *opt, double *scores,
                                         uint32_t *meet_counts,
                                         uint64_t *weight_sums,
                                         void *cuda_stream) {
  clear_error();
  if (!g) return fail(SRK_EINVAL, "null graph");
  if (!scores) return fail(SRK_EINVAL, "scores is null");
  if (opt && (opt->flags & ~(SRK_OPT_WARMUP_RULE | SRK_OPT_LITERAL_SHUFFLE |
                             SRK_OPT_SHARED_WALKS)))
    return fail(SRK_EINVAL, "unsupported opts.flags 0x%x", opt->flags);
  uint32_t *step_counts = opt ? opt->step_counts : nullptr;
  QueryTab t;
  int rc = build_table(g->n, s, c, eps, seed, opt, &t);
  if (rc) return rc;
  int32_t u_begin = 0, u_end = g->n;
  rc = target_range(g, opt, &u_begin, &u_end);
  if (rc) return rc;
  DeviceGuard guard(g->device);
  // host outputs would need a device staging buffer: only device memory here
  if (!is_device_ptr(scores) || (meet_counts && !is_device_ptr(meet_counts)) ||
      (weight_sums && !is_device_ptr(weight_sums)) ||
      (step_counts && !is_device_ptr(step_counts)))
    return fail(SRK_EINVAL, "srk_single_source_noalloc takes device output pointers only");
  Workspace w;
  const size_t need = plan(t, &w, nullptr);
  if (need > (size_t)SRK_NOALLOC_SCRATCH_BYTES)
    return fail(SRK_EINVAL,
                "query needs %zu bytes of scratch (N_tot = %d walks, L = %d); the "
                "static scratch of srk_single_source_noalloc holds %zu bytes",
                need, t.N_tot, t.L, (size_t)SRK_NOALLOC_SCRATCH_BYTES);
  char *base = nullptr;
  rc = scratch_address(g->device, &base);
  if (rc) return rc;
  plan(t, &w, base);
  Outputs o;
  o.scores = scores;
  o.counts = meet_counts;
  o.wsums = reinterpret_cast<unsigned long long *>(weight_sums);
  o.steps = step_counts;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  rc = enqueue_query(g, t, w, o, st,
                     opt ? (const cudaEvent_t *)opt->timing_events : nullptr, u_begin, u_end);
  if (!rc && opt && opt->stats) rc = read_stats(t, w, st, opt->stats, false);
  return rc;
}
