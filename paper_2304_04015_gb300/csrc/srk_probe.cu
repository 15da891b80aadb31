// Random-gather probe: the achievable rate of independent random 4-byte loads
// from a device array, the ceiling of a walk step's memory work.  The
// benchmark runs it on an array the size of the graph (L2-resident) and on
// one far larger than L2 (HBM) to report the walk kernel's fraction of the
// gather roofline.  Each thread draws indices with a 32-bit linear
// congruential generator (x <- 1664525 x + 1013904223 mod 2^32, the
// "quick" generator of Numerical Recipes) and maps them to [0, n) with a
// multiply-high; four loads per iteration are independent of the loaded
// values, so the memory system sees as many requests in flight as it accepts.
#include "srk_internal.h"

namespace srk {

// One 4-byte load with the cache operator OP: 0 default (ld.global),
// 1 .cg (cache in L2 only), 2 .nc (read-only path), 3 .ca (all levels).
template <int OP>
__device__ __forceinline__ int32_t probe_load(const int32_t *p) {
  int32_t v;
  if (OP == 0) v = *p;
  else if (OP == 1) asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(p));
  else if (OP == 2) asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  else asm volatile("ld.global.ca.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

template <int OP>
__global__ void __launch_bounds__(256)
k_probe_gather(const int32_t *__restrict__ data, uint32_t n, int64_t iters,
               uint32_t seed, unsigned long long *__restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x0 = seed ^ (tid * 0x9E3779B9u), x1 = x0 ^ 0x85EBCA6Bu,
           x2 = x0 ^ 0xC2B2AE35u, x3 = x0 ^ 0x27D4EB2Fu;
  uint32_t acc = 0;
  for (int64_t it = 0; it < iters; ++it) {
    x0 = x0 * 1664525u + 1013904223u;
    x1 = x1 * 1664525u + 1013904223u;
    x2 = x2 * 1664525u + 1013904223u;
    x3 = x3 * 1664525u + 1013904223u;
    acc += probe_load<OP>(data + __umulhi(x0, n)) ^ probe_load<OP>(data + __umulhi(x1, n)) ^
           probe_load<OP>(data + __umulhi(x2, n)) ^ probe_load<OP>(data + __umulhi(x3, n));
  }
  if (acc == 0x7FFFFFFFu) atomicAdd(sink, 1ull);  // keeps the loads alive
}

template <int OP>
static int launch_probe(const int32_t *data, int64_t n, int64_t iters, uint32_t seed,
                        unsigned long long *sink, int64_t *loads, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "srk_probe_gather");
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_gather<OP>, 256, 0) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int blocks = sm_count(dev) * per_sm;
  k_probe_gather<OP><<<blocks, 256, 0, st>>>(data, (uint32_t)n, iters, seed, sink);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "srk_probe_gather launch");
  if (loads) *loads = (int64_t)blocks * 256 * iters * 4;
  return SRK_OK;
}

}  // namespace srk

using namespace srk;

extern "C" int srk_probe_gather_ex(const int32_t *data, int64_t n, int64_t iters,
                                   uint32_t seed, int32_t cache_op, unsigned long long *sink,
                                   int64_t *loads, void *cuda_stream) {
  clear_error();
  if (!data || !sink || n < 1 || n > (int64_t)UINT32_MAX || iters < 1)
    return fail(SRK_EINVAL, "srk_probe_gather: bad arguments");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  switch (cache_op) {
    case SRK_PROBE_DEFAULT: return launch_probe<0>(data, n, iters, seed, sink, loads, st);
    case SRK_PROBE_CG: return launch_probe<1>(data, n, iters, seed, sink, loads, st);
    case SRK_PROBE_NC: return launch_probe<2>(data, n, iters, seed, sink, loads, st);
    case SRK_PROBE_CA: return launch_probe<3>(data, n, iters, seed, sink, loads, st);
    default: return fail(SRK_EINVAL, "srk_probe_gather_ex: unknown cache_op %d", cache_op);
  }
}

extern "C" int srk_probe_gather(const int32_t *data, int64_t n, int64_t iters,
                                uint32_t seed, unsigned long long *sink,
                                int64_t *loads, void *cuda_stream) {
  return srk_probe_gather_ex(data, n, iters, seed, SRK_PROBE_DEFAULT, sink, loads,
                             cuda_stream);
}
