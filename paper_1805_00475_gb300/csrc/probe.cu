// Microbenchmark of the modular multiply-accumulate primitive used by every
// step kernel: four residues per thread, u32 x u32 products accumulated in 64
// bits, reduced after every 16th product as the step kernels do for the
// default primes (just below 2^30: mod_reduce_near30).  Operands live in
// registers and are scrambled every iteration (xor-shift) so that no product
// is loop-invariant.  It gives a measured ceiling for steps bound by the
// integer pipes, next to the ceiling derived from unit counts and clocks.
#include <cuda_runtime.h>

#include <string>

#include <algorithm>

#include "modarith.cuh"
#include "tnc_internal.h"

namespace {

__global__ void __launch_bounds__(256) modmac_probe_kernel(uint32_t seed, uint32_t iters, tnc_dev::ModGroup mg,
                                                           unsigned long long never, unsigned long long* sink) {
  uint32_t x[8];
  uint32_t h = seed ^ (blockIdx.x * 0x9E3779B9u + threadIdx.x * 0x85EBCA6Bu);
#pragma unroll
  for (int i = 0; i < 8; i++) {
    h ^= h << 13;
    h ^= h >> 17;
    h ^= h << 5;
    x[i] = h & 0x3FFFFFFFu;  // below 2^30
  }
  uint64_t acc[4] = {0, 0, 0, 0};
  for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
      for (int r = 0; r < 4; r++) acc[r] += (uint64_t)x[(u + r) & 7] * x[(u + r + 3) & 7];
    }
    if ((it & 3u) == 3u) {
#pragma unroll
      for (int r = 0; r < 4; r++) acc[r] = tnc_dev::reduce64<true>(acc[r], mg, r);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = (x[i] ^ (x[(i + 1) & 7] >> 3)) & 0x3FFFFFFFu;
  }
  const uint64_t s = acc[0] + acc[1] + acc[2] + acc[3];
  if (s == never) atomicAdd(sink, 1ull);  // a runtime value no sum reaches: keeps the work observable
}

}  // namespace

extern "C" int tnc_probe_modmac(void* cuda_stream, int32_t iters, double* macs_per_s) {
  using namespace tnc;
  clear_error();
  if (!macs_per_s || iters <= 0) return set_error(TNC_ERR_INVALID, "bad probe arguments");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, modmac_probe_kernel, 256, 0);
  if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("probe setup: ") + cudaGetErrorString(e));
  const uint32_t ps[4] = {1073741789u, 1073741783u, 1073741741u, 1073741723u};
  const tnc_dev::ModGroup mg = tnc_dev::make_mod_group(ps);
  const int blocks = sms * occ;
  cudaEvent_t a = nullptr, b = nullptr;
  unsigned long long* sink = nullptr;
  // the probe is a diagnostic, not part of the counting path: it may use the
  // runtime's allocator for its 8-byte sink
  e = cudaMallocAsync((void**)&sink, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    modmac_probe_kernel<<<blocks, 256, 0, st>>>(1u, (uint32_t)std::max(1, iters / 8), mg, ~0ull, sink);  // warm-up
    cudaEventRecord(a, st);
    modmac_probe_kernel<<<blocks, 256, 0, st>>>(7u, (uint32_t)iters, mg, ~0ull, sink);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
  }
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (sink) cudaFreeAsync(sink, st);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("probe: ") + cudaGetErrorString(e));
  const double macs = (double)blocks * 256.0 * (double)iters * 16.0;
  *macs_per_s = macs / (ms * 1e-3);
  return TNC_OK;
}
