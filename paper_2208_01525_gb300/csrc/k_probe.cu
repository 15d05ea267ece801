// Throughput probe of the FP64 arithmetic pipe, the ceiling of the FP64
// step (which is bound by GB300's FP64 rate, not by HBM).  Every thread runs
// eight independent chains of dependent fused multiply-adds, so that enough
// operations are in flight to keep the pipe busy at full occupancy; the rate
// is timed with CUDA events on the caller's stream.  It changes no device
// setting and allocates nothing (the sink is a static device word).
#include <cuda_runtime.h>

#include "../../include/u1u1.h"
#include "host_internal.h"

namespace u1u1 {
namespace {

__device__ double g_fma_sink;

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;
constexpr int PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS) k_fp64_fma(long long iters, double a, double b) {
  double x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  if (s == 1.25e300) g_fma_sink = s;  // never true for these inputs; keeps every chain live
}

}  // namespace
}  // namespace u1u1

using namespace u1u1;

extern "C" int u1u1_fp64_fma_rate(double* tflops, void* stream) {
  if (!tflops) return fail(U1U1_ERR_INVALID_ARG, "tflops is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  U1U1_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  U1U1_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  U1U1_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, PROBE_THREADS, 0), "occupancy");
  if (per_sm < 1) per_sm = 1;
  const long long blocks = (long long)sms * per_sm;
  // a = 1 - 2^-20, b = 2^-30: the chains stay finite and never reach the sink's value
  const double a = 1.0 - 9.5367431640625e-07, b = 9.313225746154785e-10;
  cudaEvent_t e0, e1;
  U1U1_CUDA_TRY(cudaEventCreate(&e0), "event");
  U1U1_CUDA_TRY(cudaEventCreate(&e1), "event");
  int rc = U1U1_OK;
  long long iters = 64;
  double best = 0.0;
  for (int pass = 0; pass < 8 && !rc; ++pass) {
    cudaEventRecord(e0, st);
    k_fp64_fma<<<(unsigned)blocks, PROBE_THREADS, 0, st>>>(iters, a, b);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "FP64 probe kernel");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * CHAINS * UNROLL * (double)iters * (double)blocks * PROBE_THREADS;
    if (ms < 50.0f) {  // grow the run to at least 50 ms before it counts
      iters *= ms > 0.5f ? (long long)(100.0f / ms) + 1 : 64;
      continue;
    }
    const double r = flops / (ms * 1e-3) / 1e12;
    if (r > best) best = r;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc && best <= 0.0) rc = fail(U1U1_ERR_CUDA, "FP64 probe did not reach a timed run");
  if (!rc) *tflops = best;
  return rc;
}
