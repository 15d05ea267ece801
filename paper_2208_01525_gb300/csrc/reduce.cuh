// Deterministic block reductions for the measuring kernels: warp shuffles in
// a fixed order, then a fixed-order compensated (Neumaier) merge across warps.
#pragma once

#include "u1u1_internal.cuh"

namespace u1u1 {

// Neumaier compensated accumulation: s + c carries the exact running sum to
// about twice the working precision.
__device__ __forceinline__ void neumaier_add(double& s, double& c, double v) {
  double t = s + v;
  if (fabs(s) >= fabs(v)) c += (s - t) + v;
  else c += (v - t) + s;
  s = t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Per-thread accumulator of the diagnostic sums, extrema and counts.
struct ThreadAcc {
  double s[NSUM];
  double mx[NMAX];
  long long cnt[NCNT];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < NSUM; ++k) s[k] = 0.0;
#pragma unroll
    for (int k = 0; k < NMAX; ++k) mx[k] = -INFINITY;
#pragma unroll
    for (int k = 0; k < NCNT; ++k) cnt[k] = 0;
  }
};

// Scratch for block_reduce: one slot per warp per quantity.
template <int NWARPS>
struct ReduceSmem {
  double s[NWARPS][NSUM];
  double mx[NWARPS][NMAX];
  long long cnt[NWARPS][NCNT];
};

// Reduce every thread's accumulator into *out (one BlockPartial).  Must be
// called by all threads of the block.
template <int NWARPS>
__device__ void block_reduce(const ThreadAcc& a, ReduceSmem<NWARPS>& sm, BlockPartial* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NSUM; ++k) {
    double v = warp_sum(a.s[k]);
    if (lane == 0) sm.s[warp][k] = v;
  }
#pragma unroll
  for (int k = 0; k < NMAX; ++k) {
    double v = warp_max(a.mx[k]);
    if (lane == 0) sm.mx[warp][k] = v;
  }
#pragma unroll
  for (int k = 0; k < NCNT; ++k) {
    long long v = (k == C_MAXW) ? warp_max_ll(a.cnt[k]) : warp_sum_ll(a.cnt[k]);
    if (lane == 0) sm.cnt[warp][k] = v;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < NSUM) {
    double s = 0.0, c = 0.0;
    for (int w = 0; w < NWARPS; ++w) neumaier_add(s, c, sm.s[w][t]);
    out->sum[t] = s;
    out->comp[t] = c;
  } else if (t < NSUM + NMAX) {
    int k = t - NSUM;
    double m = -INFINITY;
    for (int w = 0; w < NWARPS; ++w) m = fmax(m, sm.mx[w][k]);
    out->mx[k] = m;
  } else if (t < NSUM + NMAX + NCNT) {
    int k = t - NSUM - NMAX;
    long long v = 0;
    for (int w = 0; w < NWARPS; ++w) v = (k == C_MAXW) ? max(v, sm.cnt[w][k]) : v + sm.cnt[w][k];
    out->cnt[k] = v;
  }
}

}  // namespace u1u1
