// Block and grid reductions of the Hartree energy (FP64, deterministic order).
#pragma once

#include "common.cuh"

namespace ps {

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// Deterministic grid reduction: every CTA stores its partial; the CTA that
// arrives last sums all partials in index order and resets the counter.
__device__ inline void energy_finish(double part, double* partials, unsigned* counter,
                              double scale, double* E) {
  __shared__ double sh[32];
  __shared__ unsigned s_last;
  const int nblk = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  double bs = block_sum(part, sh);
  if (threadIdx.x == 0) {
    partials[bid] = bs;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned)(nblk - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += __ldcg(partials + i);
    double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) {
      *E = scale * tot;
      *counter = 0u;
    }
  }
}

// The same grid reduction for an FP32 per-thread partial: FP32 within each
// warp, the warp sums added in FP64 by one thread, FP64 across CTAs. Keeps
// the (slow) FP64 pipe out of the per-warp shuffles; two barriers.
__device__ inline void energy_finish_f32(float part, double* partials, unsigned* counter, double scale,
                                         double* E) {
  __shared__ float wsum[32];
  __shared__ double sh[32];
  __shared__ unsigned s_last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wsum[wid] = part;
  __syncthreads();
  const int nblk = gridDim.x * gridDim.y;
  if (threadIdx.x == 0) {
    double bs = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) bs += (double)wsum[w];
    partials[blockIdx.y * gridDim.x + blockIdx.x] = bs;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned)(nblk - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += __ldcg(partials + i);
    double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) {
      *E = scale * tot;
      *counter = 0u;
    }
  }
}

}  // namespace ps
