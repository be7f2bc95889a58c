// Block reductions and the last-block ticket used by every reduction kernel.
// Sums are formed in a fixed order (per-block partials, then one block adds
// the partials by a fixed strided pattern), so results are bit-reproducible
// for a given launch shape.
#pragma once

#include <cuda_runtime.h>

namespace mfg {

__device__ __forceinline__ int flat_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int flat_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }
__device__ __forceinline__ int flat_bid() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }
__device__ __forceinline__ int flat_nblocks() { return gridDim.x * gridDim.y * gridDim.z; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of `v` over the block; the result is valid in thread 0.  Up to 1024 threads.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double ws[NV][32];
  const int tid = flat_tid(), lane = tid & 31, w = tid >> 5, nw = (flat_nthreads() + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) ws[q][w] = v[q];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = lane < nw ? ws[q][lane] : 0.0;
      v[q] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Publishes this block's partial sums (valid in thread 0) and returns true in
// every thread of the block that finishes last.  partials holds NV arrays of
// flat_nblocks() entries.
template <int NV>
__device__ __forceinline__ bool publish_and_check_last(const double (&v)[NV], double* partials,
                                                       unsigned int* counter) {
  __shared__ bool am_last;
  const int nb = flat_nblocks(), bid = flat_bid();
  if (flat_tid() == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[q * nb + bid] = v[q];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == (unsigned int)(nb - 1));
  }
  __syncthreads();
  return am_last;
}

// In the last block: adds the partials in a fixed order; result in thread 0.
template <int NV>
__device__ __forceinline__ void gather_partials(const double* partials, double (&out)[NV]) {
  __threadfence();
  const int nb = flat_nblocks();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
    for (int i = flat_tid(); i < nb; i += flat_nthreads()) s += __ldcg(partials + q * nb + i);
    out[q] = s;
  }
  block_sum<NV>(out);
}

}  // namespace mfg
