// reduce.cuh -- deterministic block reductions shared by the Krylov solvers
// (internal).  Fixed block size RED_THREADS; every sum is taken in a fixed
// order, so results are reproducible run to run on the same device.
#pragma once

#include "common.cuh"

namespace cpm {

constexpr int RED_THREADS = 256;

// sum of v over the block (the result is valid in thread 0)
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int q = 0; q < RED_THREADS / 32; ++q) t += sh[q];
  return t;
}

// Sum NV per-lane values over a warp with NV - 1 + log2(32 / NV) shuffles
// instead of 5 NV: at each halving step a lane keeps one half of its values
// and receives its partner's copy of the same half.  On return lane l (and,
// for NV < 32, every lane congruent to l modulo NV) holds in a[0] the warp
// sum of value l % NV.
template <int NV>
__device__ __forceinline__ void warp_transpose_sum(double (&a)[NV], int lane) {
#pragma unroll
  for (int half = NV / 2; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const double send = up ? a[k] : a[k + half];
      const double keep = up ? a[k + half] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
#pragma unroll
  for (int o = NV; o < 32; o <<= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
}

// Block partial sums of NV per-thread values: partial[t * gridDim.x + b] for
// t < nv, summed over the block's warps in a fixed order.
template <int NV>
__device__ __forceinline__ void block_partials(double (&a)[NV], int nv, double* partial) {
  __shared__ double sh[RED_THREADS / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  warp_transpose_sum<NV>(a, lane);
  if (lane < NV) sh[wid][lane] = a[0];
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0;
#pragma unroll
    for (int q = 0; q < RED_THREADS / 32; ++q) t += sh[q][threadIdx.x];
    partial[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

}  // namespace cpm
