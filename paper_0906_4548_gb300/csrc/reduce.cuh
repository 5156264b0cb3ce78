// Warp and block sums in FP64 (deterministic two-stage reductions: each block
// writes its partials, one block adds them in a fixed order).
#pragma once

namespace dgp {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NC values per thread; thread 0 returns the totals in v.
template <int NC>
__device__ __forceinline__ void block_sum(double (&v)[NC]) {
  __shared__ double s_part[NC][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    v[c] = warp_sum(v[c]);
    if (lane == 0) s_part[c][wid] = v[c];
  }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double t = lane < nw ? s_part[c][lane] : 0.0;
      v[c] = warp_sum(t);
    }
  }
}

}  // namespace dgp
