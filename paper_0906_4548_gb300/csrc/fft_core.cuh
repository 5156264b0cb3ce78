// In-register DFT building block of the mesh transforms.
//
// Every 1D transform of length N = N1 * N2 is done as the Cooley-Tukey
// "four-step" split: each of N2 lanes transforms the N1 elements
// x[N2*j1 + j2] held in its registers, multiplies by W_N^{j2 k1}, and the
// result is transposed through shared memory so that each of N1 lanes holds
// the N2 elements of a k1 and transforms them; output index k1 + N1*k2.
// Twiddles W_N^t = exp(-2 pi i t / N), t < N, live in a shared-memory table
// (computed on the host in FP64 by calling sin/cos, rounded once).
// Inverse transforms use conj(DFT(conj(x))).
#pragma once

#include "common.cuh"

namespace dgp {

template <int R> struct Log2;
template <> struct Log2<1> { static constexpr int v = 0; };
template <> struct Log2<2> { static constexpr int v = 1; };
template <> struct Log2<4> { static constexpr int v = 2; };
template <> struct Log2<8> { static constexpr int v = 3; };
template <> struct Log2<16> { static constexpr int v = 4; };
template <> struct Log2<32> { static constexpr int v = 5; };

__host__ __device__ constexpr int bitrev_c(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// Forward DFT of the R values in v (natural order in and out), radix-2
// decimation in time.  tw is the W_N table, TWS = N / R so that
// W_R^m = tw[m * TWS].
template <int R, int TWS, typename V>
__device__ __forceinline__ void dft_regs(V (&v)[R], const V* __restrict__ tw) {
  constexpr int L = Log2<R>::v;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = bitrev_c(i, L);
    if (i < j) { V t = v[i]; v[i] = v[j]; v[j] = t; }
  }
#pragma unroll
  for (int st = 0; st < L; ++st) {
    const int len = 2 << st;
    const int half = 1 << st;
#pragma unroll
    for (int g = 0; g < R / 2; ++g) {
      const int k = g % half;          // position inside the butterfly group
      const int i = (g / half) * len;  // group start
      V u = v[i + k];
      V t = v[i + k + half];
      if (k != 0) {
        if (4 * k == len) {
          t = cmake<V>(t.y, -t.x);  // times W_4^1 = -i
        } else {
          t = cmul(t, tw[k * (R / len) * TWS]);
        }
      }
      v[i + k] = cadd(u, t);
      v[i + k + half] = csub(u, t);
    }
  }
}

template <int R, typename V>
__device__ __forceinline__ void conj_regs(V (&v)[R]) {
#pragma unroll
  for (int i = 0; i < R; ++i) v[i].y = -v[i].y;
}

// Twiddle tables, 3N entries: [0, N) W_N^t; [N, 2N) the forward phase table
// A[k1 * N2 + j2] = W_N^{j2 k1}; [2N, 3N) the transposed phase table
// B[m1 * N1 + k1] = W_N^{k1 m1}.  With A and B, the lane-dependent twiddle of
// the four-step split is read at consecutive addresses by consecutive lanes.
constexpr int kTwiddleTables = 3;

template <typename V>
__device__ __forceinline__ void load_twiddles(V* __restrict__ s_tw, const V* __restrict__ g_tw, int n) {
  for (int i = threadIdx.x; i < kTwiddleTables * n; i += blockDim.x) s_tw[i] = g_tw[i];
}

}  // namespace dgp
