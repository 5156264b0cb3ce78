// Shared types and small helpers of the DGP CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace dgp {

// Raise the dynamic shared-memory limit of kernel K to `bytes` (its largest
// launch) once per device.  Setting the attribute before every launch would
// let one host thread lower it between another thread's set and launch; a
// failure is returned and also left for the launch check that follows.
template <auto K>
inline cudaError_t raise_smem_limit(size_t bytes) {
  static std::mutex mu;
  static uint64_t done = 0;  // bit d: set on device d
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (dev < 64 && ((done >> dev) & 1u)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using vec2_t = typename Vec2<T>::type;

template <typename V> __host__ __device__ __forceinline__ V cmake(decltype(V::x) a, decltype(V::x) b) {
  V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmake<V>(a.x, -a.y); }
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) {
  return cmake<V>(a.x * s, a.y * s);
}

// Signed wavenumber index of FFT bin i on an n-point axis; the Nyquist bin
// n/2 maps to -n/2 and is flagged.
__device__ __forceinline__ int signed_index(int i, int n) { return i < n / 2 ? i : i - n; }

// Launch geometry of the two-level pencil FFT: N = N1 * N2, N1 >= N2.
template <int N> struct Split;
// N = N1 * N2 with N1 a power of two (the lane count of a pencil) and N2 <= N1
// a power of two, 3 or 6 (meshes of 2^a 3^b points).
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Split<48> { static constexpr int N1 = 16, N2 = 3; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<96> { static constexpr int N1 = 16, N2 = 6; };
template <> struct Split<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct Split<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct Split<512> { static constexpr int N1 = 32, N2 = 16; };

// Per-point statistics of one relaxation update, reduced in FP64.
struct RelaxStats {
  double sum_abs_r;   // sum |R| over the mesh
  double sum_dnew;    // sum of D_new (its mean is projected out next time)
  double nbad;        // number of points with Delta < 0
  double sum_nonfinite;  // count of non-finite R (NaN guard)
};

}  // namespace dgp
