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

// cos(pi j / 16) for any integer j, from its values on [0, pi/2] (decimal
// expansions of the exact constants) and the symmetries of cos.
__host__ __device__ constexpr double cos_pi16(int j) {
  j = ((j % 32) + 32) % 32;
  if (j > 16) j = 32 - j;
  if (j > 8) return -cos_pi16(16 - j);
  return j == 0 ? 1.0
       : j == 1 ? 0.98078528040323044913
       : j == 2 ? 0.92387953251128675613
       : j == 3 ? 0.83146961230254523708
       : j == 4 ? 0.70710678118654752440
       : j == 5 ? 0.55557023301960222474
       : j == 6 ? 0.38268343236508977173
       : j == 7 ? 0.19509032201612826785
       : 0.0;
}

// W_32^j = exp(-2 pi i j / 32) = (cos(pi j / 16), -sin(pi j / 16)) in constant
// memory; with a compile-time index the FMA reads it as a constant-bank operand.
#define DGP_W32(j) {cos_pi16(j), -cos_pi16((j) - 8)}
#define DGP_W32F(j) {(float)cos_pi16(j), (float)-cos_pi16((j) - 8)}
static __constant__ double2 c_w32d[32] = {
    DGP_W32(0),  DGP_W32(1),  DGP_W32(2),  DGP_W32(3),  DGP_W32(4),  DGP_W32(5),  DGP_W32(6),  DGP_W32(7),
    DGP_W32(8),  DGP_W32(9),  DGP_W32(10), DGP_W32(11), DGP_W32(12), DGP_W32(13), DGP_W32(14), DGP_W32(15),
    DGP_W32(16), DGP_W32(17), DGP_W32(18), DGP_W32(19), DGP_W32(20), DGP_W32(21), DGP_W32(22), DGP_W32(23),
    DGP_W32(24), DGP_W32(25), DGP_W32(26), DGP_W32(27), DGP_W32(28), DGP_W32(29), DGP_W32(30), DGP_W32(31)};
static __constant__ float2 c_w32f[32] = {
    DGP_W32F(0),  DGP_W32F(1),  DGP_W32F(2),  DGP_W32F(3),  DGP_W32F(4),  DGP_W32F(5),  DGP_W32F(6),
    DGP_W32F(7),  DGP_W32F(8),  DGP_W32F(9),  DGP_W32F(10), DGP_W32F(11), DGP_W32F(12), DGP_W32F(13),
    DGP_W32F(14), DGP_W32F(15), DGP_W32F(16), DGP_W32F(17), DGP_W32F(18), DGP_W32F(19), DGP_W32F(20),
    DGP_W32F(21), DGP_W32F(22), DGP_W32F(23), DGP_W32F(24), DGP_W32F(25), DGP_W32F(26), DGP_W32F(27),
    DGP_W32F(28), DGP_W32F(29), DGP_W32F(30), DGP_W32F(31)};
#undef DGP_W32
#undef DGP_W32F

// W_R^m for R dividing 32.
template <typename V, int R>
__device__ __forceinline__ V twiddle_c(int m) {
  const int j = ((32 / R) * m) & 31;
  if constexpr (sizeof(V) == 16) return c_w32d[j];
  else return c_w32f[j];
}

// Radix-2 decimation in time, natural order in and out, R a power of two <= 32.
template <int R, typename V>
__device__ __forceinline__ void dft_regs_pow2(V (&v)[R]) {
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
        } else if (8 * k == len) {
          // times W_8^1 = (1 - i) / sqrt(2)
          const auto c = (decltype(V::x))0.70710678118654752440;
          t = cmake<V>((t.x + t.y) * c, (t.y - t.x) * c);
        } else if (8 * k == 3 * len) {
          // times W_8^3 = -(1 + i) / sqrt(2)
          const auto c = (decltype(V::x))0.70710678118654752440;
          t = cmake<V>((t.y - t.x) * c, -(t.x + t.y) * c);
        } else {
          t = cmul(t, twiddle_c<V, R>(k * (R / len)));
        }
      }
      v[i + k] = cadd(u, t);
      v[i + k + half] = csub(u, t);
    }
  }
}

// 3-point DFT in place: with W_3 = -1/2 - i h, h = sqrt(3)/2,
// X0 = a + s, X1 = t - i h d, X2 = t + i h d, where s = b + c, d = b - c,
// t = a - s/2.
template <typename V>
__device__ __forceinline__ void dft3(V& a, V& b, V& c) {
  using S = decltype(V::x);
  const S h = (S)0.86602540378443864676;  // sqrt(3) / 2
  const V s = cadd(b, c), d = csub(b, c);
  const V t = cmake<V>(a.x - (S)0.5 * s.x, a.y - (S)0.5 * s.y);
  a = cadd(a, s);
  b = cmake<V>(t.x + h * d.y, t.y - h * d.x);
  c = cmake<V>(t.x - h * d.y, t.y + h * d.x);
}

// Forward DFT of the R values in v (natural order in and out): R = 3 directly,
// R = 6 as two 3-point DFTs of the even and odd elements combined with
// W_6^k = 1/2 - i h, -1/2 - i h (decimation in time), otherwise radix-2
// decimation in time for R <= 32 with compile-time twiddle constants.
template <int R, int TWS, typename V>
__device__ __forceinline__ void dft_regs(V (&v)[R], const V* __restrict__ tw) {
  if constexpr (R == 3) {
    dft3(v[0], v[1], v[2]);
  } else if constexpr (R == 6) {
    using S = decltype(V::x);
    const S h = (S)0.86602540378443864676, half = (S)0.5;
    V e0 = v[0], e1 = v[2], e2 = v[4], o0 = v[1], o1 = v[3], o2 = v[5];
    dft3(e0, e1, e2);
    dft3(o0, o1, o2);
    const V t1 = cmake<V>(half * o1.x + h * o1.y, half * o1.y - h * o1.x);    // W_6^1 o1
    const V t2 = cmake<V>(-half * o2.x + h * o2.y, -half * o2.y - h * o2.x);  // W_6^2 o2
    v[0] = cadd(e0, o0);
    v[3] = csub(e0, o0);
    v[1] = cadd(e1, t1);
    v[4] = csub(e1, t1);
    v[2] = cadd(e2, t2);
    v[5] = csub(e2, t2);
  } else {
    dft_regs_pow2<R>(v);
  }
  (void)tw;
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
