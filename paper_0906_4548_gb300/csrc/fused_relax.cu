// Fused z pass of one relaxation iteration for FP64 mesh data (Secs. III.B-C);
// FP32 mesh data take relax_tma.cu.
//
// A CTA owns TY consecutive rows (x, y0..y0+TY-1) of the mesh.  It
//   1. inverse-transforms along z the six y-inverted spectra H_xx, H_yy, H_xy,
//      H_xz, H_yz, N of those rows, two fields of the same row packed into one
//      complex pencil (A + i B: three transforms per row), and folds them into
//      per-point accumulators held in registers:
//        q = H_xy^2 + H_xz^2 + H_yz^2 + a^2 + a b + b^2 - (a + b) d,
//      (a = H_xx, b = H_yy, d the mean-free D; this is
//      sum_{i<j} (H_ij^2 - H_ii H_jj) with H_zz = d - a - b eliminated), then
//        R = alpha d - 2 q + c2 N - S                    (Eq. FullDGP2, LHS - RHS)
//        B' = (1 - w) d^2 + alpha d - R                  (Eq. Bwpara)
//        Delta = alpha^2 + 4 (1 - w) B', bad points take Delta = 0 (Sec. III.C)
//        D_new = 2 B' / (alpha + sqrt(Delta))            (Eq. nabla^2Cwpara, '+' root)
//   2. writes D_new and forward-transforms it along z into the transposed half
//      spectrum, ready for the next iteration's y pass;
//   3. emits FP64 block partials of sum |R|, sum D_new, bad points, non-finite R.
// The six real Hessian fields, D_new's re-read and two launches never exist.
//
// B' and Delta are formed with the identities
//        B' = d ((1 - w) d + alpha) - R,  Delta = (alpha + 2 (1 - w) d)^2 - 4 (1 - w) R,
// so Delta has no cancellation except where it is genuinely near zero.
// The six spectra arrive as three field pairs; the next pair's tile is copied
// to shared memory with cp.async while the current pair is transformed.
#include <math.h>

#include <type_traits>

#include "fft_core.cuh"
#include "kernels.cuh"

namespace dgp {

// ---------------------------------------------------------------- arithmetic
// Arithmetic of q, R, B' and Delta (FP64).  d is the mean-free D at a point;
// q accumulates sum_{i<j} (H_ij^2 - H_ii H_jj); R, B', Delta as in the file header.
struct ArF64 {
  using Acc = double;
  __device__ static Acc d_of(double D, float, float, double mean) { return D - mean; }
  __device__ static void q_init(Acc& q) { q = 0.0; }
  __device__ static void q_add_sq(Acc& q, double x, double y) { q = fma(x, y, q); }
  __device__ static void q_sub_d(Acc& q, Acc d, double x) { q = fma(-x, d, q); }
  __device__ static Acc residual(Acc q, Acc d, double n, double s, const RelaxParams& rp) {
    return fma(rp.alpha, d, fma(rp.c2, n, -s)) - 2.0 * q;
  }
  __device__ static double bprime(Acc d, Acc R, const RelaxParams& rp) {
    return d * fma(1.0 - rp.w, d, rp.alpha) - R;
  }
  __device__ static double disc(Acc d, Acc R, const RelaxParams& rp, bool& neg) {
    const double s = fma(2.0 * (1.0 - rp.w), d, rp.alpha);
    const double v = fma(s, s, -4.0 * (1.0 - rp.w) * R);
    neg = v < 0.0;
    return v;
  }
  __device__ static double to_f(Acc x) { return x; }
  __device__ static void acc_abs(Acc& a, Acc x) { a += fabs(x); }
  __device__ static double to_d(Acc x) { return x; }
};

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// ---------------------------------------------------------------- geometry
template <typename T, int N> struct FGeom {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int TYW = (sizeof(T) == 8 && N >= 512) ? 4 : 16;
  static constexpr int TY = TYW < N ? TYW : N;          // rows per CTA
  static constexpr int THREADS = TY * N1;
  static constexpr int NK = N / 2 + 1;
  static constexpr int GSZ = 2 * NK * (TY + 1);         // one field pair's half-spectrum tile
  static constexpr int TSZ = TY * N1 * (N2 + 1);        // four-step transpose
  static constexpr int P = TY / 2;                       // row pairs in the forward transform
  // G1 is reused after the second pair: D_new rows (TY x N) then the prefetched
  // S rows (TY x SS, padded when it fits so two rows of a warp use other banks)
  static constexpr int SS_PAD = N + 16;
  static constexpr bool PAD_FITS = (2 * TY * N + TY * 16) * sizeof(T) <= GSZ * 2 * sizeof(T);
  static constexpr int SS = PAD_FITS ? SS_PAD : N;
};

template <typename T> struct FusedArgs {
  const vec2_t<T>* spec[6];  // y-inverted spectra of H_xx, H_yy, H_xy, H_xz, H_yz, N
  const T* D;                // current iterate (its mean = dsum / N^3)
  const double* dsum;
  const T* S;                // source field
  T* Dnew;                   // next iterate
  vec2_t<T>* Snew;           // z-transformed next iterate, layout S[kz][x][y]
  double* partials;          // [blocks][4]
  RelaxParams rp;
  const int* skip;
};

// Start copying the TY-row tile of spectra A and B into G (layout
// [field][kz][TY + 1], complex).
template <typename T, int N>
__device__ __forceinline__ void issue_pair(const vec2_t<T>* __restrict__ A, const vec2_t<T>* __restrict__ B, int x,
                                           int y0, vec2_t<T>* G) {
  using G_ = FGeom<T, N>;
  constexpr int TY = G_::TY, NK = G_::NK, THREADS = G_::THREADS;
  static_assert(THREADS % TY == 0, "each thread copies one column of the tile");
  constexpr int KZS = THREADS / TY;               // kz rows per round
  constexpr int ROUNDS = (NK + KZS - 1) / KZS;
  const int yl = threadIdx.x % TY, kz0 = threadIdx.x / TY;
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const vec2_t<T>* src = (f == 0 ? A : B) + ((int64_t)kz0 * N + x) * N + y0 + yl;
    vec2_t<T>* dst = G + f * NK * (TY + 1) + kz0 * (TY + 1) + yl;
#pragma unroll
    for (int i = 0; i < ROUNDS; ++i) {
      if (i < ROUNDS - 1 || kz0 + i * KZS < NK) {
        if constexpr (sizeof(T) == 8) cp_async_16(dst + i * KZS * (TY + 1), src + (int64_t)i * KZS * N * N);
        else cp_async_8(dst + i * KZS * (TY + 1), src + (int64_t)i * KZS * N * N);
      }
    }
  }
  cp_commit();
}

// Start copying the TY rows of the source S (16-byte pieces) into s_S with row stride SS.
template <typename T, int N>
__device__ __forceinline__ void issue_source(const T* __restrict__ S, int64_t rbase0, T* s_S) {
  constexpr int TY = FGeom<T, N>::TY, SS = FGeom<T, N>::SS;
  constexpr int PER = 16 / sizeof(T);  // elements per 16-byte copy
  for (int item = threadIdx.x; item < TY * N / PER; item += blockDim.x) {
    const int r = item / (N / PER), c = (item % (N / PER)) * PER;
    cp_async_16(s_S + r * SS + c, S + rbase0 + (int64_t)r * N + c);
  }
  cp_commit();
}

// Inverse z transform of the tile in G: per row Z = A + i B rebuilt over all
// k from the half spectra (imaginary parts of k = 0 and N/2 dropped), read in
// place by phase 1.  Thread (row, lane) ends with A (ra) and B (rb) of its row
// at z = lane + N1 k2.
template <typename T, int N>
__device__ __forceinline__ void pair_c2r(const vec2_t<T>* G, vec2_t<T>* s_T, const vec2_t<T>* s_tw,
                                         T (&ra)[Split<N>::N2], T (&rb)[Split<N>::N2]) {
  using V = vec2_t<T>;
  using G_ = FGeom<T, N>;
  constexpr int N1 = G_::N1, N2 = G_::N2, TY = G_::TY, NK = G_::NK;
  const V* GA = G;
  const V* GB = G + NK * (TY + 1);
  const int lane = threadIdx.x % N1, row = threadIdx.x / N1;
  V* Tp = s_T + row * (N1 * (N2 + 1));
  if (lane < N2) {
    V v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int k = N2 * j1 + lane;
      V A, B;
      // j1 is a compile-time index: whole blocks of k below or above N/2 need no test
      if (N2 * j1 + N2 - 1 < N / 2) {
        A = GA[k * (TY + 1) + row];
        B = GB[k * (TY + 1) + row];
        if (j1 == 0 && lane == 0) { A.y = 0; B.y = 0; }
      } else if (N2 * j1 > N / 2) {
        A = cconj(GA[(N - k) * (TY + 1) + row]);
        B = cconj(GB[(N - k) * (TY + 1) + row]);
      } else if (k <= N / 2) {
        A = GA[k * (TY + 1) + row];
        B = GB[k * (TY + 1) + row];
        if (k == 0 || k == N / 2) { A.y = 0; B.y = 0; }
      } else {
        A = cconj(GA[(N - k) * (TY + 1) + row]);
        B = cconj(GB[(N - k) * (TY + 1) + row]);
      }
      v[j1] = cmake<V>(A.x - B.y, -(A.y + B.x));  // conj(A + i B)
    }
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      Tp[k1 * (N2 + 1) + lane] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + lane]);
  }
  __syncthreads();
  V u[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[lane * (N2 + 1) + j2];
  dft_regs<N2, N / N2>(u, s_tw);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    ra[k2] = u[k2].x;
    rb[k2] = -u[k2].y;
  }
}

template <typename T, int N, class AR>
__global__ void __launch_bounds__(FGeom<T, N>::THREADS, 2)
    k_fused_relax(const __grid_constant__ FusedArgs<T> args, const vec2_t<T>* __restrict__ g_tw) {
  if (args.skip && *args.skip) return;
  using V = vec2_t<T>;
  using G_ = FGeom<T, N>;
  using Acc = typename AR::Acc;
  constexpr int N1 = G_::N1, N2 = G_::N2, TY = G_::TY, NK = G_::NK, P = G_::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s_tw = reinterpret_cast<V*>(smem_raw);
  V* G0 = s_tw + kTwiddleTables * N;
  V* G1 = G0 + G_::GSZ;
  V* s_T = G1 + G_::GSZ;
  const int x = blockIdx.y, y0 = blockIdx.x * TY;
  const int lane = threadIdx.x % N1, row = threadIdx.x / N1;
  const int64_t rbase = ((int64_t)x * N + y0 + row) * N;
  const RelaxParams& rp = args.rp;
  // pairs (H_xx, H_yy) -> G0 and (H_xy, H_xz) -> G1 start loading now
  issue_pair<T, N>(args.spec[0], args.spec[1], x, y0, G0);
  issue_pair<T, N>(args.spec[2], args.spec[3], x, y0, G1);
  load_twiddles(s_tw, g_tw, N);
  // mean of D, split once per CTA into a float pair (no per-point FP64 work)
  __shared__ double s_mean;
  __shared__ float s_mpair[2];
  if (threadIdx.x == 0) {
    const double m = args.dsum ? args.dsum[0] * rp.inv_m : 0.0;
    s_mean = m;
    s_mpair[0] = (float)m;
    s_mpair[1] = (float)(m - (double)s_mpair[0]);
  }
  __syncthreads();
  const double mean = s_mean;
  const float m_hi = s_mpair[0], m_lo = s_mpair[1];
  Acc d[N2], q[N2];
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    d[k2] = AR::d_of(args.D[rbase + lane + N1 * k2], m_hi, m_lo, mean);
    AR::q_init(q[k2]);
  }
  T ra[N2], rb[N2];
#pragma unroll 1
  for (int pr = 0; pr < 3; ++pr) {
    cp_wait<1>();  // groups: pair 0, pair 1, pair 2 (issued at pr 0), S (issued at pr 1)
    __syncthreads();  // tile pr visible; s_T free
    pair_c2r<T, N>((pr & 1) ? G1 : G0, s_T, s_tw, ra, rb);
    // pair_c2r's barrier follows its last read of the tile, so the buffer is free
    if (pr == 0) issue_pair<T, N>(args.spec[4], args.spec[5], x, y0, G0);
    if (pr == 1) issue_source<T, N>(args.S, ((int64_t)x * N + y0) * N, reinterpret_cast<T*>(G1) + TY * N);
    if (pr == 0) {
      // a = H_xx, b = H_yy:  q = a^2 + a b + b^2 - (a + b) d
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        AR::q_add_sq(q[k2], ra[k2], ra[k2]);
        AR::q_add_sq(q[k2], ra[k2], rb[k2]);
        AR::q_add_sq(q[k2], rb[k2], rb[k2]);
        AR::q_sub_d(q[k2], d[k2], ra[k2]);
        AR::q_sub_d(q[k2], d[k2], rb[k2]);
      }
    } else if (pr == 1) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        AR::q_add_sq(q[k2], ra[k2], ra[k2]);
        AR::q_add_sq(q[k2], rb[k2], rb[k2]);
      }
    } else {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) AR::q_add_sq(q[k2], ra[k2], ra[k2]);
    }
  }
  // residual, update, statistics (rb holds N)
  T alpha_t, bad_bp;
  if constexpr (sizeof(T) == 8) {
    alpha_t = rp.alpha;
    bad_bp = -rp.alpha * rp.alpha / (4.0 * (1.0 - rp.w));
  } else {
    alpha_t = rp.alpha_f;
    bad_bp = rp.bad_bp_f;
  }
  T* s_dn = reinterpret_cast<T*>(G1);  // TY rows of D_new (G1 is free: pair 1 is done)
  const T* s_S = s_dn + TY * N;
  cp_wait<0>();
  __syncthreads();  // S rows visible
  Acc acc_r;
  AR::q_init(acc_r);
  // the sum of D_new sets the mean removed next iteration: double for double data
  T acc_d = (T)0;
  float nbad = 0.f, nonfin = 0.f;
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const int z = lane + N1 * k2;
    const int64_t idx = rbase + z;
    const Acc R = AR::residual(q[k2], d[k2], rb[k2], s_S[row * G_::SS + z], rp);
    T bpt = (T)AR::bprime(d[k2], R, rp);
    bool neg;
    T dt = (T)AR::disc(d[k2], R, rp, neg);
    if (neg) {
      nbad += 1.f;
      bpt = bad_bp;
      dt = (T)0;
    }
    const T dn = (T)2 * bpt / (alpha_t + sqrt(dt));
    args.Dnew[idx] = dn;
    s_dn[row * N + z] = dn;
    if (isfinite(AR::to_f(R))) AR::acc_abs(acc_r, R);
    else nonfin += 1.f;
    acc_d += dn;
  }
  __syncthreads();
  // forward z transform of D_new (two rows per pencil, as fft_z.cu), written transposed
  V* s_Zf = G0;  // N * (P + 1) complex
  constexpr int FT = P * N1;
  const int fl = threadIdx.x % N1, fp = threadIdx.x / N1;
  V* Tp = s_T + fp * (N1 * (N2 + 1));
  if (threadIdx.x < FT && fl < N2) {
    V v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      v[j1].x = s_dn[(2 * fp) * N + N2 * j1 + fl];
      v[j1].y = s_dn[(2 * fp + 1) * N + N2 * j1 + fl];
    }
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      Tp[k1 * (N2 + 1) + fl] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + fl]);
  }
  __syncthreads();
  if (threadIdx.x < FT) {
    V u[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[fl * (N2 + 1) + j2];
    dft_regs<N2, N / N2>(u, s_tw);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) s_Zf[(fl + N1 * k2) * (P + 1) + fp] = u[k2];
  }
  __syncthreads();
  {
    // thread (kz0, yl) writes kz = kz0, kz0 + KZS, ... of column yl
    constexpr int THREADS = G_::THREADS, KZS = THREADS / TY, ROUNDS = (NK + KZS - 1) / KZS;
    const int yl = threadIdx.x % TY, kz0 = threadIdx.x / TY, p = yl >> 1;
    const bool odd = yl & 1;
    V* dst = args.Snew + ((int64_t)kz0 * N + x) * N + y0 + yl;
#pragma unroll
    for (int i = 0; i < ROUNDS; ++i) {
      const int kz = kz0 + i * KZS;
      if (i < ROUNDS - 1 || kz < NK) {
        const V zk = s_Zf[kz * (P + 1) + p];
        const V zm = s_Zf[((N - kz) % N) * (P + 1) + p];
        V r;
        if (!odd) r = cmake<V>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
        else r = cmake<V>((T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x));
        dst[(int64_t)i * KZS * N * N] = r;
      }
    }
  }
  // block statistics in FP64
  __shared__ double s_part[4][32];
  const int wl = threadIdx.x & 31, wid = threadIdx.x >> 5;
  {
    double v4[4] = {AR::to_d(acc_r), (double)acc_d, (double)nbad, (double)nonfin};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v4[c] += __shfl_xor_sync(0xffffffffu, v4[c], o);
      if (wl == 0) s_part[c][wid] = v4[c];
    }
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int nw = (blockDim.x + 31) >> 5;
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += s_part[threadIdx.x][w];
    args.partials[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = t;
  }
}

template <typename T, int N> int fused_relax_blocks() { return (N / FGeom<T, N>::TY) * N; }

template <typename T, int N, class AR>
static void launch_f(const FusedArgs<T>& a, const vec2_t<T>* tw, cudaStream_t s) {
  using G = FGeom<T, N>;
  const size_t smem = sizeof(vec2_t<T>) * (kTwiddleTables * N + 2 * G::GSZ + G::TSZ);
  raise_smem_limit<k_fused_relax<T, N, AR>>(smem);
  dim3 grid(N / G::TY, N);
  k_fused_relax<T, N, AR><<<grid, G::THREADS, smem, s>>>(a, tw);
}

template <typename T, int N>
void launch_fused_relax(int, vec2_t<T>* const* spec6, const T* D, const double* dsum, const T* S, T* Dnew,
                        vec2_t<T>* Snew, RelaxParams rp, double* partials, const vec2_t<T>* tw, cudaStream_t s,
                        const int* skip) {
  static_assert(sizeof(T) == 8, "FP32 mesh data take launch_relax_tma");
  FusedArgs<T> a;
  a.skip = skip;
  for (int i = 0; i < 6; ++i) a.spec[i] = spec6[i];
  a.D = D; a.dsum = dsum; a.S = S; a.Dnew = Dnew; a.Snew = Snew; a.partials = partials; a.rp = rp;
  launch_f<T, N, ArF64>(a, tw, s);
}

#define DGP_INST_F(T, N)                                                                                    \
  template void launch_fused_relax<T, N>(int, vec2_t<T>* const*, const T*, const double*, const T*, T*,       \
                                         vec2_t<T>*, RelaxParams, double*, const vec2_t<T>*, cudaStream_t,  \
                                         const int*);                                                       \
  template int fused_relax_blocks<T, N>();
#define DGP_INST_F_ALL(T) DGP_INST_F(T, 16) DGP_INST_F(T, 32) DGP_INST_F(T, 64) DGP_INST_F(T, 128) \
  DGP_INST_F(T, 256) DGP_INST_F(T, 512) DGP_INST_F(T, 48) DGP_INST_F(T, 96)
DGP_INST_F_ALL(double)

}  // namespace dgp
