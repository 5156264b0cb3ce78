// x pass: forward DFT along x (stride N inside a kz plane of S[kz][x][y]),
// a k-space operation, and the inverse DFT along x of each output.
//
// A CTA owns one kz plane and TY consecutive ky columns; thread (lane, yl)
// has yl fastest so every global access is TY consecutive complex values.
// After the forward transform lane k1 holds X[k1 + N1*k2] (k2 < N2) in
// registers; an output is formed there, transformed back over k2 in the same
// registers (the inverse four-step with the roles of N1 and N2 swapped),
// transposed through shared memory once and finished over k1.
//
// Operations (all multipliers real-even or i*odd, so outputs stay Hermitian):
//  HESSIAN    D(k) -> (k_i k_j / k^2) D(k) for xx, yy, xy, xz, yz and
//             N(k) = -D(k) / kbar   (Sec. III.B: nabla_ij C(k) = -k_i k_j C(k);
//             sqrt(-lapbar) C = kbar C = -D / kbar).  Off-diagonal pairs with a
//             component on its Nyquist index use |k_i k_j| / k^2.
//  SOURCE     S(k) = s (1 - beta / kbar) delta(k)        (RHS of Eq. FullDGP2)
//  SOURCE_LIN S(k) and D_lin(k) = S(k) / (alpha - c2 / kbar)  (Sec. III.B)
//  PHI_FORCE  phi(k) from Eq. FullDGP1 (or Eq. LinearDGP / GRPoisson) and
//             g_i(k) = -i k_i phi(k), Nyquist component of axis i set to 0.
//  PK         |delta_k|^2 binned in shells (Sec. IV), per-block FP64 partials.
//  SHELL      delta_k and 1 restricted to a |k| shell (bispectrum, Sec. VI).
//  RC         derivative-in-r_c contractions of the solve's adjoint (adjoint_rc.cuh).
// Every output carries the 1 / N^3 of the three inverse transforms.
#include <math.h>

#include <cooperative_groups.h>

#include "adjoint_rc.cuh"
#include "fft_core.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "xy.cuh"

namespace dgp {

template <typename T, int N> struct XGeom {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int TYW = sizeof(T) == 4 ? 16 : 8;
  static constexpr int TY = TYW < N ? TYW : N;
  static constexpr int THREADS = TY * N1;
  // at least two CTAs per SM so one CTA's transposes overlap another's loads
  static constexpr int MIN_BLOCKS = THREADS <= 256 ? 2 : 1;
};

template <typename T> struct XArgs {
  const vec2_t<T>* in0;
  const vec2_t<T>* in1;
  FieldSet<T> out;
  int nout_mask;
  KParams kp;
  double* pk_partials;
  int nbins;
  double shell_lo, shell_hi;
  const int* skip;
  FieldSet<T> in;  // adjoint ops: input spectra
  int in_mask;
  RcDeriv rc;      // XOP_RC: derivatives of the coefficients in r_c H0
};

template <typename T, int N>
__device__ __forceinline__ void x_forward(const vec2_t<T>* __restrict__ in, int kz, int ky0, int lane, int yl,
                                          vec2_t<T>* s_T, const vec2_t<T>* s_tw,
                                          vec2_t<T> (&X)[Split<N>::N2]) {
  using V = vec2_t<T>;
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, TY = XGeom<T, N>::TY;
  const V* plane = in + (int64_t)kz * N * N;
  if (lane < N2) {
    V v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = plane[(int64_t)(N2 * j1 + lane) * N + ky0 + yl];
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      s_T[(k1 * N2 + lane) * TY + yl] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + lane]);
  }
  __syncthreads();
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) X[j2] = s_T[(lane * N2 + j2) * TY + yl];
  dft_regs<N2, N / N2>(X, s_tw);
  __syncthreads();
}

// trailing: end with a barrier so the next call may reuse s_T; callers that alternate
// two transpose buffers between consecutive calls pass false.
template <typename T, int N, bool trailing = true>
__device__ __forceinline__ void x_inverse(vec2_t<T> (&Y)[Split<N>::N2], vec2_t<T>* __restrict__ out, int kz,
                                          int ky0, int lane, int yl, vec2_t<T>* s_T, const vec2_t<T>* s_tw) {
  using V = vec2_t<T>;
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, TY = XGeom<T, N>::TY;
  conj_regs(Y);
  dft_regs<N2, N / N2>(Y, s_tw);
#pragma unroll
  for (int m1 = 0; m1 < N2; ++m1)
    s_T[(m1 * N1 + lane) * TY + yl] = (m1 == 0) ? Y[m1] : cmul(Y[m1], s_tw[2 * N + m1 * N1 + lane]);
  __syncthreads();
  if (lane < N2) {
    V w[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) w[k1] = s_T[(lane * N1 + k1) * TY + yl];
    dft_regs<N1, N / N1>(w, s_tw);
    V* plane = out + (int64_t)kz * N * N;
#pragma unroll
    for (int m2 = 0; m2 < N1; ++m2) plane[(int64_t)(lane + N2 * m2) * N + ky0 + yl] = cconj(w[m2]);
  }
  if (trailing) __syncthreads();
}

// A coefficient in the element type: the host-rounded float for FP32 data, the double otherwise.
template <typename T> __device__ __forceinline__ T kc(double d, float f) {
  if constexpr (sizeof(T) == 8) return d;
  else return f;
}

// G_eff / G of Eq. Geff at |k| (h/Mpc).
__device__ __forceinline__ double geff_dev(const KParams& kp, double kmag) {
  const double eta = kp.eta, q = kp.q;
  const double t1 = (2 * eta * (2 + q) - 3) / (2 * eta * (2 + q) - 4);
  const double r = (eta * (1 + q) - 1) / (eta * (2 + q) - 2);
  const double t2 = 3.0 * kp.a / (kmag * kp.rc_H0 * (kp.kbar_fac * kp.aE)) * r * r;
  return 1.0 / (t1 + t2);
}

// The Hessian spectra (Sec. III.B): H_ab(k) = (n_a n_b / |n|^2) D(k) for (a, b) = xx, yy, xy,
// xz, yz (outputs 0..4), with the absolute value where a component of an off-diagonal pair is
// on its Nyquist index (on the diagonal the product is a square anyway), and N = -D / kbar
// (output 5).  1/|n|^2 and the 1/N^3 of the inverse transforms are folded into the spectrum
// once (hessian_prescale); each output's multiplier is then a product of the wavenumber
// components, formed in registers, and its pair is chosen once per output, so the multiplier
// is branch-free per element.  X[k2] holds kx = lane + N1 k2.
template <typename T, int N>
__device__ __forceinline__ void hessian_prescale(vec2_t<T> (&X)[Split<N>::N2], int lane, T fy, T fz, T inv_m) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  const T nyz2 = fy * fy + fz * fz;
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const T fx = (T)signed_index(lane + N1 * k2, N);
    const T n2 = fx * fx + nyz2;
    X[k2] = cscale(X[k2], n2 != (T)0 ? inv_m / n2 : (T)0);
  }
}

// Output o of the prescaled spectrum X; ikf = 1 / (kbar_fac k_f) (0 in the local-only mode),
// so that |n|^2 / kbar = |n| ikf.
template <typename T, int N>
__device__ __forceinline__ void hessian_output(const vec2_t<T> (&X)[Split<N>::N2], int o, int lane, T fy, T fz,
                                               bool nyq_y, bool nyq_z, T ikf, vec2_t<T> (&Y)[Split<N>::N2]) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  if (o == 5) {
    const T nyz2 = fy * fy + fz * fz;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const T fx = (T)signed_index(lane + N1 * k2, N);
      Y[k2] = cscale(X[k2], -sqrt(fx * fx + nyz2) * ikf);
    }
    return;
  }
  const bool a_is_x = o == 0 || o == 2 || o == 3;             // first component x, else y
  const int b_sel = o == 0 ? 0 : (o == 1 || o == 2 ? 1 : 2);  // second: x, y or z
  const T fb_fixed = b_sel == 1 ? fy : fz;
  const bool nyq_fixed = (!a_is_x && nyq_y) || (b_sel == 1 && nyq_y) || (b_sel == 2 && nyq_z);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const int kx = lane + N1 * k2;
    const T fx = (T)signed_index(kx, N);
    const T fa = a_is_x ? fx : fy;
    const T fb = b_sel == 0 ? fx : fb_fixed;
    T prod = fa * fb;
    const bool nyq = nyq_fixed || ((a_is_x || b_sel == 0) && kx == N / 2);
    if (nyq) prod = fabs(prod);
    Y[k2] = cscale(X[k2], prod);
  }
}

template <typename T, int RB> struct XBatch {
  XArgs<T> a[RB];
};

template <typename T, int N, int OP, int RB>
__global__ void __launch_bounds__(XGeom<T, N>::THREADS, XGeom<T, N>::MIN_BLOCKS)
    k_fft_x(const __grid_constant__ XBatch<T, RB> xb, const vec2_t<T>* __restrict__ g_tw) {
  const XArgs<T>& args = xb.a[RB > 1 ? blockIdx.z : 0];  // realisation of this CTA
  if (args.skip && *args.skip) return;
  using V = vec2_t<T>;
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, TY = XGeom<T, N>::TY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s_tw = reinterpret_cast<V*>(smem_raw);
  V* s_T = s_tw + kTwiddleTables * N;  // N * TY
  // per-thread 1/|n|^2 and 1/kbar for each of the N2 register slots, kept in
  // shared memory so the output loop does not hold 2 * N2 extra registers
  T* s_inv = reinterpret_cast<T*>(s_T + N * TY);               // N2 * THREADS
  T* s_ikb = s_inv + N2 * XGeom<T, N>::THREADS;                // N2 * THREADS
  // P(k) operations (which use neither table): per-warp shell sums
  // [warp][NBS][nbins] and a per-warp staging row [warp][32][NBS]
  constexpr int NW = XGeom<T, N>::THREADS / 32;
  constexpr int NBS = OP == XOP_PK_BRANE ? 4 : 3;  // sums per shell
  double* s_bins = reinterpret_cast<double*>(s_inv);
  V* s_T2 = reinterpret_cast<V*>(s_inv);  // the Hessian op's second transpose buffer (N * TY)
  double* s_stage = s_bins + NW * NBS * args.nbins;
  load_twiddles(s_tw, g_tw, N);
  if (OP == XOP_PK || OP == XOP_PK_BRANE)
    for (int i = threadIdx.x; i < NW * NBS * args.nbins; i += blockDim.x) s_bins[i] = 0.0;
  const int yl = threadIdx.x % TY;
  const int lane = threadIdx.x / TY;
  const int kz = blockIdx.y;
  const int ky0 = blockIdx.x * TY;
  const int ky = ky0 + yl;
  const int nz = kz == N / 2 ? -(N / 2) : kz;
  const int ny = signed_index(ky, N);
  const bool nyq_y = ky == N / 2, nyq_z = kz == N / 2;
  const KParams& kp = args.kp;
  const T kf = kc<T>(2.0 * M_PI / kp.box, kp.kf_f);
  __syncthreads();

  V X0[N2], X1[N2];
  constexpr bool ADJ = OP == XOP_ADJ_PHI || OP == XOP_ADJ_COMBINE || OP == XOP_ZEL_ADJ || OP == XOP_RC;
  if (!ADJ) x_forward<T, N>(args.in0, kz, ky0, lane, yl, s_T, s_tw, X0);
  if (OP == XOP_PHI_FORCE && kp.gravity == 0) x_forward<T, N>(args.in1, kz, ky0, lane, yl, s_T, s_tw, X1);

  if (OP == XOP_PK || OP == XOP_PK_BRANE) {
    // Shell sums in a fixed order, so that P(k) is the same bits on every run:
    // per register slot, the lanes of a warp that fall in one shell are summed
    // by the lowest of them in lane order into that warp's own shell row (the
    // shells of different groups differ, so no two lanes write one address);
    // the warps' rows are then added in warp order.
    const double norm = kp.box * kp.box * kp.box * kp.inv_m * kp.inv_m;
    const double w = (kz == 0 || kz == N / 2) ? 1.0 : 2.0;
    const int wl = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* wbins = s_bins + wid * NBS * args.nbins;
    double* stage = s_stage + wid * 32 * NBS;
    __syncthreads();  // the bins are zeroed
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int nx = signed_index(lane + N1 * k2, N);
      const int n2 = nx * nx + ny * ny + nz * nz;
      const double nm = sqrt((double)n2);
      int b = (int)floor(nm + 0.5);
      if (n2 == 0 || b < 1 || b > args.nbins) b = 0;
      const double p = ((double)X0[k2].x * X0[k2].x + (double)X0[k2].y * X0[k2].y) * norm;
      stage[wl * NBS + 0] = w;
      stage[wl * NBS + 1] = w * nm * (2.0 * M_PI / kp.box);
      stage[wl * NBS + 2] = w * p;
      if (OP == XOP_PK_BRANE) stage[wl * NBS + 3] = n2 ? w * p / ((double)n2 * (double)n2) : 0.0;
      const unsigned group = __match_any_sync(0xffffffffu, b);
      __syncwarp();
      if (b != 0 && wl == __ffs(group) - 1) {
        double acc[NBS];
#pragma unroll
        for (int c = 0; c < NBS; ++c) acc[c] = 0.0;
        for (unsigned g = group; g; g &= g - 1) {
          const int l = __ffs(g) - 1;
#pragma unroll
          for (int c = 0; c < NBS; ++c) acc[c] += stage[l * NBS + c];
        }
#pragma unroll
        for (int c = 0; c < NBS; ++c) wbins[c * args.nbins + b - 1] += acc[c];
      }
      __syncwarp();
    }
    __syncthreads();
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    for (int i = threadIdx.x; i < NBS * args.nbins; i += blockDim.x) {
      double t = 0.0;
      for (int v = 0; v < NW; ++v) t += s_bins[v * NBS * args.nbins + i];
      args.pk_partials[blk * NBS * args.nbins + i] = t;
    }
    return;
  }

  constexpr int NT = XGeom<T, N>::THREADS;
  const T inv_m = kc<T>(kp.inv_m, kp.inv_m_f);
#pragma unroll
  for (int k2 = 0; k2 < N2 && OP != XOP_HESSIAN && OP != XOP_PHI_FORCE; ++k2) {
    const int nx = signed_index(lane + N1 * k2, N);
    const int n2 = nx * nx + ny * ny + nz * nz;
    T inv = (T)0, ikb = (T)0;
    if (n2 != 0) {
      inv = (T)1 / (T)n2;
      if (!kp.local_only) ikb = (T)1 / (kc<T>(kp.kbar_fac * 2.0 * M_PI / kp.box, kp.kbkf_f) * sqrt((T)n2));
    }
    // the Hessian outputs use 1 / (|n|^2 N^3) directly
    s_inv[k2 * NT + threadIdx.x] = OP == XOP_HESSIAN ? inv * inv_m : inv;
    s_ikb[k2 * NT + threadIdx.x] = ikb;
  }

  if constexpr (OP == XOP_RC) {
    // acc: phibar_tot (phase of phibar) or lam (phase of lam); then delta and D in turn
    V acc[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) acc[k2] = cmake<V>((T)0, (T)0);
    const bool lam_phase = (args.in_mask >> 6) & 1;
    if (lam_phase) {
      x_forward<T, N>(args.in.p[6], kz, ky0, lane, yl, s_T, s_tw, acc);
    } else {
#pragma unroll 1
      for (int f = 0; f < 4; ++f) {
        if (!((args.in_mask >> f) & 1)) continue;  // uniform over the block
        x_forward<T, N>(args.in.p[f], kz, ky0, lane, yl, s_T, s_tw, X0);
        const int nfix = f == 2 ? ny : nz;
        const bool nyq_fix = f == 2 ? nyq_y : nyq_z;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          if (f == 0) {
            acc[k2] = cadd(acc[k2], X0[k2]);
          } else {
            const int kx = lane + N1 * k2;
            const bool nyq = f == 1 ? kx == N / 2 : nyq_fix;
            const T ki = kf * (T)(f == 1 ? signed_index(kx, N) : nfix);
            if (!nyq) acc[k2] = cadd(acc[k2], cmake<V>(-ki * X0[k2].y, ki * X0[k2].x));  // i k_i X
          }
        }
      }
    }
    const RcDeriv& d = args.rc;
    const double eta = kp.eta, kfd = 2.0 * M_PI / kp.box;
    const double om = (eta - 1.0) / eta, dom = d.deta / (eta * eta);
    double t = 0.0;
#pragma unroll 1
    for (int f = 4; f < 6; ++f) {  // delta, then D
      x_forward<T, N>(args.in.p[f], kz, ky0, lane, yl, s_T, s_tw, X0);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int nx = signed_index(lane + N1 * k2, N);
        const int n2 = nx * nx + ny * ny + nz * nz;
        if (n2 == 0) continue;
        const double kmag = kfd * sqrt((double)n2);
        const double ikb = kp.local_only ? 0.0 : 1.0 / (kp.kbar_fac * kmag);
        const double dikb = ikb * d.dE_over_E;  // 1/kbar = a E / (C_H |k|)
        double m;
        if (!lam_phase) {
          const double pref = -kp.aE * kp.aE / (kmag * kmag), dpref = 2.0 * pref * d.dE_over_E;
          const double den = 1.0 + ikb / eta, dden = dikb / eta - ikb * d.deta / (eta * eta);
          if (f == 4) {  // A' = d/drc [1.5 pref om / den]
            m = 1.5 * (dpref * om / den + pref * dom / den - pref * om * dden / (den * den));
          } else {       // B' = d/drc [pref (-1/(2 eta) + c3 / kbar) / den]
            const double b = -0.5 / eta + kp.c3 * ikb;
            const double db = d.deta / (2.0 * eta * eta) + d.dc3 * ikb + kp.c3 * dikb;
            m = dpref * b / den + pref * db / den - pref * b * dden / (den * den);
          }
        } else if (f == 4) {  // S' = d/drc [s (1 - beta / kbar)]
          m = d.ds * (1.0 - kp.beta * ikb) - kp.s * (d.dbeta * ikb + kp.beta * dikb);
        } else {              // -(alpha' + c2' N + c2 N'), N = -1/kbar
          m = -d.dalpha + d.dc2 * ikb + kp.c2 * dikb;
        }
        t += m * ((double)acc[k2].x * (double)X0[k2].x + (double)acc[k2].y * (double)X0[k2].y);
      }
    }
    if (kz != 0 && kz != N / 2) t *= 2.0;
    double v[1] = {t};
    block_sum<1>(v);
    if (threadIdx.x == 0) args.pk_partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = v[0];
    return;
  }

  if (OP == XOP_ADJ_PHI || OP == XOP_ZEL_ADJ) {
    const T inv_m = kc<T>(kp.inv_m, kp.inv_m_f);
    V acc[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) acc[k2] = cmake<V>((T)0, (T)0);
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      if (!((args.in_mask >> f) & 1)) continue;  // uniform over the block
      x_forward<T, N>(args.in.p[f], kz, ky0, lane, yl, s_T, s_tw, X0);
      const int nfix = f == 2 ? ny : nz;            // component of axis f - 1 when it is y or z
      const bool nyq_fix = f == 2 ? nyq_y : nyq_z;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        if (f == 0) {
          acc[k2] = cadd(acc[k2], X0[k2]);
        } else {
          const int kx = lane + N1 * k2;
          const bool nyq = f == 1 ? kx == N / 2 : nyq_fix;
          const T ki = kf * (T)(f == 1 ? signed_index(kx, N) : nfix);
          if (!nyq) acc[k2] = cadd(acc[k2], cmake<V>(-ki * X0[k2].y, ki * X0[k2].x));  // i k_i X
        }
      }
    }
    const T om15 = kc<T>(1.5 * (kp.eta - 1.0) / kp.eta, kp.om15_f);
#pragma unroll 1
    for (int o = 0; o < (OP == XOP_ZEL_ADJ ? 1 : 2); ++o) {
      V Y[N2];
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int nx = signed_index(lane + N1 * k2, N);
        const int n2 = nx * nx + ny * ny + nz * nz;
        Y[k2] = cmake<V>((T)0, (T)0);
        if (n2 != 0) {
          const T kmag = kf * sqrt((T)n2);
          T m;
          if (OP == XOP_ZEL_ADJ) {
            m = (T)-1 / (kmag * kmag);
          } else {
            const T ikb = s_ikb[k2 * NT + threadIdx.x];
            const T pref = -kc<T>(kp.aE * kp.aE, kp.aE2_f) / (kmag * kmag);
            const T den = (T)1 + ikb * kc<T>(1.0 / kp.eta, kp.inv_eta_f);
            const T cd = -kc<T>(0.5 / kp.eta, kp.half_inv_eta_f) + kc<T>(kp.c3, kp.c3_f) * ikb;
            m = (o == 0 ? cd : om15) * pref / den;
          }
          Y[k2] = cscale(acc[k2], m * inv_m);
        }
      }
      x_inverse<T, N>(Y, args.out.p[o], kz, ky0, lane, yl, s_T, s_tw);
    }
    return;
  }

  if (OP == XOP_ADJ_COMBINE) {
    const T inv_m = kc<T>(kp.inv_m, kp.inv_m_f);
    const T fy = (T)ny, fz = (T)nz;
    V acc[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) acc[k2] = cmake<V>((T)0, (T)0);
#pragma unroll 1
    for (int f = 0; f < 7; ++f) {
      x_forward<T, N>(args.in.p[f], kz, ky0, lane, yl, s_T, s_tw, X0);
      // pair (a, b) of input f: xx, yy, zz, xy, xz, yz; weight -2 (diagonal) or -4 (twice off-diagonal)
      const int ca = f == 0 || f == 3 || f == 4 ? 0 : (f == 1 || f == 5 ? 1 : 2);
      const int cb = f == 0 ? 0 : (f == 1 || f == 3 ? 1 : 2);
      const T wgt = f < 3 ? (T)-2 : (T)-4;
      const T fa_fix = ca == 1 ? fy : fz, fb_fix = cb == 1 ? fy : fz;
      const bool nyq_fix = (ca != 0 && (ca == 1 ? nyq_y : nyq_z)) || (cb != 0 && (cb == 1 ? nyq_y : nyq_z));
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int kx = lane + N1 * k2;
        const T fx = (T)signed_index(kx, N);
        const T inv_n2 = s_inv[k2 * NT + threadIdx.x];
        T m;
        if (f == 6) {
          m = -kc<T>(kp.c2, kp.c2_f) * s_ikb[k2 * NT + threadIdx.x];  // c2 N = c2 (-1/kbar)
        } else {
          T prod = (ca == 0 ? fx : fa_fix) * (cb == 0 ? fx : fb_fix);
          if (ca != cb && (nyq_fix || ((ca == 0 || cb == 0) && kx == N / 2))) prod = fabs(prod);
          m = wgt * prod * inv_n2;
        }
        acc[k2] = cadd(acc[k2], cscale(X0[k2], m));
      }
    }
    V Y[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) Y[k2] = cscale(acc[k2], inv_m);
    x_inverse<T, N>(Y, args.out.p[0], kz, ky0, lane, yl, s_T, s_tw);
    return;
  }

  if (OP == XOP_HESSIAN) {
    const T fy = (T)ny, fz = (T)nz;
    hessian_prescale<T, N>(X0, lane, fy, fz, inv_m);
    const T ikf = kp.local_only ? (T)0 : (T)1 / kc<T>(kp.kbar_fac * 2.0 * M_PI / kp.box, kp.kbkf_f);
#pragma unroll 1
    for (int o = 0; o < 6; ++o) {
      V Y[N2];
      hessian_output<T, N>(X0, o, lane, fy, fz, nyq_y, nyq_z, ikf, Y);
      // the outputs alternate between two transpose buffers: one barrier per output
      x_inverse<T, N, false>(Y, args.out.p[o], kz, ky0, lane, yl, (o & 1) ? s_T2 : s_T, s_tw);
    }
    return;
  }

  if constexpr (OP == XOP_PHI_FORCE) {
    // phi(k) once per slot, in place of X0 (Eq. FullDGP1 with the D spectrum X1; Eq. LinearDGP
    // with G_eff of Eq. Geff; Eq. GRPoisson), with the 1/N^3 of the inverse transforms; then each
    // requested output: phi (bit 0) or g_i = -i k_i phi (bits 1..3, Nyquist component of axis
    // i zero).  The outputs alternate between two transpose buffers.
    const T fy = (T)ny, fz = (T)nz;
    const T nyz2 = fy * fy + fz * fz;
    const T om15 = kc<T>(1.5 * (kp.eta - 1.0) / kp.eta, kp.om15_f);
    const T aE2m = kc<T>(kp.aE * kp.aE, kp.aE2_f) * inv_m;
    const T kf2 = kf * kf;
    const T ikf = kp.local_only ? (T)0 : (T)1 / kc<T>(kp.kbar_fac * 2.0 * M_PI / kp.box, kp.kbkf_f);
    const T inv_eta = kc<T>(1.0 / kp.eta, kp.inv_eta_f);
    const T half_inv_eta = kc<T>(0.5 / kp.eta, kp.half_inv_eta_f);
    const T c3 = kc<T>(kp.c3, kp.c3_f);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const T fx = (T)signed_index(lane + N1 * k2, N);
      const T n2 = fx * fx + nyz2;
      if (n2 == (T)0) {
        X0[k2] = cmake<V>((T)0, (T)0);
        continue;
      }
      const T pref = -aE2m / (kf2 * n2);
      if (kp.gravity == 0) {
        const T ikb = ikf / sqrt(n2);  // 1 / kbar
        const T cd = -half_inv_eta + c3 * ikb;
        const T f = pref / ((T)1 + ikb * inv_eta);
        X0[k2] = cmake<V>(f * (om15 * X0[k2].x + cd * X1[k2].x), f * (om15 * X0[k2].y + cd * X1[k2].y));
      } else if (kp.gravity == 1) {
        X0[k2] = cscale(X0[k2], pref * om15 * (T)geff_dev(kp, (double)(kf * sqrt(n2))));
      } else {
        X0[k2] = cscale(X0[k2], pref * om15);
      }
    }
    int cnt = 0;
#pragma unroll 1
    for (int o = 0; o < 4; ++o) {
      if (!((args.nout_mask >> o) & 1)) continue;  // uniform over the block
      V Y[N2];
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        if (o == 0) {
          Y[k2] = X0[k2];
        } else {
          const int kx = lane + N1 * k2;
          const bool nyq = o == 1 ? kx == N / 2 : (o == 2 ? nyq_y : nyq_z);
          const T ki = kf * (o == 1 ? (T)signed_index(kx, N) : (o == 2 ? fy : fz));
          // g = -grad phi -> -i k_i phi
          Y[k2] = nyq ? cmake<V>((T)0, (T)0) : cmake<V>(ki * X0[k2].y, -ki * X0[k2].x);
        }
      }
      x_inverse<T, N, false>(Y, args.out.p[o], kz, ky0, lane, yl, (cnt & 1) ? s_T2 : s_T, s_tw);
      ++cnt;
    }
    return;
  }

  if (OP == XOP_PK_ADJ) {
    V Y[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int nx = signed_index(lane + N1 * k2, N);
      const int n2 = nx * nx + ny * ny + nz * nz;
      Y[k2] = cmake<V>((T)0, (T)0);
      if (n2 != 0) {
        const int b = (int)floor(sqrt((double)n2) + 0.5);  // the shell of the P(k) estimator
        if (b >= 1 && b <= args.nbins) Y[k2] = cscale(X0[k2], (T)(2.0 * args.pk_partials[b - 1]));
      }
    }
    x_inverse<T, N>(Y, args.out.p[0], kz, ky0, lane, yl, s_T, s_tw);
    return;
  }
  if (OP == XOP_ZEL) {
    const T inv_m = kc<T>(kp.inv_m, kp.inv_m_f);
#pragma unroll 1
    for (int o = 0; o < 3; ++o) {
      const int nfix = o == 1 ? ny : nz;
      const bool nyq_fix = o == 1 ? nyq_y : nyq_z;
      V Y[N2];
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int kx = lane + N1 * k2;
        const int nx = signed_index(kx, N);
        const int n2 = nx * nx + ny * ny + nz * nz;
        const bool nyq = o == 0 ? kx == N / 2 : nyq_fix;
        Y[k2] = cmake<V>((T)0, (T)0);
        if (n2 != 0 && !nyq) {
          const T ki = kf * (T)(o == 0 ? nx : nfix);
          const T m = ki / (kf * kf * (T)n2) * inv_m;
          Y[k2] = cmake<V>(-m * X0[k2].y, m * X0[k2].x);  // (i k_j / k^2) X
        }
      }
      x_inverse<T, N>(Y, args.out.p[o], kz, ky0, lane, yl, s_T, s_tw);
    }
    return;
  }

  int nout;
  if (OP == XOP_HESSIAN) nout = 6;
  else if (OP == XOP_SOURCE) nout = 1;
  else if (OP == XOP_SOURCE_LIN || OP == XOP_SHELL) nout = 2;
  else nout = 4;
  for (int o = 0; o < nout; ++o) {
    if (OP == XOP_PHI_FORCE && !((args.nout_mask >> o) & 1)) continue;
    V Y[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int kx = lane + N1 * k2;
      const int nx = signed_index(kx, N);
      const bool nyq_x = kx == N / 2;
      const int n2 = nx * nx + ny * ny + nz * nz;
      V r = cmake<V>((T)0, (T)0);
      if (n2 != 0) {
        const T inv_n2 = s_inv[k2 * NT + threadIdx.x];
        // 1 / kbar = 1 / (kbar_fac * kf * |n|)
        const T ikb = s_ikb[k2 * NT + threadIdx.x];
        if (OP == XOP_HESSIAN) {
          T m;
          switch (o) {
            case 0: m = (T)(nx * nx) * inv_n2; break;
            case 1: m = (T)(ny * ny) * inv_n2; break;
            case 2: m = (T)((nyq_x || nyq_y) ? abs(nx * ny) : nx * ny) * inv_n2; break;
            case 3: m = (T)((nyq_x || nyq_z) ? abs(nx * nz) : nx * nz) * inv_n2; break;
            case 4: m = (T)((nyq_y || nyq_z) ? abs(ny * nz) : ny * nz) * inv_n2; break;
            default: m = -ikb; break;
          }
          r = cscale(X0[k2], m * inv_m);
        } else if (OP == XOP_SOURCE || OP == XOP_SOURCE_LIN) {
          const T sfac = kc<T>(kp.s, kp.s_f) * ((T)1 - kc<T>(kp.beta, kp.beta_f) * ikb) * inv_m;
          r = cscale(X0[k2], sfac);
          if (o == 1) r = cscale(r, (T)1 / (kc<T>(kp.alpha, kp.alpha_f) - kc<T>(kp.c2, kp.c2_f) * ikb));
        } else if (OP == XOP_SHELL) {
          const double nm = sqrt((double)n2);
          if (nm > args.shell_lo && nm < args.shell_hi)
            r = (o == 0) ? cscale(X0[k2], inv_m) : cmake<V>(inv_m, (T)0);
        } else {  // XOP_PHI_FORCE
          const T kmag = kf * sqrt((T)n2);
          const T pref = -kc<T>(kp.aE * kp.aE, kp.aE2_f) / (kmag * kmag);
          const T om15 = kc<T>(1.5 * (kp.eta - 1.0) / kp.eta, kp.om15_f);
          V phi;
          if (kp.gravity == 0) {
            const T cd = -kc<T>(0.5 / kp.eta, kp.half_inv_eta_f) + kc<T>(kp.c3, kp.c3_f) * ikb;
            const T den = (T)1 + ikb * kc<T>(1.0 / kp.eta, kp.inv_eta_f);
            const V rhs = cadd(cscale(X0[k2], om15), cscale(X1[k2], cd));
            phi = cscale(rhs, pref / den);
          } else if (kp.gravity == 1) {
            phi = cscale(X0[k2], pref * om15 * (T)geff_dev(kp, (double)kmag));
          } else {
            phi = cscale(X0[k2], pref * om15);
          }
          phi = cscale(phi, inv_m);
          if (o == 0) {
            r = phi;
          } else {
            const int ni = o == 1 ? nx : (o == 2 ? ny : nz);
            const bool nyq = o == 1 ? nyq_x : (o == 2 ? nyq_y : nyq_z);
            const T ki = kf * (T)ni;
            // g = -grad phi -> -i k_i phi
            r = nyq ? cmake<V>((T)0, (T)0) : cmake<V>(ki * phi.y, -ki * phi.x);
          }
        }
      }
      Y[k2] = r;
    }
    x_inverse<T, N>(Y, args.out.p[o], kz, ky0, lane, yl, s_T, s_tw);
  }
}

// ---------------------------------------------------------------------------
// Hessian x pass for FP32 data with the spectrum in shared memory (N <= 256).
//
// The same work as k_fft_x's Hessian operation for one kz plane and TY ky columns, with the
// x transforms done as in-place four-step stages on a [x][ky] tile in shared memory: the
// forward transform leaves X[k1 + N1 k2] at row N2 k1 + k2 (digit order), and each output's
// inverse reads that order back, forming the multiplier as it reads.  No thread holds the
// spectrum in registers, so a thread needs about half the registers of the register-resident
// version, and three CTAs fit on an SM instead of two (more warps to hide the latency of the
// transposes and the stores).
template <int N> struct XSGeom {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int TY = 16 < N ? 16 : N;
  static constexpr int THREADS = TY * N1;
  static constexpr int TILE = N * TY;  // complex
  static constexpr size_t SMEM = sizeof(float2) * ((size_t)kTwiddleTables * N + 2 * (size_t)TILE);
  static constexpr int MINB = THREADS <= 256 ? 3 : 1;
};

template <int N, int RB>
__global__ void __launch_bounds__(XSGeom<N>::THREADS, XSGeom<N>::MINB)
    k_x_hessian_smem(const __grid_constant__ XBatch<float, RB> xb, const float2* __restrict__ g_tw) {
  using G = XSGeom<N>;
  using V = float2;
  constexpr int N1 = G::N1, N2 = G::N2, TY = G::TY;
  const XArgs<float>& args = xb.a[RB > 1 ? blockIdx.z : 0];
  if (args.skip && *args.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s_tw = reinterpret_cast<V*>(smem_raw);
  V* A = s_tw + kTwiddleTables * N;  // the spectrum, rows in digit order
  V* B = A + G::TILE;                // one output at a time
  load_twiddles(s_tw, g_tw, N);
  const int tid = threadIdx.x;
  const int yl = tid % TY, q = tid / TY;  // q: j2 / n2 (stages 1 and 4) or k1 (stages 2 and 3)
  const int kz = blockIdx.y, ky0 = blockIdx.x * TY, ky = ky0 + yl;
  const int nz = kz == N / 2 ? -(N / 2) : kz;
  const bool nyq_y = ky == N / 2, nyq_z = kz == N / 2;
  const KParams& kp = args.kp;
  const float fy = (float)signed_index(ky, N), fz = (float)nz;
  const bool st14 = q < N2;  // stages over N1 points: TY x N2 tasks
  __syncthreads();
  // forward, stage 1: x = N2 j1 + j2 from global, transform over j1, twiddle, rows N2 k1 + j2
  if (st14) {
    const V* plane = args.in0 + (int64_t)kz * N * N;
    V v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = plane[(int64_t)(N2 * j1 + q) * N + ky];
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) A[(N2 * k1 + q) * TY + yl] = k1 == 0 ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + q]);
  }
  __syncthreads();
  // forward, stage 2 (k1 = q): transform over j2; X[k1 + N1 k2] to row N2 k1 + k2, prescaled
  {
    V X[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) X[j2] = A[(N2 * q + j2) * TY + yl];
    dft_regs<N2, N / N2>(X, s_tw);
    hessian_prescale<float, N>(X, q, fy, fz, kp.inv_m_f);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) A[(N2 * q + k2) * TY + yl] = X[k2];
  }
  __syncthreads();
  const float ikf = kp.local_only ? 0.f : 1.f / kp.kbkf_f;
#pragma unroll 1
  for (int o = 0; o < 6; ++o) {
    // inverse, stage 1 (k1 = q): multiplier as read, conj, transform over k2, twiddle
    {
      V X[N2], Y[N2];
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) X[k2] = A[(N2 * q + k2) * TY + yl];
      hessian_output<float, N>(X, o, q, fy, fz, nyq_y, nyq_z, ikf, Y);
      conj_regs(Y);
      dft_regs<N2, N / N2>(Y, s_tw);
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) B[(N2 * q + n2) * TY + yl] = n2 == 0 ? Y[n2] : cmul(Y[n2], s_tw[N + q * N2 + n2]);
    }
    __syncthreads();
    // inverse, stage 2 (n2 = q): transform over k1, conj, x = N2 n1 + n2 to global
    if (st14) {
      V w[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) w[k1] = B[(N2 * k1 + q) * TY + yl];
      dft_regs<N1, N / N1>(w, s_tw);
      V* plane = args.out.p[o] + (int64_t)kz * N * N;
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) plane[(int64_t)(N2 * n1 + q) * N + ky] = cconj(w[n1]);
    }
    __syncthreads();
  }
}

template <int N, int RB>
static void launch_xs(const XArgs<float>* a, int count, const float2* tw, cudaStream_t s) {
  using G = XSGeom<N>;
  raise_smem_limit<k_x_hessian_smem<N, RB>>(G::SMEM);
  XBatch<float, RB> xb;
  for (int r = 0; r < count; ++r) xb.a[r] = a[r];
  k_x_hessian_smem<N, RB><<<dim3(N / G::TY, N / 2 + 1, count), G::THREADS, G::SMEM, s>>>(xb, tw);
}

template <typename T, int N> int x_pass_blocks() { return (N / XGeom<T, N>::TY) * (N / 2 + 1); }

template <typename T, int N, int OP, int RB = 1>
static void launch_x(const XArgs<T>* a, int count, const vec2_t<T>* tw, cudaStream_t s) {
  using G = XGeom<T, N>;
  // the P(k) operations put their per-warp shell sums where the others keep
  // their per-thread multiplier tables
  constexpr bool PK = OP == XOP_PK || OP == XOP_PK_BRANE;
  constexpr int NBS = OP == XOP_PK_BRANE ? 4 : 3, NW = G::THREADS / 32;
  const size_t base = sizeof(vec2_t<T>) * (kTwiddleTables * N + (size_t)N * G::TY);
  const size_t tables = PK ? sizeof(double) * NW * 32 * NBS
                            : ((OP == XOP_HESSIAN || OP == XOP_PHI_FORCE) ? sizeof(vec2_t<T>) * (size_t)N * G::TY
                                                                          : sizeof(T) * 2 * Split<N>::N2 * G::THREADS);
  const size_t per_bin = PK ? sizeof(double) * NW * NBS : 0;
  const size_t smem = base + tables + per_bin * a[0].nbins;
  raise_smem_limit<k_fft_x<T, N, OP, RB>>(base + tables + per_bin * (N / 2));
  if constexpr (OP == XOP_HESSIAN && sizeof(T) == 4 && N <= 256) {
    launch_xs<N, RB>(a, count, tw, s);  // the shared-memory version of the same pass
    return;
  }
  XBatch<T, RB> xb;
  for (int r = 0; r < count; ++r) xb.a[r] = a[r];
  dim3 grid(N / G::TY, N / 2 + 1, count);
  k_fft_x<T, N, OP, RB><<<grid, G::THREADS, smem, s>>>(xb, tw);
}

template <typename T, int N>
void launch_fft_x_batch(int op, const XReal<T>* rz, int count, const vec2_t<T>* tw, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  XArgs<T> a[kBatchMax];
  for (int r = 0; r < count; ++r) {
    a[r] = XArgs<T>{};
    a[r].in0 = rz[r].in0;
    a[r].in1 = rz[r].in1;
    a[r].out = rz[r].out;
    a[r].nout_mask = rz[r].nout_mask;
    a[r].kp = rz[r].kp;
    a[r].skip = rz[r].skip;
    for (int i = 0; i < kMaxFields; ++i) a[r].in.p[i] = nullptr;
  }
  switch (op) {
    case XOP_HESSIAN: launch_x<T, N, XOP_HESSIAN, kBatchMax>(a, count, tw, s); break;
    case XOP_SOURCE: launch_x<T, N, XOP_SOURCE, kBatchMax>(a, count, tw, s); break;
    case XOP_SOURCE_LIN: launch_x<T, N, XOP_SOURCE_LIN, kBatchMax>(a, count, tw, s); break;
    case XOP_PHI_FORCE: launch_x<T, N, XOP_PHI_FORCE, kBatchMax>(a, count, tw, s); break;
    default: break;
  }
}

template <typename T, int N>
void launch_fft_x_op(int op, const vec2_t<T>* in0, const vec2_t<T>* in1, const FieldSet<T>& out, int nout_mask,
                     const KParams& kp, double* pk_partials, int nbins, double shell_lo, double shell_hi,
                     const vec2_t<T>* tw, cudaStream_t s, const int* skip) {
  XArgs<T> a{};
  a.skip = skip;
  a.in0 = in0; a.in1 = in1; a.out = out; a.nout_mask = nout_mask; a.kp = kp;
  a.pk_partials = pk_partials; a.nbins = nbins; a.shell_lo = shell_lo; a.shell_hi = shell_hi;
  a.in_mask = 0;
  for (int i = 0; i < kMaxFields; ++i) a.in.p[i] = nullptr;
  switch (op) {
    case XOP_HESSIAN: launch_x<T, N, XOP_HESSIAN>(&a, 1, tw, s); break;
    case XOP_SOURCE: launch_x<T, N, XOP_SOURCE>(&a, 1, tw, s); break;
    case XOP_SOURCE_LIN: launch_x<T, N, XOP_SOURCE_LIN>(&a, 1, tw, s); break;
    case XOP_PHI_FORCE: launch_x<T, N, XOP_PHI_FORCE>(&a, 1, tw, s); break;
    case XOP_PK: launch_x<T, N, XOP_PK>(&a, 1, tw, s); break;
    case XOP_PK_BRANE: launch_x<T, N, XOP_PK_BRANE>(&a, 1, tw, s); break;
    case XOP_ZEL: launch_x<T, N, XOP_ZEL>(&a, 1, tw, s); break;
    case XOP_PK_ADJ: launch_x<T, N, XOP_PK_ADJ>(&a, 1, tw, s); break;
    case XOP_SHELL: launch_x<T, N, XOP_SHELL>(&a, 1, tw, s); break;
    default: break;
  }
}

template <typename T, int N>
void launch_fft_x_adj(int op, const FieldSet<T>& in, int in_mask, const FieldSet<T>& out, const KParams& kp,
                      const vec2_t<T>* tw, cudaStream_t s) {
  XArgs<T> a{};
  a.skip = nullptr;
  a.in0 = nullptr; a.in1 = nullptr; a.out = out; a.nout_mask = 0; a.kp = kp;
  a.pk_partials = nullptr; a.nbins = 0; a.shell_lo = 0; a.shell_hi = 0;
  a.in = in; a.in_mask = in_mask;
  if (op == XOP_ADJ_PHI) launch_x<T, N, XOP_ADJ_PHI>(&a, 1, tw, s);
  else if (op == XOP_ADJ_COMBINE) launch_x<T, N, XOP_ADJ_COMBINE>(&a, 1, tw, s);
  else if (op == XOP_ZEL_ADJ) launch_x<T, N, XOP_ZEL_ADJ>(&a, 1, tw, s);
}

template <typename T, int N>
void launch_fft_x_rc(const FieldSet<T>& in, int in_mask, const KParams& kp, const RcDeriv& d, double* partials,
                     const vec2_t<T>* tw, cudaStream_t s) {
  XArgs<T> a{};
  a.skip = nullptr;
  a.in0 = nullptr; a.in1 = nullptr; a.nout_mask = 0; a.kp = kp;
  for (int i = 0; i < kMaxFields; ++i) a.out.p[i] = nullptr;
  a.pk_partials = partials; a.nbins = 0; a.shell_lo = 0; a.shell_hi = 0;
  a.in = in; a.in_mask = in_mask; a.rc = d;
  launch_x<T, N, XOP_RC>(&a, 1, tw, s);
}

// ---------------------------------------------------------------------------
// Hessian x pass fused with the inverse y transforms of its six outputs (FP32, N = 128 or 256).
//
// The CTAs of one kz plane (N / TY of them, the ky blocks) form one thread-block cluster.  Each
// does what the Hessian x pass does for its TY ky columns, but keeps every output's x inverse
// in its own shared memory (all x, its TY ky) instead of writing it out.  After a cluster
// barrier each CTA takes TY x rows of the plane: it reads their N ky values from the CTAs of
// the cluster (distributed shared memory, TY consecutive values from each), transforms them
// back along y and writes the rows of the output in the layout (kz, x, y) that the relaxation
// pass reads.  An iteration then needs no six-field inverse y pass: its 12 S of memory traffic
// (read and write of six half spectra) are gone and the six outputs cross memory once.  Two
// alternating exchange buffers let one cluster barrier per output order the writes of one
// output after the reads of the output before it; a last barrier keeps every CTA resident
// until the others have read its buffers.  Measured on a GB300 at 256^3 (clusters of 16):
// 352 us per launch against 240 us for the x pass and six-field y pass it replaces.  The x
// pass is latency-bound at 16 warps per SM and the y work adds to its time rather than
// hiding in it, so the fused pass is opt-in (dgp_set_hessian_fusion).
template <int N> struct XYGeom {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int TY = 16;                  // ky columns per CTA; x rows per CTA in the y stage
  static constexpr int CS = N / TY;              // CTAs per cluster: one kz plane
  static constexpr int THREADS = TY * N1;
  static constexpr int XT = N * TY;              // x transpose (complex)
  static constexpr int YT = TY * N1 * (N2 + 1);  // y transpose (complex)
  static constexpr int TBUF = XT > YT ? XT : YT;
  static constexpr int EX = N * TY;              // one exchange buffer: [x][ky in the block]
  static constexpr size_t SMEM = sizeof(float2) * ((size_t)kTwiddleTables * N + TBUF + 2 * (size_t)EX);
  static_assert(THREADS == 256, "TY rows of N1 lanes in both stages");
};

template <int N, int RB>
__global__ void __launch_bounds__(256, 2) k_xy_hessian(const __grid_constant__ XBatch<float, RB> xb,
                                                       const float2* __restrict__ g_tw) {
  namespace cg = cooperative_groups;
  using G = XYGeom<N>;
  using V = float2;
  constexpr int N1 = G::N1, N2 = G::N2, TY = G::TY;
  const XArgs<float>& args = xb.a[RB > 1 ? blockIdx.z : 0];
  // the flag was set by an earlier launch, so every CTA of a cluster takes the same branch
  if (args.skip && *args.skip) return;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s_tw = reinterpret_cast<V*>(smem_raw);
  V* s_T = s_tw + kTwiddleTables * N;  // the x transpose, then the y transpose
  V* s_E = s_T + G::TBUF;              // two exchange buffers
  load_twiddles(s_tw, g_tw, N);
  const int tid = threadIdx.x;
  const int yl = tid % TY, lane = tid / TY;  // x stage: the TY columns fastest
  const int kz = blockIdx.y;
  const int rank = blockIdx.x;  // the CTA's rank in its cluster (cluster dims CS x 1 x 1, gridDim.x = CS)
  const int ky0 = rank * TY;
  const int ky = ky0 + yl;
  const int nz = kz == N / 2 ? -(N / 2) : kz;
  const int ny = signed_index(ky, N);
  const bool nyq_y = ky == N / 2, nyq_z = kz == N / 2;
  const KParams& kp = args.kp;
  __syncthreads();
  V X0[N2];
  x_forward<float, N>(args.in0, kz, ky0, lane, yl, s_T, s_tw, X0);
  const float fy = (float)ny, fz = (float)nz;
  hessian_prescale<float, N>(X0, lane, fy, fz, kp.inv_m_f);
  const float ikf = kp.local_only ? 0.f : 1.f / kp.kbkf_f;
  // y stage: thread (row, j) of TY rows x N1; stage one's TY x N2 tasks on the first threads
  const int row = tid / N1, j = tid % N1;
  const int r1 = tid / N2, c1 = tid % N2;
  const bool act1 = tid < TY * N2;
  const int xr0 = rank * TY;  // first x row of this CTA's y stage
#pragma unroll 1
  for (int o = 0; o < 6; ++o) {
    V Y[N2];
    hessian_output<float, N>(X0, o, lane, fy, fz, nyq_y, nyq_z, ikf, Y);
    // x inverse as in x_inverse; the result stays conjugated in the exchange buffer
    conj_regs(Y);
    dft_regs<N2, N / N2>(Y, s_tw);
#pragma unroll
    for (int m1 = 0; m1 < N2; ++m1)
      s_T[(m1 * N1 + lane) * TY + yl] = (m1 == 0) ? Y[m1] : cmul(Y[m1], s_tw[2 * N + m1 * N1 + lane]);
    __syncthreads();
    V* E = s_E + (o & 1) * G::EX;
    if (lane < N2) {
      V w[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) w[k1] = s_T[(lane * N1 + k1) * TY + yl];
      dft_regs<N1, N / N1>(w, s_tw);
#pragma unroll
      for (int m2 = 0; m2 < N1; ++m2) E[(lane + N2 * m2) * TY + yl] = w[m2];
    }
    cluster.sync();  // every CTA's block of this output is in its exchange buffer
    // y inverse of rows xr0 + r as conj(DFT(conj(x))), conj(x) being what the buffers hold
    if (act1) {
      V v[N1];
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) {
        const int kyy = N2 * j1 + c1;
        const V* Ep = cluster.map_shared_rank(E, kyy / TY);
        v[j1] = Ep[(xr0 + r1) * TY + kyy % TY];
      }
      dft_regs<N1, N / N1>(v, s_tw);
      V* T1 = s_T + r1 * (N1 * (N2 + 1));
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) T1[k1 * (N2 + 1) + c1] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + c1]);
    }
    __syncthreads();
    {
      const V* Tp = s_T + row * (N1 * (N2 + 1));
      V u[N2];
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[j * (N2 + 1) + j2];
      dft_regs<N2, N / N2>(u, s_tw);
      V* dst = args.out.p[o] + ((int64_t)kz * N + xr0 + row) * N;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) dst[j + N1 * k2] = cconj(u[k2]);
    }
    __syncthreads();  // the y transpose is read before the next output's x transpose reuses it
  }
  cluster.sync();  // no CTA leaves while another may still read its exchange buffers
}

template <int N, int RB>
static void xy_launch_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int count, cudaStream_t s) {
  using G = XYGeom<N>;
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(G::CS, N / 2 + 1, count);
  cfg.blockDim = dim3(G::THREADS, 1, 1);
  cfg.dynamicSmemBytes = G::SMEM;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G::CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

// Shared-memory limit and (for clusters above 8) the non-portable cluster size, once per
// instantiation and device.
template <int N, int RB>
static cudaError_t xy_prepare() {
  using G = XYGeom<N>;
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (dev < 64 && ((done >> dev) & 1u)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_xy_hessian<N, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e == cudaSuccess && G::CS > 8)
    e = cudaFuncSetAttribute(k_xy_hessian<N, RB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

template <int N, int RB>
static void launch_xy(const XArgs<float>* a, int count, const float2* tw, cudaStream_t s) {
  if (xy_prepare<N, RB>() != cudaSuccess) return;  // the launch error check reports it
  XBatch<float, RB> xb;
  for (int r = 0; r < count; ++r) xb.a[r] = a[r];
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  xy_launch_config<N, RB>(cfg, attr, count, s);
  cudaLaunchKernelEx(&cfg, k_xy_hessian<N, RB>, xb, tw);
}

template <int N>
static int xy_probe() {
  if (xy_prepare<N, 1>() != cudaSuccess || xy_prepare<N, kBatchMax>() != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  xy_launch_config<N, 1>(cfg, attr, 1, nullptr);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, k_xy_hessian<N, 1>, &cfg) != cudaSuccess) return 0;
  return nc > 0 ? 1 : 0;
}

bool xy_hessian_available(int n) {
  if (n != 128 && n != 256) return false;
  static std::mutex mu;
  static int ok[2][64];
  static bool init = false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return false;
  std::lock_guard<std::mutex> g(mu);
  if (!init) {
    for (auto& r : ok)
      for (int& v : r) v = -1;
    init = true;
  }
  int& v = ok[n == 256 ? 1 : 0][dev];
  if (v < 0) {
    v = n == 256 ? xy_probe<256>() : xy_probe<128>();
    cudaGetLastError();
  }
  return v == 1;
}

template <typename T, int N>
void launch_xy_hessian(const vec2_t<T>* in, const FieldSet<T>& out, const KParams& kp, const vec2_t<T>* tw,
                       cudaStream_t s, const int* skip) {
  if constexpr (sizeof(T) == 4 && (N == 128 || N == 256)) {
    XArgs<float> a{};
    a.in0 = in;
    a.out = out;
    a.kp = kp;
    a.skip = skip;
    launch_xy<N, 1>(&a, 1, tw, s);
  }
}

template <typename T, int N>
void launch_xy_hessian_batch(const XReal<T>* rz, int count, const vec2_t<T>* tw, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && (N == 128 || N == 256)) {
    if (count < 1 || count > kBatchMax) return;
    XArgs<float> a[kBatchMax];
    for (int r = 0; r < count; ++r) {
      a[r] = XArgs<float>{};
      a[r].in0 = rz[r].in0;
      a[r].out = rz[r].out;
      a[r].kp = rz[r].kp;
      a[r].skip = rz[r].skip;
    }
    launch_xy<N, kBatchMax>(a, count, tw, s);
  }
}

#define DGP_INST_XY(N)                                                                                       \
  template void launch_xy_hessian<float, N>(const float2*, const FieldSet<float>&, const KParams&,            \
                                            const float2*, cudaStream_t, const int*);                          \
  template void launch_xy_hessian<double, N>(const double2*, const FieldSet<double>&, const KParams&,         \
                                             const double2*, cudaStream_t, const int*);                        \
  template void launch_xy_hessian_batch<float, N>(const XReal<float>*, int, const float2*, cudaStream_t);
DGP_INST_XY(16) DGP_INST_XY(32) DGP_INST_XY(48) DGP_INST_XY(64) DGP_INST_XY(96) DGP_INST_XY(128) DGP_INST_XY(256)
DGP_INST_XY(512)

#define DGP_INST_X(T, N)                                                                            \
  template void launch_fft_x_op<T, N>(int, const vec2_t<T>*, const vec2_t<T>*, const FieldSet<T>&, int, \
                                      const KParams&, double*, int, double, double, const vec2_t<T>*,   \
                                      cudaStream_t, const int*);                                        \
  template void launch_fft_x_adj<T, N>(int, const FieldSet<T>&, int, const FieldSet<T>&, const KParams&,  \
                                       const vec2_t<T>*, cudaStream_t);                                  \
  template void launch_fft_x_rc<T, N>(const FieldSet<T>&, int, const KParams&, const RcDeriv&, double*,   \
                                      const vec2_t<T>*, cudaStream_t);
#define DGP_INST_XB(N) \
  template void launch_fft_x_batch<float, N>(int, const XReal<float>*, int, const float2*, cudaStream_t);
DGP_INST_XB(16) DGP_INST_XB(32) DGP_INST_XB(48) DGP_INST_XB(64) DGP_INST_XB(96) DGP_INST_XB(128)
#define DGP_INST_X_ALL(T) DGP_INST_X(T, 16) DGP_INST_X(T, 32) DGP_INST_X(T, 64) DGP_INST_X(T, 128) \
  DGP_INST_X(T, 256) DGP_INST_X(T, 512) DGP_INST_X(T, 48) DGP_INST_X(T, 96)
DGP_INST_X_ALL(float)
DGP_INST_X_ALL(double)
#define DGP_INST_XB(T) template int x_pass_blocks<T, 16>(); template int x_pass_blocks<T, 32>(); \
  template int x_pass_blocks<T, 64>(); template int x_pass_blocks<T, 128>(); \
  template int x_pass_blocks<T, 256>(); template int x_pass_blocks<T, 512>(); \
  template int x_pass_blocks<T, 48>(); template int x_pass_blocks<T, 96>();
DGP_INST_XB(float)
DGP_INST_XB(double)

}  // namespace dgp
