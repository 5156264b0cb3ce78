// Fused z pass of one relaxation iteration for FP32 mesh data (Secs. III.B-C).
//
// A CTA owns TY = 16 consecutive rows (x, y0 .. y0 + 15) of the mesh.  It
//   1. inverse-transforms along z the six y-inverted spectra of those rows as
//      three field pairs (two real fields per complex pencil), in the order
//        A = (H_xy, H_xz),  B = (H_yz, N),  C = (H_xx, H_yy),
//      and folds them into one accumulator per point,
//        after A and B:  r = -2 (H_xy^2 + H_xz^2 + H_yz^2) + c2 N,
//      then with a = H_xx, b = H_yy, the mean-free d = D - <D>, u = a + b and
//      H_zz = d - u (the trace identity):
//        R  = r + 2 a b + 2 u H_zz + alpha d - S            (Eq. FullDGP2, LHS - RHS)
//      (-2 sum_{i<j} (H_ij^2 - H_ii H_jj) = -2 (H_xy^2 + H_xz^2 + H_yz^2) + 2 a b + 2 u H_zz);
//        B' = d ((1 - w) d + alpha) - R                     (Eq. Bwpara)
//        Delta = (alpha + 2 (1 - w) d)^2 - 4 (1 - w) R      (= alpha^2 + 4 (1 - w) B')
//      bad points (Delta < 0) take Delta = 0 (Sec. III.C), and
//        D_new = 2 B' / (alpha + sqrt(Delta))              (Eq. nabla^2Cwpara, '+' root);
//   2. writes D_new and forward-transforms it along z into the transposed half
//      spectrum, ready for the next iteration's y pass;
//   3. emits FP64 block partials of sum |R|, sum D_new, bad points, non-finite R.
// The arithmetic of r, R, B' and Delta is a policy: FP32; FP32 with an exact
// discriminant and pair sums (the mixed default); pairs of floats with
// error-free transformations for R and Delta (about 48 significant bits); or FP64.
//
// Data movement.  The spectra are read as TMA tiles (one tensor map per
// spectrum; a tile is 16 complex values along y, 128 bytes, for every kz),
// landed with the 128-byte swizzle so that the transform's column reads are
// free of bank conflicts, and completed on an mbarrier.  Two tile buffers
// alternate: while one pair is transformed the next lands in the other; the
// four-step transpose of a pair reuses the bytes of the tile it came from.
// The rows of D and S come in by plain bulk copies into padded rows.  Every
// wait is bounded (tma.cuh): on expiry the CTA records a fault that stops the
// solve with DGP_E_TIMEOUT, waits for the copies it issued and returns.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "eft.cuh"
#include "fft_core.cuh"
#include "kernels.cuh"
#include "tma.cuh"

namespace dgp {

// ---------------------------------------------------------------- arithmetic policies
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fdiv_full(float a, float b) {
  float r;
  asm("div.full.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

struct PointOut {
  float bp, dt;  // B' and Delta, rounded to float
  bool neg;      // Delta < 0 (a bad point)
};

struct RxF32 {
  using Acc = float;
  using Sum = float;
  static constexpr bool kApproxRoot = true;
  __device__ static void pair_a(Acc& r, float x, float y) { r = fmaf(-2.f * x, x, (-2.f * y) * y); }
  __device__ static void pair_b(Acc& r, float x, float n, const RelaxParams& rp) {
    r = fmaf(-2.f * x, x, fmaf(rp.c2_hi, n, r));
  }
  __device__ static PointOut finish(Acc r, float a, float b, float D, float S, float m_hi, float, double,
                                    const RelaxParams& rp, Sum& rsum, float& nonfin) {
    const float d = D - m_hi, u = a + b, c = d - u;
    const float R = fmaf(2.f * a, b, fmaf(2.f * u, c, fmaf(rp.alpha_hi, d, r - S)));
    PointOut o;
    o.bp = fmaf(d, fmaf(rp.omw, d, rp.alpha_hi), -R);
    const float s = fmaf(rp.two_omw, d, rp.alpha_hi);
    o.dt = fmaf(s, s, -rp.four_omw_hi * R);
    o.neg = o.dt < 0.f;
    if (isfinite(R)) rsum += fabsf(R);
    else nonfin += 1.f;
    return o;
  }
  __device__ static double sum_d(Sum s) { return (double)s; }
};

// Config-3 mixed arithmetic: R, B' and D_new in FP32 (the FP32 data's own
// rounding already leaves a residual floor of order 1e-8 of <|S|>, which
// pair arithmetic cannot go below); the discriminant's sign from Delta formed
// exactly for the FP32 s = alpha + 2 (1 - w) d and R (a pair); the per-thread
// sum of D_new (its mean is removed next iteration) as a pair; every
// cross-thread sum in FP64.
struct RxM32 {
  using Acc = float;
  using Sum = float;
  static constexpr bool kApproxRoot = true;
  __device__ static void pair_a(Acc& r, float x, float y) { RxF32::pair_a(r, x, y); }
  __device__ static void pair_b(Acc& r, float x, float n, const RelaxParams& rp) { RxF32::pair_b(r, x, n, rp); }
  __device__ static PointOut finish(Acc r, float a, float b, float D, float S, float m_hi, float, double,
                                    const RelaxParams& rp, Sum& rsum, float& nonfin) {
    const float d = D - m_hi, u = a + b, c = d - u;
    const float R = fmaf(2.f * a, b, fmaf(2.f * u, c, fmaf(rp.alpha_hi, d, r - S)));
    PointOut o;
    o.bp = fmaf(d, fmaf(rp.omw, d, rp.alpha_hi), -R);
    const float s = fmaf(rp.two_omw, d, rp.alpha_hi);
    FP v = fp_prod(s, s);
    FP t = fp_prod(-rp.four_omw_hi, R);
    t.lo = fmaf(-rp.four_omw_lo, R, t.lo);
    fp_acc(v, t);
    v = fp_fast(v.hi, v.lo);
    o.neg = v.hi < 0.f || (v.hi == 0.f && v.lo < 0.f);
    o.dt = v.hi + v.lo;
    if (isfinite(R)) rsum += fabsf(R);
    else nonfin += 1.f;
    return o;
  }
  __device__ static double sum_d(Sum s) { return (double)s; }
};

struct RxEFT {
  using Acc = FP;
  using Sum = FP;
  static constexpr bool kApproxRoot = false;
  __device__ static void pair_a(Acc& r, float x, float y) {
    r = fp_prod(-2.f * x, x);
    fp_acc(r, fp_prod(-2.f * y, y));
  }
  __device__ static void pair_b(Acc& r, float x, float n, const RelaxParams& rp) {
    fp_acc(r, fp_prod(-2.f * x, x));
    FP c = fp_prod(rp.c2_hi, n);
    c.lo = fmaf(rp.c2_lo, n, c.lo);
    fp_acc(r, c);
  }
  __device__ static PointOut finish(Acc r, float a, float b, float D, float S, float m_hi, float m_lo, double,
                                    const RelaxParams& rp, Sum& rsum, float& nonfin) {
    FP d = fp_two_sum(D, -m_hi);
    d.lo -= m_lo;
    d = fp_fast(d.hi, d.lo);
    const FP u = fp_two_sum(a, b);  // a + b exactly
    FP c = fp_two_sum(d.hi, -u.hi);  // H_zz = d - u
    c.lo += d.lo - u.lo;
    fp_acc(r, fp_prod(2.f * a, b));
    {
      FP p = fp_prod(2.f * u.hi, c.hi);
      p.lo = fmaf(2.f * u.hi, c.lo, fmaf(2.f * u.lo, c.hi, p.lo));
      fp_acc(r, p);
    }
    {
      FP p = fp_prod(rp.alpha_hi, d.hi);
      p.lo = fmaf(rp.alpha_hi, d.lo, fmaf(rp.alpha_lo, d.hi, p.lo));
      fp_acc(r, p);
    }
    fp_acc(r, FP{-S, 0.f});
    const FP R = fp_fast(r.hi, r.lo);
    PointOut o;
    // B' only feeds D_new, an FP32 datum: FP32 from the pair-accurate R and d suffices
    o.bp = fmaf(d.hi, fmaf(rp.omw, d.hi, rp.alpha_hi), -R.hi);
    {
      const float s = fmaf(rp.two_omw, d.hi, rp.alpha_hi);
      FP v = fp_prod(s, s);
      FP t = fp_prod(-rp.four_omw_hi, R.hi);
      t.lo = fmaf(-rp.four_omw_hi, R.lo, fmaf(-rp.four_omw_lo, R.hi, t.lo));
      fp_acc(v, t);
      v = fp_fast(v.hi, v.lo);
      o.neg = v.hi < 0.f || (v.hi == 0.f && v.lo < 0.f);
      o.dt = v.hi + v.lo;
    }
    if (isfinite(R.hi)) fp_acc(rsum, R.hi < 0.f ? FP{-R.hi, -R.lo} : R);
    else nonfin += 1.f;
    return o;
  }
  __device__ static double sum_d(Sum s) { return (double)s.hi + (double)s.lo; }
};

struct RxF64 {
  using Acc = double;
  using Sum = double;
  static constexpr bool kApproxRoot = false;
  __device__ static void pair_a(Acc& r, float x, float y) { r = -2.0 * ((double)x * x + (double)y * y); }
  __device__ static void pair_b(Acc& r, float x, float n, const RelaxParams& rp) {
    r = fma(-2.0 * x, (double)x, fma(rp.c2, (double)n, r));
  }
  __device__ static PointOut finish(Acc r, float a, float b, float D, float S, float, float, double mean,
                                    const RelaxParams& rp, Sum& rsum, float& nonfin) {
    const double d = (double)D - mean, u = (double)a + (double)b, c = d - u;
    const double R = fma(2.0 * a, (double)b, fma(2.0 * u, c, fma(rp.alpha, d, r - (double)S)));
    const double omw = 1.0 - rp.w;
    PointOut o;
    o.bp = (float)(d * fma(omw, d, rp.alpha) - R);
    const double s = fma(2.0 * omw, d, rp.alpha);
    const double v = fma(s, s, -4.0 * omw * R);
    o.neg = v < 0.0;
    o.dt = (float)v;
    if (isfinite(R)) rsum += fabs(R);
    else nonfin += 1.f;
    return o;
  }
  __device__ static double sum_d(Sum s) { return s; }
};

// ---------------------------------------------------------------- geometry
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int align1k(int b) { return (b + 1023) / 1024 * 1024; }

template <int N> struct RGeom {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int TY = 16;                           // rows per CTA: 128 bytes of complex floats per kz
  static constexpr int THREADS = TY * N1;
  static constexpr int NK = N / 2 + 1;
  static constexpr int NBOX = (NK + 255) / 256;           // TMA boxes along kz (at most 256 rows each)
  static constexpr int BOXK = (NK + NBOX - 1) / NBOX;
  static constexpr int ROWB = TY * 8;                     // bytes of one kz row of a tile
  static constexpr int BSTRIDE = align1k(BOXK * ROWB);    // each box starts on a swizzle period
  static constexpr int FIELD = NBOX * BSTRIDE;            // one spectrum's tile
  // row stride of the four-step transpose (complex): N1 (N2 + 1), padded when N2 < N1 so that
  // it is N2 mod 16 and the rows a half-warp writes in the packed first stage (N2 columns
  // each) fall on different banks
  static constexpr int RS0 = N1 * (N2 + 1);
  static constexpr int RS = N2 < N1 ? RS0 + ((N2 - RS0 % 16) % 16 + 16) % 16 : RS0;
  static constexpr int TSZ = TY * RS * 8;                 // four-step transpose of a pair
  // the second buffer receives TMA tiles with the 128-byte swizzle: it starts on 1024 bytes
  static constexpr int BUF0 = align1k(cmax(2 * FIELD, TSZ));
  static constexpr int ROWP = N + 16;                     // padded real row (floats)
  static constexpr int P = TY / 2;                        // row pairs of the forward transform
  // tiles of a pair, then their transpose; the D and S rows; the forward spectrum of D_new
  static constexpr int BUF1 = cmax(cmax(cmax(2 * FIELD, TSZ), 2 * TY * ROWP * 4), N * (P + 1) * 8);
  static constexpr int TW = N * 8;                        // the phase table W_N^{j2 k1}
  static constexpr int EXTRA = 64 + 4 * 32 * 8 + 32;      // mbarriers, warp partials, the mean
  static constexpr size_t SMEM = 1024 + BUF0 + BUF1 + TW + EXTRA;
  static constexpr int MINB = THREADS <= 256 ? 3 : 1;
  static_assert(2 * ROWB == 256 && TY * 8 == 128, "a tile row is one 128-byte swizzle row");
  static_assert(P * RS * 8 <= BUF0, "forward transpose fits the first buffer");
  static_assert(BUF0 % 1024 == 0 && BSTRIDE % 1024 == 0, "TMA tiles start on 1024-byte boundaries");
  static_assert(TSZ <= BUF0 && TSZ <= BUF1, "a pair's transpose fits the buffer that held its tiles");
};

// byte offset of complex (kz, y) in a swizzled tile (relative to a 1024-aligned base)
template <int N>
__device__ __forceinline__ unsigned tile_off(int kz, int y) {
  using G = RGeom<N>;
  const int b = G::NBOX == 1 ? 0 : kz / G::BOXK;
  const unsigned off = (unsigned)(b * G::BSTRIDE + (kz - b * G::BOXK) * G::ROWB + y * 8);
  return off ^ (((off >> 7) & 7u) << 4);
}

template <int N>
__device__ __forceinline__ void issue_spectra(unsigned char* dst, const CUtensorMap* ma, const CUtensorMap* mb,
                                              int x, int y0, uint64_t* bar) {
  using G = RGeom<N>;
  mbar_expect_tx(bar, 2u * G::NBOX * G::BOXK * G::ROWB);
#pragma unroll
  for (int b = 0; b < G::NBOX; ++b) {
    tma_load_3d(dst + b * G::BSTRIDE, ma, 2 * y0, x, b * G::BOXK, bar);
    tma_load_3d(dst + G::FIELD + b * G::BSTRIDE, mb, 2 * y0, x, b * G::BOXK, bar);
  }
}

// Inverse z transform of the field pair in buf: per row Z = A + i B rebuilt
// over all k from the half spectra (imaginary parts of k = 0 and N/2 dropped).
// Thread (row, lane) ends with A (ra) and B (rb) of its row at z = lane + N1 k2.
// The transpose reuses buf, so every thread reads its tile values first.
//
// Stage one (pair_load, pair_stage1) has TY x N2 tasks (a row r1 and one of its N2 columns c1);
// stage two (pair_stage2) has TY x N1 (a row and lane k1).

// stage one's reads: v[j1] = conj(Z) at k = N2 j1 + c1 of row r1
template <int N>
__device__ __forceinline__ void pair_load(const unsigned char* buf, int r1, int c1, float2 (&v)[Split<N>::N1]) {
  using G = RGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2;
  const unsigned char* TA = buf;
  const unsigned char* TB = buf + G::FIELD;
  // With N2 a multiple of 8 and one box, row kk of a read satisfies kk = +-c1 (mod 8) for
  // every j1, so the swizzle term is one constant per thread and direction.
  constexpr bool HOIST = N2 % 8 == 0 && G::NBOX == 1;
  const unsigned off_d = (unsigned)c1 * G::ROWB + (((unsigned)r1 * 8u) ^ (((unsigned)c1 & 7u) << 4));
  const unsigned off_m = (unsigned)(N - c1) * G::ROWB + (((unsigned)r1 * 8u) ^ (((unsigned)(N - c1) & 7u) << 4));
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) {
    const int k = N2 * j1 + c1;
    float2 A, B;
    bool mirror;
    if (N2 * j1 + N2 - 1 < N / 2) mirror = false;  // j1 is a compile-time index
    else if (N2 * j1 > N / 2) mirror = true;
    else mirror = k > N / 2;
    const int kk = mirror ? N - k : k;
    unsigned off;
    if constexpr (HOIST) off = mirror ? off_m - (unsigned)(N2 * j1 * G::ROWB) : off_d + (unsigned)(N2 * j1 * G::ROWB);
    else off = tile_off<N>(kk, r1);
    A = *reinterpret_cast<const float2*>(TA + off);
    B = *reinterpret_cast<const float2*>(TB + off);
    if (mirror) {
      A.y = -A.y;
      B.y = -B.y;
    } else if (kk == 0 || kk == N / 2) {
      A.y = 0.f;
      B.y = 0.f;
    }
    v[j1] = make_float2(A.x - B.y, -(A.y + B.x));  // conj(A + i B)
  }
}

// stage one's transform over j1 and its twiddled transpose into buf (row r1, column c1)
template <int N>
__device__ __forceinline__ void pair_stage1(unsigned char* buf, const float2* s_tw, int r1, int c1,
                                            float2 (&v)[Split<N>::N1]) {
  using G = RGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2;
  float2* T1 = reinterpret_cast<float2*>(buf) + r1 * G::RS;
  dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) T1[k1 * (N2 + 1) + c1] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[k1 * N2 + c1]);
}

// stage two: transform over j2 of (row, lane), A and B at z = lane + N1 k2
template <int N>
__device__ __forceinline__ void pair_stage2(const unsigned char* buf, const float2* s_tw, int row, int lane,
                                            float (&ra)[Split<N>::N2], float (&rb)[Split<N>::N2]) {
  using G = RGeom<N>;
  constexpr int N2 = G::N2;
  const float2* Tp = reinterpret_cast<const float2*>(buf) + row * G::RS;
  float2 u[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[lane * (N2 + 1) + j2];
  dft_regs<N2, N / N2>(u, s_tw);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    ra[k2] = u[k2].x;
    rb[k2] = -u[k2].y;
  }
}

template <int N>
__device__ __forceinline__ void pair_inverse(unsigned char* buf, const float2* s_tw, int row, int lane,
                                             float (&ra)[Split<N>::N2], float (&rb)[Split<N>::N2]) {
  using G = RGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2;
  // When N2 < N1 stage one's tasks go to the first TY x N2 threads, so that whole warps
  // idle instead of every warp running with lanes masked off.
  constexpr bool PACK = N2 < N1;
  const int t1 = threadIdx.x;
  const bool act1 = !PACK || t1 < G::TY * N2;
  const int r1 = PACK ? t1 / N2 : row, c1 = PACK ? t1 % N2 : lane;
  float2 v[N1];
  if (act1) pair_load<N>(buf, r1, c1, v);
  __syncthreads();  // the tile is read: its bytes become the transpose buffer
  if (act1) pair_stage1<N>(buf, s_tw, r1, c1, v);
  __syncthreads();
  pair_stage2<N>(buf, s_tw, row, lane, ra, rb);
}

// Two pairs at once (tiles in bufA and bufB) when N2 < N1: stage one of both on the first
// 2 x TY x N2 threads, then stage two of each on every thread.
template <int N>
__device__ __forceinline__ void pair2_inverse(unsigned char* bufA, unsigned char* bufB, const float2* s_tw, int row,
                                              int lane, float (&ra)[Split<N>::N2], float (&rb)[Split<N>::N2],
                                              float (&ra2)[Split<N>::N2], float (&rb2)[Split<N>::N2]) {
  using G = RGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2, TN = G::TY * N2;
  const int t = threadIdx.x;
  const bool act1 = t < 2 * TN;
  const int sel = t >= TN ? 1 : 0;
  const int t1 = t - sel * TN;
  const int r1 = t1 / N2, c1 = t1 % N2;
  unsigned char* buf = sel ? bufB : bufA;
  float2 v[N1];
  if (act1) pair_load<N>(buf, r1, c1, v);
  __syncthreads();  // both tiles are read
  if (act1) pair_stage1<N>(buf, s_tw, r1, c1, v);
  __syncthreads();
  pair_stage2<N>(bufA, s_tw, row, lane, ra, rb);
  pair_stage2<N>(bufB, s_tw, row, lane, ra2, rb2);
}

template <int N, class AR, int RB>
__global__ void __launch_bounds__(RGeom<N>::THREADS, RGeom<N>::MINB)
    k_relax_tma(const __grid_constant__ RelaxTmaBatch<RB> batch, const float2* __restrict__ g_tw) {
  const RelaxTmaArgs& args = batch.a[RB > 1 ? blockIdx.z : 0];  // realisation of this CTA
  if (args.skip && *args.skip) return;
  using G = RGeom<N>;
  using Acc = typename AR::Acc;
  using Sum = typename AR::Sum;
  constexpr int N1 = G::N1, N2 = G::N2, TY = G::TY, NK = G::NK, P = G::P, ROWP = G::ROWP;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* buf0 = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* buf1 = buf0 + G::BUF0;
  float2* s_tw = reinterpret_cast<float2*>(buf1 + G::BUF1);
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_tw + N);  // [2]
  double* s_part = reinterpret_cast<double*>(bars + 8);    // [4][32]
  double* s_mean = s_part + 4 * 32;                          // mean, then its float pair
  const int tid = threadIdx.x, lane = tid % N1, row = tid / N1;
  const int x = blockIdx.y, y0 = blockIdx.x * TY;
  const RelaxParams& rp = args.rp;
  const uint64_t lim = args.wait_ns;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init_fence();
    // pair A -> buf0, pair B -> buf1 (phase 0 of each barrier)
    if (!args.withhold) issue_spectra<N>(buf0, &args.map[2], &args.map[3], x, y0, &bars[0]);
    issue_spectra<N>(buf1, &args.map[4], &args.map[5], x, y0, &bars[1]);
    const double m = args.dsum ? args.dsum[0] * rp.inv_m : 0.0;
    s_mean[0] = m;
    float* mp = reinterpret_cast<float*>(s_mean + 1);
    mp[0] = (float)m;
    mp[1] = (float)(m - (double)mp[0]);
  }
  for (int i = tid; i < N; i += blockDim.x) s_tw[i] = g_tw[N + i];
  __syncthreads();
  const double mean = s_mean[0];
  const float m_hi = reinterpret_cast<const float*>(s_mean + 1)[0];
  const float m_lo = reinterpret_cast<const float*>(s_mean + 1)[1];

  // phases issued on each barrier (A and C on bars[0]; B, then the D and S rows on bars[1])
  int issued0 = args.withhold ? 0 : 1, issued1 = 1, done0 = 0, done1 = 0;
  // On a wait that gave up: record the fault, wait (bounded) for every copy this
  // CTA issued, and leave.  The decision is made by the whole CTA at once.
  auto give_up = [&]() {
    if (tid == 0) {
      atomicExch(args.fault, 1);
      for (int p = done0; p < issued0; ++p) mbar_wait_bounded(&bars[0], p & 1, 4 * lim + 1000000000ull);
      for (int p = done1; p < issued1; ++p) mbar_wait_bounded(&bars[1], p & 1, 4 * lim + 1000000000ull);
    }
  };

  Acc r[N2];
  float ra[N2], rb[N2];
  float* sD = reinterpret_cast<float*>(buf1);
  float* sS = sD + TY * ROWP;
  // pairs A = (H_xy, H_xz) from buf0, B = (H_yz, N) from buf1, C = (H_xx, H_yy) from buf0 again.
  // When N2 < N1 and stage one of two pairs fits the CTA's threads, A and B are transformed
  // together and C and the D and S rows are issued once both buffers are read.
  constexpr bool PACK2 = N2 < N1 && 2 * TY * N2 <= G::THREADS;
  if constexpr (PACK2) {
    const bool ok0 = mbar_wait_bounded(&bars[0], 0u, lim);
    const bool ok = ok0 && mbar_wait_bounded(&bars[1], 0u, lim);
    if (__syncthreads_or(!ok)) {
      give_up();
      return;
    }
    done0 = 1;
    done1 = 1;
    float ra2[N2], rb2[N2];
    pair2_inverse<N>(buf0, buf1, s_tw, row, lane, ra, rb, ra2, rb2);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      AR::pair_a(r[k2], ra[k2], rb[k2]);
      AR::pair_b(r[k2], ra2[k2], rb2[k2], rp);
    }
    fence_proxy_async();  // this thread's accesses to both buffers precede the copies into them
    __syncthreads();
    if (tid == 0) issue_spectra<N>(buf0, &args.map[0], &args.map[1], x, y0, &bars[0]);
    issued0 = 2;
    if (tid < 32) {
      if (tid == 0) mbar_expect_tx(&bars[1], 2u * TY * N * 4);
      __syncwarp();
      const int64_t rbase0 = ((int64_t)x * N + y0) * N;
      for (int i = tid; i < 2 * TY; i += 32) {
        const int rr = i % TY;
        const float* src = (i < TY ? args.D : args.S) + rbase0 + (int64_t)rr * N;
        bulk_load((i < TY ? sD : sS) + rr * ROWP, src, N * 4, &bars[1]);
      }
    }
    issued1 = 2;
    if (__syncthreads_or(!mbar_wait_bounded(&bars[0], 1u, lim))) {
      give_up();
      return;
    }
    done0 = 2;
    pair_inverse<N>(buf0, s_tw, row, lane, ra, rb);
  }
  // otherwise one barrier per pair: after it every thread is done with the previous pair's
  // buffer, which then receives its next copy (C after A, the D and S rows after B)
#pragma unroll 1
  for (int pr = 0; pr < (PACK2 ? 0 : 3); ++pr) {
    uint64_t* bar = &bars[pr == 1 ? 1 : 0];
    unsigned char* buf = pr == 1 ? buf1 : buf0;
    fence_proxy_async();  // this thread's accesses to the previous buffer precede the copy into it
    if (__syncthreads_or(!mbar_wait_bounded(bar, pr == 2 ? 1u : 0u, lim))) {
      give_up();
      return;
    }
    if (pr == 0) done0 = 1;
    else if (pr == 1) done1 = 1;
    else done0 = 2;
    if (pr == 1) {
      if (tid == 0) issue_spectra<N>(buf0, &args.map[0], &args.map[1], x, y0, &bars[0]);
      issued0 = 2;
    } else if (pr == 2) {
      if (tid < 32) {
        if (tid == 0) mbar_expect_tx(&bars[1], 2u * TY * N * 4);
        __syncwarp();
        const int64_t rbase0 = ((int64_t)x * N + y0) * N;
        for (int i = tid; i < 2 * TY; i += 32) {
          const int rr = i % TY;
          const float* src = (i < TY ? args.D : args.S) + rbase0 + (int64_t)rr * N;
          bulk_load((i < TY ? sD : sS) + rr * ROWP, src, N * 4, &bars[1]);
        }
      }
      issued1 = 2;
    }
    pair_inverse<N>(buf, s_tw, row, lane, ra, rb);
    if (pr == 0) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) AR::pair_a(r[k2], ra[k2], rb[k2]);
    } else if (pr == 1) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) AR::pair_b(r[k2], ra[k2], rb[k2], rp);
    }
  }
  // ra, rb hold a = H_xx and b = H_yy
  if (__syncthreads_or(!mbar_wait_bounded(&bars[1], 1, lim))) {
    give_up();
    return;
  }
  // ---- residual and update; D_new replaces D in shared memory for the forward transform
  Sum rsum{};
  FP acc_d{0.f, 0.f};  // sum of D_new: its mean is removed next iteration
  float nbad = 0.f, nonfin = 0.f;
  const int64_t rbase = ((int64_t)x * N + y0 + row) * N;
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const int z = lane + N1 * k2;
    const PointOut o = AR::finish(r[k2], ra[k2], rb[k2], sD[row * ROWP + z], sS[row * ROWP + z], m_hi, m_lo, mean,
                                  rp, rsum, nonfin);
    float bpt = o.bp, dt = o.dt;
    if (o.neg) {
      nbad += 1.f;
      bpt = rp.bad_bp_f;
      dt = 0.f;
    }
    float dn;
    if constexpr (AR::kApproxRoot) {
      // D_new is an FP32 datum: the hardware square root and the full-range division (a few
      // ulp, far below the FFTs' rounding of the fields it is computed from)
      dn = fdiv_full(2.f * bpt, rp.alpha_f + sqrt_approx(dt));
    } else {
      dn = 2.f * bpt / (rp.alpha_f + sqrtf(dt));
    }
    args.Dnew[rbase + z] = dn;
    sD[row * ROWP + z] = dn;
    if constexpr (std::is_same<AR, RxF32>::value) acc_d.hi += dn;
    else fp_acc(acc_d, FP{dn, 0.f});
  }
  __syncthreads();
  // ---- forward z transform of D_new (two rows per pencil), written transposed
  {
    constexpr int FT = P * N1;
    const int fl = tid % N1, fp = tid / N1;
    float2* Tp = reinterpret_cast<float2*>(buf0) + fp * G::RS;
    if (tid < P * N2) {  // first stage: P x N2 tasks on the first threads
      const int q1 = tid / N2, l1 = tid % N2;
      float2* T1 = reinterpret_cast<float2*>(buf0) + q1 * G::RS;
      float2 v[N1];
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) {
        v[j1].x = sD[(2 * q1) * ROWP + N2 * j1 + l1];
        v[j1].y = sD[(2 * q1 + 1) * ROWP + N2 * j1 + l1];
      }
      dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) T1[k1 * (N2 + 1) + l1] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[k1 * N2 + l1]);
    }
    __syncthreads();
    float2* s_Zf = reinterpret_cast<float2*>(buf1);  // N x (P + 1); D_new has been read
    if (tid < FT) {
      float2 u[N2];
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[fl * (N2 + 1) + j2];
      dft_regs<N2, N / N2>(u, s_tw);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) s_Zf[(fl + N1 * k2) * (P + 1) + fp] = u[k2];
    }
    __syncthreads();
    // thread (kz0, yl) writes kz = kz0, kz0 + KZS, ... of column yl
    constexpr int KZS = G::THREADS / TY, ROUNDS = (NK + KZS - 1) / KZS;
    const int yl = tid % TY, kz0 = tid / TY, p = yl >> 1;
    const bool odd = yl & 1;
    float2* dst = args.Snew + ((int64_t)kz0 * N + x) * N + y0 + yl;
#pragma unroll
    for (int i = 0; i < ROUNDS; ++i) {
      const int kz = kz0 + i * KZS;
      if (i < ROUNDS - 1 || kz < NK) {
        const float2 zk = s_Zf[kz * (P + 1) + p];
        const float2 zm = s_Zf[((N - kz) % N) * (P + 1) + p];
        float2 o;
        if (!odd) o = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        else o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        dst[(int64_t)i * KZS * N * N] = o;
      }
    }
  }
  // ---- block statistics: within a warp float pairs (FP64 for the FP64 policy), across warps FP64
  const int wl = tid & 31, wid = tid >> 5;
  if constexpr (std::is_same<Sum, double>::value) {
    double v4[4] = {rsum, (double)acc_d.hi + (double)acc_d.lo, (double)nbad, (double)nonfin};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v4[c] += __shfl_xor_sync(0xffffffffu, v4[c], o);
      if (wl == 0) s_part[c * 32 + wid] = v4[c];
    }
  } else {
    FP r2 = pair_of(rsum), d2 = acc_d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      fp_acc(r2, FP{__shfl_xor_sync(0xffffffffu, r2.hi, o), __shfl_xor_sync(0xffffffffu, r2.lo, o)});
      fp_acc(d2, FP{__shfl_xor_sync(0xffffffffu, d2.hi, o), __shfl_xor_sync(0xffffffffu, d2.lo, o)});
    }
    const unsigned nb = __reduce_add_sync(0xffffffffu, (unsigned)nbad);
    const unsigned nf = __reduce_add_sync(0xffffffffu, (unsigned)nonfin);
    if (wl == 0) {
      s_part[0 * 32 + wid] = (double)r2.hi + (double)r2.lo;
      s_part[1 * 32 + wid] = (double)d2.hi + (double)d2.lo;
      s_part[2 * 32 + wid] = (double)nb;
      s_part[3 * 32 + wid] = (double)nf;
    }
  }
  __syncthreads();
  if (tid < 4) {
    const int nw = (blockDim.x + 31) >> 5;
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += s_part[tid * 32 + w];
    args.partials[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + tid] = t;
  }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

template <int N>
int relax_maps(float2* const* spec6, RelaxMaps* out) {
  using G = RGeom<N>;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return 1;
  // the half spectrum S[kz][x][y] as floats: dim 0 = 2N floats along y, dim 1 = x, dim 2 = kz
  const cuuint64_t dims[3] = {(cuuint64_t)2 * N, (cuuint64_t)N, (cuuint64_t)G::NK};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * N * 4, (cuuint64_t)N * 2 * N * 4};
  const cuuint32_t box[3] = {(cuuint32_t)2 * G::TY, 1, (cuuint32_t)G::BOXK};
  const cuuint32_t es[3] = {1, 1, 1};
  for (int f = 0; f < 6; ++f) {
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(&out->map[f]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                           spec6[f], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return 1;
  }
  return 0;
}

template <int N> int relax_tma_blocks() { return (N / RGeom<N>::TY) * N; }

template <int N, class AR, int RB>
static void launch_rt(const RelaxTmaArgs* a, int count, const float2* tw, cudaStream_t s) {
  using G = RGeom<N>;
  RelaxTmaBatch<RB> b;
  for (int r = 0; r < count; ++r) b.a[r] = a[r];
  raise_smem_limit<k_relax_tma<N, AR, RB>>(G::SMEM);
  dim3 grid(N / G::TY, N, count);
  k_relax_tma<N, AR, RB><<<grid, G::THREADS, G::SMEM, s>>>(b, tw);
}

template <int N, class AR>
static void launch_rt(const RelaxTmaArgs* a, int count, const float2* tw, cudaStream_t s) {
  if (count == 1) launch_rt<N, AR, 1>(a, 1, tw, s);
  else launch_rt<N, AR, kBatchMax>(a, count, tw, s);
}

template <int N>
void launch_relax_tma(int arith, const RelaxMaps& maps, const float* D, const double* dsum, const float* S,
                      float* Dnew, float2* Snew, RelaxParams rp, double* partials, const float2* tw, cudaStream_t s,
                      const int* skip, int* fault, unsigned long long wait_ns, int withhold) {
  RelaxTmaArgs a;
  memcpy(a.map, maps.map, sizeof(a.map));
  a.D = D; a.dsum = dsum; a.S = S; a.Dnew = Dnew; a.Snew = Snew; a.partials = partials; a.rp = rp;
  a.skip = skip; a.fault = fault; a.wait_ns = wait_ns; a.withhold = withhold;
  launch_relax_tma_batch<N>(arith, &a, 1, tw, s);
}

template <int N>
void launch_relax_tma_batch(int arith, const RelaxTmaArgs* a, int count, const float2* tw, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  if (arith == ARITH_F64) launch_rt<N, RxF64>(a, count, tw, s);
  else if (arith == ARITH_EFT) launch_rt<N, RxEFT>(a, count, tw, s);
  else if (arith == ARITH_M32) launch_rt<N, RxM32>(a, count, tw, s);
  else launch_rt<N, RxF32>(a, count, tw, s);
}

#define DGP_INST_RT(N)                                                                                          \
  template int relax_maps<N>(float2* const*, RelaxMaps*);                                                     \
  template int relax_tma_blocks<N>();                                                                         \
  template void launch_relax_tma<N>(int, const RelaxMaps&, const float*, const double*, const float*, float*,  \
                                    float2*, RelaxParams, double*, const float2*, cudaStream_t, const int*, int*, \
                                    unsigned long long, int);                                                 \
  template void launch_relax_tma_batch<N>(int, const RelaxTmaArgs*, int, const float2*, cudaStream_t);
DGP_INST_RT(16)
DGP_INST_RT(32)
DGP_INST_RT(48)
DGP_INST_RT(64)
DGP_INST_RT(96)
DGP_INST_RT(128)
DGP_INST_RT(256)
DGP_INST_RT(512)

}  // namespace dgp
