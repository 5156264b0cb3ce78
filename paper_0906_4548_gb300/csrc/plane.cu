// Plane-resident Hessian pass for small meshes (FP32 data, realisations of one class).
//
// One CTA owns one kz plane of one realisation.  It reads the plane of the z spectrum of
// the iterate D (layout S[kz][x][y]) once, transforms it forward along y and along x in
// shared memory, and for each of the six outputs of the relaxation (H_xx, H_yy, H_xy, H_xz,
// H_yz and N, Sec. III.B: nabla_ij C(k) = -k_i k_j C(k), sqrt(-lapbar) C = -D / kbar)
// forms the multiplier, transforms back along x and y and writes the plane of the output
// (kz, x, y), ready for the relaxation pass's inverse z transform.  This replaces the
// y pass of D_new, the Hessian x pass and the six-field inverse y pass of an iteration: per
// iteration the six output spectra cross HBM once (written here, read by the relaxation)
// instead of three times.  A plane of N x N complex floats must fit twice in shared
// memory, so the pass serves N <= 96.
//
// Transforms are the four-step split N = N1 * N2 done in place on a line of the plane:
// forward, stage 1 takes the N1 elements N2*j1 + j2 of a line, transforms them, multiplies
// by W_N^{j2 k1} and puts them back at N2*k1 + j2; stage 2 transforms the N2 contiguous
// elements N2*k1 + j2 (j2 < N2) and leaves X[k1 + N1*k2] at position N2*k1 + k2 (digit
// order).  The inverse runs the stages in the opposite order, from digit order back to
// natural order, as conj(DFT(conj(.))).  The plane's row pitch is N + 1 (odd): within a
// stage consecutive threads take consecutive lines of the same stage index, so a half-warp
// touches 16 different banks along either axis.
#include "fft_core.cuh"
#include "kernels.cuh"

namespace dgp {

template <int N> struct PGeom {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int PITCH = N + 1;
  static constexpr int PLANE = N * PITCH;  // complex elements of one plane buffer
  static constexpr int THREADS = N == 96 ? 768 : N == 64 ? 256 : N == 48 ? 192 : N == 32 ? 128 : 64;
  static constexpr int MINB = N == 96 ? 1 : N == 64 ? 2 : N == 48 ? 4 : N == 32 ? 4 : 8;
  static constexpr size_t SMEM = sizeof(float2) * ((size_t)2 * PLANE + (size_t)kTwiddleTables * N);
  static_assert(N % 16 == 0 || N < 16, "lines of a stage are taken 16 at a time");
};

// Forward stage 1 on the lines of a plane buffer: line stride LS, element stride ES.
template <int N, int LS, int ES>
__device__ __forceinline__ void fwd_stage1(float2* __restrict__ b, const float2* __restrict__ s_tw) {
  using G = PGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2;
#pragma unroll 1
  for (int q = threadIdx.x; q < N * N2; q += G::THREADS) {
    const int line = q % N, j2 = q / N;
    float2* L = b + line * LS;
    float2 v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = L[(N2 * j1 + j2) * ES];
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) L[(N2 * k1 + j2) * ES] = k1 == 0 ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + j2]);
  }
}

// Forward stage 2; MUL(line, k1, k2, value) may scale each output before it is stored.
template <int N, int LS, int ES, class Mul>
__device__ __forceinline__ void fwd_stage2(float2* __restrict__ b, const float2* __restrict__ s_tw, Mul mul) {
  using G = PGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2;
#pragma unroll 1
  for (int q = threadIdx.x; q < N * N1; q += G::THREADS) {
    const int line = q % N, k1 = q / N;
    float2* L = b + line * LS + N2 * k1 * ES;
    float2 u[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) u[j2] = L[j2 * ES];
    dft_regs<N2, N / N2>(u, s_tw);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) L[k2 * ES] = mul(line, k1, k2, u[k2]);
  }
}

// Inverse stage 1 from src (digit order) into dst: CONJ_IN conjugates on entry, and
// MUL(line, k1, k2, value) forms the input (a k-space multiplier) as it is read.
template <int N, int LS, int ES, bool CONJ_IN, class Mul>
__device__ __forceinline__ void inv_stage1(const float2* src, float2* dst,  // may be the same buffer
                                           const float2* __restrict__ s_tw, Mul mul) {
  using G = PGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2;
#pragma unroll 1
  for (int q = threadIdx.x; q < N * N1; q += G::THREADS) {
    const int line = q % N, k1 = q / N;
    const int o = line * LS + N2 * k1 * ES;
    float2 u[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const float2 x = mul(line, k1, k2, src[o + k2 * ES]);
      u[k2] = CONJ_IN ? cconj(x) : x;
    }
    dft_regs<N2, N / N2>(u, s_tw);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) dst[o + n2 * ES] = n2 == 0 ? u[n2] : cmul(u[n2], s_tw[N + k1 * N2 + n2]);
  }
}

// Inverse stage 2 in place, natural order out; CONJ_OUT conjugates on exit.
template <int N, int LS, int ES, bool CONJ_OUT>
__device__ __forceinline__ void inv_stage2(float2* __restrict__ b, const float2* __restrict__ s_tw) {
  using G = PGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2;
#pragma unroll 1
  for (int q = threadIdx.x; q < N * N2; q += G::THREADS) {
    const int line = q % N, n2 = q / N;
    float2* L = b + line * LS;
    float2 w[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) w[k1] = L[(N2 * k1 + n2) * ES];
    dft_regs<N1, N / N1>(w, s_tw);
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) L[(N2 * n1 + n2) * ES] = CONJ_OUT ? cconj(w[n1]) : w[n1];
  }
}

template <int RB> struct PlaneBatch {
  PlaneArgs a[RB];
};

// Plane <-> shared-memory copies (row pitch PITCH): TY rows of N at a time when the CTA's
// threads divide into whole rows, so no thread divides its index by N per element.
template <int N, bool TO_SMEM>
__device__ __forceinline__ void copy_plane(float2* __restrict__ sm, float2* __restrict__ g) {
  using G = PGeom<N>;
  if constexpr (G::THREADS % N == 0) {
    constexpr int RPI = G::THREADS / N;  // rows per round
    const int col = threadIdx.x % N, r0 = threadIdx.x / N;
#pragma unroll 4
    for (int r = r0; r < N; r += RPI) {
      if (TO_SMEM) sm[r * G::PITCH + col] = g[r * N + col];
      else g[r * N + col] = sm[r * G::PITCH + col];
    }
  } else {
    for (int i = threadIdx.x; i < N * N; i += G::THREADS) {
      if (TO_SMEM) sm[(i / N) * G::PITCH + i % N] = g[i];
      else g[i] = sm[(i / N) * G::PITCH + i % N];
    }
  }
}

template <int N, int RB>
__global__ void __launch_bounds__(PGeom<N>::THREADS, PGeom<N>::MINB)
    k_plane_hessian(const __grid_constant__ PlaneBatch<RB> pb, const float2* __restrict__ g_tw) {
  using G = PGeom<N>;
  constexpr int N1 = G::N1, N2 = G::N2, PITCH = G::PITCH;
  const PlaneArgs& args = pb.a[RB > 1 ? blockIdx.y : 0];
  if (args.skip && *args.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* A = reinterpret_cast<float2*>(smem_raw);  // the spectrum of D, then scaled
  float2* B = A + G::PLANE;                          // one output at a time
  float2* s_tw = B + G::PLANE;
  load_twiddles(s_tw, g_tw, N);
  const int kz = blockIdx.x;
  copy_plane<N, true>(A, const_cast<float2*>(args.in) + (int64_t)kz * N * N);
  __syncthreads();
  // forward along y (lines = rows x), then along x (lines = columns)
  fwd_stage1<N, PITCH, 1>(A, s_tw);
  __syncthreads();
  auto keep = [](int, int, int, float2 v) { return v; };
  fwd_stage2<N, PITCH, 1>(A, s_tw, keep);
  __syncthreads();
  fwd_stage1<N, 1, PITCH>(A, s_tw);
  __syncthreads();
  // column py holds ky = k1y + N1 k2y at py = N2 k1y + k2y; the x stage 2 output of (k1, k2)
  // is kx = k1 + N1 k2.  Scale by 1 / (|n|^2 N^3) there (0 at k = 0).
  const KParams& kp = args.kp;
  const float inv_m = kp.inv_m_f;
  const int nz = kz == N / 2 ? -(N / 2) : kz;
  const bool nyq_z = kz == N / 2;
  const float fz = (float)nz;
  auto ky_of = [](int py) { return py / N2 + N1 * (py % N2); };
  auto scale = [&](int py, int k1, int k2, float2 v) {
    const int ky = ky_of(py);
    const float fx = (float)signed_index(k1 + N1 * k2, N), fy = (float)signed_index(ky, N);
    const float n2 = fx * fx + fy * fy + fz * fz;
    return cscale(v, n2 != 0.f ? inv_m / n2 : 0.f);
  };
  fwd_stage2<N, 1, PITCH>(A, s_tw, scale);
  __syncthreads();
  const float ikf = kp.local_only ? 0.f : 1.f / kp.kbkf_f;
#pragma unroll 1
  for (int o = 0; o < 6; ++o) {
    // multiplier of output o at (kx, ky, kz), formed as the x inverse reads A
    const bool a_is_x = o == 0 || o == 2 || o == 3;
    const int b_sel = o == 0 ? 0 : (o == 1 || o == 2 ? 1 : 2);
    auto mul = [&](int py, int k1, int k2, float2 v) {
      const int kx = k1 + N1 * k2, ky = ky_of(py);
      const float fx = (float)signed_index(kx, N), fy = (float)signed_index(ky, N);
      float m;
      if (o == 5) {
        m = -sqrtf(fx * fx + fy * fy + fz * fz) * ikf;
      } else {
        const float fa = a_is_x ? fx : fy;
        const float fb = b_sel == 0 ? fx : (b_sel == 1 ? fy : fz);
        m = fa * fb;
        const bool nyq = (!a_is_x && ky == N / 2) || (b_sel == 1 && ky == N / 2) || (b_sel == 2 && nyq_z) ||
                         ((a_is_x || b_sel == 0) && kx == N / 2);
        if (nyq) m = fabsf(m);
      }
      return cscale(v, m);
    };
    // inverse along x (lines = columns): conj on entry; along y (lines = rows): conj on exit
    inv_stage1<N, 1, PITCH, true>(A, B, s_tw, mul);
    __syncthreads();
    inv_stage2<N, 1, PITCH, false>(B, s_tw);
    __syncthreads();
    inv_stage1<N, PITCH, 1, false>(B, B, s_tw, keep);
    __syncthreads();
    inv_stage2<N, PITCH, 1, true>(B, s_tw);
    __syncthreads();
    copy_plane<N, false>(B, args.out.p[o] + (int64_t)kz * N * N);
    __syncthreads();
  }
}

template <int N>
static void launch_plane(const PlaneArgs* a, int count, const float2* tw, cudaStream_t s) {
  using G = PGeom<N>;
  PlaneBatch<kBatchMax> pb;
  for (int r = 0; r < count; ++r) pb.a[r] = a[r];
  raise_smem_limit<k_plane_hessian<N, kBatchMax>>(G::SMEM);
  k_plane_hessian<N, kBatchMax><<<dim3((unsigned)(N / 2 + 1), (unsigned)count), G::THREADS, G::SMEM, s>>>(pb, tw);
}

bool plane_hessian_supported(int n) { return n == 16 || n == 32 || n == 48 || n == 64 || n == 96; }

void launch_plane_hessian_batch(int n, const PlaneArgs* a, int count, const float2* tw, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  switch (n) {
    case 16: launch_plane<16>(a, count, tw, s); break;
    case 32: launch_plane<32>(a, count, tw, s); break;
    case 48: launch_plane<48>(a, count, tw, s); break;
    case 64: launch_plane<64>(a, count, tw, s); break;
    case 96: launch_plane<96>(a, count, tw, s); break;
    default: break;
  }
}

}  // namespace dgp
