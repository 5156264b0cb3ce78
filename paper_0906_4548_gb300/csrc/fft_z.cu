// z transforms: real rows f[x][y][0..N) <-> half spectra S[kz][x][y].
//
// A CTA owns TY consecutive rows y0..y0+TY-1 at one x.  Two real rows are
// packed into one complex pencil (a + i b), transformed with the four-step
// split, and separated with A(k) = (Z(k) + conj Z(N-k))/2,
// B(k) = (Z(k) - conj Z(N-k))/(2i).  Output goes to S[kz][x][y0 + yl] so that
// consecutive threads write consecutive y (TY * 8 bytes per kz).  The inverse
// gathers S[kz][x][y-tile] the same way, rebuilds Z(k) = A(k) + i B(k) over all
// k by Hermitian symmetry (the imaginary parts of the kz = 0 and kz = N/2
// coefficients are dropped, as a real-output transform must), and writes rows.
#include "fft_core.cuh"
#include "kernels.cuh"

namespace dgp {

template <typename T, int N> struct ZGeom {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int TYW0 = (sizeof(T) == 8 || N >= 512) ? 16 : 32;
  static constexpr int TYW = N % TYW0 == 0 ? TYW0 : 16;  // rows per CTA divide N
  static constexpr int TY = TYW < N ? TYW : N;
  static constexpr int P = TY / 2;
  static constexpr int THREADS = P * N1;
};

// Prologue as v * scale + shift, the two coefficients formed once per CTA:
// kind 1 (rho -> rho / mean - 1): scale = 1 / mean, shift = -1;
// kind 2 (v - mean): scale = 1, shift = -mean.
template <typename T>
__device__ __forceinline__ void prologue_coeffs(const ZPrologue& pro, T* s_ss) {
  if (threadIdx.x == 0) {
    T sc = (T)1, sh = (T)0;
    if (pro.kind != 0) {
      const double mean = pro.mean_src[0] * pro.inv_count;
      if (pro.kind == 1) { sc = (T)(1.0 / mean); sh = (T)-1; }
      else sh = (T)(-mean);
    }
    s_ss[0] = sc;
    s_ss[1] = sh;
  }
}

template <typename T, int RB> struct ZR2CBatch {
  const T* in[RB];
  vec2_t<T>* out[RB];
  ZPrologue pro[RB];
};

template <typename T, int N, int RB>
__global__ void __launch_bounds__(ZGeom<T, N>::THREADS, 3)
k_fft_z_r2c(const __grid_constant__ ZR2CBatch<T, RB> zb, int64_t in_stride, int64_t out_stride,
            const vec2_t<T>* __restrict__ g_tw) {
  // fields on blockIdx.z (one realisation), or realisations on blockIdx.z (one field each)
  const int rz = RB > 1 ? blockIdx.z : 0;
  const T* __restrict__ in = zb.in[rz];
  vec2_t<T>* __restrict__ out = zb.out[rz];
  const ZPrologue& pro = zb.pro[rz];
  using V = vec2_t<T>;
  using G = ZGeom<T, N>;
  constexpr int N1 = G::N1, N2 = G::N2, TY = G::TY, P = G::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s_tw = reinterpret_cast<V*>(smem_raw);
  V* s_T = s_tw + kTwiddleTables * N;                        // P * N1 * (N2 + 1)
  V* s_Z = s_T + P * N1 * (N2 + 1);         // N * (P + 1)
  load_twiddles(s_tw, g_tw, N);
  const int lane = threadIdx.x % N1;
  const int pl = threadIdx.x / N1;
  const int x = blockIdx.y;
  const int y0 = blockIdx.x * TY;
  const T* src = in + (RB > 1 ? 0 : (int64_t)blockIdx.z * in_stride);
  V* dst = out + (RB > 1 ? 0 : (int64_t)blockIdx.z * out_stride);
  __shared__ T s_ss[2];
  prologue_coeffs<T>(pro, s_ss);
  const T* rowa = src + ((int64_t)x * N + y0 + 2 * pl) * N;
  const T* rowb = rowa + N;
  V* Tp = s_T + pl * (N1 * (N2 + 1));
  __syncthreads();
  const T sc = s_ss[0], sh = s_ss[1];
  // stage one has P x N2 tasks (a row pair and its column j2): when N2 < N1 they go to the
  // first P x N2 threads, so that whole warps idle rather than lanes of every warp
  constexpr bool PACK = N2 < N1;
  const int p1 = PACK ? (int)threadIdx.x / N2 : pl, c1 = PACK ? (int)threadIdx.x % N2 : lane;
  if (!PACK || p1 < P) {
    const T* ra1 = PACK ? src + ((int64_t)x * N + y0 + 2 * p1) * N : rowa;
    const T* rb1 = ra1 + N;
    V* T1 = PACK ? s_T + p1 * (N1 * (N2 + 1)) : Tp;
    V v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      v[j1].x = ra1[N2 * j1 + c1] * sc + sh;
      v[j1].y = rb1[N2 * j1 + c1] * sc + sh;
    }
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      T1[k1 * (N2 + 1) + c1] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + c1]);
  }
  __syncthreads();
  {
    V u[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[lane * (N2 + 1) + j2];
    dft_regs<N2, N / N2>(u, s_tw);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) s_Z[(lane + N1 * k2) * (P + 1) + pl] = u[k2];
  }
  __syncthreads();
  constexpr int NK = N / 2 + 1;
  for (int item = threadIdx.x; item < NK * TY; item += blockDim.x) {
    const int kz = item / TY, yl = item % TY;
    const int p = yl >> 1;
    const V zk = s_Z[kz * (P + 1) + p];
    const V zm = s_Z[((N - kz) % N) * (P + 1) + p];
    V r;
    if ((yl & 1) == 0) r = cmake<V>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
    else r = cmake<V>((T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x));
    dst[((int64_t)kz * N + x) * N + y0 + yl] = r;
  }
}

template <typename T, int RB> struct ZC2RBatch {
  FieldSet<T> in[RB];
  FieldSet<T> out[RB];
};

template <typename T, int N, int RB>
__global__ void __launch_bounds__(ZGeom<T, N>::THREADS, 3)
k_fft_z_c2r(const __grid_constant__ ZC2RBatch<T, RB> zb, int nfields, const vec2_t<T>* __restrict__ g_tw) {
  const int rz = RB > 1 ? (int)blockIdx.z / nfields : 0, fz = RB > 1 ? (int)blockIdx.z % nfields : blockIdx.z;
  const FieldSet<T>& in = zb.in[rz];
  const FieldSet<T>& outp = zb.out[rz];
  using V = vec2_t<T>;
  using G = ZGeom<T, N>;
  constexpr int N1 = G::N1, N2 = G::N2, TY = G::TY, P = G::P;
  constexpr int NK = N / 2 + 1;
  constexpr int HSZ = NK * (TY + 1);
  constexpr int TSZ = P * N1 * (N2 + 1);
  constexpr int BUF = HSZ > TSZ ? HSZ : TSZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s_tw = reinterpret_cast<V*>(smem_raw);
  V* s_H = s_tw + kTwiddleTables * N;        // NK * (TY + 1); later reused as s_T
  V* s_T = s_H;
  V* s_Z = s_H + BUF;       // N * (P + 1)
  load_twiddles(s_tw, g_tw, N);
  const int x = blockIdx.y;
  const int y0 = blockIdx.x * TY;
  const V* src = in.p[fz];
  T* dst = reinterpret_cast<T*>(outp.p[fz]);
  // the CTA's NK rows of TY values, one 8- or 16-byte segment per kz plane: for FP32 all of a
  // thread's loads are issued before its stores, so they are in flight together
  constexpr int ITEMS = (NK * TY + G::THREADS - 1) / G::THREADS;
  if constexpr (sizeof(T) == 4 && ITEMS <= 24) {
    V tmp[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int item = threadIdx.x + i * G::THREADS;
      if (item < NK * TY) tmp[i] = src[((int64_t)(item / TY) * N + x) * N + y0 + item % TY];
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int item = threadIdx.x + i * G::THREADS;
      if (item < NK * TY) s_H[(item / TY) * (TY + 1) + item % TY] = tmp[i];
    }
  } else {
    for (int item = threadIdx.x; item < NK * TY; item += blockDim.x) {
      const int kz = item / TY, yl = item % TY;
      s_H[kz * (TY + 1) + yl] = src[((int64_t)kz * N + x) * N + y0 + yl];
    }
  }
  __syncthreads();
  for (int item = threadIdx.x; item < N * P; item += blockDim.x) {
    const int k = item / P, p = item % P;
    V A, B;
    if (k <= N / 2) {
      A = s_H[k * (TY + 1) + 2 * p];
      B = s_H[k * (TY + 1) + 2 * p + 1];
      if (k == 0 || k == N / 2) { A.y = 0; B.y = 0; }
    } else {
      A = cconj(s_H[(N - k) * (TY + 1) + 2 * p]);
      B = cconj(s_H[(N - k) * (TY + 1) + 2 * p + 1]);
    }
    // Z = A + i B, stored conjugated for the inverse
    s_Z[k * (P + 1) + p] = cmake<V>(A.x - B.y, -(A.y + B.x));
  }
  __syncthreads();
  const int lane = threadIdx.x % N1;
  const int pl = threadIdx.x / N1;
  V* Tp = s_T + pl * (N1 * (N2 + 1));
  constexpr bool PACK = N2 < N1;  // stage one on the first P x N2 threads, as in the r2c pass
  const int p1 = PACK ? (int)threadIdx.x / N2 : pl, c1 = PACK ? (int)threadIdx.x % N2 : lane;
  if (!PACK || p1 < P) {
    V* T1 = PACK ? s_T + p1 * (N1 * (N2 + 1)) : Tp;
    V v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = s_Z[(N2 * j1 + c1) * (P + 1) + p1];
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      T1[k1 * (N2 + 1) + c1] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + c1]);
  }
  __syncthreads();
  {
    V u[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[lane * (N2 + 1) + j2];
    dft_regs<N2, N / N2>(u, s_tw);
    T* rowa = dst + ((int64_t)x * N + y0 + 2 * pl) * N;
    T* rowb = rowa + N;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      rowa[lane + N1 * k2] = u[k2].x;    // conj of the result: real part unchanged
      rowb[lane + N1 * k2] = -u[k2].y;
    }
  }
}

template <typename T, int N> static size_t r2c_smem() {
  using G = ZGeom<T, N>;
  return sizeof(vec2_t<T>) * (kTwiddleTables * N + G::P * G::N1 * (G::N2 + 1) + N * (G::P + 1));
}
template <typename T, int N> static size_t c2r_smem() {
  using G = ZGeom<T, N>;
  const size_t hsz = (size_t)(N / 2 + 1) * (G::TY + 1), tsz = (size_t)G::P * G::N1 * (G::N2 + 1);
  return sizeof(vec2_t<T>) * (kTwiddleTables * N + (hsz > tsz ? hsz : tsz) + (size_t)N * (G::P + 1));
}

template <typename T, int N>
void launch_fft_z_r2c(const T* in, int64_t in_stride, vec2_t<T>* out, int64_t out_stride, int nfields,
                      ZPrologue pro, const vec2_t<T>* tw, cudaStream_t s) {
  using G = ZGeom<T, N>;
  const size_t smem = r2c_smem<T, N>();
  raise_smem_limit<k_fft_z_r2c<T, N, 1>>(smem);
  ZR2CBatch<T, 1> zb;
  zb.in[0] = in;
  zb.out[0] = out;
  zb.pro[0] = pro;
  dim3 grid(N / G::TY, N, nfields);
  k_fft_z_r2c<T, N, 1><<<grid, G::THREADS, smem, s>>>(zb, in_stride, out_stride, tw);
}

template <typename T, int N>
void launch_fft_z_r2c_batch(const T* const* in, vec2_t<T>* const* out, const ZPrologue* pro, int count,
                            const vec2_t<T>* tw, cudaStream_t s) {
  using G = ZGeom<T, N>;
  if (count < 1 || count > kBatchMax) return;
  const size_t smem = r2c_smem<T, N>();
  raise_smem_limit<k_fft_z_r2c<T, N, kBatchMax>>(smem);
  ZR2CBatch<T, kBatchMax> zb;
  for (int r = 0; r < count; ++r) {
    zb.in[r] = in[r];
    zb.out[r] = out[r];
    zb.pro[r] = pro[r];
  }
  dim3 grid(N / G::TY, N, count);
  k_fft_z_r2c<T, N, kBatchMax><<<grid, G::THREADS, smem, s>>>(zb, 0, 0, tw);
}

template <typename T, int N>
void launch_fft_z_c2r(const FieldSet<T>& in, T* const* out, int nfields, const vec2_t<T>* tw,
                      cudaStream_t s) {
  using G = ZGeom<T, N>;
  ZC2RBatch<T, 1> zb;
  zb.in[0] = in;
  for (int i = 0; i < kMaxFields; ++i) zb.out[0].p[i] = i < nfields ? reinterpret_cast<vec2_t<T>*>(out[i]) : nullptr;
  const size_t smem = c2r_smem<T, N>();
  raise_smem_limit<k_fft_z_c2r<T, N, 1>>(smem);
  dim3 grid(N / G::TY, N, nfields);
  k_fft_z_c2r<T, N, 1><<<grid, G::THREADS, smem, s>>>(zb, nfields, tw);
}

template <typename T, int N>
void launch_fft_z_c2r_batch(const FieldSet<T>* in, const FieldSet<T>* out, int nfields, int count,
                            const vec2_t<T>* tw, cudaStream_t s) {
  using G = ZGeom<T, N>;
  if (count < 1 || count > kBatchMax) return;
  ZC2RBatch<T, kBatchMax> zb;
  for (int r = 0; r < count; ++r) {
    zb.in[r] = in[r];
    zb.out[r] = out[r];
  }
  const size_t smem = c2r_smem<T, N>();
  raise_smem_limit<k_fft_z_c2r<T, N, kBatchMax>>(smem);
  dim3 grid(N / G::TY, N, nfields * count);
  k_fft_z_c2r<T, N, kBatchMax><<<grid, G::THREADS, smem, s>>>(zb, nfields, tw);
}

#define DGP_INST_Z(T, N)                                                                          \
  template void launch_fft_z_r2c<T, N>(const T*, int64_t, vec2_t<T>*, int64_t, int, ZPrologue,     \
                                       const vec2_t<T>*, cudaStream_t);                            \
  template void launch_fft_z_c2r<T, N>(const FieldSet<T>&, T* const*, int, const vec2_t<T>*, cudaStream_t);
#define DGP_INST_ZB(N)                                                                                  \
  template void launch_fft_z_r2c_batch<float, N>(const float* const*, float2* const*, const ZPrologue*, int,  \
                                                 const float2*, cudaStream_t);                               \
  template void launch_fft_z_c2r_batch<float, N>(const FieldSet<float>*, const FieldSet<float>*, int, int,     \
                                                 const float2*, cudaStream_t);
DGP_INST_ZB(16) DGP_INST_ZB(32) DGP_INST_ZB(48) DGP_INST_ZB(64) DGP_INST_ZB(96) DGP_INST_ZB(128)
#define DGP_INST_Z_ALL(T) DGP_INST_Z(T, 16) DGP_INST_Z(T, 32) DGP_INST_Z(T, 64) DGP_INST_Z(T, 128) \
  DGP_INST_Z(T, 256) DGP_INST_Z(T, 512) DGP_INST_Z(T, 48) DGP_INST_Z(T, 96)
DGP_INST_Z_ALL(float)
DGP_INST_Z_ALL(double)

}  // namespace dgp
