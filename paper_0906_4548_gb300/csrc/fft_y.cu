// y transform: in-place complex DFT along the contiguous rows of S[kz][x][y].
//
// Each CTA of B threads (B = 128, 256 or 512, chosen per context by timing, see
// api.cu) owns P = B / N1 rows.  Phase 1: one thread per row and j2 < N2
// reads x[N2*j1 + j2] straight from global memory (consecutive lanes,
// consecutive addresses), transforms over j1 and stores the twiddled result
// to shared memory; phase 2: lane k1 reads its N2 values back with an odd
// row pitch (N2 + 1, no bank conflicts), transforms and writes
// X[k1 + N1*k2] back to global memory (again consecutive lanes, consecutive
// addresses).  HBM traffic: one read and one write of the rows.
#include "fft_core.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "relax_control.cuh"

namespace dgp {

// 64 registers per thread for FP32 rows of up to 256 points, 128 otherwise
template <typename T, int N, bool INV, int B, bool CTL, int RB>
__global__ void __launch_bounds__(B, (sizeof(T) == 8 || N >= 512 ? 512 : 1024) / B)
    k_fft_y(const __grid_constant__ YBatch<T, RB> yb, int64_t npencils, const vec2_t<T>* __restrict__ g_tw) {
  const int rz = RB > 1 ? blockIdx.z : 0;  // realisation of this CTA
  const FieldSet<T>& f = yb.f[rz];
  const int* skip = yb.skip[rz];
  const YControl& yc = yb.yc[rz];
  if (skip && *skip) return;
  if constexpr (CTL) {
    // the extra CTA, first in launch order so that it overlaps the transform's CTAs:
    // statistics and stop rules of the iteration
    if (blockIdx.x == 0) {
      double v[4] = {0.0, 0.0, 0.0, 0.0};
      for (int b = threadIdx.x; b < yc.nblocks; b += blockDim.x) {
        const double* pb = yc.partials + 4 * (int64_t)b;
        v[0] += pb[0];
        v[1] += pb[1];
        v[2] += pb[2];
        v[3] += pb[3];
      }
      block_sum<4>(v);
      if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) yc.stats[k] = v[k];
        relax_control_step(yc.ctl, yc.stats, yc.abs_src_sum, yc.hist, yc.max_iter, yc.patience, yc.tol, yc.inv_m);
      }
      return;
    }
  }
  using V = vec2_t<T>;
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  constexpr int P = B / N1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s_tw = reinterpret_cast<V*>(smem_raw);
  V* s_T = s_tw + kTwiddleTables * N;
  load_twiddles(s_tw, g_tw, N);
  const int lane = threadIdx.x % N1;
  const int pl = threadIdx.x / N1;
  const int64_t pencil = (int64_t)(blockIdx.x - (CTL ? 1 : 0)) * P + pl;
  const bool active = pencil < npencils;
  V* base = f.p[blockIdx.y] + (active ? pencil : 0) * N;
  V* Tp = s_T + pl * (N1 * (N2 + 1));
  // Phase 1 has P x N2 tasks (a row and its column j2); when N2 < N1 they go to the first
  // P x N2 threads, so that whole warps idle rather than lanes of every warp.
  constexpr bool PACK = N2 < N1;
  const int p1 = PACK ? (int)threadIdx.x / N2 : pl, c1 = PACK ? (int)threadIdx.x % N2 : lane;
  const int64_t pencil1 = PACK ? (int64_t)(blockIdx.x - (CTL ? 1 : 0)) * P + p1 : pencil;
  const bool act1 = PACK ? (p1 < P && pencil1 < npencils) : active;
  const V* base1 = PACK ? f.p[blockIdx.y] + (act1 ? pencil1 : 0) * N : base;
  V* T1 = PACK ? s_T + p1 * (N1 * (N2 + 1)) : Tp;
  __syncthreads();
  if (act1) {
    V v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = base1[N2 * j1 + c1];
    if (INV) conj_regs(v);
    dft_regs<N1, N / N1>(v, s_tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      T1[k1 * (N2 + 1) + c1] = (k1 == 0) ? v[k1] : cmul(v[k1], s_tw[N + k1 * N2 + c1]);
  }
  __syncthreads();
  if (active) {
    V u[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) u[j2] = Tp[lane * (N2 + 1) + j2];
    dft_regs<N2, N / N2>(u, s_tw);
    if (INV) conj_regs(u);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) base[lane + N1 * k2] = u[k2];
  }
}

template <typename T, int N, int B, int RB>
static void launch_y(const YBatch<T, RB>& yb, int count, int nfields, bool inverse, bool ctl, const vec2_t<T>* tw,
                     cudaStream_t s) {
  using V = vec2_t<T>;
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  constexpr int P = B / N1;
  const int64_t npencils = (int64_t)(N / 2 + 1) * N;
  const size_t smem = sizeof(V) * (kTwiddleTables * N + P * N1 * (N2 + 1));
  // with the stop rules: one extra CTA, and the fields on grid.x only (one field)
  dim3 grid((unsigned)((npencils + P - 1) / P) + (ctl ? 1u : 0u), (unsigned)nfields, (unsigned)count);
  if (inverse) {
    raise_smem_limit<k_fft_y<T, N, true, B, false, RB>>(smem);
    k_fft_y<T, N, true, B, false, RB><<<grid, B, smem, s>>>(yb, npencils, tw);
  } else if (ctl) {
    raise_smem_limit<k_fft_y<T, N, false, B, true, RB>>(smem);
    k_fft_y<T, N, false, B, true, RB><<<grid, B, smem, s>>>(yb, npencils, tw);
  } else {
    raise_smem_limit<k_fft_y<T, N, false, B, false, RB>>(smem);
    k_fft_y<T, N, false, B, false, RB><<<grid, B, smem, s>>>(yb, npencils, tw);
  }
}

template <typename T, int N, int RB>
static void launch_y_threads(const YBatch<T, RB>& yb, int count, int nfields, bool inverse, bool ctl,
                             const vec2_t<T>* tw, cudaStream_t s, int threads) {
  if (threads == 128) launch_y<T, N, 128, RB>(yb, count, nfields, inverse, ctl, tw, s);
  else if (threads == 512) launch_y<T, N, 512, RB>(yb, count, nfields, inverse, ctl, tw, s);
  else launch_y<T, N, 256, RB>(yb, count, nfields, inverse, ctl, tw, s);
}

template <typename T, int N>
void launch_fft_y(const FieldSet<T>& f, int nfields, bool inverse, const vec2_t<T>* tw, cudaStream_t s,
                  const int* skip, int threads, const YControl* ctl) {
  if (ctl && (inverse || nfields != 1)) return;  // the stop rules ride on a one-field forward pass only
  YBatch<T, 1> yb;
  yb.f[0] = f;
  yb.skip[0] = skip;
  yb.yc[0] = ctl ? *ctl : YControl{};
  launch_y_threads<T, N, 1>(yb, 1, nfields, inverse, ctl != nullptr, tw, s, threads);
}

template <typename T, int N>
void launch_fft_y_batch(const FieldSet<T>* f, const int* const* skip, const YControl* ctl, int count, int nfields,
                        bool inverse, const vec2_t<T>* tw, cudaStream_t s, int threads) {
  if (count < 1 || count > kBatchMax || (ctl && (inverse || nfields != 1))) return;
  YBatch<T, kBatchMax> yb;
  for (int r = 0; r < count; ++r) {
    yb.f[r] = f[r];
    yb.skip[r] = skip ? skip[r] : nullptr;
    yb.yc[r] = ctl ? ctl[r] : YControl{};
  }
  launch_y_threads<T, N, kBatchMax>(yb, count, nfields, inverse, ctl != nullptr, tw, s, threads);
}

#define DGP_INST_Y(T, N) \
  template void launch_fft_y<T, N>(const FieldSet<T>&, int, bool, const vec2_t<T>*, cudaStream_t, const int*, int, \
                                   const YControl*);
#define DGP_INST_YB(N) \
  template void launch_fft_y_batch<float, N>(const FieldSet<float>*, const int* const*, const YControl*, int, int, \
                                             bool, const float2*, cudaStream_t, int);
#define DGP_INST_Y_ALL(T) DGP_INST_Y(T, 16) DGP_INST_Y(T, 32) DGP_INST_Y(T, 64) DGP_INST_Y(T, 128) \
  DGP_INST_Y(T, 256) DGP_INST_Y(T, 512) DGP_INST_Y(T, 48) DGP_INST_Y(T, 96)
DGP_INST_Y_ALL(float)
DGP_INST_Y_ALL(double)
DGP_INST_YB(16) DGP_INST_YB(32) DGP_INST_YB(48) DGP_INST_YB(64) DGP_INST_YB(96) DGP_INST_YB(128)

}  // namespace dgp
