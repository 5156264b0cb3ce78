// Pointwise and particle kernels of the DGP library.
//
// Reductions are two-stage and deterministic: each block writes FP64 partial
// sums (grid-stride loop, warp-shuffle tree), and a single block adds the
// partials in a fixed order.  No FP64 atomics.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"
#include "cic.cuh"
#include "reduce.cuh"
#include "relax_control.cuh"

namespace dgp {

int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ partials, int nblocks, int ncomp,
                                                  double* __restrict__ out, const int* __restrict__ skip) {
  if (skip && *skip) return;
  if (ncomp == 4) {  // the relaxation statistics: one pass over the partials
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double4_32a p = reinterpret_cast<const double4_32a*>(partials)[b];
      v[0] += p.x;
      v[1] += p.y;
      v[2] += p.z;
      v[3] += p.w;
    }
    block_sum<4>(v);
    if (threadIdx.x == 0)
      for (int c = 0; c < 4; ++c) out[c] = v[c];
    return;
  }
  for (int c = 0; c < ncomp; ++c) {
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v[0] += partials[(int64_t)b * ncomp + c];
    block_sum<1>(v);
    if (threadIdx.x == 0) out[c] = v[0];
    __syncthreads();
  }
}

void launch_finalize(const double* partials, int nblocks, int ncomp, double* out, cudaStream_t s,
                     const int* skip) {
  k_finalize<<<1, 256, 0, s>>>(partials, nblocks, ncomp, out, skip);
}

// Batched one-component sums: realisation r = blockIdx.y (k_sum) or blockIdx.x (finalize).
struct SumBatch {
  const float* a[kBatchMax];
  double* partials[kBatchMax];
  double* out[kBatchMax];
};
__global__ void __launch_bounds__(256) k_sum_batch(const __grid_constant__ SumBatch b, int64_t m, int absval) {
  const float* __restrict__ a = b.a[blockIdx.y];
  float s = 0.f, c = 0.f;
  auto add = [&](float v) {  // compensated (TwoSum) accumulation in the thread
    v = absval ? fabsf(v) : v;
    const float t = s + v;
    const float bb = t - s;
    c += (s - (t - bb)) + (v - bb);
    s = t;
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((m & 3) == 0 && (reinterpret_cast<uintptr_t>(a) & 15) == 0) {
    // 16-byte loads, four in flight per thread
    const float4* __restrict__ a4 = reinterpret_cast<const float4*>(a);
    const int64_t m4 = m >> 2;
    int64_t i = i0;
    for (; i + 3 * stride < m4; i += 4 * stride) {
      float4 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = a4[i + u * stride];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        add(q[u].x);
        add(q[u].y);
        add(q[u].z);
        add(q[u].w);
      }
    }
    for (; i < m4; i += stride) {
      const float4 q = a4[i];
      add(q.x);
      add(q.y);
      add(q.z);
      add(q.w);
    }
  } else {
    for (int64_t i = i0; i < m; i += stride) add(a[i]);
  }
  double v[1] = {(double)s + (double)c};
  block_sum<1>(v);
  if (threadIdx.x == 0) b.partials[blockIdx.y][blockIdx.x] = v[0];
}
__global__ void __launch_bounds__(256) k_finalize_batch(const __grid_constant__ SumBatch b, int nblocks) {
  double v[1] = {0.0};
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) v[0] += b.partials[blockIdx.x][k];
  block_sum<1>(v);
  if (threadIdx.x == 0) b.out[blockIdx.x][0] = v[0];
}
void launch_sum_batch(const float* const* a, int64_t m, bool absval, double* const* partials, int nblocks,
                      double* const* out, int count, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  SumBatch b;
  for (int r = 0; r < count; ++r) {
    b.a[r] = a[r];
    b.partials[r] = partials[r];
    b.out[r] = out[r];
  }
  // about nblocks CTAs in all, shared among the realisations
  const int nb = nblocks / count > 0 ? nblocks / count : 1;
  k_sum_batch<<<dim3((unsigned)nb, (unsigned)count), 256, 0, s>>>(b, m, absval ? 1 : 0);
  k_finalize_batch<<<count, 256, 0, s>>>(b, nb);
}

struct FillBatch {
  float* a[kBatchMax];
};
__global__ void k_fill_batch(const __grid_constant__ FillBatch b, int64_t m) {
  float* __restrict__ a = b.a[blockIdx.y];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 0.f;
}
void launch_zero_batch(float* const* a, int64_t m, int count, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  FillBatch b;
  for (int r = 0; r < count; ++r) b.a[r] = a[r];
  k_fill_batch<<<dim3((unsigned)(num_sms() * 4 / count + 1), (unsigned)count), 256, 0, s>>>(b, m);
}

struct ControlBatch {
  YControl c[kBatchMax];
  const int* skip[kBatchMax];
};
__global__ void __launch_bounds__(256) k_control_batch(const __grid_constant__ ControlBatch b) {
  const YControl& yc = b.c[blockIdx.x];
  const int* skip = b.skip[blockIdx.x];
  if (skip && *skip) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < yc.nblocks; k += blockDim.x) {
    const double* pk = yc.partials + 4 * (int64_t)k;
    v[0] += pk[0];
    v[1] += pk[1];
    v[2] += pk[2];
    v[3] += pk[3];
  }
  block_sum<4>(v);
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; ++c) yc.stats[c] = v[c];
    relax_control_step(yc.ctl, yc.stats, yc.abs_src_sum, yc.hist, yc.max_iter, yc.patience, yc.tol, yc.inv_m);
  }
}
void launch_control_batch(const YControl* ctl, const int* const* skip, int count, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  ControlBatch b;
  for (int r = 0; r < count; ++r) {
    b.c[r] = ctl[r];
    b.skip[r] = skip ? skip[r] : nullptr;
  }
  k_control_batch<<<count, 256, 0, s>>>(b);
}

// The stop rules as a launch of their own (relax_control.cuh).
__global__ void k_relax_control(SolveCtl* __restrict__ c, const double* __restrict__ stats,
                                const double* __restrict__ abs_src_sum, double* __restrict__ hist,
                                int max_iter, int patience, double tol, double inv_m) {
  if (threadIdx.x != 0) return;
  relax_control_step(c, stats, abs_src_sum, hist, max_iter, patience, tol, inv_m);
}

void launch_relax_control(SolveCtl* ctl, const double* stats, const double* abs_src_sum, double* hist,
                          int max_iter, int patience, double tol, double inv_m, cudaStream_t s) {
  k_relax_control<<<1, 32, 0, s>>>(ctl, stats, abs_src_sum, hist, max_iter, patience, tol, inv_m);
}

__global__ void __launch_bounds__(256)
    k_finalize_control(const double* __restrict__ partials, int nblocks, double* __restrict__ stats,
                       SolveCtl* __restrict__ c, const double* __restrict__ abs_src_sum, double* __restrict__ hist,
                       int max_iter, int patience, double tol, double inv_m, const int* __restrict__ skip) {
  if (skip && *skip) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double4_32a p = reinterpret_cast<const double4_32a*>(partials)[b];
    v[0] += p.x;
    v[1] += p.y;
    v[2] += p.z;
    v[3] += p.w;
  }
  block_sum<4>(v);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) stats[k] = v[k];
    relax_control_step(c, stats, abs_src_sum, hist, max_iter, patience, tol, inv_m);
  }
}

void launch_finalize_control(const double* partials, int nblocks, double* stats, SolveCtl* ctl,
                             const double* abs_src_sum, double* hist, int max_iter, int patience, double tol,
                             double inv_m, cudaStream_t s, const int* skip) {
  k_finalize_control<<<1, 256, 0, s>>>(partials, nblocks, stats, ctl, abs_src_sum, hist, max_iter, patience, tol,
                                       inv_m, skip);
}

// Per-thread sums of FP32 data run on the FP32 pipe as an unevaluated pair:
// Knuth's TwoSum keeps every rounding error of the running sum s in c, so
// s + c is the thread's sum to about 2^-44 relative; the cross-thread and
// cross-block stages are FP64.  (Per-element FP64 conversion and addition
// would make the pass FP64-pipe bound on GB300.)
template <typename T>
__global__ void __launch_bounds__(256) k_sum(const T* __restrict__ a, int64_t m, int absval,
                                             double* __restrict__ partials) {
  double acc = 0.0;
  if constexpr (sizeof(T) == 4) {
    float s = 0.f, c = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
      const float v = absval ? fabsf(a[i]) : a[i];
      const float t = s + v;
      const float bb = t - s;
      c += (s - (t - bb)) + (v - bb);
      s = t;
    }
    acc = (double)s + (double)c;
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double v = (double)a[i];
      acc += absval ? fabs(v) : v;
    }
  }
  double v[1] = {acc};
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

template <typename T>
void launch_sum(const T* a, int64_t m, bool absval, double* partials, int nblocks, cudaStream_t s) {
  k_sum<T><<<nblocks, 256, 0, s>>>(a, m, absval ? 1 : 0, partials);
}

template <typename T>
__global__ void __launch_bounds__(256) k_product3(const T* __restrict__ a, const T* __restrict__ b,
                                                  const T* __restrict__ c, int64_t m, double* __restrict__ partials) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)a[i] * (double)b[i];
    if (c) v *= (double)c[i];
    acc += v;
  }
  double v[1] = {acc};
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

template <typename T>
void launch_product3_sum(const T* a, const T* b, const T* c, int64_t m, double* partials, int nblocks,
                         cudaStream_t s) {
  k_product3<T><<<nblocks, 256, 0, s>>>(a, b, c, m, partials);
}

// delta = rho / mean - 1; FP32 data use 1 / mean as a float pair (hi + lo),
// formed once per block, so the per-element work stays on the FP32 pipe.
template <typename T>
__global__ void k_density_contrast(const T* __restrict__ rho, T* __restrict__ delta, int64_t m,
                                   const double* __restrict__ sum) {
  if constexpr (sizeof(T) == 4) {
    __shared__ float s_inv[2];
    if (threadIdx.x == 0) {
      const double inv = (double)m / sum[0];
      s_inv[0] = (float)inv;
      s_inv[1] = (float)(inv - (double)s_inv[0]);
    }
    __syncthreads();
    const float hi = s_inv[0], lo = s_inv[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
      delta[i] = fmaf(rho[i], hi, fmaf(rho[i], lo, -1.f));
  } else {
    const double inv_mean = (double)m / sum[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
      delta[i] = (T)((double)rho[i] * inv_mean - 1.0);
  }
}

template <typename T>
void launch_density_contrast(const T* rho, T* delta, int64_t m, const double* sum, cudaStream_t s) {
  k_density_contrast<T><<<num_sms() * 4, 256, 0, s>>>(rho, delta, m, sum);
}

template <typename T>
__global__ void k_fill(T* __restrict__ a, int64_t m, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

template <typename T>
void launch_fill(T* a, int64_t m, T v, cudaStream_t s) {
  k_fill<T><<<num_sms() * 4, 256, 0, s>>>(a, m, v);
}

template <typename T>
__global__ void k_sub_mean(const T* __restrict__ in, T* __restrict__ out, int64_t m, const double* __restrict__ sum) {
  if constexpr (sizeof(T) == 4) {
    __shared__ float s_mean[2];
    if (threadIdx.x == 0) {
      const double mean = sum[0] / (double)m;
      s_mean[0] = (float)mean;
      s_mean[1] = (float)(mean - (double)s_mean[0]);
    }
    __syncthreads();
    const float hi = s_mean[0], lo = s_mean[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
      out[i] = (in[i] - hi) - lo;
  } else {
    const double mean = sum[0] / (double)m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
      out[i] = (T)((double)in[i] - mean);
  }
}

template <typename T>
void launch_sub_mean(const T* in, T* out, int64_t m, const double* sum, cudaStream_t s) {
  k_sub_mean<T><<<num_sms() * 4, 256, 0, s>>>(in, out, m, sum);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sph_update(const T* __restrict__ S, T* __restrict__ D, int64_t m, T alpha,
                                                    T alpha2, double* __restrict__ partials) {
  const T eight_thirds = (T)8 / (T)3, bad_d = (T)-0.75 * alpha;
  double nbad = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const T s = S[i];
    const T disc = alpha2 + eight_thirds * s;
    if (disc < (T)0) {
      D[i] = bad_d;
      nbad += 1.0;
    } else {
      D[i] = (T)2 * s / (alpha + sqrt(disc));
    }
  }
  double v[1] = {nbad};
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

template <typename T>
void launch_sph_update(const T* S, T* D, int64_t m, double alpha, double* partials, int nblocks, cudaStream_t s) {
  k_sph_update<T><<<nblocks, 256, 0, s>>>(S, D, m, (T)alpha, (T)(alpha * alpha), partials);
}

// ---- adjoint relaxation (see kernels.cuh)
template <typename T>
__device__ __forceinline__ T block_mean_d(const double* dsum, int64_t m) {
  __shared__ T s_mean;
  if (threadIdx.x == 0) s_mean = (T)(dsum[0] / (double)m);
  __syncthreads();
  return s_mean;
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_products(const T* __restrict__ lam, const T* __restrict__ D,
                                                      const double* __restrict__ dsum, const T* __restrict__ hxx,
                                                      const T* __restrict__ hyy, const T* __restrict__ hxy,
                                                      const T* __restrict__ hxz, const T* __restrict__ hyz,
                                                      T* __restrict__ P, int64_t m) {
  const T mean = block_mean_d<T>(dsum, m);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const T l = lam[i], a = hxx[i], b = hyy[i];
    P[i] = a * l;
    P[m + i] = b * l;
    P[2 * m + i] = ((D[i] - mean) - a - b) * l;
    P[3 * m + i] = hxy[i] * l;
    P[4 * m + i] = hxz[i] * l;
    P[5 * m + i] = hyz[i] * l;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_update_a(const T* __restrict__ lam, const T* __restrict__ D,
                                                      const double* __restrict__ dsum, const T* __restrict__ g,
                                                      const T* __restrict__ Q, T* __restrict__ u, int64_t m,
                                                      T alpha, T w, double* __restrict__ partials) {
  const T mean = block_mean_d<T>(dsum, m);
  double su = 0.0, sr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const T d = D[i] - mean, l = lam[i];
    const T diag = (T)2 * ((T)1 - w) * d + alpha;
    const T ui = (g[i] - (T)2 * w * d * l - Q[i]) / diag;
    u[i] = ui;
    su += (double)ui;
    sr += (double)(diag * (l - ui));
  }
  double v[2] = {su, sr};
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = v[0];
    partials[2 * blockIdx.x + 1] = v[1];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_update_b(T* __restrict__ lam, const T* __restrict__ D,
                                                      const double* __restrict__ dsum, const T* __restrict__ u,
                                                      int64_t m, T alpha, T w, const double* __restrict__ sums,
                                                      double* __restrict__ partials) {
  const T mean = block_mean_d<T>(dsum, m);
  const T c = (T)(-(sums[0] / (double)m) / (sums[2] / (double)m));
  const T rmean = (T)(sums[1] / (double)m);
  double sa = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const T d = D[i] - mean;
    const T diag = (T)2 * ((T)1 - w) * d + alpha;
    const T ui = u[i];
    sa += (double)fabs(diag * (lam[i] - ui) - rmean);
    lam[i] = ui + c / diag;
  }
  double v[1] = {sa};
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_inv_diag(const T* __restrict__ D, const double* __restrict__ dsum,
                                                      int64_t m, T alpha, T w, double* __restrict__ partials) {
  const T mean = block_mean_d<T>(dsum, m);
  double s = 0.0, nbad = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const T diag = (T)2 * ((T)1 - w) * (D[i] - mean) + alpha;
    if (diag > (T)0) s += 1.0 / (double)diag;
    else nbad += 1.0;
  }
  double v[2] = {s, nbad};
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = v[0];
    partials[2 * blockIdx.x + 1] = v[1];
  }
}

template <typename T>
__global__ void k_axpy(const T* __restrict__ x, const T* __restrict__ y, T* __restrict__ out, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x[i] + y[i];
}

template <typename T>
void launch_adj_products(const T* lam, const T* D, const double* dsum, T* const* H5, T* P, int64_t m,
                         cudaStream_t s) {
  k_adj_products<T><<<num_sms() * 4, 256, 0, s>>>(lam, D, dsum, H5[0], H5[1], H5[2], H5[3], H5[4], P, m);
}
template <typename T>
void launch_adj_update_a(const T* lam, const T* D, const double* dsum, const T* g, const T* Q, T* u, int64_t m,
                         double alpha, double w, double* partials, int nblocks, cudaStream_t s) {
  k_adj_update_a<T><<<nblocks, 256, 0, s>>>(lam, D, dsum, g, Q, u, m, (T)alpha, (T)w, partials);
}
template <typename T>
void launch_adj_update_b(T* lam, const T* D, const double* dsum, const T* u, int64_t m, double alpha, double w,
                         const double* sums, double* partials, int nblocks, cudaStream_t s) {
  k_adj_update_b<T><<<nblocks, 256, 0, s>>>(lam, D, dsum, u, m, (T)alpha, (T)w, sums, partials);
}
template <typename T>
void launch_adj_inv_diag(const T* D, const double* dsum, int64_t m, double alpha, double w, double* partials,
                         int nblocks, cudaStream_t s) {
  k_adj_inv_diag<T><<<nblocks, 256, 0, s>>>(D, dsum, m, (T)alpha, (T)w, partials);
}
template <typename T>
void launch_axpy(const T* x, const T* y, T* out, int64_t m, cudaStream_t s) {
  k_axpy<T><<<num_sms() * 4, 256, 0, s>>>(x, y, out, m);
}

#define DGP_INST_PW(T)                                                                         \
  template void launch_adj_products<T>(const T*, const T*, const double*, T* const*, T*, int64_t, cudaStream_t); \
  template void launch_adj_update_a<T>(const T*, const T*, const double*, const T*, const T*, T*, int64_t,     \
                                       double, double, double*, int, cudaStream_t);                           \
  template void launch_adj_update_b<T>(T*, const T*, const double*, const T*, int64_t, double, double,         \
                                       const double*, double*, int, cudaStream_t);                            \
  template void launch_adj_inv_diag<T>(const T*, const double*, int64_t, double, double, double*, int,         \
                                       cudaStream_t);                                                          \
  template void launch_axpy<T>(const T*, const T*, T*, int64_t, cudaStream_t);                                 \
  template void launch_sph_update<T>(const T*, T*, int64_t, double, double*, int, cudaStream_t); \
  template void launch_sum<T>(const T*, int64_t, bool, double*, int, cudaStream_t);            \
  template void launch_product3_sum<T>(const T*, const T*, const T*, int64_t, double*, int,    \
                                       cudaStream_t);                                          \
  template void launch_density_contrast<T>(const T*, T*, int64_t, const double*, cudaStream_t); \
  template void launch_fill<T>(T*, int64_t, T, cudaStream_t);                                  \
  template void launch_sub_mean<T>(const T*, T*, int64_t, const double*, cudaStream_t);
DGP_INST_PW(float)
DGP_INST_PW(double)

// --------------------------------------------------------------------------
// CIC (Eq. CIC): grid point i at x = i d; lower index floor(x/d), weights
// (1 - f, f) per axis, periodic.  In FP32 x/d is formed as an exact product
// with N/box held as an unevaluated pair (hi + lo), so the fractional offset
// carries no more error than the position itself.
template <typename T>
__device__ __forceinline__ T wrap_periodic(T v, T box, T inv_box) {
  v -= box * floor(v * inv_box);
  if (v >= box) v -= box;
  if (v < (T)0) v = (T)0;
  return v;
}

// Force interpolation with the deposit's window (Sec. III.A), kick, optional drift.
// One particle of the gather-kick-drift: the mesh force at the particle with the CIC
// window (8 corners, 3 components), p += kick g, then x += drift p (wrapped) if asked.
template <typename T>
struct GatherOne {
  int64_t r00, r01, r10, r11;
  int iz0, iz1;
  T w[8];
  __device__ __forceinline__ void locate(T xp, T yp, T zp, const CicParams& cp) {
    const int64_t n = cp.n;
    int ix0, ix1, iy0, iy1;
    T fx, fy, fz;
    cic_axis(xp, cp, ix0, ix1, fx);
    cic_axis(yp, cp, iy0, iy1, fy);
    cic_axis(zp, cp, iz0, iz1, fz);
    const T hx = (T)1 - fx, hy = (T)1 - fy, hz = (T)1 - fz;
    r00 = (ix0 * n + iy0) * n;
    r01 = (ix0 * n + iy1) * n;
    r10 = (ix1 * n + iy0) * n;
    r11 = (ix1 * n + iy1) * n;
    w[0] = hx * hy * hz; w[1] = hx * hy * fz; w[2] = hx * fy * hz; w[3] = hx * fy * fz;
    w[4] = fx * hy * hz; w[5] = fx * hy * fz; w[6] = fx * fy * hz; w[7] = fx * fy * fz;
  }
  __device__ __forceinline__ T at(const T* __restrict__ G) const {
    return w[0] * G[r00 + iz0] + w[1] * G[r00 + iz1] + w[2] * G[r01 + iz0] + w[3] * G[r01 + iz1] +
           w[4] * G[r10 + iz0] + w[5] * G[r10 + iz1] + w[6] * G[r11 + iz0] + w[7] * G[r11 + iz1];
  }
};

// Two particles per iteration (p and p + stride): their 48 mesh loads are independent, which
// doubles the loads in flight of this latency-bound gather.
template <typename T>
__device__ __forceinline__ void gather_kick_body(T* __restrict__ x, T* __restrict__ y, T* __restrict__ z,
                                                 T* __restrict__ px, T* __restrict__ py, T* __restrict__ pz,
                                                 int64_t np, const T* __restrict__ gx, const T* __restrict__ gy,
                                                 const T* __restrict__ gz, const CicParams& cp, T kick, T drift,
                                                 int do_drift, int64_t blk, int64_t nblk) {
  T box, inv_box;
  if constexpr (sizeof(T) == 8) {
    box = cp.box;
    inv_box = 1.0 / cp.box;
  } else {
    box = cp.box_f;
    inv_box = cp.inv_box_f;
  }
  const int64_t stride = nblk * blockDim.x;
  for (int64_t p = blk * blockDim.x + threadIdx.x; p < np; p += 2 * stride) {
    const int64_t q = p + stride;
    const bool two = q < np;
    const T xp = x[p], yp = y[p], zp = z[p];
    const T xq = two ? x[q] : xp, yq = two ? y[q] : yp, zq = two ? z[q] : zp;
    GatherOne<T> A, B;
    A.locate(xp, yp, zp, cp);
    B.locate(xq, yq, zq, cp);
    const T ga0 = A.at(gx), ga1 = A.at(gy), ga2 = A.at(gz);
    const T gb0 = B.at(gx), gb1 = B.at(gy), gb2 = B.at(gz);
    {
      const T qx = px[p] + kick * ga0, qy = py[p] + kick * ga1, qz = pz[p] + kick * ga2;
      px[p] = qx;
      py[p] = qy;
      pz[p] = qz;
      if (do_drift) {
        x[p] = wrap_periodic(xp + drift * qx, box, inv_box);
        y[p] = wrap_periodic(yp + drift * qy, box, inv_box);
        z[p] = wrap_periodic(zp + drift * qz, box, inv_box);
      }
    }
    if (two) {
      const T qx = px[q] + kick * gb0, qy = py[q] + kick * gb1, qz = pz[q] + kick * gb2;
      px[q] = qx;
      py[q] = qy;
      pz[q] = qz;
      if (do_drift) {
        x[q] = wrap_periodic(xq + drift * qx, box, inv_box);
        y[q] = wrap_periodic(yq + drift * qy, box, inv_box);
        z[q] = wrap_periodic(zq + drift * qz, box, inv_box);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gather_kick(T* __restrict__ x, T* __restrict__ y, T* __restrict__ z,
                                                     T* __restrict__ px, T* __restrict__ py, T* __restrict__ pz,
                                                     int64_t np, const T* __restrict__ gx, const T* __restrict__ gy,
                                                     const T* __restrict__ gz, CicParams cp, T kick, T drift,
                                                     int do_drift) {
  gather_kick_body<T>(x, y, z, px, py, pz, np, gx, gy, gz, cp, kick, drift, do_drift, blockIdx.x, gridDim.x);
}

template <typename T>
void launch_gather_kick(T* x, T* y, T* z, T* px, T* py, T* pz, int64_t np, const T* gx, const T* gy,
                        const T* gz, CicParams cp, double kick, double drift, int do_drift, cudaStream_t s) {
  if (np <= 0) return;
  int64_t blocks = (np + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_gather_kick<T><<<(unsigned)blocks, 256, 0, s>>>(x, y, z, px, py, pz, np, gx, gy, gz, cp, (T)kick, (T)drift,
                                                    do_drift);
}

// Batched: realisation r = blockIdx.y
struct GatherBatch {
  GatherArgs a[kBatchMax];
};
__global__ void __launch_bounds__(256) k_gather_kick_batch(const __grid_constant__ GatherBatch b) {
  const GatherArgs& a = b.a[blockIdx.y];
  gather_kick_body<float>(a.p[0], a.p[1], a.p[2], a.p[3], a.p[4], a.p[5], a.np, a.g[0], a.g[1], a.g[2], a.cp,
                          a.kick, a.drift, a.do_drift, blockIdx.x, gridDim.x);
}
void launch_gather_kick_batch(const GatherArgs* a, int count, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  GatherBatch b;
  int64_t npmax = 0;
  for (int r = 0; r < count; ++r) {
    b.a[r] = a[r];
    npmax = a[r].np > npmax ? a[r].np : npmax;
  }
  if (npmax <= 0) return;
  int64_t blocks = (npmax + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16 / count + 1;
  if (blocks > cap) blocks = cap;
  k_gather_kick_batch<<<dim3((unsigned)blocks, (unsigned)count), 256, 0, s>>>(b);
}

template <typename T>
__global__ void k_zel_particles(const T* __restrict__ p0, const T* __restrict__ p1, const T* __restrict__ p2, T vf,
                                CicParams cp, T* __restrict__ x, T* __restrict__ y, T* __restrict__ z,
                                T* __restrict__ px, T* __restrict__ py, T* __restrict__ pz) {
  const int64_t n = cp.n, m = n * n * n;
  T box, inv_box;
  if constexpr (sizeof(T) == 8) {
    box = cp.box;
    inv_box = 1.0 / cp.box;
  } else {
    box = cp.box_f;
    inv_box = cp.inv_box_f;
  }
  const T d = box / (T)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = i / (n * n), iy = (i / n) % n, iz = i % n;
    x[i] = wrap_periodic((T)ix * d + p0[i], box, inv_box);
    y[i] = wrap_periodic((T)iy * d + p1[i], box, inv_box);
    z[i] = wrap_periodic((T)iz * d + p2[i], box, inv_box);
    px[i] = vf * p0[i];
    py[i] = vf * p1[i];
    pz[i] = vf * p2[i];
  }
}

template <typename T>
__global__ void k_zel_cot(const T* __restrict__ xb, const T* __restrict__ yb, const T* __restrict__ zb,
                          const T* __restrict__ pxb, const T* __restrict__ pyb, const T* __restrict__ pzb, T vf,
                          int64_t m, T* __restrict__ o0, T* __restrict__ o1, T* __restrict__ o2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    o0[i] = xb[i] + vf * pxb[i];
    o1[i] = yb[i] + vf * pyb[i];
    o2[i] = zb[i] + vf * pzb[i];
  }
}

template <typename T>
void launch_zel_particles(T* const* psi, double vf, CicParams cp, T* const* out, cudaStream_t s) {
  k_zel_particles<T><<<num_sms() * 4, 256, 0, s>>>(psi[0], psi[1], psi[2], (T)vf, cp, out[0], out[1], out[2],
                                                   out[3], out[4], out[5]);
}
template <typename T>
void launch_zel_cot(T* const* cot, double vf, int64_t m, T* const* psibar, cudaStream_t s) {
  k_zel_cot<T><<<num_sms() * 4, 256, 0, s>>>(cot[0], cot[1], cot[2], cot[3], cot[4], cot[5], (T)vf, m, psibar[0],
                                             psibar[1], psibar[2]);
}

#define DGP_INST_P(T)                                                                              \
  template void launch_zel_particles<T>(T* const*, double, CicParams, T* const*, cudaStream_t);     \
  template void launch_zel_cot<T>(T* const*, double, int64_t, T* const*, cudaStream_t);            \
  template void launch_gather_kick<T>(T*, T*, T*, T*, T*, T*, int64_t, const T*, const T*, const T*,  \
                                      CicParams, double, double, int, cudaStream_t);
DGP_INST_P(float)
DGP_INST_P(double)

}  // namespace dgp
