// Particle side of the step adjoint (pm_step_adjoint in include/dgp.h).
//
// CIC (Eq. CIC) is piecewise linear in the positions: for the corner c of a
// particle the weight is W = w_x w_y w_z with w = 1 - f (lower corner) or f
// (upper corner) per axis, and dW/dx_a = (-1 or +1) / d times the other two
// factors.  With the forces interpolated as F_p = sum_c W G(c) and the density
// rho(c) = sum_p W, a cotangent fbar_p of F_p gives
//   Gbar_i(c) = sum_p W fbar_i,p                      (k_deposit_vec)
//   xbar_p   += sum_c grad W (G(c) . fbar_p + s rbar(c))  (k_force_vjp_gather)
// where rbar is the cotangent of the density contrast and s = N^3 / Np its
// derivative in rho (the particle count is conserved, so the mean is fixed).
// The same gather can also sum F_p . fbar_p (the kick factors' derivatives in
// r_c H0 multiply it).
#include "adjoint_rc.cuh"
#include "cic.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace dgp {

template <typename T>
__global__ void __launch_bounds__(256) k_deposit_vec(const __grid_constant__ ParticleSet<T> pp, T scale, int64_t np,
                                                     T* __restrict__ gx, T* __restrict__ gy, T* __restrict__ gz,
                                                     CicParams cp) {
  const int64_t n = cp.n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    int i0[3], i1[3];
    T f[3];
    cic_axis(pp.p[0][p], cp, i0[0], i1[0], f[0]);
    cic_axis(pp.p[1][p], cp, i0[1], i1[1], f[1]);
    cic_axis(pp.p[2][p], cp, i0[2], i1[2], f[2]);
    const T v[3] = {scale * pp.p[3][p], scale * pp.p[4][p], scale * pp.p[5][p]};
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int dx = t >> 2, dy = (t >> 1) & 1, dz = t & 1;
      const T wgt = (dx ? f[0] : (T)1 - f[0]) * (dy ? f[1] : (T)1 - f[1]) * (dz ? f[2] : (T)1 - f[2]);
      const int64_t idx = ((int64_t)(dx ? i1[0] : i0[0]) * n + (dy ? i1[1] : i0[1])) * n + (dz ? i1[2] : i0[2]);
      atomicAdd(gx + idx, wgt * v[0]);
      atomicAdd(gy + idx, wgt * v[1]);
      atomicAdd(gz + idx, wgt * v[2]);
    }
  }
}

// pp.p[0..2]: positions; pp.p[3..5]: the cotangent fbar / scale; xb: accumulated position cotangents.
template <typename T>
__global__ void __launch_bounds__(256) k_force_vjp_gather(const __grid_constant__ ParticleSet<T> pp, T scale,
                                                          int64_t np, const T* __restrict__ G0,
                                                          const T* __restrict__ G1, const T* __restrict__ G2,
                                                          const T* __restrict__ rbar, T rscale,
                                                          const __grid_constant__ ParticleSet<T> xb, CicParams cp,
                                                          double* __restrict__ fdot) {
  const int64_t n = cp.n;
  T inv_d;
  if constexpr (sizeof(T) == 8) inv_d = cp.inv_d;
  else inv_d = cp.inv_d_hi;
  double dot = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    int i0[3], i1[3];
    T f[3];
    cic_axis(pp.p[0][p], cp, i0[0], i1[0], f[0]);
    cic_axis(pp.p[1][p], cp, i0[1], i1[1], f[1]);
    cic_axis(pp.p[2][p], cp, i0[2], i1[2], f[2]);
    const T raw[3] = {pp.p[3][p], pp.p[4][p], pp.p[5][p]};
    const T fb[3] = {scale * raw[0], scale * raw[1], scale * raw[2]};
    T acc[3] = {(T)0, (T)0, (T)0}, F[3] = {(T)0, (T)0, (T)0};
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int dx = t >> 2, dy = (t >> 1) & 1, dz = t & 1;
      const T wx = dx ? f[0] : (T)1 - f[0], wy = dy ? f[1] : (T)1 - f[1], wz = dz ? f[2] : (T)1 - f[2];
      const T sx = dx ? inv_d : -inv_d, sy = dy ? inv_d : -inv_d, sz = dz ? inv_d : -inv_d;
      const int64_t idx = ((int64_t)(dx ? i1[0] : i0[0]) * n + (dy ? i1[1] : i0[1])) * n + (dz ? i1[2] : i0[2]);
      const T v = G0[idx] * fb[0] + G1[idx] * fb[1] + G2[idx] * fb[2] + rscale * rbar[idx];
      acc[0] += sx * wy * wz * v;
      acc[1] += wx * sy * wz * v;
      acc[2] += wx * wy * sz * v;
      if (fdot) {
        const T wgt = wx * wy * wz;
        F[0] += wgt * G0[idx];
        F[1] += wgt * G1[idx];
        F[2] += wgt * G2[idx];
      }
    }
    xb.p[0][p] += acc[0];
    xb.p[1][p] += acc[1];
    xb.p[2][p] += acc[2];
    dot += (double)F[0] * raw[0] + (double)F[1] * raw[1] + (double)F[2] * raw[2];
  }
  if (fdot) {  // uniform over the grid
    double v[1] = {dot};
    block_sum<1>(v);
    if (threadIdx.x == 0) fdot[blockIdx.x] = v[0];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_dot3(const T* __restrict__ a0, const T* __restrict__ a1,
                                              const T* __restrict__ a2, const T* __restrict__ b0,
                                              const T* __restrict__ b1, const T* __restrict__ b2, int64_t m,
                                              double* __restrict__ partials) {
  double t = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    t += (double)a0[i] * b0[i] + (double)a1[i] * b1[i] + (double)a2[i] * b2[i];
  double v[1] = {t};
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

// out[c][p] += a * in[c][p] for c = 0..2 (pbar += Dr xbar in the step adjoint)
template <typename T>
__global__ void k_particle_axpy(const __grid_constant__ ParticleSet<T> in, T a, int64_t np,
                                const __grid_constant__ ParticleSet<T> out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) out.p[c][p] += a * in.p[c][p];
  }
}

static int64_t pblocks(int64_t np) {
  int64_t b = (np + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  return b > cap ? cap : (b < 1 ? 1 : b);
}

template <typename T>
void launch_deposit_vec(const ParticleSet<T>& pp, double scale, int64_t np, T* const* g, CicParams cp,
                        cudaStream_t s) {
  if (np <= 0) return;
  k_deposit_vec<T><<<(unsigned)pblocks(np), 256, 0, s>>>(pp, (T)scale, np, g[0], g[1], g[2], cp);
}
template <typename T>
void launch_force_vjp_gather(const ParticleSet<T>& pp, double scale, int64_t np, T* const* G, const T* rbar,
                             double rscale, const ParticleSet<T>& xb, CicParams cp, cudaStream_t s) {
  if (np <= 0) return;
  k_force_vjp_gather<T><<<(unsigned)pblocks(np), 256, 0, s>>>(pp, (T)scale, np, G[0], G[1], G[2], rbar, (T)rscale,
                                                              xb, cp, nullptr);
}
template <typename T>
int launch_force_vjp_gather_dot(const ParticleSet<T>& pp, double scale, int64_t np, T* const* G, const T* rbar,
                                double rscale, const ParticleSet<T>& xb, CicParams cp, double* fdot_partials,
                                cudaStream_t s) {
  const int nb = (int)pblocks(np);
  k_force_vjp_gather<T><<<(unsigned)nb, 256, 0, s>>>(pp, (T)scale, np, G[0], G[1], G[2], rbar, (T)rscale, xb, cp,
                                                     fdot_partials);
  return nb;
}
template <typename T>
int launch_dot3(T* const* a, T* const* b, int64_t m, double* partials, cudaStream_t s) {
  const int nb = (int)pblocks(m);
  k_dot3<T><<<(unsigned)nb, 256, 0, s>>>(a[0], a[1], a[2], b[0], b[1], b[2], m, partials);
  return nb;
}
template <typename T>
void launch_particle_axpy(const ParticleSet<T>& in, double a, int64_t np, const ParticleSet<T>& out,
                          cudaStream_t s) {
  if (np <= 0) return;
  k_particle_axpy<T><<<(unsigned)pblocks(np), 256, 0, s>>>(in, (T)a, np, out);
}

#define DGP_INST_PA(T)                                                                                      \
  template void launch_deposit_vec<T>(const ParticleSet<T>&, double, int64_t, T* const*, CicParams,          \
                                      cudaStream_t);                                                        \
  template void launch_force_vjp_gather<T>(const ParticleSet<T>&, double, int64_t, T* const*, const T*,       \
                                           double, const ParticleSet<T>&, CicParams, cudaStream_t);          \
  template void launch_particle_axpy<T>(const ParticleSet<T>&, double, int64_t, const ParticleSet<T>&,        \
                                        cudaStream_t);                                                      \
  template int launch_force_vjp_gather_dot<T>(const ParticleSet<T>&, double, int64_t, T* const*, const T*,    \
                                              double, const ParticleSet<T>&, CicParams, double*, cudaStream_t); \
  template int launch_dot3<T>(T* const*, T* const*, int64_t, double*, cudaStream_t);
DGP_INST_PA(float)
DGP_INST_PA(double)

}  // namespace dgp
