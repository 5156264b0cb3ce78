// Launchers of the derivative in the crossover scale r_c H0 (gradients of a
// loss through the solve's coefficients, E(a) and the step's time factors).
#pragma once
#include "kernels.cuh"

namespace dgp {

// Derivatives in r_c H0 of the scalars of the field equations (Sec. II):
// E, eta, alpha, beta, s, c2, c3.
constexpr int XOP_RC = 12;  // x-pass operation id (after those of kernels.cuh)

struct RcDeriv {
  double dE_over_E, deta, dalpha, dbeta, ds, dc2, dc3;
};

// x pass op (one block partial per CTA into partials[blockIdx.y * gridDim.x + blockIdx.x]):
//   in_mask bits 0-3 (phibar, gbar_x, gbar_y, gbar_z; the phase of phibar):
//     sum_k w(k) Re[conj(phibar_tot) (A'(k) delta(k) + B'(k) D(k))]
//   in_mask bit 6 (lam; the phase of lam):
//     sum_k w(k) Re[conj(lam) (S'(k) delta(k) - (alpha' + c2' N(k) + c2 N'(k)) D(k))]
// with delta = in.p[4], D = in.p[5], lam = in.p[6]; phibar_tot = phibar + sum_i i k_i gbar_i
// (Nyquist component zero); w = 1 on the kz = 0 and Nyquist planes, else 2.  Multiply the
// total by 1 / N^3 to get the real-space inner products.  ' = d/d(r_c H0).
template <typename T, int N>
void launch_fft_x_rc(const FieldSet<T>& in, int in_mask, const KParams& kp, const RcDeriv& d, double* partials,
                     const vec2_t<T>* tw, cudaStream_t s);

// launch_force_vjp_gather plus, when fdot_partials is set, per-block FP64 partials of
// sum_p F(x_p) . pp.p[3..5][p] (the forces interpolated from G, the unscaled cotangent);
// returns the number of blocks written.
template <typename T>
int launch_force_vjp_gather_dot(const ParticleSet<T>& pp, double scale, int64_t np, T* const* G, const T* rbar,
                                double rscale, const ParticleSet<T>& xb, CicParams cp, double* fdot_partials,
                                cudaStream_t s);

// Per-block FP64 partials of sum_{c < 3} sum_i a[c][i] b[c][i]; returns the number of blocks.
template <typename T>
int launch_dot3(T* const* a, T* const* b, int64_t m, double* partials, cudaStream_t s);

}  // namespace dgp
