// Launchers of the DGP mesh and particle kernels (definitions in the .cu files,
// explicit instantiations for T in {float, double} and N in {16..512}).
//
// Spectral layout.  A real field f[x][y][z] (z fastest) is transformed along z
// first (real-to-complex, kz = 0..N/2) and stored TRANSPOSED as
// S[kz][x][y] (y fastest), (N/2+1) * N * N complex values; the y transform
// acts in place on contiguous rows, and the x transform (stride N) is always
// fused with a k-space operation and its inverse, so the fully transformed
// spectrum never touches memory.  The Nyquist plane kz = N/2 is simply the
// last plane.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace dgp {

constexpr int kMaxFields = 8;
// Batched launches: one launch runs a stage for up to kBatchMax realisations of
// the same mesh size, realisation r on blockIdx.z = r with its own arguments.
constexpr int kBatchMax = 16;

template <typename T> struct FieldSet {
  vec2_t<T>* p[kMaxFields];
};

// Prologue applied to real values before the z transform.
struct ZPrologue {
  const double* mean_src;  // device scalar: sum of the source field (nullptr: identity)
  double inv_count;        // 1 / number of points
  int kind;                // 0: identity; 1: rho -> rho / mean - 1; 2: v - mean
};

// Parameters of the fused x-pass k-space operations.
struct KParams {
  double box;        // Mpc/h
  double inv_m;      // 1 / N^3 (inverse-transform normalisation)
  double kbar_fac;   // C_H / (a E): kbar = kbar_fac |k|
  int local_only;
  // coefficients (Sec. II)
  double eta, alpha, beta, s, c2, c3, aE, q, rc_H0, a;
  int gravity;
  // the per-mode constants rounded once (FP32 paths read these, never the doubles)
  float kf_f, kbkf_f, inv_m_f;   // 2 pi / box, kbar_fac * 2 pi / box, 1 / N^3
  float s_f, beta_f, alpha_f, c2_f, c3_f, inv_eta_f, half_inv_eta_f, om15_f, aE2_f;
};

enum XOp { XOP_HESSIAN = 0, XOP_SOURCE = 1, XOP_SOURCE_LIN = 2, XOP_PHI_FORCE = 3, XOP_PK = 4,
           XOP_SHELL = 5, XOP_PK_BRANE = 6, XOP_ADJ_PHI = 7, XOP_ADJ_COMBINE = 8, XOP_ZEL = 9, XOP_ZEL_ADJ = 10,
           XOP_PK_ADJ = 11 };
// XOP_ZEL: the Zel'dovich displacements Psi_j = (i k_j / k^2) delta_L (Nyquist component of
//   k_j zero), three outputs.  XOP_PK_ADJ: out0 = 2 c_b delta(k) on shell b (the P(k)
//   estimator's transpose; c = pk_partials[b - 1], nbins shells); the inverse
//   transforms' 1/N^3 is not applied, so the real output is 2 sum_k c delta_k e^{ikx}.

// Every launcher of a kernel that can run inside a relaxation iteration takes
// skip: NULL, or a device flag read at kernel entry; when it is nonzero the
// whole grid returns at once (iterations enqueued past the solver's stop).
// threads: 128, 256 or 512 per CTA (threads / N1 rows per CTA).
// ctl (may be null): one extra CTA of the launch sums the relaxation's block
// partials and applies the stop rules, as launch_finalize_control does (the
// y pass that follows the relaxation pass carries them, one launch fewer per
// iteration).
struct SolveCtl;
struct YControl {
  const double* partials;
  int nblocks;
  double* stats;
  SolveCtl* ctl;
  const double* abs_src_sum;
  double* hist;
  int max_iter, patience;
  double tol, inv_m;
};
template <typename T, int N>
void launch_fft_y(const FieldSet<T>& f, int nfields, bool inverse, const vec2_t<T>* tw, cudaStream_t s,
                  const int* skip = nullptr, int threads = 256, const YControl* ctl = nullptr);
// Batched y pass: realisation r of count (<= kBatchMax, same N) with fields f[r],
// skip flag skip[r] and, when ctl is not null, stop rules ctl[r] (FP32 data, N <= 128).
template <typename T, int RB> struct YBatch {
  FieldSet<T> f[RB];
  const int* skip[RB];
  YControl yc[RB];
};
template <typename T, int N>
void launch_fft_y_batch(const FieldSet<T>* f, const int* const* skip, const YControl* ctl, int count, int nfields,
                        bool inverse, const vec2_t<T>* tw, cudaStream_t s, int threads);

template <typename T, int N>
void launch_fft_z_r2c(const T* in, int64_t in_stride, vec2_t<T>* out, int64_t out_stride, int nfields,
                      ZPrologue pro, const vec2_t<T>* tw, cudaStream_t s);

template <typename T, int N>
void launch_fft_z_c2r(const FieldSet<T>& in, T* const* out, int nfields, const vec2_t<T>* tw,
                      cudaStream_t s);
// Batched z passes over count <= kBatchMax realisations of one mesh size (FP32,
// N <= 128): one field each for the forward transform; nfields each (the
// fields of realisation r in in[r].p / out[r].p) for the inverse.
template <typename T, int N>
void launch_fft_z_r2c_batch(const T* const* in, vec2_t<T>* const* out, const ZPrologue* pro, int count,
                            const vec2_t<T>* tw, cudaStream_t s);
template <typename T, int N>
void launch_fft_z_c2r_batch(const FieldSet<T>* in, const FieldSet<T>* out, int nfields, int count,
                            const vec2_t<T>* tw, cudaStream_t s);

// x-pass: forward x transform of nin input spectra, op, inverse x transform of
// each of the op's outputs.  For XOP_PK, outputs are the per-block bin
// partials (pk_partials, 3 * nbins doubles per block: modes, sum |k|,
// sum |X|^2 box^3 / N^6); XOP_PK_BRANE adds sum |X|^2 box^3 / N^6 / |n|^4
// (4 * nbins per block).  For XOP_SHELL the
// op is a shell indicator on |k| (shell_lo <= |k|/k_f < shell_hi) applied to
// input 0 (out 0) and the indicator itself (out 1).
template <typename T, int N>
void launch_fft_x_op(int op, const vec2_t<T>* in0, const vec2_t<T>* in1, const FieldSet<T>& out,
                     int nout_mask, const KParams& kp, double* pk_partials, int nbins, double shell_lo,
                     double shell_hi, const vec2_t<T>* tw, cudaStream_t s, const int* skip = nullptr);

// Adjoint x-passes (several y-transformed input spectra):
//  XOP_ADJ_PHI: inputs (mask bit f) phibar, gbar_x, gbar_y, gbar_z; with
//    phibar_tot = phibar + sum_i i k_i gbar_i (the transpose of g_i = -i k_i phi,
//    Nyquist component zero), out0 = B phibar_tot and out1 = A phibar_tot, where
//    phi = A delta + B D is Eq. FullDGP1.
//  XOP_ZEL_ADJ: inputs (mask bits 1..3) Psibar_x, Psibar_y, Psibar_z; out0 =
//    -(1/k^2) sum_j i k_j Psibar_j, the transpose of the Zel'dovich multiplier.
//  XOP_ADJ_COMBINE: inputs P_xx, P_yy, P_zz, P_xy, P_xz, P_yz (spectra of
//    H_ij(D) lam) and lam; out0 = -2 sum_ij h_ij P_ij + c2 (-1/kbar) lam over all
//    nine i, j (off-diagonals twice), h_ij the Hessian multipliers.
template <typename T, int N>
void launch_fft_x_adj(int op, const FieldSet<T>& in, int in_mask, const FieldSet<T>& out, const KParams& kp,
                      const vec2_t<T>* tw, cudaStream_t s);

template <typename T, int N> int x_pass_blocks();

// Batched x pass (XOP_HESSIAN, XOP_SOURCE, XOP_SOURCE_LIN, XOP_PHI_FORCE) for
// count <= kBatchMax realisations of one mesh size (FP32 data, N <= 128).
template <typename T> struct XReal {
  const vec2_t<T>* in0;
  const vec2_t<T>* in1;
  FieldSet<T> out;
  int nout_mask;
  KParams kp;
  const int* skip;
};
template <typename T, int N>
void launch_fft_x_batch(int op, const XReal<T>* r, int count, const vec2_t<T>* tw, cudaStream_t s);

// Parameters of the relaxation update (Eqs. nabla^2Cwpara, Bwpara and the
// residual of FullDGP2).
struct RelaxParams {
  double alpha, w, c2;
  double inv_m;
  // the same constants as float pairs (hi + lo), split on the host
  float alpha_hi, alpha_lo, c2_hi, c2_lo;
  float omw, two_omw;            // 1 - w, 2 (1 - w) (float; see fused_relax.cu)
  float four_omw_hi, four_omw_lo;
  float alpha_f, bad_bp_f;       // alpha and the bad-point B' = -alpha^2 / (4 (1 - w)), rounded once
};

// Fused z pass of a relaxation iteration for FP64 mesh data (fused_relax.cu):
// inverse z transform of the six y-inverted spectra (H_xx, H_yy, H_xy, H_xz,
// H_yz, N), residual and update (FP64), forward z transform of D_new into
// Snew; partials: fused_relax_blocks() x 4 doubles.  arith selects the
// arithmetic of FP32 mesh data and is not read here (FP32 data take
// launch_relax_tma below).
enum { ARITH_F32 = 0, ARITH_EFT = 1, ARITH_F64 = 2, ARITH_M32 = 3 };
template <typename T, int N>
void launch_fused_relax(int arith, vec2_t<T>* const* spec6, const T* D, const double* dsum, const T* S, T* Dnew,
                        vec2_t<T>* Snew, RelaxParams rp, double* partials, const vec2_t<T>* tw, cudaStream_t s,
                        const int* skip = nullptr);
template <typename T, int N> int fused_relax_blocks();

// The same pass for FP32 mesh data with TMA tile loads (relax_tma.cu): one
// tensor map per y-inverted spectrum (H_xx, H_yy, H_xy, H_xz, H_yz, N), built
// once per context by relax_maps (nonzero when the driver cannot encode them).
// Every wait inside is bounded by wait_ns; a wait that gives up sets *fault
// to 1 and its CTA returns.  withhold (a test hook) leaves the first pair's
// copy unissued, so that the first wait runs out.
struct RelaxMaps {
  CUtensorMap map[6];
};
// Arguments of one realisation's relaxation pass (relax_tma.cu).
struct RelaxTmaArgs {
  CUtensorMap map[6];   // y-inverted spectra of H_xx, H_yy, H_xy, H_xz, H_yz, N
  const float* D;       // current iterate (its mean = dsum / N^3)
  const double* dsum;
  const float* S;       // source field
  float* Dnew;          // next iterate
  float2* Snew;         // z-transformed next iterate, layout S[kz][x][y]
  double* partials;     // [blocks][4]
  RelaxParams rp;
  const int* skip;
  int* fault;           // set to 1 when a wait gave up
  unsigned long long wait_ns;
  int withhold;         // test hook: the first pair's copy is never issued
};
template <int RB> struct RelaxTmaBatch {
  RelaxTmaArgs a[RB];
};
template <int N>
void launch_relax_tma_batch(int arith, const RelaxTmaArgs* a, int count, const float2* tw, cudaStream_t s);

// Plane-resident Hessian pass (plane.cu) for count <= kBatchMax realisations of one mesh size
// n (FP32 data; plane_hessian_supported(n)): from the z spectrum in (layout S[kz][x][y]) of
// each realisation, the six relaxation inputs H_xx, H_yy, H_xy, H_xz, H_yz, N transformed back
// along x and y, in out.p[0..5] (same layout).  Replaces the y pass of the iterate, the Hessian
// x pass and the six-field inverse y pass of an iteration.  skip as for the other passes.
struct PlaneArgs {
  const float2* in;
  FieldSet<float> out;
  KParams kp;
  const int* skip;
};
bool plane_hessian_supported(int n);
void launch_plane_hessian_batch(int n, const PlaneArgs* a, int count, const float2* tw, cudaStream_t s);
// The stop rules of count <= kBatchMax realisations after a relaxation pass: block r sums
// realisation r's block partials and applies its stop rules (as the control CTA of the y pass);
// realisations whose skip flag is set are left alone.
void launch_control_batch(const YControl* ctl, const int* const* skip, int count, cudaStream_t s);
template <int N> int relax_maps(float2* const* spec6, RelaxMaps* out);
template <int N> int relax_tma_blocks();
template <int N>
void launch_relax_tma(int arith, const RelaxMaps& maps, const float* D, const double* dsum, const float* S,
                      float* Dnew, float2* Snew, RelaxParams rp, double* partials, const float2* tw, cudaStream_t s,
                      const int* skip, int* fault, unsigned long long wait_ns, int withhold);

// Spherical approximation (Eq. FullDGP2sph): the w = 1/3 update from C = 0,
// D = 2 S / (alpha + sqrt(alpha^2 + (8/3) S)), bad points (Delta < 0) take
// D = -3 alpha / 4.  partials[b] = bad points of block b (nblocks blocks).
template <typename T>
void launch_sph_update(const T* S, T* D, int64_t m, double alpha, double* partials, int nblocks, cudaStream_t s);

// Adjoint relaxation (J^T lam = g on mean-free fields, w-split as the forward
// iteration).  d = D - mean(D) (mean = dsum / m), diag = 2 (1 - w) d + alpha.
//  products: P[f m + i] = H_f lam for f = xx, yy, zz (= d - xx - yy), xy, xz, yz.
//  update_a: u = (g - 2 w d lam - Q) / diag; partials[b][2] = (sum u, sum diag (lam - u)).
//  update_b: sums = [sum u, sum diag (lam - u), sum 1/diag]; lam <- u + c / diag with
//    c = -mean(u) / mean(1/diag) (lam stays mean-free); partials[b] = sum |diag (lam_old - u)
//    - mean| (the projected residual of the previous lam).
//  inv_diag: partials[b][2] = (sum 1/diag, number of points with diag <= 0).
template <typename T>
void launch_adj_products(const T* lam, const T* D, const double* dsum, T* const* H5, T* P, int64_t m,
                         cudaStream_t s);
template <typename T>
void launch_adj_update_a(const T* lam, const T* D, const double* dsum, const T* g, const T* Q, T* u, int64_t m,
                         double alpha, double w, double* partials, int nblocks, cudaStream_t s);
template <typename T>
void launch_adj_update_b(T* lam, const T* D, const double* dsum, const T* u, int64_t m, double alpha, double w,
                         const double* sums, double* partials, int nblocks, cudaStream_t s);
template <typename T>
void launch_adj_inv_diag(const T* D, const double* dsum, int64_t m, double alpha, double w, double* partials,
                         int nblocks, cudaStream_t s);
template <typename T>
void launch_axpy(const T* x, const T* y, T* out, int64_t m, cudaStream_t s);  // out = x + y

// partials[nblocks][ncomp] -> out[ncomp], fixed summation order.
void launch_finalize(const double* partials, int nblocks, int ncomp, double* out, cudaStream_t s,
                     const int* skip = nullptr);

// Stop rules of the relaxation (Eq. normres, Sec. III.C), applied on the device
// after each iteration so the host need not wait for every residual.
enum { CTL_RUNNING = 0, CTL_CONVERGED = 1, CTL_STOPPED = 2, CTL_NONFINITE = 3, CTL_FAULT = 4 };
struct SolveCtl {
  int done;      // nonzero once a rule has stopped the solve (the skip flag)
  int fault;     // set by a kernel of the iteration whose bounded wait gave up
  int next_it;   // index of the iteration the controller examines next
  int status;    // CTL_*
  int stop_it;   // last iteration whose residual was examined
  int best_it;   // iteration whose incoming iterate has the smallest residual
  double rbest, rprev, prev_nbad, last_bad;
  double eps, rnorm;  // <|S|> and the normalisation of the residual
};
// stats: [sum |R|, sum D_new, bad points, non-finite R] of the iteration
// it = ctl->next_it (counted on the device, so the same launch serves every
// iteration of a captured graph); abs_src_sum: sum |S| (read at it = 0);
// hist[it] receives <|R|> / rnorm.
void launch_relax_control(SolveCtl* ctl, const double* stats, const double* abs_src_sum, double* hist,
                          int max_iter, int patience, double tol, double inv_m, cudaStream_t s);

template <typename T>
void launch_sum(const T* a, int64_t m, bool absval, double* partials, int nblocks, cudaStream_t s);

template <typename T>
void launch_density_contrast(const T* rho, T* delta, int64_t m, const double* sum, cudaStream_t s);

template <typename T>
void launch_fill(T* a, int64_t m, T v, cudaStream_t s);

// out = in - sum / m
template <typename T>
void launch_sub_mean(const T* in, T* out, int64_t m, const double* sum, cudaStream_t s);

template <typename T>
void launch_product3_sum(const T* a, const T* b, const T* c, int64_t m, double* partials,
                         int nblocks, cudaStream_t s);

// Particles.
struct CicParams {
  int n;
  float inv_d_hi, inv_d_lo;  // N / box as an unevaluated float pair
  double inv_d;              // N / box (FP64 path)
  double box;
  float box_f, inv_box_f;    // box and 1 / box rounded once
};

template <typename T>
void launch_gather_kick(T* x, T* y, T* z, T* px, T* py, T* pz, int64_t np, const T* gx,
                        const T* gy, const T* gz, CicParams cp, double kick, double drift, int do_drift,
                        cudaStream_t s);

// Batched particle and reduction stages (count <= kBatchMax realisations of one
// mesh size, FP32): CIC deposit, gather-kick(-drift), one-component FP64 sums
// (out[r][0] = sum of a[r], partials[r] with nblocks entries), zeroing of fields.
template <typename T> struct DepositArgs {
  const T* x;
  const T* y;
  const T* z;
  int64_t np;
  T* rho;
  CicParams cp;
};
template <typename T>
void launch_cic_deposit_batch(const DepositArgs<T>* a, int count, cudaStream_t s);
struct GatherArgs {
  float* p[6];         // x, y, z, px, py, pz
  int64_t np;
  const float* g[3];   // force meshes
  CicParams cp;
  float kick, drift;
  int do_drift;
};
void launch_gather_kick_batch(const GatherArgs* a, int count, cudaStream_t s);
void launch_sum_batch(const float* const* a, int64_t m, bool absval, double* const* partials, int nblocks,
                      double* const* out, int count, cudaStream_t s);
void launch_zero_batch(float* const* a, int64_t m, int count, cudaStream_t s);

// Counting sort of particles by CIC cell (sort_deposit.cu).
template <typename T>
struct ParticleSet {
  T* p[6];  // x, y, z, px, py, pz
};
struct SortWork {
  int* key;     // [np] cell of each particle
  int* count;   // [N^3] particles per cell
  int* start;   // [N^3] exclusive scan of count: first slot of each cell
  int* cursor;  // [N^3] scatter cursors
  int* sums;    // [sort_scan_blocks(N^3)] chunk sums of the scan
};
int sort_scan_blocks(int64_t m);
// Writes the particles of parts, ordered by cell, into tmp (no copy back).
template <typename T>
void launch_cell_sort(const ParticleSet<T>& parts, int64_t np, CicParams cp, const SortWork& w,
                      const ParticleSet<T>& tmp, cudaStream_t s);
// CIC deposit with warp-aggregated atomics over lanes that share a cell.
template <typename T>
void launch_cic_deposit_warp(const T* x, const T* y, const T* z, int64_t np, T* rho, CicParams cp,
                              cudaStream_t s);

// Particle side of the step adjoint (particle_adjoint.cu); pp.p[0..2] positions,
// pp.p[3..5] a per-particle 3-vector c, scaled by `scale`:
//  deposit_vec: g_i += sum_p W scale c_i,p;
//  force_vjp_gather: xb_p += sum_c grad W (G(c) . scale c_p + rscale rbar(c));
//  particle_axpy: out[0..2] += a in[0..2].
template <typename T>
void launch_deposit_vec(const ParticleSet<T>& pp, double scale, int64_t np, T* const* g, CicParams cp,
                        cudaStream_t s);
template <typename T>
void launch_force_vjp_gather(const ParticleSet<T>& pp, double scale, int64_t np, T* const* G, const T* rbar,
                             double rscale, const ParticleSet<T>& xb, CicParams cp, cudaStream_t s);
template <typename T>
void launch_particle_axpy(const ParticleSet<T>& in, double a, int64_t np, const ParticleSet<T>& out,
                          cudaStream_t s);

// Zel'dovich particles on the lattice (x index slowest): pos = (q + Psi) wrapped,
// mom = vf Psi; and the transpose: psibar_j = xbar_j + vf pbar_j as n^3 fields.
template <typename T>
void launch_zel_particles(T* const* psi, double vf, CicParams cp, T* const* out, cudaStream_t s);
template <typename T>
void launch_zel_cot(T* const* cot, double vf, int64_t m, T* const* psibar, cudaStream_t s);

int num_sms();

}  // namespace dgp
