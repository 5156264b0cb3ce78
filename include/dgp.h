/*
 * dgp.h -- C ABI of the GB300 DGP particle-mesh library.
 *
 * The library implements the hot path of the particle-mesh N-body method for
 * brane-induced (DGP) gravity of Chan & Scoccimarro, "Large-Scale Structure in
 * Brane-Induced Gravity II. Numerical Simulations":
 *   - the nonlinear field equation for the brane-bending mode C (Eq. FullDGP2)
 *     solved for D = lapbar^2 C by FFT-relaxation with the w-splitting of
 *     Eqs. FullDGP2wpara, nabla^2Cwpara and Bwpara (Secs. III.B-C);
 *   - the modified Poisson equation for phi (Eq. FullDGP1), solved in Fourier
 *     space, and the spectral force i k phi (Sec. III.A);
 *   - CIC mass assignment (Eq. CIC) and CIC force interpolation, and the
 *     second-order leapfrog in uniform steps of ln a (Sec. III.A);
 *   - the power-spectrum and bispectrum estimators of Secs. IV and VI.
 *
 * Conventions used by every call
 *   Units: lengths in Mpc/h, time in 1/H0 (H0 = 1).  c/H0 is
 *   dgp_cosmology.c_over_H0 (2997.92458 Mpc/h).  Mesh: n^3 points at x = i d,
 *   d = box / n, periodic.  A real mesh field is n^3 contiguous elements in
 *   C order [x][y][z] (z fastest).  Element type: float when the context
 *   precision is DGP_FP32 or one of the DGP_MIXED modes, double when it is DGP_FP64.
 *   Particles: struct-of-arrays, same element type; p = a^2 dx/dt.
 *   Streams: every call enqueues its GPU work on the stream given to
 *   dgp_init (NULL = the legacy default stream).  Calls that return host
 *   values (solve info, spectra) synchronise that stream before returning.
 *   Ownership: the caller owns every buffer it passes; the library never
 *   frees or retains them past the call.  The context owns its workspace,
 *   allocated in dgp_init and freed in dgp_destroy.
 *   Errors: every int-returning call returns a dgp_status; no call throws or
 *   aborts.  After DGP_E_CUDA the context should be destroyed.
 *   Threads: a context is not thread safe; use one context per host thread.
 */
#ifndef DGP_H
#define DGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DGP_OK = 0,
  DGP_E_INVALID = 1,       /* bad argument (size, pointer, parameter range) */
  DGP_E_CUDA = 2,          /* a CUDA runtime call failed */
  DGP_E_NOMEM = 3,         /* device or host allocation failed */
  DGP_E_NONFINITE = 4,     /* NaN or Inf in an input field or in the solve */
  DGP_E_NOT_CONVERGED = 5, /* tolerance not met: best iterate used, info filled */
  DGP_E_BAD_POINTS = 6,    /* discriminant clamped at some points (informational) */
  DGP_E_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  DGP_E_STATE = 8          /* call not valid in the context's current state */
} dgp_status;

/* Precision of a context.
 *   DGP_FP32      all arithmetic FP32 (FP64 only for cross-block sums).
 *   DGP_MIXED     FP32 mesh fields, FFTs and particles; the residual R, the
 *                 split source B' and the discriminant Delta in FP64; norms and
 *                 global means reduced in FP64.
 *   DGP_FP64      everything FP64 (double buffers).
 *   DGP_MIXED_EFT as DGP_MIXED, but R and Delta are evaluated on pairs of
 *                 floats with error-free transformations (TwoSum, FMA TwoProd),
 *                 ~48 significant bits, without the FP64 pipe; B' (which only
 *                 feeds the FP32 D_new) is formed in FP32 from the pair R.
 *   DGP_MIXED_F32R FP32 mesh fields, FFTs, particles and pointwise residual
 *                 R, B' and D_new; the discriminant Delta formed exactly (a pair)
 *                 for the FP32 operands, so its sign (the bad-point test) is
 *                 exact; the sums behind the residual norm and the mean of D
 *                 carried as float pairs within a thread and reduced in FP64
 *                 across threads and blocks, as every global mean.  Rounding the
 *                 converged fields to FP32 alone leaves <|R|> of order 1e-8 of
 *                 <|S|>, which no residual arithmetic can go below; the FP32
 *                 evaluation of R adds an error of the same order. */
enum { DGP_FP32 = 0, DGP_MIXED = 1, DGP_FP64 = 2, DGP_MIXED_EFT = 3, DGP_MIXED_F32R = 4 };
/* Gravity modes: the full nonlinear DGP equations (Eqs. FullDGP1-2), the
 * linearised DGP Poisson equation (Eq. LinearDGP), GR with the DGP expansion
 * (Eq. GRPoisson), and the spherical approximation of Sec. IV: Eq. FullDGP2sph
 * solved by one w = 1/3 relaxation update from C = 0 (Eq. SphPoi locally;
 * the nonlocal factor of the source is kept, N[C = 0] = 0), then Eq. FullDGP1. */
enum { DGP_GRAVITY_NL = 0, DGP_GRAVITY_LDGP = 1, DGP_GRAVITY_GRH = 2, DGP_GRAVITY_SPH = 3 };

typedef struct dgp_ctx dgp_ctx;

typedef struct {
  double omega_m0;   /* present matter density parameter */
  double c_over_H0;  /* c / H0 in Mpc/h (2997.92458) */
} dgp_cosmology;

typedef struct {
  double box;        /* side of the periodic box, Mpc/h, > 0 */
  int n;             /* mesh points per side: 16, 32, 48, 64, 96, 128, 256 or 512 */
  double rc_H0;      /* crossover scale r_c in units of c/H0, > 0 (Sec. II) */
  double w;          /* splitting parameter of Eq. FullDGP2wpara, 0 <= w < 1 */
  int precision;     /* DGP_FP32, DGP_MIXED, DGP_FP64, DGP_MIXED_EFT or DGP_MIXED_F32R */
  int gravity;       /* DGP_GRAVITY_NL (Eqs. FullDGP1-2), _LDGP (Eq. LinearDGP), _GRH (Eq. GRPoisson),
                        _SPH (spherical approximation, Sec. IV) */
  int local_only;    /* nonzero: drop the sqrt(-lapbar) terms (Appendix Eq. FullDGP2simp) */
  int max_iter;      /* relaxation updates per solve before giving up, >= 0 */
  double tol;        /* normalised-residual tolerance used by pm_step (Eq. normres) */
  int sort_every;    /* >= 0; nonzero: every sort_every-th pm_step call cell-sorts the
                        particles after its drift (dgp_sort_particles); 0: never */
  double a_nonlinear; /* >= 0; with DGP_GRAVITY_NL, solves at a < a_nonlinear use the
                        linearised equation (Sec. III.D switches at a ~ 0.1); 0: never */
} dgp_params;

typedef struct {
  int iters;            /* relaxation updates before the accepted iterate */
  double norm_res;      /* <|R|>/eps of the accepted iterate (Eq. normres) */
  double min_norm_res;  /* smallest <|R|>/eps seen */
  double bad_fraction;  /* bad points / n^3 in the last update (Sec. III.C) */
  double eps;           /* <|S|>, the normalisation of Eq. normres */
  int status;           /* DGP_OK or DGP_E_NOT_CONVERGED */
} dgp_solve_info;

typedef struct {
  void *x, *y, *z;      /* device positions in [0, box) */
  void *px, *py, *pz;   /* device momenta p = a^2 dx/dt */
  int64_t n;            /* number of particles, >= 0 */
} dgp_particles;

typedef struct {
  double E, eta, alpha, beta, s, c2, c3, q, omega_m;
  double geff_local;    /* k -> infinity limit of Eq. Geff */
  double growth_D;      /* linear growth factor, D = a deep in matter domination */
  double growth_f;      /* dlnD/dlna */
} dgp_background_t;

/* Host-only.  DGP background at scale factor a (Sec. II): E = H/H0 is the
 * self-accelerating root of Eq. DGPFriedmann, eta = r_c H, and alpha, beta,
 * q, the coefficients s = 3(eta-1)/eta, c2 = 3 beta (eta-1)/(2 eta - 1),
 * c3 = (3 eta^2 - 5 eta + 1)/(2 eta^2 (2 eta - 1)) of Eqs. FullDGP1-2, plus the
 * linear growth rate with the local G_eff (used for Zel'dovich velocities).
 * Returns DGP_E_INVALID for a <= 0, rc_H0 <= 0, omega_m0 < 0 or out == NULL. */
int dgp_background(const dgp_cosmology *cosmo, double rc_H0, double a, dgp_background_t *out);

/* Create a context for the problem of Sec. III: a periodic box of side p->box
 * (Mpc/h) with an n^3 mesh (Sec. III.A: mesh points at i box / n), the DGP
 * crossover scale p->rc_H0 and the cosmology of Sec. II (Omega_m0, c / H0).
 * Validates p, allocates all device workspace for the mesh (the fields of
 * Eqs. FullDGP1-2, the spectra of the relaxation, the warm-start iterates of
 * Sec. III.B), and binds cuda_stream (a cudaStream_t, may be NULL).  *out is
 * set to NULL on failure: DGP_E_INVALID for bad parameters (n must be one of
 * the sizes listed in dgp_params), DGP_E_NOMEM or DGP_E_CUDA. */
int dgp_init(dgp_ctx **out, const dgp_params *p, const dgp_cosmology *cosmo, void *cuda_stream);

/* Free everything the context owns.  NULL is accepted. */
void dgp_destroy(dgp_ctx *c);

/* Static description of a status code. */
const char *dgp_strerror(int status);

/* Forget the warm-start solution and the cached mesh force. */
int dgp_reset(dgp_ctx *c);

/* Solve Eqs. FullDGP2 and FullDGP1 for phi at scale factor a (Secs. III.B-C).
 *   delta: device n^3 density contrast (its mean is ignored);
 *   phi:   device n^3 output, code units (phi(k = 0) = 0); may be NULL when
 *          only the info or the warm start is wanted.
 * The relaxation starts from the context's previous accepted solution if
 * there is one (Sec. III.B, warm start), else from the linear solution, and
 * stops when <|R|>/eps < tol or after max_iter updates; without convergence
 * phi is built from the minimum-residual iterate and DGP_E_NOT_CONVERGED is
 * returned.  info (host, may be NULL) is filled in every case that reaches
 * the solver.  DGP_E_NONFINITE if delta holds NaN/Inf. */
int dgp_solve_phi(dgp_ctx *c, double a, const void *delta, void *phi, double tol,
                  dgp_solve_info *info);

/* Same solve; writes the mesh force g = -grad(phi) (Sec. III.A: i k phi
 * transformed back) into three device n^3 fields gx, gy, gz (the Nyquist
 * component of each derivative is zero).  phi may be NULL. */
int dgp_solve_forces(dgp_ctx *c, double a, const void *delta, void *phi, void *gx, void *gy,
                     void *gz, double tol, dgp_solve_info *info);

/* Normalised residual <|R|>/eps of every iterate of the last nonlinear solve,
 * in order (the first is the starting iterate).  Copies min(count, max_n)
 * values to out (host) and returns the count; a negative status on error. */
int dgp_solve_history(dgp_ctx *c, double *out, int max_n);

/* Copy the accepted solution D = lapbar^2 C of the last nonlinear solve
 * (the warm start of the next one, Sec. III.B) into the device n^3 field D,
 * with its mean removed (the solver works with mean-free D).
 * DGP_E_STATE if no nonlinear solve has completed since init/reset. */
int dgp_get_solution(dgp_ctx *c, void *D);

/* CIC mass assignment (Eq. CIC) of unit-mass particles and the density
 * contrast delta = rho / rho_bar - 1 (rho_bar: FP64 mean of the mesh).
 * delta: device n^3 output.  Positions outside [0, box) are wrapped. */
int dgp_deposit(dgp_ctx *c, const dgp_particles *parts, void *delta);

/* Adjoint of the context's last accepted nonlinear solve (gravity NL), for
 * gradients through the field solve (the differentiation pattern of the
 * method; the paper has no adjoint).  With delta -> D defined by R(D, delta) = 0
 * (Eq. FullDGP2) on mean-free fields and phi = A delta + B D (Eq. FullDGP1),
 * a cotangent phibar of phi (and/or gbar_i of the forces g_i = -d_i phi, which
 * add sum_i d_i gbar_i to phibar) gives
 *   deltabar = A phibar + S lam,  J^T lam = B phibar,
 * J the Jacobian of R in D (J^T lam = (2D + alpha) lam - 2 sum_ij H_ij[H_ij(D) lam]
 * + c2 N[lam]) and S the source multiplier s (1 - beta/kbar).  J^T lam = B phibar
 * is solved by the relaxation's w-splitting (Sec. III.C) to <|P(J^T lam - g)|> /
 * <|g|> < tol, P the mean projection, at most params.max_iter updates.
 *   phibar, gbar_x, gbar_y, gbar_z: device n^3 fields (phibar may be NULL; the
 *     three gbar all NULL or all set); deltabar: device n^3 output.
 * info (host, may be NULL): iters = updates, norm_res = last residual, eps =
 * <|B phibar|>.  Returns DGP_OK, DGP_E_NOT_CONVERGED (deltabar from the last
 * iterate), DGP_E_STATE (no nonlinear solve accepted since init/reset),
 * DGP_E_BAD_POINTS (2(1-w)D + alpha <= 0 somewhere: the splitting is not
 * defined), DGP_E_INVALID (bad arguments or a gravity mode other than NL). */
int dgp_solve_adjoint(dgp_ctx *c, const void *phibar, const void *gbar_x, const void *gbar_y,
                      const void *gbar_z, void *deltabar, double tol, dgp_solve_info *info);

/* Transpose of the Jacobian of one pm_step (gravity NL): for cotangents
 * (xbar1, pbar1) of the positions and momenta after the step from a to a + da,
 * returns those of the state before it, given that state in `start` (device
 * arrays, unchanged).  cot holds (xbar1, pbar1) on entry (x, y, z, px, py, pz
 * members, device arrays of n values) and (xbar0, pbar0) on return.  The step
 * is recomputed from `start`; with p_h = p0 + K1 F(x0), x1 = x0 + Dr p_h and
 * p1 = p_h + K2 F(x1):
 *   xbar = xbar1 + F'(x1)^T (K2 pbar1),  pbar0 = pbar1 + Dr xbar,
 *   xbar0 = xbar + F'(x0)^T (K1 pbar0),
 * where F'(x)^T fbar is the force VJP: the gather's transpose with the CIC
 * weights' derivatives, plus the deposit of fbar -> dgp_solve_adjoint (force
 * cotangents) -> the density contrast's cotangent -> the deposit's transpose.
 * Three nonlinear solves (x0, x1, x0) and two adjoint solves at params.tol.
 * The periodic wrap is the identity on the cotangents (positions differ by
 * lattice vectors only).  The context's warm start and force cache are
 * replaced.  DGP_E_INVALID for bad arguments or a gravity mode other than NL. */
int pm_step_adjoint(dgp_ctx *c, const dgp_particles *start, double a, double da, dgp_particles *cot);

/* Zel'dovich initial conditions from a device n^3 linear field delta_L (Sec. III.A
 * uses 2LPT; this is the first-order map the synthetic inputs use): one particle
 * per mesh cell in lattice order (x index slowest), Psi_j = IFFT(i k_j / k^2
 * delta_L(k)) with the Nyquist component of k_j dropped, pos = q + Psi wrapped
 * into [0, box), mom = vel_factor Psi.  out->n must be n^3. */
int dgp_zeldovich(dgp_ctx *c, const void *delta_l, double vel_factor, dgp_particles *out);

/* Transpose of dgp_zeldovich: delta_l_bar = sum_j (-i k_j / k^2)[xbar_j + vel_factor pbar_j]
 * for the cotangents in cot (lattice order, n^3 particles). */
int dgp_zeldovich_adjoint(dgp_ctx *c, const dgp_particles *cot, double vel_factor, void *delta_l_bar);

/* Transpose of particles -> CIC deposit -> density contrast -> power_spectrum for
 * the host gradient dl_dp[nbins] = dL/dP_b: the density contrast's cotangent is
 * 2 sum_k c(k) delta_k e^{ikx}, c = dL/dP_b box^3 / (n^6 n_b) on shell b, and its
 * transpose through the deposit is added to the position cotangents of cot
 * (its momentum members are not touched). */
int dgp_power_spectrum_adjoint(dgp_ctx *c, const dgp_particles *parts, int nbins, const double *dl_dp,
                               dgp_particles *cot);

/* Derivatives in the crossover scale r_c H0 (Sec. II: r_c enters through
 * E(a) of Eq. DGPFriedmann, eta = r_c H and every coefficient of Eqs.
 * FullDGP1-2, the step's kick and drift factors, and the growth rate of the
 * initial velocities).  The context's own r_c H0 is the point of evaluation;
 * ' below is d/d(r_c H0).
 *
 * dgp_solve_adjoint_rc: dgp_solve_adjoint plus *rc_bar (host) = the explicit
 * derivative of <phibar_tot, phi> with delta fixed and D through the solve:
 *   rc_bar = <phibar_tot, A' delta + B' D> - <lam, alpha' D + c2' N[D] + c2 N'[D] - S' delta>,
 * phibar_tot = phibar + sum_i d_i gbar_i.  Needs the accepted solve's delta,
 * so the last field solve must have been nonlinear (else DGP_E_STATE).  rc_bar
 * is a host double the call writes (NULL: DGP_E_INVALID); other arguments and
 * return codes as dgp_solve_adjoint. */
int dgp_solve_adjoint_rc(dgp_ctx *c, const void *phibar, const void *gbar_x, const void *gbar_y,
                         const void *gbar_z, void *deltabar, double tol, double *rc_bar, dgp_solve_info *info);

/* pm_step_adjoint plus *rc_bar (host) = the step's explicit derivative of
 * <xbar1, x1> + <pbar1, p1> in r_c H0 with (x0, p0) fixed:
 *   K2' <pbar1, F(x1)> + rc_solve(x1) + Dr' <xbar1_tot, p_h> + K1' <pbar_h, F(x0)> + rc_solve(x0),
 * xbar1_tot the cotangent of x1 after the second kick's transpose and rc_solve the
 * dgp_solve_adjoint_rc term of each force VJP.  The K' and Dr' are taken by
 * complex-step differentiation of the 8-point Gauss-Legendre rules.  Summed
 * over the steps of a run (with the cotangents passed backwards) this is the
 * run's derivative in r_c H0 at fixed initial particles.  rc_bar is a host double
 * the call writes (NULL: DGP_E_INVALID); other arguments and return codes as
 * pm_step_adjoint. */
int pm_step_adjoint_rc(dgp_ctx *c, const dgp_particles *start, double a, double da, dgp_particles *cot,
                       double *rc_bar);

/* Cotangent of vel_factor in dgp_zeldovich: *vf_bar (host) = sum_j <pbar_j, Psi_j(delta_L)>
 * for the momentum cotangents of cot (lattice order, n^3 particles); delta_l is the device
 * n^3 linear field (read only); vf_bar is a host double the call writes.  The cached mesh
 * force is discarded.  DGP_E_INVALID for NULL arguments or cot->n != n^3. */
int dgp_zeldovich_vf_adjoint(dgp_ctx *c, const void *delta_l, const dgp_particles *cot, double *vf_bar);

/* Host-only.  The Zel'dovich velocity factor vf = a^2 E f (local G_eff, as
 * dgp_background's growth_f) and d vf / d(r_c H0), by complex-step
 * differentiation of the growth ODE's RK4 steps.  DGP_E_INVALID as
 * dgp_background. */
int dgp_velocity_factor(const dgp_cosmology *cosmo, double rc_H0, double a, double *vf, double *dvf_drc);

/* Host-only.  d/d(r_c H0) of every member of dgp_background at scale factor a (the
 * derivatives the r_c adjoint uses), by complex-step differentiation of the same
 * code; errors as dgp_background. */
int dgp_background_drc(const dgp_cosmology *cosmo, double rc_H0, double a, dgp_background_t *out);

/* Host-only.  The leapfrog's time factors between a0 and a1 (Sec. III.A with
 * p = a^2 dx/dt; 8-point Gauss-Legendre in ln a, as pm_step uses them):
 *   out[0] = int dlna / E            (kick),   out[1] = int dlna / (a^2 E)   (drift),
 *   out[2], out[3] = their derivatives in r_c H0 (complex-step differentiation of the rule).
 * pm_step kicks with out[0] over each half step (a0 -> sqrt(a0 a1) -> a1) and drifts with
 * out[1] over the whole step.  DGP_E_INVALID for a0, a1 <= 0 or not finite, rc_H0 <= 0,
 * omega_m0 < 0 or NULL. */
int dgp_time_factors(const dgp_cosmology *cosmo, double rc_H0, double a0, double a1, double *out);

/* Host-only.  Device bytes a context with parameters p requests from cudaMalloc
 * (sums of the requested sizes; the allocator's rounding and the CUDA context
 * itself are not included), without creating one:
 *   base:      at dgp_init (14 real fields, 9 half spectra, twiddles, reduction
 *              partials, residual history);
 *   sort:      added by the first dgp_sort_particles / sorting pm_step of np
 *              particles (keys, six permuted arrays, three int32 fields per cell);
 *   adjoint:   added by the first pm_step_adjoint of np particles (products,
 *              spectra, cotangent grids, the recomputed particle state);
 *   host_step: added by the first pm_step_host of np particles.
 * The reduction partials depend on the device's SM count (1 when no device is
 * visible; a few KB either way).  Only p->n, p->precision and p->max_iter are
 * read.  DGP_E_INVALID for an unsupported n or precision, np < 0 or NULL. */
typedef struct {
  size_t base, sort, adjoint, host_step;
} dgp_workspace;
int dgp_workspace_size(const dgp_params *p, int64_t np, dgp_workspace *out);

/* Tile configuration of the context (not part of the paper's method): the y
 * pass's threads per CTA, 128, 256 or 512 (that many / N1 rows per CTA), picked
 * at dgp_init by timing the three variants on the context's own buffers.  The
 * results do not depend on the choice.  dgp_set_tile_config forces a value
 * (DGP_E_INVALID for any other). */
int dgp_tile_config(dgp_ctx *c, int *y_threads);
int dgp_set_tile_config(dgp_ctx *c, int y_threads);

/* Fused Hessian pass of the relaxation (Sec. III.B, Eq. FullDGP2: the second
 * derivatives of C and the non-local term N, each iteration).  For FP32 mesh
 * data at n = 128 or 256, when the device co-schedules a thread-block cluster
 * of n / 16 CTAs, an iteration forms the six spectra and transforms them back
 * along x and y in one launch (a cluster per kz plane exchanging through
 * distributed shared memory) instead of an x pass and a six-field y pass; the
 * six spectra then cross memory once instead of three times.  The results
 * are the same up to rounding order.  On a GB300 at 256^3 the fused launch
 * took 352 us against 240 us for the two passes it replaces, so it is off by
 * default.  dgp_set_hessian_fusion turns it on (on != 0) or off (0, the
 * default); dgp_hessian_fusion sets *active to 1 when the context's solves
 * use it.  DGP_E_INVALID for a NULL argument. */
int dgp_set_hessian_fusion(dgp_ctx *c, int on);
int dgp_hessian_fusion(dgp_ctx *c, int *active);

/* Bound of the waits inside the relaxation kernel (not part of the paper's
 * method).  The FP32-data relaxation pass waits on its own asynchronous tile
 * copies; each wait gives up after `seconds` (default 2; 0 < seconds <= 60),
 * and the solve then returns DGP_E_TIMEOUT with the context still usable (the
 * warm start is left as it was before the solve).  withhold_first_copy != 0 is
 * a test hook: the pass leaves the first of its copies unissued, so its first
 * wait runs out; set it back to 0 to solve again.  DGP_E_INVALID for a NULL
 * context or a bound out of range. */
int dgp_set_wait_limit(dgp_ctx *c, double seconds, int withhold_first_copy);

/* Host waits of the context (the relaxation's stop-rule verdicts, host outputs)
 * block on an event and yield the CPU (on != 0) instead of spinning (0, the
 * default).  For callers that drive many contexts from many host threads. */
int dgp_set_blocking_sync(dgp_ctx *c, int on);

/* ---- Batches of independent realisations --------------------------------
 * Not part of the paper's method: many small boxes (e.g. 48 realisations of
 * 48^3, 64^3 and 96^3 meshes with different boxes and r_c) stepped together.
 * The realisations are grouped into classes: those with the same mesh size
 * and precision, in the nonlinear mode (no local_only, no a_nonlinear), with
 * FP32 mesh data and n <= 128, at most 16 to a class, in order of appearance.
 * A class shares one non-blocking stream; its step launches each kernel stage
 * once for all members (one launch of every FFT pass, relaxation pass, deposit
 * and gather for the whole class), its members iterate in lockstep, each
 * stopping by its own rules (members that have stopped skip at kernel entry),
 * and its relaxation iterations replay as one CUDA graph.  Every member ends
 * each step exactly as its own pm_step would leave it.  A realisation that
 * forms no class is a context stepped alone on a stream of its own.  Each
 * class or lone context has one host worker thread, so classes run
 * concurrently; the contexts use blocking host waits.
 *   dgp_batch_create: count contexts from params[count] (sizes may differ)
 *     and one cosmology; DGP_E_INVALID, DGP_E_NOMEM or DGP_E_CUDA on failure,
 *     *out = NULL then.
 *   dgp_batch_context: the i-th context (for deposit, P(k), reset, ...); the
 *     batch keeps ownership (do not destroy it).  Contexts of one class share
 *     their stream.
 *   dgp_batch_step: pm_step of every realisation i with parts[i], a[i], da[i]
 *     (info[i] filled when info != NULL).  The batch streams first wait for
 *     the work enqueued so far on cuda_stream (may be NULL); the call returns
 *     when every realisation's step has completed on the device.  Returns
 *     the first non-OK status of a realisation.  A class whose step is refused
 *     for a bad argument (e.g. an empty particle set) steps its members one by
 *     one instead, so the valid ones still step.
 *   dgp_batch_classes: class_of[count] receives the class of each realisation
 *     and *nclasses the number of classes and lone contexts.
 *   dgp_batch_set_plane_pass: for classes of n <= 96 (on != 0, the default)
 *     an iteration's Hessian spectra come from one plane-resident pass: a CTA
 *     per kz plane and realisation transforms the iterate's z spectrum along
 *     y and x in shared memory and writes the six relaxation inputs
 *     transformed back along x and y (Sec. III.B, Eq. FullDGP2: the second
 *     derivatives of C and the non-local term), so each crosses HBM once;
 *     on = 0 uses the separate x and y passes of a single context.  Both
 *     compute the same spectra up to rounding order.
 * Calls on one batch must not overlap. */
typedef struct dgp_batch dgp_batch;
int dgp_batch_create(dgp_batch **out, int count, const dgp_params *params, const dgp_cosmology *cosmo);
int dgp_batch_context(dgp_batch *b, int i, dgp_ctx **out);
int dgp_batch_step(dgp_batch *b, dgp_particles *parts, const double *a, const double *da, dgp_solve_info *info,
                   void *cuda_stream);
int dgp_batch_classes(dgp_batch *b, int *class_of, int *nclasses);
int dgp_batch_set_plane_pass(dgp_batch *b, int on);
void dgp_batch_destroy(dgp_batch *b);

/* Spectra of the brane-bending mode C of the context's accepted nonlinear
 * solution D = lapbar^2 C, at the scale factor of that solve (Sec. IV):
 *   pc[b]:  P_c of c = alpha eta / (3 (eta - 1)) D (Eq. cdef; P_c / P_m -> 1 on
 *           linear scales, suppressed by the Vainshtein mechanism);
 *   pC[b]:  P_C of C, C(k) = -D(k) / kbar^2 with kbar = (c/H0) |k| / (a E);
 *   delta_gradc[b]: 4 pi k^5 P_C(k) (Eq. DGradC; C dimensionless, k the
 *           shell's mean |k| in h/Mpc).
 * Shells, k[b] and nmodes[b] as power_spectrum (host outputs, 1 <= nbins <= n/2).
 * DGP_E_STATE if no nonlinear solve has been accepted since init/reset. */
int dgp_brane_spectra(dgp_ctx *c, int nbins, double *k, double *pc, double *pC, double *delta_gradc,
                      int64_t *nmodes);

/* Counting sort of the particles by mesh cell, in place (support for the CIC
 * assignment of Sec. III.A; the paper deposits particles in storage order).
 * The key of a particle is the cell of its lower CIC corner,
 * (ix n + iy) n + iz with i = floor(x n / box) mod n per axis, the index the
 * deposit and the gather use.  After the call the six arrays are permuted
 * together so that keys are nondecreasing; the order of particles that share
 * a cell is not specified (it can differ between calls).  Particles carry no
 * identity in this interface, so the permutation is not returned.
 *   parts:      device arrays of the context precision, n <= 2^31 - 1;
 *   cell_start: NULL, or device int32[n^3 + 1] receiving the first slot of
 *               each cell (cell c holds slots cell_start[c] .. cell_start[c+1]-1;
 *               cell_start[n^3] = parts->n); synchronised on return when given.
 * The first call, and any call with more particles than before, allocates
 * 4 + 6 sizeof(real) bytes per particle and 12 n^3 bytes of workspace; the
 * sort itself goes through those copies (the six arrays are copied back).
 * DGP_E_INVALID for a bad argument, DGP_E_NOMEM, DGP_E_CUDA. */
int dgp_sort_particles(dgp_ctx *c, dgp_particles *parts, int32_t *cell_start);

/* One kick-drift-kick step from a to a + da, uniform in ln a (Sec. III.A):
 * p += g(x, a) K(a, a_h); x += p Dr(a, a + da); p += g(x', a + da) K(a_h, a + da)
 * with a_h the midpoint in ln a, K = int dlna / E and Dr = int dlna / (a^2 E).
 * The force at the start reuses the mesh force the previous call left when
 * that call ended at the same a with the same particle buffers; otherwise it
 * is computed first.  The solve uses params.tol and the warm start.  info
 * (host, may be NULL) describes the solve at a + da.  With params.sort_every
 * = K > 0, every K-th call (counted since init or dgp_reset) reorders the
 * particles by cell after the drift, as dgp_sort_particles does. */
int pm_step(dgp_ctx *c, dgp_particles *parts, double a, double da, dgp_solve_info *info);

/* pm_step on host particle arrays (pageable or pinned): copies them to the
 * context's device buffers, steps, and copies them back before returning.
 * The positions are final after the drift, so their copy back runs on a
 * second stream during the field solve (overlapped when the host arrays are
 * pinned).  The host arrays are float or double per the context precision.
 * The force at the start is reused only when the previous call on this
 * context was a pm_step_host that ended at the same a on the same host arrays
 * (same host_parts->x pointer and n); stepping another set of host arrays, or
 * a pm_step on device arrays in between, makes the step compute it afresh.
 * The caller must not change the host arrays between two such calls unless it
 * calls dgp_reset. */
int pm_step_host(dgp_ctx *c, dgp_particles *host_parts, double a, double da, dgp_solve_info *info);

/* Power spectrum of a device n^3 field (Sec. IV):
 * P(k_b) = box^3 <|delta_k / n^3|^2> over shells b = 1..nbins of width
 * k_f = 2 pi / box centred on b k_f (a mode belongs to shell round(|k|/k_f)),
 * no window deconvolution, no shot-noise subtraction.  Host outputs
 * k[nbins] (mean |k| of the shell), pk[nbins], nmodes[nbins] (all n^3 modes
 * counted once).  1 <= nbins <= n/2. */
int power_spectrum(dgp_ctx *c, const void *delta, int nbins, double *k, double *pk, int64_t *nmodes);

/* Bispectrum by the FFT shell-filter estimator (Sec. VI, Eq. Qdef): for each
 * theta[i] (angle between k1 and k2), k3 = |k1 + k2|, shells of width dk
 * (<= 0 means k_f) around k1, k2, k3; B = box^6/n^9 * sum_x d1 d2 d3 /
 * sum_x I1 I2 I3 and Q = B / (P1 P2 + P2 P3 + P3 P1) with the shell powers.
 * Host outputs b[ntheta], q[ntheta]. */
int bispectrum(dgp_ctx *c, const void *delta, double k1, double k2, int ntheta, const double *theta,
               double dk, double *b, double *q);

/* ---- P(k) for callers that cannot allocate device memory --------------------
 * The paper has no counterpart to this call.  Some callers cannot call
 * cudaMalloc: a host framework that reserved the whole device for its own
 * pooling allocator, or a long-running loop that must not allocate once it has
 * started.  dgp_init allocates a workspace, so power_spectrum is closed to
 * them; this variant needs no context and allocates nothing.  It computes the
 * same estimator as power_spectrum (same kernels, same shells) for an FP32
 * field of n^3 points, n in {16, 32, 64} (n <= DGP_NOALLOC_MAX_N), using one
 * file-scope device array of DGP_NOALLOC_SCRATCH_BYTES bytes that every GPU
 * loading the library holds until the process exits.
 *   delta:  device n^3 floats, [x][y][z];  box: side in Mpc/h;  1 <= nbins <= n/2;
 *   k, pk, nmodes: host outputs of length nbins (as power_spectrum);
 *   cuda_stream: stream for the work (NULL = legacy default); synchronised on return.
 * The first call on a device, with that device current, resolves the array's
 * device address and writes the twiddle tables into it (a copy on cuda_stream
 * that completes before the call goes on); make that first call before any
 * stream capture.  Every call on a device uses
 * the same array and overwrites it entirely, so calls that overlap on the GPU
 * (other streams, other host threads) race: serialise them.
 * Returns DGP_E_INVALID for n outside {16, 32, 64} (larger meshes do not fit
 * the array: use power_spectrum with a context) or a bad argument,
 * DGP_E_CUDA if a CUDA call fails. */
#define DGP_NOALLOC_MAX_N 64
#define DGP_NOALLOC_SCRATCH_BYTES 1188096
int dgp_power_spectrum_noalloc(const float *delta, int n, double box, int nbins, double *k, double *pk,
                               int64_t *nmodes, void *cuda_stream);

/* Kernel accounting (not part of the paper's method; used to measure it).
 * Every kernel launch of a context is counted per kind together with its
 * algorithmic bytes (one read of each input and one write of each output).
 * dgp_profile resets the counters; with timing != 0 each later launch is
 * also bracketed by two CUDA events on the context's stream (adding two
 * event records per launch).  dgp_profile_read synchronises on the pending
 * events and returns, for kind in [0, DGP_KERNEL_KINDS): launches and bytes
 * since the reset, and the timed launches, their summed duration (ms) and
 * their bytes.  Any output pointer may be NULL. */
#define DGP_KERNEL_KINDS 11
int dgp_profile(dgp_ctx *c, int timing);
/* As dgp_profile, but only launches of the kinds whose bit is set in
 * kind_mask (bit k for kind k) are bracketed by events, so the timing of the
 * others is not perturbed by event records. */
int dgp_profile_kinds(dgp_ctx *c, unsigned kind_mask);
/* As dgp_profile_kinds, but the iterations of a solve keep running as CUDA
 * graphs (dgp_profile and dgp_profile_kinds turn graph replay off), so the
 * timed launches are those of the production path.  Only launches outside a
 * graph that are certain to do their work are bracketed by events: the first
 * relaxation iteration of each solve, replays of an earlier iterate, and every
 * launch outside the iteration loop; their bytes are the full algorithmic
 * bytes of one executed launch. */
int dgp_profile_sampled(dgp_ctx *c, unsigned kind_mask);
int dgp_profile_read(dgp_ctx *c, int kind, int64_t *launches, double *bytes, int64_t *timed, double *ms,
                     double *timed_bytes);
/* Name of a kernel kind ("fft_z_r2c", "fft_y", "relax", ...), NULL if out of range. */
const char *dgp_kernel_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* DGP_H */
