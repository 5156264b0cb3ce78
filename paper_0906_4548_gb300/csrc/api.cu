// C ABI of the DGP library: context, host background, and the orchestration of
// the FFT-relaxation solve (Secs. III.B-C), phi and forces (Eq. FullDGP1,
// Sec. III.A), the kick-drift-kick step, and the estimators (Secs. IV, VI).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <functional>
#include <new>
#include <utility>
#include <vector>

#include "../../include/dgp.h"
#include "adjoint_rc.cuh"
#include "fft_core.cuh"
#include "kernels.cuh"
#include "relax_control.cuh"
#include "xy.cuh"

namespace dgp {

// ---------------------------------------------------------------- background
// The background is written once for a scalar type S: double for the values,
// std::complex<double> for their derivatives in r_c H0 by complex-step
// differentiation (Squire & Trapp 1998): for f analytic in r, evaluated at
// r + i h, f'(r) = Im f(r + i h) / h + O(h^2), with no difference taken, so
// h = 1e-20 r gives the derivative to rounding.  Every operation on an S below
// is analytic (no abs, no comparison); a and ln a stay real.
using cplx = std::complex<double>;

// Eq. DGPFriedmann with H0 = 1: E^2 - E / rc - Om a^-3 = 0, '+' root.
template <typename S> static S hubble_E_t(double a, double om, S rc) {
  using std::sqrt;
  const S eps = 1.0 / rc;
  return 0.5 * (eps + sqrt(eps * eps + 4.0 * om / (a * a * a)));
}
static double hubble_E(double a, double om, double rc) { return hubble_E_t<double>(a, om, rc); }

template <typename S> struct CoefT {
  double a;
  S E, eta, alpha, beta, s, c2, c3, q, omega_m;
};
using Coef = CoefT<double>;

template <typename S> static CoefT<S> coefficients_t(double a, double om, S rc) {
  CoefT<S> c;
  c.a = a;
  c.E = hubble_E_t<S>(a, om, rc);
  const S eta = rc * c.E;
  c.eta = eta;
  const S den = eta * (2.0 * eta - 1.0);
  c.alpha = 3.0 * (2.0 * eta * eta - 2.0 * eta + 1.0) / den;
  c.beta = (2.0 * eta * eta - 2.0 * eta - 1.0) / den;
  c.s = 3.0 * (eta - 1.0) / eta;
  c.c2 = 3.0 * c.beta * (eta - 1.0) / (2.0 * eta - 1.0);
  c.c3 = (3.0 * eta * eta - 5.0 * eta + 1.0) / (2.0 * eta * eta * (2.0 * eta - 1.0));
  c.q = (2.0 - eta) / (2.0 * eta - 1.0);
  c.omega_m = om / (a * a * a * c.E * c.E);
  return c;
}
static Coef coefficients(double a, double om, double rc) { return coefficients_t<double>(a, om, rc); }

template <typename S> static S geff_local_t(const CoefT<S>& c) {
  const S t = 2.0 * c.eta * (2.0 + c.q);
  return (t - 4.0) / (t - 3.0);
}
static double geff_local(const Coef& c) { return geff_local_t<double>(c); }

static double cs_step(double rc) { return 1e-20 * rc; }

// d/d(r_c H0) of every coefficient (fields of the returned Coef hold derivatives; a is a).
static Coef coefficients_drc(double a, double om, double rc) {
  const double h = cs_step(rc);
  const CoefT<cplx> z = coefficients_t<cplx>(a, om, cplx(rc, h));
  Coef d;
  d.a = a;
  d.E = z.E.imag() / h; d.eta = z.eta.imag() / h; d.alpha = z.alpha.imag() / h; d.beta = z.beta.imag() / h;
  d.s = z.s.imag() / h; d.c2 = z.c2.imag() / h; d.c3 = z.c3.imag() / h; d.q = z.q.imag() / h;
  d.omega_m = z.omega_m.imag() / h;
  return d;
}

// Linear growth D'' + (2 + dlnE/dlna) D' = 1.5 Omega_m(a) Geff_local D in ln a,
// growing mode D = a at a = 1e-5, classical RK4 with 400 steps per e-fold.
template <typename S> static void growth_t(double a_out, double om, S rc, S* D_out, S* f_out) {
  auto rhs = [&](double lna, const S y[2], S dy[2]) {
    const double a = exp(lna);
    const CoefT<S> c = coefficients_t<S>(a, om, rc);
    const S dlnE = -3.0 * om / (a * a * a) / ((2.0 * c.E - 1.0 / rc) * c.E);
    dy[0] = y[1];
    dy[1] = -(2.0 + dlnE) * y[1] + 1.5 * c.omega_m * geff_local_t<S>(c) * y[0];
  };
  const double x0 = log(1e-5), x1 = log(a_out);
  int n = (int)ceil((x1 - x0) * 400.0);
  if (n < 1) n = 1;
  const double h = (x1 - x0) / n;
  S y[2] = {S(1e-5), S(1e-5)}, k1[2], k2[2], k3[2], k4[2], t[2];
  double x = x0;
  for (int i = 0; i < n; ++i) {
    rhs(x, y, k1);
    for (int j = 0; j < 2; ++j) t[j] = y[j] + 0.5 * h * k1[j];
    rhs(x + 0.5 * h, t, k2);
    for (int j = 0; j < 2; ++j) t[j] = y[j] + 0.5 * h * k2[j];
    rhs(x + 0.5 * h, t, k3);
    for (int j = 0; j < 2; ++j) t[j] = y[j] + h * k3[j];
    rhs(x + h, t, k4);
    for (int j = 0; j < 2; ++j) y[j] += h / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
    x += h;
  }
  *D_out = y[0];
  *f_out = y[1] / y[0];
}
static void growth(double a_out, double om, double rc, double* D_out, double* f_out) {
  growth_t<double>(a_out, om, rc, D_out, f_out);
}

// Zel'dovich velocity factor vf = a^2 E f and its derivative in r_c H0.
static void velocity_factor(double a, double om, double rc, double* vf, double* dvf) {
  const double h = cs_step(rc);
  cplx D, f;
  growth_t<cplx>(a, om, cplx(rc, h), &D, &f);
  const cplx v = a * a * hubble_E_t<cplx>(a, om, cplx(rc, h)) * f;
  double Dr, fr;
  growth(a, om, rc, &Dr, &fr);
  *vf = a * a * hubble_E(a, om, rc) * fr;
  *dvf = v.imag() / h;
}

// 8-point Gauss-Legendre nodes and weights by Newton iteration on P_8.
static void gauss_legendre8(double xs[8], double ws[8]) {
  const int n = 8;
  for (int i = 0; i < n; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    xs[i] = x;
    ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// int_{ln a0}^{ln a1} dlna / (a^pw E): pw = 0 kick, pw = 2 drift (Sec. III.A
// with p = a^2 dx/dt: dp/dlna = -grad phi / E, dx/dlna = p / (a^2 E)).
template <typename S> static S time_integral_t(double a0, double a1, double om, S rc, int pw) {
  double xs[8], ws[8];
  gauss_legendre8(xs, ws);
  const double l0 = log(a0), l1 = log(a1);
  const double xm = 0.5 * (l0 + l1), xr = 0.5 * (l1 - l0);
  S acc = S(0.0);
  for (int i = 0; i < 8; ++i) {
    const double a = exp(xm + xr * xs[i]);
    acc += ws[i] / (pow(a, pw) * hubble_E_t<S>(a, om, rc));
  }
  return xr * acc;
}
static double time_integral(double a0, double a1, double om, double rc, int pw) {
  return time_integral_t<double>(a0, a1, om, rc, pw);
}
// d/d(r_c H0) of time_integral (complex step)
static double time_integral_drc(double a0, double a1, double om, double rc, int pw) {
  const double h = cs_step(rc);
  return time_integral_t<cplx>(a0, a1, om, cplx(rc, h), pw).imag() / h;
}

// ---------------------------------------------------------------- engine
// Kernel-level accounting.  Launches and algorithmic bytes are always counted;
// when timing is on, each launch is bracketed by two events on the context's
// stream and the durations are resolved when read.
enum KernelKind { KK_Z_R2C = 0, KK_Z_C2R, KK_Y, KK_X_HESSIAN, KK_X_OTHER, KK_RELAX, KK_REDUCE, KK_DEPOSIT,
                  KK_GATHER, KK_MISC, KK_SORT, KK_COUNT };
static const char* const kKernelNames[KK_COUNT] = {
    "fft_z_r2c", "fft_z_c2r", "fft_y", "fft_x_hessian", "fft_x_other", "relax", "reduce", "cic_deposit",
    "cic_gather_kick", "misc", "cell_sort"};

struct Profiler {
  unsigned timing = 0;  // bit k: launches of kind k are bracketed by events
  // sampled: CUDA-graph replay of the iterations stays on, and only launches
  // outside graphs that are sure to do their work (the first iteration of a
  // solve, replays, everything outside the iteration loop) are timed
  bool sampled = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, double>> pending;  // (kind, bytes) per event pair
  int64_t launches[KK_COUNT] = {};
  double bytes[KK_COUNT] = {};
  double ms[KK_COUNT] = {};
  int64_t timed[KK_COUNT] = {};
  double timed_bytes[KK_COUNT] = {};

  void reset(unsigned t, bool smp = false) {
    resolve();
    timing = t;
    sampled = smp;
    for (int k = 0; k < KK_COUNT; ++k) { launches[k] = 0; bytes[k] = 0; ms[k] = 0; timed[k] = 0; timed_bytes[k] = 0; }
  }
  cudaEvent_t ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  int resolve() {
    for (size_t i = 0; i < pending.size(); ++i) {
      float t = 0.f;
      if (cudaEventSynchronize(pool[2 * i + 1]) != cudaSuccess) return DGP_E_CUDA;
      if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) != cudaSuccess) return DGP_E_CUDA;
      ms[pending[i].first] += t;
      timed[pending[i].first] += 1;
      timed_bytes[pending[i].first] += pending[i].second;
    }
    pending.clear();
    used = 0;
    return DGP_OK;
  }
  void count(int kind, int64_t n) { launches[kind] += n; }
  // bytes of work that launches already counted (with 0 bytes) turned out to do
  void credit(int kind, double b) {
    bytes[kind] += b;
    if (((timing >> kind) & 1u) && !sampled) timed_bytes[kind] += b;
  }
  bool capturing = false;  // launches recorded into a graph are counted when the graph runs
  template <class F>
  void run(int kind, double b, cudaStream_t s, F&& f) {
    run_it(kind, b, b, s, static_cast<F&&>(f));
  }
  // A launch of a relaxation iteration: b bytes are counted now (the rest is
  // credited once the solve has stopped); sure_b >= 0 when the launch is sure
  // to do its work (sure_b bytes), < 0 when it may return at entry.
  template <class F>
  void run_it(int kind, double b, double sure_b, cudaStream_t s, F&& f) {
    if (capturing) { f(); return; }
    launches[kind] += 1;
    bytes[kind] += b;
    if (!((timing >> kind) & 1u) || (sampled && sure_b < 0)) { f(); return; }
    if (pending.size() >= 8192) resolve();
    cudaEventRecord(ev(), s);
    f();
    cudaEventRecord(ev(), s);
    pending.push_back({kind, sampled ? sure_b : b});
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

class EngineBase {
 public:
  dgp_params p;
  dgp_cosmology cosmo;
  cudaStream_t stream = nullptr;
  virtual ~EngineBase() {}
  virtual int init() = 0;
  virtual int solve(double a, const void* delta, void* phi, void* gx, void* gy, void* gz, double tol,
                    dgp_solve_info* info) = 0;
  virtual int deposit(const dgp_particles* parts, void* delta) = 0;
  virtual int sort(dgp_particles* parts, int* cell_start) = 0;
  virtual int brane(int nbins, double* k, double* pc, double* pC, double* dgc, int64_t* nmodes) = 0;
  virtual int adjoint(const void* phibar, const void* const* gbar, void* deltabar, double tol,
                      dgp_solve_info* info, double* rcbar) = 0;
  virtual int step_adjoint(const dgp_particles* start, double a, double da, dgp_particles* cot,
                           double* rcbar) = 0;
  virtual int zeldovich_vf_adjoint(const void* dl, const dgp_particles* cot, double* vfbar) = 0;
  virtual int zeldovich(const void* dl, double vf, dgp_particles* out) = 0;
  virtual int zeldovich_adjoint(const dgp_particles* cot, double vf, void* dlbar) = 0;
  virtual int pk_adjoint(const dgp_particles* pp, int nbins, const double* dldp, dgp_particles* cot) = 0;
  virtual int step(dgp_particles* parts, double a, double da, dgp_solve_info* info) = 0;
  virtual int step_host(dgp_particles* parts, double a, double da, dgp_solve_info* info) = 0;
  // One pm_step of every member of a class of realisations (this engine first; all
  // of the same type and stream), each kernel stage launched once for the class.
  virtual int step_class(EngineBase* const* members, int count, dgp_particles* parts, const double* a,
                         const double* da, dgp_solve_info* info) = 0;
  virtual int pk(const void* delta, int nbins, double* k, double* pk, int64_t* nmodes) = 0;
  virtual int bispec(const void* delta, double k1, double k2, int ntheta, const double* theta, double dk,
                     double* b, double* q) = 0;
  virtual void reset() = 0;
  virtual int get_solution(void* D) = 0;
  Profiler prof;
  std::vector<double> history;  // normalised residual of each iterate of the last solve
  cudaEvent_t sync_event = nullptr;  // set: host waits block on this event instead of spinning
  int y_threads = 256;          // y-pass CTA size, chosen at init by timing (tile autotuning)
  unsigned long long wait_ns = 2000000000ull;  // bound of every in-kernel wait
  int withhold = 0;             // test hook: the relaxation pass leaves its first copy unissued
  bool plane_pass = true;       // class solves of small meshes: the plane-resident Hessian pass
  bool xy_on = false;           // the Hessian x pass fused with the inverse y pass (opt-in: slower)
  bool xy_ok = false;           // set at init: the mesh and device allow the fused pass

  // Host wait for the work enqueued so far on the context's stream.
  cudaError_t wait_stream() {
    if (!sync_event) return cudaStreamSynchronize(stream);
    const cudaError_t e = cudaEventRecord(sync_event, stream);
    return e != cudaSuccess ? e : cudaEventSynchronize(sync_event);
  }
  int set_blocking(bool on) {
    if (on && !sync_event) {
      if (cudaEventCreateWithFlags(&sync_event, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
        sync_event = nullptr;
        return DGP_E_CUDA;
      }
    } else if (!on && sync_event) {
      cudaEventDestroy(sync_event);
      sync_event = nullptr;
    }
    return DGP_OK;
  }
};

#define DGP_CUDA(call)                          \
  do {                                          \
    if ((call) != cudaSuccess) return DGP_E_CUDA; \
  } while (0)
#define DGP_CHECK_LAUNCH()                                 \
  do {                                                     \
    if (cudaGetLastError() != cudaSuccess) return DGP_E_CUDA; \
  } while (0)

template <typename T, int N>
class Engine : public EngineBase {
  using V = vec2_t<T>;
  static constexpr int64_t M = (int64_t)N * N * N;
  static constexpr int64_t SPEC = (int64_t)(N / 2 + 1) * N * N;

  T* rD[3] = {nullptr, nullptr, nullptr};
  T* rS = nullptr;
  T* rH[6] = {};
  T* rRho = nullptr;
  T* rG[3] = {};
  V* sD = nullptr;
  V* sD2 = nullptr;             // ping-pong partner of sD during the iteration
  V* sDelta = nullptr;
  V* s6[6] = {};
  V* tw = nullptr;
  double* partials = nullptr;
  int nblocks = 0;              // grid of the grid-stride reductions
  int fblocks = 0;              // grid of the fused relaxation pass
  double* d_rstats = nullptr;   // [3][4]: sum|R|, sum D, nbad, nonfinite per D buffer
  double* d_misc = nullptr;     // [8]: sum rho, sum |S|, ...
  double* h_stats = nullptr;    // pinned host [8]
  double* pk_partials = nullptr;
  double* d_pk = nullptr;
  int pk_blocks = 0;
  int wcur = -1;                // buffer of the warm-start solution
  bool force_valid = false;
  double force_a = 0.0;
  const void* force_x = nullptr;
  int64_t force_np = -1;
  const void* force_host = nullptr;  // pm_step_host: host x array of the state the forces belong to
  RelaxMaps rmaps;              // tensor maps of s6[0..5] for the FP32 relaxation pass
  SolveCtl* d_ctl = nullptr;    // stop-rule state of the running solve
  SolveCtl* h_ctl = nullptr;    // pinned host copy
  double* d_hist = nullptr;     // [max_iter + 1] normalised residuals of the running solve
  int last_stop_it = -1;        // last iteration examined by the previous solve
  double last_nl_a = -1.0;      // scale factor of the last nonlinear solve
  static constexpr int kPatience = 10;  // iterations without a new minimum before stopping
  static constexpr int kChunk = 4;      // iterations enqueued per verdict after the first chunk
  // CUDA graph of two consecutive iterations (it odd, it + 1), one per buffer
  // holding the starting iterate; updated with each solve's parameters
  cudaGraphExec_t pair_exec[3] = {nullptr, nullptr, nullptr};
  // pm_step_host: three copy streams, so that several copy engines move the six arrays at once
  // (one array per stream), and the events that order them against the context's stream
  static constexpr int kCopyStreams = 3;
  cudaStream_t copy_streams[kCopyStreams] = {};
  cudaEvent_t copy_ev[kCopyStreams + 1] = {};  // [j]: stream j's copies in; [kCopyStreams]: a fence on stream
  // pm_step_host works on kHostChunks particle ranges, so that each range's kick overlaps the
  // copies of the others: per range, its copy in, its first kick, its second kick
  static constexpr int kHostChunks = 4;
  cudaEvent_t chunk_ev[3][kHostChunks] = {};
  T* hp[6] = {};                // device copies for pm_step_host
  int64_t hp_n = 0;
  // cell sort: key and permuted copies per particle, counts / starts / cursors per cell
  int* srt_key = nullptr;
  T* srt_tmp[6] = {};
  int64_t srt_np = 0;
  int* srt_cell = nullptr;      // [3][M]: count, start, cursor
  int* srt_sums = nullptr;
  int64_t nsteps = 0;           // pm_step calls since init / reset
  // adjoint workspace (allocated on the first dgp_solve_adjoint)
  T* aP = nullptr;              // [7][M]: H_f(D) lam for six pairs, then lam
  T* aF = nullptr;              // [4][M]: u, Q, Dbar, A phibar
  V* aS = nullptr;              // [7][SPEC]
  double* d_adj = nullptr;      // [12]: sum u, sum r, sum 1/diag, nonpositive diag, sum |res|, sum |g|,
                                // then the r_c terms: phibar and lam contractions, F . fbar, a dot product
  bool delta_nl = false;        // sDelta holds the spectrum of the last nonlinear solve's delta
  T* ap[6] = {};                // step adjoint: the recomputed particle state
  int64_t ap_n = 0;
  T* aFb = nullptr;             // [3][M] force-cotangent grids

 public:
  ~Engine() override {
    cudaStreamSynchronize(stream);
    for (int i = 0; i < 3; ++i) cudaFree(rD[i]);
    cudaFree(rS);
    for (int i = 0; i < 6; ++i) { cudaFree(rH[i]); cudaFree(s6[i]); cudaFree(hp[i]); }
    cudaFree(rRho);
    for (int i = 0; i < 3; ++i) cudaFree(rG[i]);
    cudaFree(sD); cudaFree(sD2); cudaFree(sDelta); cudaFree(tw);
    cudaFree(partials); cudaFree(d_rstats); cudaFree(d_misc);
    cudaFree(pk_partials); cudaFree(d_pk);
    cudaFree(srt_key); cudaFree(srt_cell); cudaFree(srt_sums);
    cudaFree(aP); cudaFree(aF); cudaFree(aS); cudaFree(d_adj); cudaFree(aFb);
    for (int i = 0; i < 6; ++i) cudaFree(ap[i]);
    cudaFree(d_ctl); cudaFree(d_hist); cudaFreeHost(h_ctl);
    for (int j = 0; j < kCopyStreams; ++j)
      if (copy_streams[j]) cudaStreamDestroy(copy_streams[j]);
    for (int j = 0; j <= kCopyStreams; ++j)
      if (copy_ev[j]) cudaEventDestroy(copy_ev[j]);
    for (auto& row : chunk_ev)
      for (cudaEvent_t& e : row)
        if (e) cudaEventDestroy(e);
    for (int i = 0; i < 3; ++i)
      if (pair_exec[i]) cudaGraphExecDestroy(pair_exec[i]);
    if (class_exec) cudaGraphExecDestroy(class_exec);
    set_blocking(false);
    for (int i = 0; i < 6; ++i) cudaFree(srt_tmp[i]);
    cudaFreeHost(h_stats);
  }

  int init() override {
    const size_t rb = sizeof(T) * M, sb = sizeof(V) * SPEC;
    for (int i = 0; i < 3; ++i) if (cudaMalloc(&rD[i], rb) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&rS, rb) != cudaSuccess) return DGP_E_NOMEM;
    for (int i = 0; i < 6; ++i) {
      if (cudaMalloc(&rH[i], rb) != cudaSuccess) return DGP_E_NOMEM;
      if (cudaMalloc(&s6[i], sb) != cudaSuccess) return DGP_E_NOMEM;
    }
    if (cudaMalloc(&rRho, rb) != cudaSuccess) return DGP_E_NOMEM;
    for (int i = 0; i < 3; ++i) if (cudaMalloc(&rG[i], rb) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&sD, sb) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&sD2, sb) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&sDelta, sb) != cudaSuccess) return DGP_E_NOMEM;
    nblocks = num_sms() * 4;
    if constexpr (sizeof(T) == 4) {
      if (relax_maps<N>(s6, &rmaps) != 0) return DGP_E_CUDA;
      fblocks = relax_tma_blocks<N>();
    } else {
      fblocks = fused_relax_blocks<T, N>();
    }
    const int pblocks = fblocks > nblocks ? fblocks : nblocks;
    if (cudaMalloc(&partials, sizeof(double) * 4 * pblocks) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&d_rstats, sizeof(double) * 12) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&d_misc, sizeof(double) * 8) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMallocHost(&h_stats, sizeof(double) * 8) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&d_ctl, sizeof(SolveCtl)) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMallocHost(&h_ctl, sizeof(SolveCtl)) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&d_hist, sizeof(double) * ((size_t)p.max_iter + 1)) != cudaSuccess) return DGP_E_NOMEM;
    pk_blocks = x_pass_blocks<T, N>();
    if (cudaMalloc(&pk_partials, sizeof(double) * 4 * (N / 2) * (size_t)pk_blocks) != cudaSuccess) return DGP_E_NOMEM;
    if (cudaMalloc(&d_pk, sizeof(double) * 4 * (N / 2)) != cudaSuccess) return DGP_E_NOMEM;
    // twiddles W_N^t = exp(-2 pi i t / N), computed in FP64 and rounded once
    // and the two phase tables of the four-step split N = N1 * N2 (see fft_core.cuh)
    constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
    std::vector<V> htw(3 * N);
    auto w = [](int t) {
      const double ang = 2.0 * M_PI * (double)(t % N) / (double)N;
      V r;
      r.x = (T)cos(ang);
      r.y = (T)(-sin(ang));
      return r;
    };
    for (int t = 0; t < N; ++t) htw[t] = w(t);
    for (int k1 = 0; k1 < N1; ++k1)
      for (int j2 = 0; j2 < N2; ++j2) htw[N + k1 * N2 + j2] = w(j2 * k1);
    for (int m1 = 0; m1 < N2; ++m1)
      for (int k1 = 0; k1 < N1; ++k1) htw[2 * N + m1 * N1 + k1] = w(k1 * m1);
    if (cudaMalloc(&tw, sizeof(V) * 3 * N) != cudaSuccess) return DGP_E_NOMEM;
    DGP_CUDA(cudaMemcpy(tw, htw.data(), sizeof(V) * 3 * N, cudaMemcpyHostToDevice));
    DGP_CUDA(cudaMemset(d_rstats, 0, sizeof(double) * 12));
    xy_ok = sizeof(T) == 4 && (N == 128 || N == 256) && xy_hessian_available(N);
    return tune_tiles();
  }

  // Tile autotuning: time the y pass's CTA sizes (128, 256, 512 threads; 128 / N1,
  // ... rows per CTA) on this context's own spectrum buffers, six inverse
  // transforms as in a relaxation iteration, and keep the fastest.  The results
  // do not depend on the choice (every row's arithmetic is the same).
  int tune_tiles() {
    for (int i = 0; i < 6; ++i) DGP_CUDA(cudaMemsetAsync(s6[i], 0, sizeof(V) * SPEC, stream));
    cudaEvent_t e0, e1;
    DGP_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      return DGP_E_CUDA;
    }
    const int cand[3] = {128, 256, 512};
    float best_ms = 1e30f;
    int best = 256, rc = DGP_OK;
    for (int c = 0; c < 3 && rc == DGP_OK; ++c) {
      launch_fft_y<T, N>(fs(s6, 6), 6, true, tw, stream, nullptr, cand[c]);  // warm-up
      cudaEventRecord(e0, stream);
      for (int r = 0; r < 3; ++r) launch_fft_y<T, N>(fs(s6, 6), 6, true, tw, stream, nullptr, cand[c]);
      cudaEventRecord(e1, stream);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
          cudaGetLastError() != cudaSuccess) {
        rc = DGP_E_CUDA;
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = cand[c];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    y_threads = best;
    return rc;
  }

  void reset() override {
    wcur = -1;
    last_nl_a = -1.0;
    last_stop_it = -1;
    force_valid = false;
    force_host = nullptr;
    nsteps = 0;
  }

  int get_solution(void* D) override {
    if (!D) return DGP_E_INVALID;
    if (wcur < 0) return DGP_E_STATE;
    // D - mean(D): the mean was reduced in FP64 when the buffer was produced
    ZPrologue pro{d_rstats + 4 * wcur + 1, 1.0 / (double)M, 2};
    prof.run(KK_MISC, 2 * RB, stream, [&] { launch_sub_mean<T>(rD[wcur], (T*)D, M, pro.mean_src, stream); });
    DGP_CHECK_LAUNCH();
    return DGP_OK;
  }

 private:
  KParams kparams(const Coef& c, int gravity) const {
    KParams kp;
    kp.box = p.box;
    kp.inv_m = 1.0 / (double)M;
    kp.kbar_fac = cosmo.c_over_H0 / (c.a * c.E);
    kp.local_only = p.local_only;
    kp.eta = c.eta; kp.alpha = c.alpha; kp.beta = c.beta; kp.s = c.s; kp.c2 = c.c2; kp.c3 = c.c3;
    kp.aE = c.a * c.E; kp.q = c.q; kp.rc_H0 = p.rc_H0; kp.a = c.a;
    // the phi operation takes the nonlinear form (with a D spectrum) for the
    // nonlinear and the spherical modes
    kp.gravity = gravity == DGP_GRAVITY_SPH ? DGP_GRAVITY_NL : gravity;
    const double kf = 2.0 * M_PI / p.box;
    kp.kf_f = (float)kf;
    kp.inv_m_f = (float)kp.inv_m;
    kp.kbkf_f = (float)(kp.kbar_fac * kf);
    kp.s_f = (float)c.s; kp.beta_f = (float)c.beta; kp.alpha_f = (float)c.alpha; kp.c2_f = (float)c.c2;
    kp.c3_f = (float)c.c3; kp.inv_eta_f = (float)(1.0 / c.eta); kp.half_inv_eta_f = (float)(0.5 / c.eta);
    kp.om15_f = (float)(1.5 * (c.eta - 1.0) / c.eta); kp.aE2_f = (float)(kp.aE * kp.aE);
    return kp;
  }

  RelaxParams relax_params(const Coef& c) const {
    RelaxParams rp;
    rp.alpha = c.alpha; rp.w = p.w; rp.c2 = c.c2; rp.inv_m = 1.0 / (double)M;
    auto split = [](double v, float& hi, float& lo) { hi = (float)v; lo = (float)(v - (double)hi); };
    split(c.alpha, rp.alpha_hi, rp.alpha_lo);
    split(c.c2, rp.c2_hi, rp.c2_lo);
    split(4.0 * (1.0 - p.w), rp.four_omw_hi, rp.four_omw_lo);
    rp.omw = (float)(1.0 - p.w);
    rp.two_omw = (float)(2.0 * (1.0 - p.w));
    rp.alpha_f = (float)c.alpha;
    rp.bad_bp_f = (float)(-c.alpha * c.alpha / (4.0 * (1.0 - p.w)));
    return rp;
  }
  int arith_mode() const {
    return p.precision == DGP_FP32         ? ARITH_F32
           : p.precision == DGP_MIXED_EFT  ? ARITH_EFT
           : p.precision == DGP_MIXED_F32R ? ARITH_M32
                                           : ARITH_F64;
  }

  static FieldSet<T> fs(V* const* ptrs, int n) {
    FieldSet<T> f;
    for (int i = 0; i < kMaxFields; ++i) f.p[i] = i < n ? ptrs[i] : nullptr;
    return f;
  }

  // real field -> S2 (z and y forward transforms)
  static constexpr double RB = (double)sizeof(T) * M;      // one real field
  static constexpr double SB = (double)sizeof(V) * SPEC;   // one half spectrum

  int forward_zy(const T* in, V* out, ZPrologue pro) {
    prof.run(KK_Z_R2C, RB + SB, stream, [&] { launch_fft_z_r2c<T, N>(in, 0, out, 0, 1, pro, tw, stream); });
    V* o[1] = {out};
    prof.run(KK_Y, 2 * SB, stream, [&] { launch_fft_y<T, N>(fs(o, 1), 1, false, tw, stream, nullptr, y_threads); });
    DGP_CHECK_LAUNCH();
    return DGP_OK;
  }

  // x-op outputs (already in s6[0..n)) -> y inverse -> z inverse into real fields
  int inverse_yz(V* const* spec, T* const* out, int n) {
    prof.run(KK_Y, 2 * SB * n, stream, [&] { launch_fft_y<T, N>(fs(spec, n), n, true, tw, stream, nullptr, y_threads); });
    prof.run(KK_Z_C2R, (RB + SB) * n, stream, [&] { launch_fft_z_c2r<T, N>(fs(spec, n), out, n, tw, stream); });
    DGP_CHECK_LAUNCH();
    return DGP_OK;
  }

  int reduce_sum(const T* a, bool absval, double* out) {
    prof.run(KK_REDUCE, RB, stream, [&] { launch_sum<T>(a, M, absval, partials, nblocks, stream); });
    prof.run(KK_REDUCE, 8.0 * nblocks, stream, [&] { launch_finalize(partials, nblocks, 1, out, stream); });
    DGP_CHECK_LAUNCH();
    return DGP_OK;
  }

  int fetch(const double* dsrc, int n) {
    DGP_CUDA(cudaMemcpyAsync(h_stats, dsrc, sizeof(double) * n, cudaMemcpyDeviceToHost, stream));
    DGP_CUDA(wait_stream());
    return DGP_OK;
  }

  // Field solve at scale factor a.  delta is a density contrast, or (from_rho)
  // a CIC mass mesh turned into rho / rho_bar - 1 on the fly.  Outputs:
  // phi (may be null) and forces g (all null or all set).
  int solve_impl(double a, const T* src, bool from_rho, T* phi, T* g0, T* g1, T* g2, double tol,
                 dgp_solve_info* info) {
    int rc;
    // Sec. III.D: the linearised DGP equation before a_nonlinear
    const int grav = (p.gravity == DGP_GRAVITY_NL && a < p.a_nonlinear) ? DGP_GRAVITY_LDGP : p.gravity;
    const Coef c = coefficients(a, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, grav);
    ZPrologue pro{nullptr, 1.0 / (double)M, 0};
    if (from_rho) {
      if ((rc = reduce_sum(src, false, d_misc + 0))) return rc;
      pro.mean_src = d_misc + 0;
      pro.kind = 1;
    }
    if ((rc = forward_zy(src, sDelta, pro))) return rc;
    delta_nl = grav == DGP_GRAVITY_NL;
    dgp_solve_info inf;
    memset(&inf, 0, sizeof(inf));
    V* sDphi = sD;  // spectrum of the accepted D for the phi operation
    int accepted = -1;
    int status = DGP_OK;

    if (grav == DGP_GRAVITY_SPH) {
      // one w = 1/3 update from C = 0 (Eq. FullDGP2sph): source, pointwise root
      prof.run(KK_X_OTHER, SB * 2, stream, [&] {
        launch_fft_x_op<T, N>(XOP_SOURCE, sDelta, nullptr, fs(s6, 1), 0, kp, nullptr, 0, 0, 0, tw, stream);
      });
      T* outs[1] = {rS};
      if ((rc = inverse_yz(s6, outs, 1))) return rc;
      prof.run(KK_RELAX, 2 * RB, stream,
               [&] { launch_sph_update<T>(rS, rH[0], M, c.alpha, partials, nblocks, stream); });
      prof.run(KK_REDUCE, 8.0 * nblocks, stream, [&] { launch_finalize(partials, nblocks, 1, d_misc + 3, stream); });
      DGP_CHECK_LAUNCH();
      if ((rc = forward_zy(rH[0], sD, ZPrologue{nullptr, 0.0, 0}))) return rc;
      if ((rc = fetch(d_misc + 3, 1))) return rc;
      sDphi = sD;
      inf.iters = 1;
      inf.bad_fraction = h_stats[0] / (double)M;
      inf.status = DGP_OK;
    }

    if (grav == DGP_GRAVITY_NL) {
      last_nl_a = a;
      const bool need_lin = wcur < 0;
      prof.run(KK_X_OTHER, SB * (need_lin ? 3 : 2), stream, [&] {
        launch_fft_x_op<T, N>(need_lin ? XOP_SOURCE_LIN : XOP_SOURCE, sDelta, nullptr, fs(s6, 2), 0, kp, nullptr, 0,
                              0, 0, tw, stream);
      });
      const int j0 = need_lin ? 0 : wcur;
      T* outs[2] = {rS, rD[j0]};
      if ((rc = inverse_yz(s6, outs, need_lin ? 2 : 1))) return rc;
      // eps = <|S|> (Eq. normres) is read by the controller at the first iteration
      if ((rc = reduce_sum(rS, true, d_misc + 1))) return rc;
      if (need_lin && (rc = reduce_sum(rD[j0], false, d_rstats + 4 * j0 + 1))) return rc;

      const RelaxParams rp = relax_params(c);
      const int arith = arith_mode();

      // Buffers: the starting iterate stays in rD[j0]; iteration it >= 1 reads
      // the previous output, and the outputs alternate between the other two.
      // The y-transformed spectrum of iteration it's input alternates sD / sD2.
      int pb[2], npb = 0;
      for (int b = 0; b < 3; ++b)
        if (b != j0) pb[npb++] = b;
      auto in_buf = [&](int it) { return it == 0 ? j0 : pb[(it - 1) & 1]; };
      auto out_buf = [&](int it) { return pb[it & 1]; };
      auto spec_in = [&](int it) { return (it & 1) ? sD2 : sD; };
      auto spec_out = [&](int it) { return (it & 1) ? sD : sD2; };
      const int* skip = &d_ctl->done;
      const bool xy = xy_ok && xy_on;  // Hessian spectra and their inverse y in one launch
      // One iteration: Hessian spectra, inverse y, fused z pass + update,
      // statistics, (stop rules), forward y of the new iterate.  With control,
      // every kernel returns at entry once the controller has stopped the solve.
      auto enqueue = [&](int it, bool control) -> int {
        const int* sk = control ? skip : nullptr;
        const int ib = in_buf(it), ob = out_buf(it);
        // the first iteration and replays always run; later ones may return at entry
        const double sure = (it == 0 || !control) ? 1.0 : -1.0;
        if (xy) {
          prof.run_it(KK_X_HESSIAN, 0, sure * 7 * SB, stream,
                      [&] { launch_xy_hessian<T, N>(spec_in(it), fs(s6, 6), kp, tw, stream, sk); });
        } else {
          prof.run_it(KK_X_HESSIAN, 0, sure * 7 * SB, stream, [&] {
            launch_fft_x_op<T, N>(XOP_HESSIAN, spec_in(it), nullptr, fs(s6, 6), 0, kp, nullptr, 0, 0, 0, tw, stream,
                                  sk);
          });
          prof.run_it(KK_Y, 0, sure * 12 * SB, stream,
                      [&] { launch_fft_y<T, N>(fs(s6, 6), 6, true, tw, stream, sk, y_threads); });
        }
        prof.run_it(KK_RELAX, 0, sure * (7 * SB + 3 * RB), stream, [&] {
          if constexpr (sizeof(T) == 4)
            launch_relax_tma<N>(arith, rmaps, rD[ib], d_rstats + 4 * ib + 1, rS, rD[ob], spec_out(it), rp, partials,
                                tw, stream, sk, &d_ctl->fault, wait_ns, withhold);
          else
            launch_fused_relax<T, N>(arith, s6, rD[ib], d_rstats + 4 * ib + 1, rS, rD[ob], spec_out(it), rp,
                                     partials, tw, stream, sk);
        });
        // the iteration's statistics: with control, summed by one extra CTA of the forward y
        // pass of the new iterate, which also applies the stop rules
        if (!control)
          prof.run_it(KK_REDUCE, 0, sure * 32.0 * fblocks, stream,
                      [&] { launch_finalize(partials, fblocks, 4, d_rstats + 4 * ob, stream, sk); });
        prof.run_it(KK_Y, 0, sure * (2 * SB + (control ? 32.0 * fblocks : 0.0)), stream, [&] {
          V* o[1] = {spec_out(it)};
          const YControl yc{partials, fblocks, d_rstats + 4 * ob, d_ctl, d_misc + 1, d_hist, p.max_iter,
                            kPatience, tol, 1.0 / (double)M};
          launch_fft_y<T, N>(fs(o, 1), 1, false, tw, stream, sk, y_threads, control ? &yc : nullptr);
        });
        DGP_CHECK_LAUNCH();
        return DGP_OK;
      };
      auto credit = [&](int iters, int yfwd) {
        prof.credit(KK_X_HESSIAN, 7 * SB * iters);
        prof.credit(KK_Y, (xy ? 0.0 : 12 * SB * iters) + (2 * SB + 32.0 * fblocks) * yfwd);
        prof.credit(KK_RELAX, (7 * SB + 3 * RB) * iters);
      };

      if ((rc = forward_zy(rD[j0], sD, ZPrologue{nullptr, 0.0, 0}))) return rc;
      DGP_CUDA(cudaMemsetAsync(d_ctl, 0, sizeof(SolveCtl), stream));
      // Iterations after the first run as a CUDA graph of two iterations (the
      // buffers alternate with period two) unless every launch is being timed.
      // (Stream capture is not available on the legacy default stream; a
      // capture that fails leaves the iterations to direct launches.)
      bool graphs = (prof.timing == 0 || prof.sampled) && stream != nullptr && stream != cudaStreamLegacy &&
                    stream != cudaStreamPerThread;
      if (graphs) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
          cudaGetLastError();
          graphs = false;
        } else {
          prof.capturing = true;
          const int r1 = enqueue(1, true), r2 = r1 ? r1 : enqueue(2, true);
          prof.capturing = false;
          const cudaError_t e = cudaStreamEndCapture(stream, &g);
          cudaGraphExec_t& ex = pair_exec[j0];
          if (r1 || r2 || e != cudaSuccess || !g) {
            graphs = false;
          } else {
            if (ex) {
              cudaGraphExecUpdateResultInfo ui;
              if (cudaGraphExecUpdate(ex, g, &ui) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(ex);
                ex = nullptr;
              }
            }
            if (!ex && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
              ex = nullptr;
              graphs = false;
            }
          }
          if (g) cudaGraphDestroy(g);
          if (!graphs) cudaGetLastError();
        }
      }
      // Iterations are enqueued in chunks and the controller's verdict is read
      // once per chunk; the first chunk covers the previous solve's length.
      int it = 0;
      int chunk = last_stop_it >= 0 ? last_stop_it + 2 : 4;
      while (true) {
        const int end = std::min(it + chunk, p.max_iter + 1);
        while (it < end) {
          if (graphs && it > 0 && (it & 1)) {
            DGP_CUDA(cudaGraphLaunch(pair_exec[j0], stream));
            prof.count(KK_X_HESSIAN, 2);
            prof.count(KK_Y, xy ? 2 : 4);
            prof.count(KK_RELAX, 2);
            it += 2;
          } else {
            if ((rc = enqueue(it, true))) return rc;
            ++it;
          }
        }
        DGP_CUDA(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, stream));
        DGP_CUDA(wait_stream());
        if (h_ctl->done || it > p.max_iter) break;
        chunk = kChunk;
      }
      const SolveCtl st = *h_ctl;
      if (!st.done) return DGP_E_STATE;  // the controller stops at it = max_iter at the latest
      const int s_it = st.stop_it;
      credit(s_it + 1, s_it);
      history.assign(s_it + 1, 0.0);
      DGP_CUDA(cudaMemcpyAsync(history.data(), d_hist, sizeof(double) * (s_it + 1), cudaMemcpyDeviceToHost, stream));
      DGP_CUDA(wait_stream());
      if (st.status == CTL_FAULT) return DGP_E_TIMEOUT;
      if (st.status == CTL_NONFINITE) return DGP_E_NONFINITE;
      last_stop_it = s_it;
      inf.eps = st.eps;
      const int best_it = st.best_it;
      if (best_it == s_it) {
        // the input of the last examined iteration: its buffer and spectrum are intact
        accepted = in_buf(s_it);
        sDphi = spec_in(s_it);
      } else {
        // an earlier iterate: the start is intact; a later one is regenerated by
        // replaying the (deterministic) iterations that produced it
        if (best_it > 0) {
          if ((rc = forward_zy(rD[j0], sD, ZPrologue{nullptr, 0.0, 0}))) return rc;
          for (int k = 0; k < best_it; ++k)
            if ((rc = enqueue(k, false))) return rc;
          credit(best_it, best_it);
        }
        accepted = in_buf(best_it);
        if ((rc = forward_zy(rD[accepted], sD, ZPrologue{nullptr, 0.0, 0}))) return rc;
        sDphi = sD;
        if (best_it > 0) {  // the replayed iterations' waits
          DGP_CUDA(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, stream));
          DGP_CUDA(wait_stream());
          if (h_ctl->fault) return DGP_E_TIMEOUT;
        }
      }
      inf.iters = best_it;
      inf.norm_res = st.rbest;
      inf.min_norm_res = st.rbest;
      inf.bad_fraction = st.last_bad / (double)M;
      status = st.status == CTL_CONVERGED ? DGP_OK : DGP_E_NOT_CONVERGED;
      inf.status = status;
      wcur = accepted;
    }

    // phi and forces (Eq. FullDGP1; g = -grad phi)
    V* outs[4] = {s6[0], s6[1], s6[2], s6[3]};
    int mask = 0;
    if (phi) mask |= 1;
    if (g0) mask |= 14;
    if (mask) {
      const int nin = (grav == DGP_GRAVITY_NL || grav == DGP_GRAVITY_SPH) ? 2 : 1;
      prof.run(KK_X_OTHER, SB * (nin + __builtin_popcount(mask)), stream, [&] {
        launch_fft_x_op<T, N>(XOP_PHI_FORCE, sDelta, sDphi, fs(outs, 4), mask, kp, nullptr, 0, 0, 0, tw, stream);
      });
      V* sp[4];
      T* rp_[4];
      int n = 0;
      if (phi) { sp[n] = s6[0]; rp_[n] = phi; ++n; }
      if (g0) {
        sp[n] = s6[1]; rp_[n] = g0; ++n;
        sp[n] = s6[2]; rp_[n] = g1; ++n;
        sp[n] = s6[3]; rp_[n] = g2; ++n;
      }
      if ((rc = inverse_yz(sp, rp_, n))) return rc;
    }
    if (info) {
      *info = inf;
      DGP_CUDA(wait_stream());
    }
    return status;
  }

  CicParams cic() const {
    CicParams cp;
    cp.n = N;
    const double inv = (double)N / p.box;
    cp.inv_d = inv;
    cp.inv_d_hi = (float)inv;
    cp.inv_d_lo = (float)(inv - (double)cp.inv_d_hi);
    cp.box = p.box;
    cp.box_f = (float)p.box;
    cp.inv_box_f = (float)(1.0 / p.box);
    return cp;
  }

  static bool valid_parts(const dgp_particles* pp) {
    if (!pp || pp->n < 0) return false;
    if (pp->n == 0) return true;
    return pp->x && pp->y && pp->z && pp->px && pp->py && pp->pz;
  }

  // Counting sort of the particles by the cell of their lower CIC corner,
  // in place (through the context's copies); cell_start (device, M + 1) optional.
  int sort_impl(const dgp_particles* pp, int* cell_start) {
    const int64_t np = pp->n;
    if (np > 0x7fffffff) return DGP_E_INVALID;
    if (!srt_cell) {
      if (cudaMalloc(&srt_cell, sizeof(int) * 3 * M) != cudaSuccess) return DGP_E_NOMEM;
      if (cudaMalloc(&srt_sums, sizeof(int) * sort_scan_blocks(M)) != cudaSuccess) return DGP_E_NOMEM;
    }
    if (np > srt_np) {
      DGP_CUDA(wait_stream());
      cudaFree(srt_key);
      srt_key = nullptr;
      for (int i = 0; i < 6; ++i) { cudaFree(srt_tmp[i]); srt_tmp[i] = nullptr; }
      srt_np = 0;
      if (cudaMalloc(&srt_key, sizeof(int) * np) != cudaSuccess) return DGP_E_NOMEM;
      for (int i = 0; i < 6; ++i)
        if (cudaMalloc(&srt_tmp[i], sizeof(T) * np) != cudaSuccess) return DGP_E_NOMEM;
      srt_np = np;
    }
    ParticleSet<T> in{{(T*)pp->x, (T*)pp->y, (T*)pp->z, (T*)pp->px, (T*)pp->py, (T*)pp->pz}};
    ParticleSet<T> out{{srt_tmp[0], srt_tmp[1], srt_tmp[2], srt_tmp[3], srt_tmp[4], srt_tmp[5]}};
    const SortWork w{srt_key, srt_cell, srt_cell + M, srt_cell + 2 * M, srt_sums};
    const double pb = sizeof(T) * 15.0 + 8.0;  // read x (3), key out/in, read 6, write 6
    prof.run(KK_SORT, pb * np + 16.0 * M, stream, [&] { launch_cell_sort<T>(in, np, cic(), w, out, stream); });
    DGP_CHECK_LAUNCH();
    for (int i = 0; i < 6 && np > 0; ++i)
      DGP_CUDA(cudaMemcpyAsync(in.p[i], out.p[i], sizeof(T) * np, cudaMemcpyDeviceToDevice, stream));
    if (cell_start) {
      const int total = (int)np;
      DGP_CUDA(cudaMemcpyAsync(cell_start, w.start, sizeof(int) * M, cudaMemcpyDeviceToDevice, stream));
      DGP_CUDA(cudaMemcpyAsync(cell_start + M, &total, sizeof(int), cudaMemcpyHostToDevice, stream));
      DGP_CUDA(wait_stream());
    }
    return DGP_OK;
  }

  int forces_at(const dgp_particles* pp, double a, dgp_solve_info* info) {
    prof.run(KK_MISC, RB, stream, [&] { launch_fill<T>(rRho, M, (T)0, stream); });
    prof.run(KK_DEPOSIT, 3.0 * sizeof(T) * pp->n + RB, stream, [&] {
      launch_cic_deposit_warp<T>((const T*)pp->x, (const T*)pp->y, (const T*)pp->z, pp->n, rRho, cic(), stream);
    });
    DGP_CHECK_LAUNCH();
    const int rc = solve_impl(a, rRho, true, nullptr, rG[0], rG[1], rG[2], p.tol, info);
    if (rc != DGP_OK && rc != DGP_E_NOT_CONVERGED) return rc;
    force_valid = true;
    force_a = a;
    force_x = pp->x;
    force_np = pp->n;
    return DGP_OK;
  }

 public:
  int solve(double a, const void* delta, void* phi, void* gx, void* gy, void* gz, double tol,
            dgp_solve_info* info) override {
    force_valid = false;
    return solve_impl(a, (const T*)delta, false, (T*)phi, (T*)gx, (T*)gy, (T*)gz, tol, info);
  }

  int sort(dgp_particles* pp, int* cell_start) override {
    if (!valid_parts(pp)) return DGP_E_INVALID;
    return sort_impl(pp, cell_start);
  }

  int deposit(const dgp_particles* pp, void* delta) override {
    if (!valid_parts(pp) || !delta) return DGP_E_INVALID;
    if (pp->n == 0) return DGP_E_INVALID;
    prof.run(KK_MISC, RB, stream, [&] { launch_fill<T>(rRho, M, (T)0, stream); });
    prof.run(KK_DEPOSIT, 3.0 * sizeof(T) * pp->n + RB, stream, [&] {
      launch_cic_deposit_warp<T>((const T*)pp->x, (const T*)pp->y, (const T*)pp->z, pp->n, rRho, cic(), stream);
    });
    int rc;
    if ((rc = reduce_sum(rRho, false, d_misc + 0))) return rc;
    prof.run(KK_MISC, 2 * RB, stream, [&] { launch_density_contrast<T>(rRho, (T*)delta, M, d_misc + 0, stream); });
    DGP_CHECK_LAUNCH();
    return DGP_OK;
  }

  // ---------------------------------------------------------------- classes of realisations
  // pm_step of every member of a class (same mesh, precision and stream; the nonlinear
  // mode), each kernel stage launched once for all members with the member on the grid's
  // z (or y) index.  Every member ends in the state its own pm_step would leave it in:
  // the same iterates, stop rules, warm start and reused end-of-step force.
  cudaGraphExec_t class_exec = nullptr;  // the class's two-iteration graph (held by its first member)

  int step_class(EngineBase* const* members, int count, dgp_particles* parts, const double* a, const double* da,
                 dgp_solve_info* info) override {
    if constexpr (sizeof(T) != 4 || N > 128) {
      return DGP_E_INVALID;
    } else {
      if (count < 1 || count > kBatchMax || !members || members[0] != this || !parts || !a || !da)
        return DGP_E_INVALID;
      std::vector<Engine*> E(count);
      std::vector<int> all(count), start;
      for (int r = 0; r < count; ++r) {
        Engine* e = dynamic_cast<Engine*>(members[r]);
        if (!e || e->stream != stream || e->p.gravity != DGP_GRAVITY_NL || e->p.local_only || e->p.a_nonlinear > 0.0 ||
            e->p.precision != p.precision)
          return DGP_E_INVALID;
        dgp_particles* pp = &parts[r];
        if (!valid_parts(pp) || pp->n == 0) return DGP_E_INVALID;
        if (!(a[r] > 0.0) || !(da[r] > 0.0) || !isfinite(a[r] + da[r])) return DGP_E_INVALID;
        E[r] = e;
        all[r] = r;
        e->force_host = nullptr;
        const bool reuse = e->force_valid && e->force_x == pp->x && e->force_np == pp->n &&
                           fabs(e->force_a - a[r]) <= 1e-12 * a[r];
        if (!reuse) start.push_back(r);
      }
      int rc;
      if (!start.empty() && (rc = class_forces(E, start, parts, a, nullptr))) return rc;
      std::vector<double> a1(count), k2(count);
      GatherArgs g[kBatchMax];
      for (int r = 0; r < count; ++r) {
        Engine* e = E[r];
        const double om = e->cosmo.omega_m0, rcH = e->p.rc_H0;
        a1[r] = a[r] + da[r];
        const double ah = exp(0.5 * (log(a[r]) + log(a1[r])));
        const dgp_particles* pp = &parts[r];
        g[r] = GatherArgs{{(float*)pp->x, (float*)pp->y, (float*)pp->z, (float*)pp->px, (float*)pp->py, (float*)pp->pz},
                          pp->n, {e->rG[0], e->rG[1], e->rG[2]}, e->cic(),
                          (float)time_integral(a[r], ah, om, rcH, 0), (float)time_integral(a[r], a1[r], om, rcH, 2), 1};
        k2[r] = time_integral(ah, a1[r], om, rcH, 0);
      }
      double gb = 0.0;  // gather bytes of the class (positions and momenta, the three force meshes)
      for (int r = 0; r < count; ++r) gb += 12.0 * sizeof(T) * parts[r].n + 3 * RB;
      prof.run(KK_GATHER, gb, stream, [&] { launch_gather_kick_batch(g, count, stream); });
      DGP_CHECK_LAUNCH();
      for (int r = 0; r < count; ++r) {
        Engine* e = E[r];
        ++e->nsteps;
        if (e->p.sort_every > 0 && e->nsteps % e->p.sort_every == 0 && (rc = e->sort_impl(&parts[r], nullptr)))
          return rc;
      }
      if ((rc = class_forces(E, all, parts, a1.data(), info))) return rc;
      for (int r = 0; r < count; ++r) {
        g[r].kick = (float)k2[r];
        g[r].drift = 0.f;
        g[r].do_drift = 0;
      }
      double gb2 = 0.0;
      for (int r = 0; r < count; ++r) gb2 += 9.0 * sizeof(T) * parts[r].n + 3 * RB;
      prof.run(KK_GATHER, gb2, stream, [&] { launch_gather_kick_batch(g, count, stream); });
      DGP_CHECK_LAUNCH();
      return DGP_OK;
    }
  }

 private:
  // Deposit and field solve at a[r] for the members in sub; forces in each member's rG.
  static int class_forces(std::vector<Engine*>& E, const std::vector<int>& sub, const dgp_particles* parts,
                          const double* a, dgp_solve_info* info) {
    const int n = (int)sub.size();
    const cudaStream_t s = E[0]->stream;
    float* rho[kBatchMax];
    DepositArgs<T> dep[kBatchMax];
    for (int k = 0; k < n; ++k) {
      Engine* e = E[sub[k]];
      const dgp_particles* pp = &parts[sub[k]];
      rho[k] = (float*)e->rRho;
      dep[k] = DepositArgs<T>{(const T*)pp->x, (const T*)pp->y, (const T*)pp->z, pp->n, e->rRho, e->cic()};
    }
    Profiler& pf = E[0]->prof;  // the class's kernels are accounted on its first member
    double db = 0.0;
    for (int k = 0; k < n; ++k) db += 3.0 * sizeof(T) * parts[sub[k]].n + RB;
    pf.run(KK_MISC, n * RB, s, [&] { launch_zero_batch(rho, M, n, s); });
    pf.run(KK_DEPOSIT, db, s, [&] { launch_cic_deposit_batch<T>(dep, n, s); });
    if (cudaGetLastError() != cudaSuccess) return DGP_E_CUDA;
    const int rc = class_solve(E, sub, a, info);
    if (rc != DGP_OK && rc != DGP_E_NOT_CONVERGED) return rc;
    for (int k = 0; k < n; ++k) {
      Engine* e = E[sub[k]];
      e->force_valid = true;
      e->force_a = a[sub[k]];
      e->force_x = parts[sub[k]].x;
      e->force_np = parts[sub[k]].n;
    }
    return DGP_OK;
  }

  // Batched one-field sums of field(k) into out(k).
  template <class FA, class FO>
  static void class_sum(Profiler& pf, std::vector<Engine*>& S, bool absval, FA field, FO out) {
    const int n = (int)S.size();
    const float* src[kBatchMax];
    double* parts[kBatchMax];
    double* dst[kBatchMax];
    for (int k = 0; k < n; ++k) {
      src[k] = (const float*)field(k);
      parts[k] = S[k]->partials;
      dst[k] = out(k);
    }
    pf.run(KK_REDUCE, n * RB, S[0]->stream,
           [&] { launch_sum_batch(src, M, absval, parts, S[0]->nblocks, dst, n, S[0]->stream); });
  }

  // The field solve of solve_impl (nonlinear mode, from a CIC mass mesh) for the members in sub.
  static int class_solve(std::vector<Engine*>& E, const std::vector<int>& sub, const double* a,
                         dgp_solve_info* info) {
    const int n = (int)sub.size();
    std::vector<Engine*> S(n);
    for (int k = 0; k < n; ++k) S[k] = E[sub[k]];
    Engine* e0 = S[0];
    const cudaStream_t st = e0->stream;
    const V* tw = e0->tw;
    const int yt = e0->y_threads;
    std::vector<KParams> kp(n);
    std::vector<RelaxParams> rp(n);
    std::vector<int> j0(n), pb0(n), pb1(n);
    for (int k = 0; k < n; ++k) {
      Engine* e = S[k];
      const Coef c = coefficients(a[sub[k]], e->cosmo.omega_m0, e->p.rc_H0);
      kp[k] = e->kparams(c, DGP_GRAVITY_NL);
      rp[k] = e->relax_params(c);
      e->delta_nl = true;
      e->last_nl_a = a[sub[k]];
    }
    auto check = [] { return cudaGetLastError() == cudaSuccess ? DGP_OK : DGP_E_CUDA; };
    Profiler& pf = E[0]->prof;  // the class's kernels are accounted on its first member
    const double nS = n * SB, nR = n * RB;
    // density contrast from the mass mesh, its z and y transforms
    class_sum(pf, S, false, [&](int k) { return S[k]->rRho; }, [&](int k) { return S[k]->d_misc + 0; });
    {
      const float* in[kBatchMax];
      V* out[kBatchMax];
      ZPrologue pro[kBatchMax];
      FieldSet<T> f[kBatchMax];
      for (int k = 0; k < n; ++k) {
        in[k] = S[k]->rRho;
        out[k] = S[k]->sDelta;
        pro[k] = ZPrologue{S[k]->d_misc + 0, 1.0 / (double)M, 1};
        f[k] = fs(&S[k]->sDelta, 1);
      }
      pf.run(KK_Z_R2C, nR + nS, st, [&] { launch_fft_z_r2c_batch<T, N>(in, out, pro, n, tw, st); });
      pf.run(KK_Y, 2 * nS, st, [&] { launch_fft_y_batch<T, N>(f, nullptr, nullptr, n, 1, false, tw, st, yt); });
    }
    // source S; the linear start D_lin for members without a warm start
    for (int lin = 0; lin < 2; ++lin) {
      XReal<T> xr[kBatchMax];
      FieldSet<T> fi[kBatchMax], fo[kBatchMax];
      int m = 0;
      for (int k = 0; k < n; ++k) {
        Engine* e = S[k];
        if ((e->wcur < 0) != (lin == 1)) continue;
        j0[k] = lin ? 0 : e->wcur;
        xr[m] = XReal<T>{e->sDelta, nullptr, fs(e->s6, lin ? 2 : 1), 0, kp[k], nullptr};
        fi[m] = fs(e->s6, lin ? 2 : 1);
        T* outs[2] = {e->rS, e->rD[j0[k]]};
        for (int i = 0; i < kMaxFields; ++i) fo[m].p[i] = i < (lin ? 2 : 1) ? reinterpret_cast<V*>(outs[i]) : nullptr;
        ++m;
      }
      if (!m) continue;
      const double nf = m * (lin ? 2 : 1);
      pf.run(KK_X_OTHER, m * SB + nf * SB, st,
             [&] { launch_fft_x_batch<T, N>(lin ? XOP_SOURCE_LIN : XOP_SOURCE, xr, m, tw, st); });
      pf.run(KK_Y, 2 * nf * SB, st, [&] { launch_fft_y_batch<T, N>(fi, nullptr, nullptr, m, lin ? 2 : 1, true, tw, st, yt); });
      pf.run(KK_Z_C2R, nf * (SB + RB), st, [&] { launch_fft_z_c2r_batch<T, N>(fi, fo, lin ? 2 : 1, m, tw, st); });
    }
    // eps = <|S|> (read by the controller at the first iteration); the mean of D_lin
    class_sum(pf, S, true, [&](int k) { return S[k]->rS; }, [&](int k) { return S[k]->d_misc + 1; });
    {
      std::vector<Engine*> L;
      std::vector<int> lk;
      for (int k = 0; k < n; ++k)
        if (S[k]->wcur < 0) {
          L.push_back(S[k]);
          lk.push_back(k);
        }
      if (!L.empty())
        class_sum(pf, L, false, [&](int i) { return L[i]->rD[0]; }, [&](int i) { return L[i]->d_rstats + 1; });
    }
    for (int k = 0; k < n; ++k) {
      int q = 0;
      int pb[2];
      for (int b = 0; b < 3; ++b)
        if (b != j0[k]) pb[q++] = b;
      pb0[k] = pb[0];
      pb1[k] = pb[1];
    }
    auto in_buf = [&](int k, int it) { return it == 0 ? j0[k] : ((it - 1) & 1 ? pb1[k] : pb0[k]); };
    auto out_buf = [&](int k, int it) { return it & 1 ? pb1[k] : pb0[k]; };
    auto spec_in = [&](int k, int it) { return (it & 1) ? S[k]->sD2 : S[k]->sD; };
    auto spec_out = [&](int k, int it) { return (it & 1) ? S[k]->sD : S[k]->sD2; };
    // With the plane pass an iteration starts from the z spectrum of its iterate (the pass
    // does the y and x transforms itself); otherwise from the z and y transformed spectrum.
    const bool plane = e0->plane_pass && plane_hessian_supported(N);
    // forward transforms of the starting iterates
    {
      const float* in[kBatchMax];
      V* out[kBatchMax];
      ZPrologue pro[kBatchMax];
      FieldSet<T> f[kBatchMax];
      for (int k = 0; k < n; ++k) {
        in[k] = S[k]->rD[j0[k]];
        out[k] = S[k]->sD;
        pro[k] = ZPrologue{nullptr, 0.0, 0};
        f[k] = fs(&S[k]->sD, 1);
      }
      pf.run(KK_Z_R2C, nR + nS, st, [&] { launch_fft_z_r2c_batch<T, N>(in, out, pro, n, tw, st); });
      if (!plane) pf.run(KK_Y, 2 * nS, st, [&] { launch_fft_y_batch<T, N>(f, nullptr, nullptr, n, 1, false, tw, st, yt); });
    }
    for (int k = 0; k < n; ++k)
      if (cudaMemsetAsync(S[k]->d_ctl, 0, sizeof(SolveCtl), st) != cudaSuccess) return DGP_E_CUDA;
    int rc;
    if ((rc = check())) return rc;
    // one iteration of the members in ks
    auto enqueue = [&](int it, bool control, const std::vector<int>& ks) {
      const int m = (int)ks.size();
      XReal<T> xr[kBatchMax];
      FieldSet<T> f6[kBatchMax], f1[kBatchMax];
      const int* sk[kBatchMax];
      RelaxTmaArgs ra[kBatchMax];
      YControl yc[kBatchMax];
      for (int i = 0; i < m; ++i) {
        const int k = ks[i];
        Engine* e = S[k];
        const int ib = in_buf(k, it), ob = out_buf(k, it);
        sk[i] = control ? &e->d_ctl->done : nullptr;
        xr[i] = XReal<T>{spec_in(k, it), nullptr, fs(e->s6, 6), 0, kp[k], sk[i]};
        f6[i] = fs(e->s6, 6);
        ra[i].map[0] = e->rmaps.map[0];
        for (int q = 0; q < 6; ++q) ra[i].map[q] = e->rmaps.map[q];
        ra[i].D = e->rD[ib];
        ra[i].dsum = e->d_rstats + 4 * ib + 1;
        ra[i].S = e->rS;
        ra[i].Dnew = e->rD[ob];
        ra[i].Snew = spec_out(k, it);
        ra[i].partials = e->partials;
        ra[i].rp = rp[k];
        ra[i].skip = sk[i];
        ra[i].fault = &e->d_ctl->fault;
        ra[i].wait_ns = e->wait_ns;
        ra[i].withhold = e->withhold;
        V* so = spec_out(k, it);
        f1[i] = fs(&so, 1);
        yc[i] = YControl{e->partials, e->fblocks, e->d_rstats + 4 * ob, e->d_ctl, e->d_misc + 1, e->d_hist,
                         e->p.max_iter, kPatience, e->p.tol, 1.0 / (double)M};
      }
      if (plane) {
        PlaneArgs pa[kBatchMax];
        for (int i = 0; i < m; ++i) pa[i] = PlaneArgs{spec_in(ks[i], it), f6[i], kp[ks[i]], sk[i]};
        pf.run(KK_X_HESSIAN, 7.0 * m * SB, st, [&] { launch_plane_hessian_batch(N, pa, m, tw, st); });
        pf.run(KK_RELAX, m * (7 * SB + 3 * RB), st, [&] { launch_relax_tma_batch<N>(e0->arith_mode(), ra, m, tw, st); });
        if (control) {
          pf.run(KK_REDUCE, 32.0 * m * e0->fblocks, st, [&] { launch_control_batch(yc, sk, m, st); });
        } else {
          for (int i = 0; i < m; ++i) {
            Engine* e = S[ks[i]];
            pf.run(KK_REDUCE, 32.0 * e->fblocks, st, [&] {
              launch_finalize(e->partials, e->fblocks, 4, e->d_rstats + 4 * out_buf(ks[i], it), st, nullptr);
            });
          }
        }
        return check();
      }
      if (e0->xy_ok && e0->xy_on) {
        pf.run(KK_X_HESSIAN, 7.0 * m * SB, st, [&] { launch_xy_hessian_batch<T, N>(xr, m, tw, st); });
      } else {
        pf.run(KK_X_HESSIAN, 7.0 * m * SB, st, [&] { launch_fft_x_batch<T, N>(XOP_HESSIAN, xr, m, tw, st); });
        pf.run(KK_Y, 12.0 * m * SB, st, [&] { launch_fft_y_batch<T, N>(f6, sk, nullptr, m, 6, true, tw, st, yt); });
      }
      pf.run(KK_RELAX, m * (7 * SB + 3 * RB), st, [&] { launch_relax_tma_batch<N>(e0->arith_mode(), ra, m, tw, st); });
      if (control) {
        pf.run(KK_Y, 2.0 * m * SB, st, [&] { launch_fft_y_batch<T, N>(f1, sk, yc, m, 1, false, tw, st, yt); });
      } else {
        for (int i = 0; i < m; ++i) {
          Engine* e = S[ks[i]];
          pf.run(KK_REDUCE, 32.0 * e->fblocks, st, [&] {
            launch_finalize(e->partials, e->fblocks, 4, e->d_rstats + 4 * out_buf(ks[i], it), st, nullptr);
          });
        }
        pf.run(KK_Y, 2.0 * m * SB, st, [&] { launch_fft_y_batch<T, N>(f1, sk, nullptr, m, 1, false, tw, st, yt); });
      }
      return check();
    };
    std::vector<int> everyone(n);
    for (int k = 0; k < n; ++k) everyone[k] = k;
    // iterations 1 and 2 as one graph for the class (buffers alternate with period two)
    bool graphs = (pf.timing == 0 || pf.sampled) && st != nullptr && st != cudaStreamLegacy &&
                  st != cudaStreamPerThread;
    if (graphs) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        graphs = false;
      } else {
        pf.capturing = true;
        const int r1 = enqueue(1, true, everyone), r2 = r1 ? r1 : enqueue(2, true, everyone);
        pf.capturing = false;
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        cudaGraphExec_t& ex = e0->class_exec;
        if (r1 || r2 || ce != cudaSuccess || !g) {
          graphs = false;
        } else {
          if (ex) {
            cudaGraphExecUpdateResultInfo ui;
            if (cudaGraphExecUpdate(ex, g, &ui) != cudaSuccess) {
              cudaGetLastError();
              cudaGraphExecDestroy(ex);
              ex = nullptr;
            }
          }
          if (!ex && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
            ex = nullptr;
            graphs = false;
          }
        }
        if (g) cudaGraphDestroy(g);
        if (!graphs) cudaGetLastError();
      }
    }
    int max_iter = 0, chunk = 4;
    for (int k = 0; k < n; ++k) {
      max_iter = std::max(max_iter, S[k]->p.max_iter);
      if (S[k]->last_stop_it >= 0) chunk = std::max(chunk, S[k]->last_stop_it + 2);
    }
    int it = 0;
    while (true) {
      const int end = std::min(it + chunk, max_iter + 1);
      while (it < end) {
        if (graphs && it > 0 && (it & 1)) {
          if (cudaGraphLaunch(e0->class_exec, st) != cudaSuccess) return DGP_E_CUDA;
          it += 2;
        } else {
          if ((rc = enqueue(it, true, everyone))) return rc;
          ++it;
        }
      }
      for (int k = 0; k < n; ++k)
        if (cudaMemcpyAsync(S[k]->h_ctl, S[k]->d_ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
          return DGP_E_CUDA;
      if (e0->wait_stream() != cudaSuccess) return DGP_E_CUDA;
      bool done = true;
      for (int k = 0; k < n; ++k) done = done && S[k]->h_ctl->done;
      if (done || it > max_iter) break;
      chunk = kChunk;
    }
    int status = DGP_OK;
    std::vector<SolveCtl> ctl(n);
    for (int k = 0; k < n; ++k) {
      ctl[k] = *S[k]->h_ctl;
      if (!ctl[k].done) return DGP_E_STATE;
      S[k]->history.assign(ctl[k].stop_it + 1, 0.0);
      if (cudaMemcpyAsync(S[k]->history.data(), S[k]->d_hist, sizeof(double) * (ctl[k].stop_it + 1),
                          cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return DGP_E_CUDA;
    }
    if (e0->wait_stream() != cudaSuccess) return DGP_E_CUDA;
    std::vector<V*> sDphi(n);
    for (int k = 0; k < n; ++k) {
      Engine* e = S[k];
      const SolveCtl& c = ctl[k];
      if (c.status == CTL_FAULT) return DGP_E_TIMEOUT;
      if (c.status == CTL_NONFINITE) return DGP_E_NONFINITE;
      const int s_it = c.stop_it, best_it = c.best_it;
      e->last_stop_it = s_it;
      int accepted;
      if (best_it == s_it) {
        accepted = in_buf(k, s_it);
        sDphi[k] = spec_in(k, s_it);
        if (plane) {  // the accepted iterate's spectrum is transformed along z only
          V* f1[1] = {sDphi[k]};
          pf.run(KK_Y, 2 * SB, st, [&] { launch_fft_y<T, N>(fs(f1, 1), 1, false, tw, st, nullptr, yt); });
        }
      } else {
        // an earlier iterate: replay the iterations that produced it for this member alone
        if (best_it > 0) {
          if (plane) {
            launch_fft_z_r2c<T, N>(e->rD[j0[k]], 0, e->sD, 0, 1, ZPrologue{nullptr, 0.0, 0}, tw, st);
            if ((rc = check())) return rc;
          } else if ((rc = e->forward_zy(e->rD[j0[k]], e->sD, ZPrologue{nullptr, 0.0, 0}))) {
            return rc;
          }
          const std::vector<int> one(1, k);
          for (int q = 0; q < best_it; ++q)
            if ((rc = enqueue(q, false, one))) return rc;
        }
        accepted = in_buf(k, best_it);
        if ((rc = e->forward_zy(e->rD[accepted], e->sD, ZPrologue{nullptr, 0.0, 0}))) return rc;
        sDphi[k] = e->sD;
        if (best_it > 0) {
          if (cudaMemcpyAsync(e->h_ctl, e->d_ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              e->wait_stream() != cudaSuccess)
            return DGP_E_CUDA;
          if (e->h_ctl->fault) return DGP_E_TIMEOUT;
        }
      }
      e->wcur = accepted;
      if (c.status != CTL_CONVERGED) status = DGP_E_NOT_CONVERGED;
      if (info) {
        dgp_solve_info& inf = info[sub[k]];
        memset(&inf, 0, sizeof(inf));
        inf.eps = c.eps;
        inf.iters = best_it;
        inf.norm_res = c.rbest;
        inf.min_norm_res = c.rbest;
        inf.bad_fraction = c.last_bad / (double)M;
        inf.status = c.status == CTL_CONVERGED ? DGP_OK : DGP_E_NOT_CONVERGED;
      }
    }
    // forces g = -grad phi (Eq. FullDGP1) of every member
    {
      XReal<T> xr[kBatchMax];
      FieldSet<T> fi[kBatchMax], fo[kBatchMax];
      for (int k = 0; k < n; ++k) {
        Engine* e = S[k];
        xr[k] = XReal<T>{e->sDelta, sDphi[k], fs(e->s6, 4), 14, kp[k], nullptr};
        V* sp[3] = {e->s6[1], e->s6[2], e->s6[3]};
        fi[k] = fs(sp, 3);
        T* outs[3] = {e->rG[0], e->rG[1], e->rG[2]};
        for (int i = 0; i < kMaxFields; ++i) fo[k].p[i] = i < 3 ? reinterpret_cast<V*>(outs[i]) : nullptr;
      }
      pf.run(KK_X_OTHER, 5.0 * nS, st, [&] { launch_fft_x_batch<T, N>(XOP_PHI_FORCE, xr, n, tw, st); });
      pf.run(KK_Y, 6.0 * nS, st, [&] { launch_fft_y_batch<T, N>(fi, nullptr, nullptr, n, 3, true, tw, st, yt); });
      pf.run(KK_Z_C2R, 3.0 * (nS + nR), st, [&] { launch_fft_z_c2r_batch<T, N>(fi, fo, 3, n, tw, st); });
    }
    if ((rc = check())) return rc;
    if (info && e0->wait_stream() != cudaSuccess) return DGP_E_CUDA;
    return status;
  }

 public:
  int step(dgp_particles* pp, double a, double da, dgp_solve_info* info) override {
    force_host = nullptr;
    return step_impl(pp, a, da, info, nullptr);
  }

  // after_drift (may be null) runs once the positions are final for the step
  // (after the drift and the cell sort), before the field solve at a + da.
  int step_impl(dgp_particles* pp, double a, double da, dgp_solve_info* info,
                const std::function<int()>* after_drift) {
    if (!valid_parts(pp) || pp->n == 0) return DGP_E_INVALID;
    if (!(a > 0.0) || !(da > 0.0) || !isfinite(a + da)) return DGP_E_INVALID;
    const double a1 = a + da;
    const double ah = exp(0.5 * (log(a) + log(a1)));
    const double om = cosmo.omega_m0, rc_ = p.rc_H0;
    int rc;
    const bool reuse = force_valid && force_x == pp->x && force_np == pp->n && fabs(force_a - a) <= 1e-12 * a;
    if (!reuse && (rc = forces_at(pp, a, nullptr))) return rc;
    const CicParams cp = cic();
    const double k1 = time_integral(a, ah, om, rc_, 0), dr = time_integral(a, a1, om, rc_, 2);
    prof.run(KK_GATHER, 12.0 * sizeof(T) * pp->n + 3 * RB, stream, [&] {
      launch_gather_kick<T>((T*)pp->x, (T*)pp->y, (T*)pp->z, (T*)pp->px, (T*)pp->py, (T*)pp->pz, pp->n, rG[0],
                            rG[1], rG[2], cp, k1, dr, 1, stream);
    });
    DGP_CHECK_LAUNCH();
    ++nsteps;
    if (p.sort_every > 0 && nsteps % p.sort_every == 0 && (rc = sort_impl(pp, nullptr))) return rc;
    if (after_drift && (rc = (*after_drift)())) return rc;
    if ((rc = forces_at(pp, a1, info))) return rc;
    const double k2 = time_integral(ah, a1, om, rc_, 0);
    prof.run(KK_GATHER, 9.0 * sizeof(T) * pp->n + 3 * RB, stream, [&] {
      launch_gather_kick<T>((T*)pp->x, (T*)pp->y, (T*)pp->z, (T*)pp->px, (T*)pp->py, (T*)pp->pz, pp->n, rG[0],
                            rG[1], rG[2], cp, k2, 0.0, 0, stream);
    });
    DGP_CHECK_LAUNCH();
    return DGP_OK;
  }

  int step_host(dgp_particles* hpp, double a, double da, dgp_solve_info* info) override {
    if (!valid_parts(hpp) || hpp->n == 0) return DGP_E_INVALID;
    if (!(a > 0.0) || !(da > 0.0) || !isfinite(a + da)) return DGP_E_INVALID;
    if (hp_n < hpp->n) {
      for (int i = 0; i < 6; ++i) {
        cudaFree(hp[i]);
        hp[i] = nullptr;
        if (cudaMalloc(&hp[i], sizeof(T) * hpp->n) != cudaSuccess) { hp_n = 0; return DGP_E_NOMEM; }
      }
      hp_n = hpp->n;
    }
    if (!copy_streams[0]) {
      for (int j = 0; j < kCopyStreams; ++j)
        DGP_CUDA(cudaStreamCreateWithFlags(&copy_streams[j], cudaStreamNonBlocking));
      for (int j = 0; j <= kCopyStreams; ++j) DGP_CUDA(cudaEventCreateWithFlags(&copy_ev[j], cudaEventDisableTiming));
      for (auto& row : chunk_ev)
        for (cudaEvent_t& e : row) DGP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    T* src[6] = {(T*)hpp->x, (T*)hpp->y, (T*)hpp->z, (T*)hpp->px, (T*)hpp->py, (T*)hpp->pz};
    const int64_t np = hpp->n;
    // every host step runs on the same device copies, so the end-of-step force
    // may be reused only for the host arrays that the previous host step wrote
    if (force_host != hpp->x) force_valid = false;
    force_host = nullptr;
    // particle ranges of whole 256-element blocks (16-byte aligned slices)
    const int64_t cs = ((np + kHostChunks - 1) / kHostChunks + 255) / 256 * 256;
    auto lo = [&](int c) { return std::min<int64_t>(np, c * cs); };
    auto hi = [&](int c) { return std::min<int64_t>(np, (c + 1) * cs); };
    // the copy streams start after the work enqueued so far on the stream
    DGP_CUDA(cudaEventRecord(copy_ev[kCopyStreams], stream));
    for (int j = 0; j < kCopyStreams; ++j) DGP_CUDA(cudaStreamWaitEvent(copy_streams[j], copy_ev[kCopyStreams], 0));
    for (int c = 0; c < kHostChunks; ++c) {
      cudaStream_t cp_s = copy_streams[c % kCopyStreams];
      const size_t b = sizeof(T) * (size_t)(hi(c) - lo(c));
      if (b)
        for (int i = 0; i < 6; ++i) DGP_CUDA(cudaMemcpyAsync(hp[i] + lo(c), src[i] + lo(c), b, cudaMemcpyHostToDevice, cp_s));
      DGP_CUDA(cudaEventRecord(chunk_ev[0][c], cp_s));
    }
    int rc = DGP_OK;
    auto finish_copies = [&]() {
      for (int j = 0; j < kCopyStreams; ++j) cudaStreamSynchronize(copy_streams[j]);
    };
    dgp_particles dp{hp[0], hp[1], hp[2], hp[3], hp[4], hp[5], np};
    // the steps of step_impl, with the two kicks taken range by range
    const double a1 = a + da;
    const double ah = exp(0.5 * (log(a) + log(a1)));
    const double om = cosmo.omega_m0, rc_ = p.rc_H0;
    const bool reuse = force_valid && force_x == dp.x && force_np == np && fabs(force_a - a) <= 1e-12 * a;
    if (!reuse) {
      for (int c = 0; c < kHostChunks; ++c) DGP_CUDA(cudaStreamWaitEvent(stream, chunk_ev[0][c], 0));
      if ((rc = forces_at(&dp, a, nullptr))) { finish_copies(); return rc; }
    }
    const CicParams cp = cic();
    const double k1 = time_integral(a, ah, om, rc_, 0), dr = time_integral(a, a1, om, rc_, 2);
    const bool sorting = p.sort_every > 0 && (nsteps + 1) % p.sort_every == 0;
    for (int c = 0; c < kHostChunks; ++c) {
      const int64_t o = lo(c), m = hi(c) - lo(c);
      if (m <= 0) continue;
      DGP_CUDA(cudaStreamWaitEvent(stream, chunk_ev[0][c], 0));
      prof.run(KK_GATHER, 12.0 * sizeof(T) * m + 3 * RB * (double)m / np, stream, [&] {
        launch_gather_kick<T>(hp[0] + o, hp[1] + o, hp[2] + o, hp[3] + o, hp[4] + o, hp[5] + o, m, rG[0], rG[1],
                              rG[2], cp, k1, dr, 1, stream);
      });
      if (!sorting) {  // the range's positions are final: copy them back during the field solve
        cudaStream_t cp_s = copy_streams[c % kCopyStreams];
        DGP_CUDA(cudaEventRecord(chunk_ev[1][c], stream));
        DGP_CUDA(cudaStreamWaitEvent(cp_s, chunk_ev[1][c], 0));
        for (int i = 0; i < 3; ++i)
          DGP_CUDA(cudaMemcpyAsync(src[i] + o, hp[i] + o, sizeof(T) * m, cudaMemcpyDeviceToHost, cp_s));
      }
    }
    if (cudaGetLastError() != cudaSuccess) { finish_copies(); return DGP_E_CUDA; }
    ++nsteps;
    if (sorting) {
      if ((rc = sort_impl(&dp, nullptr))) { finish_copies(); return rc; }
      DGP_CUDA(cudaEventRecord(copy_ev[kCopyStreams], stream));
      for (int i = 0; i < 3; ++i) {
        cudaStream_t cp_s = copy_streams[i % kCopyStreams];
        DGP_CUDA(cudaStreamWaitEvent(cp_s, copy_ev[kCopyStreams], 0));
        DGP_CUDA(cudaMemcpyAsync(src[i], hp[i], sizeof(T) * np, cudaMemcpyDeviceToHost, cp_s));
      }
    }
    if ((rc = forces_at(&dp, a1, info))) { finish_copies(); return rc; }
    const double k2 = time_integral(ah, a1, om, rc_, 0);
    for (int c = 0; c < kHostChunks; ++c) {
      const int64_t o = lo(c), m = hi(c) - lo(c);
      if (m <= 0) continue;
      prof.run(KK_GATHER, 9.0 * sizeof(T) * m + 3 * RB * (double)m / np, stream, [&] {
        launch_gather_kick<T>(hp[0] + o, hp[1] + o, hp[2] + o, hp[3] + o, hp[4] + o, hp[5] + o, m, rG[0], rG[1],
                              rG[2], cp, k2, 0.0, 0, stream);
      });
      cudaStream_t cp_s = copy_streams[c % kCopyStreams];
      DGP_CUDA(cudaEventRecord(chunk_ev[2][c], stream));
      DGP_CUDA(cudaStreamWaitEvent(cp_s, chunk_ev[2][c], 0));
      for (int i = 3; i < 6; ++i)
        DGP_CUDA(cudaMemcpyAsync(src[i] + o, hp[i] + o, sizeof(T) * m, cudaMemcpyDeviceToHost, cp_s));
    }
    if (cudaGetLastError() != cudaSuccess) { finish_copies(); return DGP_E_CUDA; }
    for (int j = 0; j < kCopyStreams; ++j) DGP_CUDA(cudaStreamSynchronize(copy_streams[j]));
    DGP_CUDA(wait_stream());
    force_host = hpp->x;
    return DGP_OK;
  }

  int pk(const void* delta, int nbins, double* k, double* pkv, int64_t* nmodes) override {
    if (!delta || !k || !pkv || !nmodes || nbins < 1 || nbins > N / 2) return DGP_E_INVALID;
    int rc;
    if ((rc = forward_zy((const T*)delta, s6[0], ZPrologue{nullptr, 0.0, 0}))) return rc;
    const Coef c = coefficients(1.0, cosmo.omega_m0, p.rc_H0);
    KParams kp = kparams(c, p.gravity);
    prof.run(KK_X_OTHER, SB, stream, [&] {
      launch_fft_x_op<T, N>(XOP_PK, s6[0], nullptr, fs(s6, 0), 0, kp, pk_partials, nbins, 0, 0, tw, stream);
    });
    prof.run(KK_REDUCE, 24.0 * nbins * pk_blocks, stream,
             [&] { launch_finalize(pk_partials, pk_blocks, 3 * nbins, d_pk, stream); });
    DGP_CHECK_LAUNCH();
    double hb[3 * 256];
    DGP_CUDA(cudaMemcpyAsync(hb, d_pk, sizeof(double) * 3 * nbins, cudaMemcpyDeviceToHost, stream));
    DGP_CUDA(wait_stream());
    for (int b = 0; b < nbins; ++b) {
      const double cnt = hb[b];
      nmodes[b] = (int64_t)llround(cnt);
      k[b] = cnt > 0 ? hb[nbins + b] / cnt : NAN;
      pkv[b] = cnt > 0 ? hb[2 * nbins + b] / cnt : NAN;
    }
    return DGP_OK;
  }

  // Spectra of the brane-bending mode of the accepted solution (Sec. IV):
  // P_c of c = alpha eta / (3 (eta - 1)) D, P_C of C = -D / kbar^2 and
  // Delta = 4 pi k^5 P_C, at the scale factor of the last nonlinear solve.
  int brane(int nbins, double* k, double* pc, double* pC, double* dgc, int64_t* nmodes) override {
    if (nbins < 1 || nbins > N / 2 || !k || !pc || !pC || !dgc || !nmodes) return DGP_E_INVALID;
    if (wcur < 0 || !(last_nl_a > 0.0)) return DGP_E_STATE;
    int rc;
    if ((rc = forward_zy(rD[wcur], s6[0], ZPrologue{nullptr, 0.0, 0}))) return rc;
    const Coef c = coefficients(last_nl_a, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, p.gravity);
    prof.run(KK_X_OTHER, SB, stream, [&] {
      launch_fft_x_op<T, N>(XOP_PK_BRANE, s6[0], nullptr, fs(s6, 0), 0, kp, pk_partials, nbins, 0, 0, tw, stream);
    });
    prof.run(KK_REDUCE, 32.0 * nbins * pk_blocks, stream,
             [&] { launch_finalize(pk_partials, pk_blocks, 4 * nbins, d_pk, stream); });
    DGP_CHECK_LAUNCH();
    double hb[4 * 256];
    DGP_CUDA(cudaMemcpyAsync(hb, d_pk, sizeof(double) * 4 * nbins, cudaMemcpyDeviceToHost, stream));
    DGP_CUDA(wait_stream());
    const double fac_c = c.alpha * c.eta / (3.0 * (c.eta - 1.0));
    const double kbf = cosmo.c_over_H0 / (c.a * c.E) * 2.0 * M_PI / p.box;  // kbar = kbf |n|
    const double kbf4 = kbf * kbf * kbf * kbf;
    for (int b = 0; b < nbins; ++b) {
      const double cnt = hb[b];
      nmodes[b] = (int64_t)llround(cnt);
      k[b] = cnt > 0 ? hb[nbins + b] / cnt : NAN;
      pc[b] = cnt > 0 ? fac_c * fac_c * hb[2 * nbins + b] / cnt : NAN;
      pC[b] = cnt > 0 ? hb[3 * nbins + b] / cnt / kbf4 : NAN;
      dgc[b] = cnt > 0 ? 4.0 * M_PI * pow(k[b], 5) * pC[b] : NAN;
    }
    return DGP_OK;
  }

  // Adjoint of the last accepted nonlinear solve (see dgp_solve_adjoint).
  int adjoint(const void* phibar, const void* const* gbar, void* deltabar, double tol,
              dgp_solve_info* info, double* rcbar) override {
    if (!deltabar || !(tol >= 0) || (!phibar && !gbar[0] && !gbar[1] && !gbar[2])) return DGP_E_INVALID;
    if ((gbar[0] != nullptr) != (gbar[1] != nullptr) || (gbar[0] != nullptr) != (gbar[2] != nullptr))
      return DGP_E_INVALID;
    if (p.gravity != DGP_GRAVITY_NL) return DGP_E_INVALID;
    if (wcur < 0 || !(last_nl_a > 0.0)) return DGP_E_STATE;
    if (rcbar && !delta_nl) return DGP_E_STATE;  // the r_c terms need that solve's delta
    if (!aP && cudaMalloc(&aP, sizeof(T) * 7 * M) != cudaSuccess) { aP = nullptr; return DGP_E_NOMEM; }
    if (!aF && cudaMalloc(&aF, sizeof(T) * 4 * M) != cudaSuccess) { aF = nullptr; return DGP_E_NOMEM; }
    if (!aS && cudaMalloc(&aS, sizeof(V) * 7 * SPEC) != cudaSuccess) { aS = nullptr; return DGP_E_NOMEM; }
    if (!adj_scalars()) return DGP_E_NOMEM;
    int rc;
    T* const lam = aP + 6 * M;
    T* const aU = aF;
    T* const aQ = aF + M;
    T* const aG = aF + 2 * M;
    T* const aA = aF + 3 * M;
    const Coef c = coefficients(last_nl_a, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, DGP_GRAVITY_NL);
    const ZPrologue none{nullptr, 0.0, 0};
    // cotangent spectra -> Dbar = B phibar_tot and A phibar_tot (real fields)
    FieldSet<T> in;
    for (int i = 0; i < kMaxFields; ++i) in.p[i] = i < 7 ? aS + i * SPEC : nullptr;
    int mask = 0;
    if (phibar) {
      if ((rc = forward_zy((const T*)phibar, in.p[0], none))) return rc;
      mask |= 1;
    }
    for (int i = 0; i < 3; ++i)
      if (gbar[i]) {
        if ((rc = forward_zy((const T*)gbar[i], in.p[1 + i], none))) return rc;
        mask |= 2 << i;
      }
    prof.run(KK_X_OTHER, SB * (__builtin_popcount(mask) + 2), stream,
             [&] { launch_fft_x_adj<T, N>(XOP_ADJ_PHI, in, mask, fs(s6, 2), kp, tw, stream); });
    T* ga[2] = {aG, aA};
    if ((rc = inverse_yz(s6, ga, 2))) return rc;
    // real Hessian fields of the accepted D: H_xx, H_yy, H_xy, H_xz, H_yz (and N)
    if ((rc = forward_zy(rD[wcur], sD2, none))) return rc;
    RcDeriv rd{};
    if (rcbar) {
      const Coef dc = coefficients_drc(last_nl_a, cosmo.omega_m0, p.rc_H0);
      rd = RcDeriv{dc.E / c.E, dc.eta, dc.alpha, dc.beta, dc.s, dc.c2, dc.c3};
      FieldSet<T> rin = in;
      rin.p[4] = sDelta;
      rin.p[5] = sD2;
      prof.run(KK_X_OTHER, SB * (__builtin_popcount(mask) + 2), stream,
               [&] { launch_fft_x_rc<T, N>(rin, mask | 0x30, kp, rd, pk_partials, tw, stream); });
      prof.run(KK_REDUCE, 8.0 * pk_blocks, stream,
               [&] { launch_finalize(pk_partials, pk_blocks, 1, d_adj + 6, stream); });
      DGP_CHECK_LAUNCH();
    }
    prof.run(KK_X_HESSIAN, 7 * SB, stream, [&] {
      launch_fft_x_op<T, N>(XOP_HESSIAN, sD2, nullptr, fs(s6, 6), 0, kp, nullptr, 0, 0, 0, tw, stream);
    });
    if ((rc = inverse_yz(s6, rH, 6))) return rc;
    const double* dsum = d_rstats + 4 * wcur + 1;
    const double alpha = c.alpha, w = p.w;
    prof.run(KK_REDUCE, RB, stream,
             [&] { launch_adj_inv_diag<T>(rD[wcur], dsum, M, alpha, w, partials, nblocks, stream); });
    prof.run(KK_REDUCE, 16.0 * nblocks, stream, [&] { launch_finalize(partials, nblocks, 2, d_adj + 2, stream); });
    if ((rc = reduce_sum(aG, true, d_adj + 5))) return rc;
    double hs[8];
    DGP_CUDA(cudaMemcpyAsync(hs, d_adj, sizeof(double) * 8, cudaMemcpyDeviceToHost, stream));
    DGP_CUDA(wait_stream());
    if (hs[3] > 0.0) return DGP_E_BAD_POINTS;  // the w-split diagonal must be positive
    const double gnorm = hs[5] > 0.0 ? hs[5] : 1.0;
    // lam_0 from rest = 0, then the w-split iteration
    DGP_CUDA(cudaMemsetAsync(lam, 0, sizeof(T) * M, stream));
    DGP_CUDA(cudaMemsetAsync(aQ, 0, sizeof(T) * M, stream));
    auto update = [&]() -> int {
      prof.run(KK_RELAX, 6 * RB, stream, [&] {
        launch_adj_update_a<T>(lam, rD[wcur], dsum, aG, aQ, aU, M, alpha, w, partials, nblocks, stream);
      });
      prof.run(KK_REDUCE, 16.0 * nblocks, stream, [&] { launch_finalize(partials, nblocks, 2, d_adj, stream); });
      prof.run(KK_RELAX, 4 * RB, stream, [&] {
        launch_adj_update_b<T>(lam, rD[wcur], dsum, aU, M, alpha, w, d_adj, partials, nblocks, stream);
      });
      prof.run(KK_REDUCE, 8.0 * nblocks, stream, [&] { launch_finalize(partials, nblocks, 1, d_adj + 4, stream); });
      DGP_CHECK_LAUNCH();
      return DGP_OK;
    };
    if ((rc = update())) return rc;
    history.clear();
    dgp_solve_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.eps = hs[5] / (double)M;
    bool converged = false;
    T* h5[5] = {rH[0], rH[1], rH[2], rH[3], rH[4]};
    FieldSet<T> aspec;
    for (int i = 0; i < kMaxFields; ++i) aspec.p[i] = i < 7 ? aS + i * SPEC : nullptr;
    int it = 0;
    for (; it <= p.max_iter; ++it) {
      prof.run(KK_MISC, 7 * RB, stream,
               [&] { launch_adj_products<T>(lam, rD[wcur], dsum, h5, aP, M, stream); });
      prof.run(KK_Z_R2C, 7 * (RB + SB), stream,
               [&] { launch_fft_z_r2c<T, N>(aP, M, aS, SPEC, 7, none, tw, stream); });
      prof.run(KK_Y, 14 * SB, stream, [&] { launch_fft_y<T, N>(aspec, 7, false, tw, stream, nullptr, y_threads); });
      prof.run(KK_X_OTHER, 8 * SB, stream,
               [&] { launch_fft_x_adj<T, N>(XOP_ADJ_COMBINE, aspec, 0x7f, fs(s6, 1), kp, tw, stream); });
      T* qo[1] = {aQ};
      if ((rc = inverse_yz(s6, qo, 1))) return rc;
      if ((rc = update())) return rc;
      DGP_CUDA(cudaMemcpyAsync(hs, d_adj + 4, sizeof(double), cudaMemcpyDeviceToHost, stream));
      DGP_CUDA(wait_stream());
      const double r = hs[0] / gnorm;  // projected residual of the iterate before this update
      history.push_back(r);
      if (!isfinite(r)) return DGP_E_NONFINITE;
      if (r < tol) {
        converged = true;
        break;
      }
    }
    // deltabar = A phibar_tot + S lam
    if ((rc = forward_zy(lam, s6[0], none))) return rc;
    if (rcbar) {
      FieldSet<T> rin;
      for (int i = 0; i < kMaxFields; ++i) rin.p[i] = nullptr;
      rin.p[4] = sDelta;
      rin.p[5] = sD2;
      rin.p[6] = s6[0];
      prof.run(KK_X_OTHER, SB * 3, stream,
               [&] { launch_fft_x_rc<T, N>(rin, 0x70, kp, rd, pk_partials, tw, stream); });
      prof.run(KK_REDUCE, 8.0 * pk_blocks, stream,
               [&] { launch_finalize(pk_partials, pk_blocks, 1, d_adj + 7, stream); });
      DGP_CHECK_LAUNCH();
      double h2[2];
      DGP_CUDA(cudaMemcpyAsync(h2, d_adj + 6, sizeof(double) * 2, cudaMemcpyDeviceToHost, stream));
      DGP_CUDA(wait_stream());
      *rcbar = (h2[0] + h2[1]) / (double)M;  // Parseval: sum_x u v = sum_k conj(U) V / N^3
    }
    prof.run(KK_X_OTHER, 2 * SB, stream, [&] {
      launch_fft_x_op<T, N>(XOP_SOURCE, s6[0], nullptr, fs(s6 + 1, 1), 0, kp, nullptr, 0, 0, 0, tw, stream);
    });
    T* so[1] = {aU};
    if ((rc = inverse_yz(s6 + 1, so, 1))) return rc;
    prof.run(KK_MISC, 3 * RB, stream, [&] { launch_axpy<T>(aA, aU, (T*)deltabar, M, stream); });
    DGP_CHECK_LAUNCH();
    inf.iters = (int)history.size();
    inf.norm_res = history.empty() ? 0.0 : history.back();
    inf.min_norm_res = inf.norm_res;
    inf.status = converged ? DGP_OK : DGP_E_NOT_CONVERGED;
    if (info) {
      *info = inf;
      DGP_CUDA(wait_stream());
    }
    return inf.status;
  }

  bool adj_scalars() {
    if (!d_adj && cudaMalloc(&d_adj, sizeof(double) * 12) != cudaSuccess) {
      d_adj = nullptr;
      return false;
    }
    return true;
  }

  // Host value of the device sum of nb per-block partials.
  int sum_partials(int nb, double* out) {
    if (!adj_scalars()) return DGP_E_NOMEM;
    prof.run(KK_REDUCE, 8.0 * nb, stream, [&] { launch_finalize(partials, nb, 1, d_adj + 8, stream); });
    DGP_CHECK_LAUNCH();
    DGP_CUDA(cudaMemcpyAsync(out, d_adj + 8, sizeof(double), cudaMemcpyDeviceToHost, stream));
    DGP_CUDA(wait_stream());
    return DGP_OK;
  }

  // VJP of the particle forces at the positions xs.p[0..2] for the cotangent
  // scale * xs.p[3..5]; accumulates into xb.p[0..2].  Solves at a first, so the
  // context's accepted D is the one the adjoint needs.  With rc_solve and fdot
  // set: the solve's explicit derivative in r_c H0 for that cotangent, and
  // sum_p F(x_p) . xs.p[3..5][p] (unscaled).
  int force_vjp(const ParticleSet<T>& xs, int64_t np, double scale, double a, const ParticleSet<T>& xb,
                double* rc_solve = nullptr, double* fdot = nullptr) {
    int rc;
    dgp_particles dp{xs.p[0], xs.p[1], xs.p[2], xs.p[0], xs.p[1], xs.p[2], np};
    if ((rc = forces_at(&dp, a, nullptr))) return rc;
    const CicParams cp = cic();
    T* fb[3] = {aFb, aFb + M, aFb + 2 * M};
    prof.run(KK_MISC, 3 * RB, stream, [&] { launch_fill<T>(aFb, 3 * M, (T)0, stream); });
    prof.run(KK_DEPOSIT, 6.0 * sizeof(T) * np + 3 * RB, stream,
             [&] { launch_deposit_vec<T>(xs, scale, np, fb, cp, stream); });
    DGP_CHECK_LAUNCH();
    const void* gb[3] = {fb[0], fb[1], fb[2]};
    rc = adjoint(nullptr, gb, rRho, p.tol, nullptr, rc_solve);
    if (rc != DGP_OK && rc != DGP_E_NOT_CONVERGED) return rc;
    if (!fdot) {
      prof.run(KK_GATHER, 9.0 * sizeof(T) * np + 4 * RB, stream, [&] {
        launch_force_vjp_gather<T>(xs, scale, np, rG, rRho, (double)M / (double)np, xb, cp, stream);
      });
      DGP_CHECK_LAUNCH();
      return DGP_OK;
    }
    int nb = 0;
    prof.run(KK_GATHER, 9.0 * sizeof(T) * np + 4 * RB, stream, [&] {
      nb = launch_force_vjp_gather_dot<T>(xs, scale, np, rG, rRho, (double)M / (double)np, xb, cp, partials, stream);
    });
    DGP_CHECK_LAUNCH();
    return sum_partials(nb, fdot);
  }

  // Transpose of one kick-drift-kick step (see pm_step_adjoint).
  int step_adjoint(const dgp_particles* st, double a, double da, dgp_particles* cot, double* rcbar) override {
    if (!valid_parts(st) || !valid_parts(cot) || st->n == 0 || cot->n != st->n) return DGP_E_INVALID;
    if (!(a > 0.0) || !(da > 0.0) || !isfinite(a + da)) return DGP_E_INVALID;
    if (p.gravity != DGP_GRAVITY_NL) return DGP_E_INVALID;
    const int64_t np = st->n;
    if (ap_n < np) {
      for (int i = 0; i < 6; ++i) {
        cudaFree(ap[i]);
        ap[i] = nullptr;
        if (cudaMalloc(&ap[i], sizeof(T) * np) != cudaSuccess) { ap_n = 0; return DGP_E_NOMEM; }
      }
      ap_n = np;
    }
    if (!aFb && cudaMalloc(&aFb, sizeof(T) * 3 * M) != cudaSuccess) return DGP_E_NOMEM;
    const double a1 = a + da;
    const double ah = exp(0.5 * (log(a) + log(a1)));
    const double om = cosmo.omega_m0, rc_ = p.rc_H0;
    const double k1 = time_integral(a, ah, om, rc_, 0), dr = time_integral(a, a1, om, rc_, 2);
    const double k2 = time_integral(ah, a1, om, rc_, 0);
    int rc;
    // recompute x1 (and p_h) from the start state on the context's copies
    const void* src[6] = {st->x, st->y, st->z, st->px, st->py, st->pz};
    for (int i = 0; i < 6; ++i)
      DGP_CUDA(cudaMemcpyAsync(ap[i], src[i], sizeof(T) * np, cudaMemcpyDeviceToDevice, stream));
    dgp_particles sp{ap[0], ap[1], ap[2], ap[3], ap[4], ap[5], np};
    if ((rc = forces_at(&sp, a, nullptr))) return rc;
    const CicParams cp = cic();
    prof.run(KK_GATHER, 12.0 * sizeof(T) * np + 3 * RB, stream, [&] {
      launch_gather_kick<T>(ap[0], ap[1], ap[2], ap[3], ap[4], ap[5], np, rG[0], rG[1], rG[2], cp, k1, dr, 1,
                            stream);
    });
    DGP_CHECK_LAUNCH();
    T* const cv[6] = {(T*)cot->x, (T*)cot->y, (T*)cot->z, (T*)cot->px, (T*)cot->py, (T*)cot->pz};
    const ParticleSet<T> xb{{cv[0], cv[1], cv[2], cv[0], cv[1], cv[2]}};
    const ParticleSet<T> pb{{cv[3], cv[4], cv[5], cv[3], cv[4], cv[5]}};
    // r_c H0: K2' <pbar1, F(x1)> + solve(x1) + Dr' <xbar1_tot, p_h> + K1' <pbar_h, F(x0)> + solve(x0)
    double rs1 = 0.0, pf1 = 0.0, dx = 0.0, rs0 = 0.0, pf0 = 0.0;
    const bool want = rcbar != nullptr;
    // x1: fbar = k2 pbar1
    if ((rc = force_vjp(ParticleSet<T>{{ap[0], ap[1], ap[2], cv[3], cv[4], cv[5]}}, np, k2, a1, xb,
                        want ? &rs1 : nullptr, want ? &pf1 : nullptr)))
      return rc;
    if (want) {
      T* xa[3] = {cv[0], cv[1], cv[2]};
      T* ph[3] = {ap[3], ap[4], ap[5]};
      int nb = 0;
      prof.run(KK_MISC, 6.0 * sizeof(T) * np, stream, [&] { nb = launch_dot3<T>(xa, ph, np, partials, stream); });
      DGP_CHECK_LAUNCH();
      if ((rc = sum_partials(nb, &dx))) return rc;
    }
    // pbar_h = pbar1 + Dr xbar
    prof.run(KK_MISC, 9.0 * sizeof(T) * np, stream, [&] { launch_particle_axpy<T>(xb, dr, np, pb, stream); });
    DGP_CHECK_LAUNCH();
    // x0: fbar = k1 pbar_h
    const ParticleSet<T> at0{{(T*)st->x, (T*)st->y, (T*)st->z, cv[3], cv[4], cv[5]}};
    if ((rc = force_vjp(at0, np, k1, a, xb, want ? &rs0 : nullptr, want ? &pf0 : nullptr))) return rc;
    force_valid = false;
    if (want) {
      const double dk1 = time_integral_drc(a, ah, om, rc_, 0), dk2 = time_integral_drc(ah, a1, om, rc_, 0);
      const double ddr = time_integral_drc(a, a1, om, rc_, 2);
      *rcbar = dk2 * pf1 + rs1 + ddr * dx + dk1 * pf0 + rs0;
    }
    return DGP_OK;
  }

  // Cotangent of vel_factor in dgp_zeldovich: sum_j <pbar_j, Psi_j(delta_L)>.
  int zeldovich_vf_adjoint(const void* dl, const dgp_particles* cot, double* vfbar) override {
    if (!dl || !vfbar || !valid_parts(cot) || cot->n != M) return DGP_E_INVALID;
    int rc;
    if ((rc = forward_zy((const T*)dl, s6[0], ZPrologue{nullptr, 0.0, 0}))) return rc;
    const Coef c = coefficients(1.0, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, p.gravity);
    prof.run(KK_X_OTHER, 4 * SB, stream, [&] {
      launch_fft_x_op<T, N>(XOP_ZEL, s6[0], nullptr, fs(s6 + 1, 3), 0, kp, nullptr, 0, 0, 0, tw, stream);
    });
    if ((rc = inverse_yz(s6 + 1, rG, 3))) return rc;
    T* pbar[3] = {(T*)cot->px, (T*)cot->py, (T*)cot->pz};
    int nb = 0;
    prof.run(KK_MISC, 6.0 * RB, stream, [&] { nb = launch_dot3<T>(rG, pbar, M, partials, stream); });
    DGP_CHECK_LAUNCH();
    force_valid = false;
    return sum_partials(nb, vfbar);
  }

  // Zel'dovich particles from a linear field (lattice order) and the map's transpose.
  int zeldovich(const void* dl, double vf, dgp_particles* out) override {
    if (!dl || !valid_parts(out) || out->n != M) return DGP_E_INVALID;
    int rc;
    if ((rc = forward_zy((const T*)dl, s6[0], ZPrologue{nullptr, 0.0, 0}))) return rc;
    const Coef c = coefficients(1.0, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, p.gravity);
    prof.run(KK_X_OTHER, 4 * SB, stream, [&] {
      launch_fft_x_op<T, N>(XOP_ZEL, s6[0], nullptr, fs(s6 + 1, 3), 0, kp, nullptr, 0, 0, 0, tw, stream);
    });
    if ((rc = inverse_yz(s6 + 1, rG, 3))) return rc;
    T* o[6] = {(T*)out->x, (T*)out->y, (T*)out->z, (T*)out->px, (T*)out->py, (T*)out->pz};
    prof.run(KK_MISC, 9 * RB, stream, [&] { launch_zel_particles<T>(rG, vf, cic(), o, stream); });
    DGP_CHECK_LAUNCH();
    force_valid = false;
    return DGP_OK;
  }

  int zeldovich_adjoint(const dgp_particles* cot, double vf, void* dlbar) override {
    if (!dlbar || !valid_parts(cot) || cot->n != M) return DGP_E_INVALID;
    int rc;
    T* cv[6] = {(T*)cot->x, (T*)cot->y, (T*)cot->z, (T*)cot->px, (T*)cot->py, (T*)cot->pz};
    prof.run(KK_MISC, 9 * RB, stream, [&] { launch_zel_cot<T>(cv, vf, M, rG, stream); });
    for (int j = 0; j < 3; ++j)
      if ((rc = forward_zy(rG[j], s6[1 + j], ZPrologue{nullptr, 0.0, 0}))) return rc;
    const Coef c = coefficients(1.0, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, p.gravity);
    FieldSet<T> in = fs(s6, 4);
    prof.run(KK_X_OTHER, 4 * SB, stream,
             [&] { launch_fft_x_adj<T, N>(XOP_ZEL_ADJ, in, 0xe, fs(s6, 1), kp, tw, stream); });
    T* o[1] = {(T*)dlbar};
    if ((rc = inverse_yz(s6, o, 1))) return rc;
    force_valid = false;
    return DGP_OK;
  }

  // Transpose of particles -> deposit -> delta -> P(k) for dL/dP_b (see dgp_power_spectrum_adjoint).
  int pk_adjoint(const dgp_particles* pp, int nbins, const double* dldp, dgp_particles* cot) override {
    if (!valid_parts(pp) || !valid_parts(cot) || pp->n == 0 || cot->n != pp->n || !dldp || nbins < 1 ||
        nbins > N / 2)
      return DGP_E_INVALID;
    int rc;
    T* delta = rH[0];
    if ((rc = deposit(pp, delta))) return rc;
    double k[256], pk[256];
    int64_t cnt[256];
    if ((rc = this->pk(delta, nbins, k, pk, cnt))) return rc;
    double hc[256];
    const double l3 = p.box * p.box * p.box;
    for (int b = 0; b < nbins; ++b)
      hc[b] = cnt[b] > 0 ? dldp[b] * l3 / ((double)M * (double)M * (double)cnt[b]) : 0.0;
    DGP_CUDA(cudaMemcpyAsync(d_pk, hc, sizeof(double) * nbins, cudaMemcpyHostToDevice, stream));
    if ((rc = forward_zy(delta, s6[0], ZPrologue{nullptr, 0.0, 0}))) return rc;
    const Coef c = coefficients(1.0, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, p.gravity);
    prof.run(KK_X_OTHER, 2 * SB, stream, [&] {
      launch_fft_x_op<T, N>(XOP_PK_ADJ, s6[0], nullptr, fs(s6 + 1, 1), 0, kp, d_pk, nbins, 0, 0, tw, stream);
    });
    T* o[1] = {rRho};
    if ((rc = inverse_yz(s6 + 1, o, 1))) return rc;
    // the deposit's transpose (the force term is absent: scale 0 on finite fields)
    T* const g3[3] = {rRho, rRho, rRho};
    const ParticleSet<T> xs{{(T*)pp->x, (T*)pp->y, (T*)pp->z, (T*)pp->x, (T*)pp->y, (T*)pp->z}};
    const ParticleSet<T> xb{{(T*)cot->x, (T*)cot->y, (T*)cot->z, (T*)cot->x, (T*)cot->y, (T*)cot->z}};
    prof.run(KK_GATHER, 6.0 * sizeof(T) * pp->n + RB, stream, [&] {
      launch_force_vjp_gather<T>(xs, 0.0, pp->n, g3, rRho, (double)M / (double)pp->n, xb, cic(), stream);
    });
    DGP_CHECK_LAUNCH();
    DGP_CUDA(wait_stream());  // hc is read by the copy above
    force_valid = false;
    return DGP_OK;
  }

  int bispec(const void* delta, double k1, double k2, int ntheta, const double* theta, double dk, double* b,
             double* q) override {
    if (!delta || ntheta < 0 || (ntheta > 0 && (!theta || !b || !q)) || !(k1 > 0) || !(k2 > 0))
      return DGP_E_INVALID;
    int rc;
    const double kf = 2.0 * M_PI / p.box;
    if (!(dk > 0)) dk = kf;
    // delta's S2 in s6[5]; each shell uses s6[0..1] and two real fields
    if ((rc = forward_zy((const T*)delta, s6[5], ZPrologue{nullptr, 0.0, 0}))) return rc;
    const Coef c = coefficients(1.0, cosmo.omega_m0, p.rc_H0);
    const KParams kp = kparams(c, p.gravity);
    auto shell = [&](double kc, T* d, T* ind) -> int {
      prof.run(KK_X_OTHER, 3 * SB, stream, [&] {
        launch_fft_x_op<T, N>(XOP_SHELL, s6[5], nullptr, fs(s6, 2), 0, kp, nullptr, 0, (kc - 0.5 * dk) / kf,
                              (kc + 0.5 * dk) / kf, tw, stream);
      });
      T* outs[2] = {d, ind};
      return inverse_yz(s6, outs, 2);
    };
    auto dot3 = [&](const T* x, const T* y, const T* z, double* hv) -> int {
      prof.run(KK_REDUCE, (z ? 3 : 2) * RB, stream,
               [&] { launch_product3_sum<T>(x, y, z, M, partials, nblocks, stream); });
      prof.run(KK_REDUCE, 8.0 * nblocks, stream, [&] { launch_finalize(partials, nblocks, 1, d_misc + 2, stream); });
      DGP_CHECK_LAUNCH();
      int r2 = fetch(d_misc + 2, 1);
      *hv = h_stats[0];
      return r2;
    };
    if ((rc = shell(k1, rH[0], rH[1]))) return rc;
    if ((rc = shell(k2, rH[2], rH[3]))) return rc;
    double d11, i11, d22, i22;
    if ((rc = dot3(rH[0], rH[0], nullptr, &d11)) || (rc = dot3(rH[1], rH[1], nullptr, &i11))) return rc;
    if ((rc = dot3(rH[2], rH[2], nullptr, &d22)) || (rc = dot3(rH[3], rH[3], nullptr, &i22))) return rc;
    const double L3M2 = p.box * p.box * p.box / ((double)M * (double)M);
    const double P1 = L3M2 * d11 / i11, P2 = L3M2 * d22 / i22;
    for (int i = 0; i < ntheta; ++i) {
      const double k3 = sqrt(k1 * k1 + k2 * k2 + 2.0 * k1 * k2 * cos(theta[i]));
      if ((rc = shell(k3, rH[4], rH[5]))) return rc;
      double ddd, iii, d33, i33;
      if ((rc = dot3(rH[0], rH[2], rH[4], &ddd)) || (rc = dot3(rH[1], rH[3], rH[5], &iii))) return rc;
      if ((rc = dot3(rH[4], rH[4], nullptr, &d33)) || (rc = dot3(rH[5], rH[5], nullptr, &i33))) return rc;
      const double P3 = L3M2 * d33 / i33;
      const double L6M3 = pow(p.box, 6) / ((double)M * (double)M * (double)M);
      b[i] = L6M3 * ddd / iii;
      q[i] = b[i] / (P1 * P2 + P2 * P3 + P3 * P1);
    }
    return DGP_OK;
  }
};

// Device bytes a context requests (the cudaMalloc sizes of init, the first sort,
// the first step adjoint and pm_step_host), without creating one.
template <typename T, int N>
static void workspace_bytes(int max_iter, int64_t np, dgp_workspace* w) {
  using V = vec2_t<T>;
  const size_t M = (size_t)N * N * N, SPEC = (size_t)(N / 2 + 1) * N * N;
  const size_t rb = sizeof(T) * M, sb = sizeof(V) * SPEC, pn = (size_t)np;
  const size_t nb = (size_t)num_sms() * 4;
  size_t fb;
  if constexpr (sizeof(T) == 4) fb = (size_t)relax_tma_blocks<N>();
  else fb = (size_t)fused_relax_blocks<T, N>();
  const size_t pblocks = fb > nb ? fb : nb;
  w->base = 14 * rb + 9 * sb + sizeof(double) * 4 * pblocks + sizeof(double) * (12 + 8) + sizeof(SolveCtl) +
            sizeof(double) * ((size_t)max_iter + 1) + sizeof(double) * 4 * (N / 2) * (size_t)x_pass_blocks<T, N>() +
            sizeof(double) * 4 * (N / 2) + sizeof(V) * 3 * N;
  w->sort = sizeof(int) * 3 * M + sizeof(int) * (size_t)sort_scan_blocks((int64_t)M) + (sizeof(int) + 6 * sizeof(T)) * pn;
  w->adjoint = sizeof(T) * (7 + 4 + 3) * M + sizeof(V) * 7 * SPEC + sizeof(double) * 12 + 6 * sizeof(T) * pn;
  w->host_step = 6 * sizeof(T) * pn;
}

template <typename T>
static bool workspace_for(int n, int max_iter, int64_t np, dgp_workspace* w) {
  switch (n) {
    case 16: workspace_bytes<T, 16>(max_iter, np, w); return true;
    case 32: workspace_bytes<T, 32>(max_iter, np, w); return true;
    case 64: workspace_bytes<T, 64>(max_iter, np, w); return true;
    case 128: workspace_bytes<T, 128>(max_iter, np, w); return true;
    case 256: workspace_bytes<T, 256>(max_iter, np, w); return true;
    case 512: workspace_bytes<T, 512>(max_iter, np, w); return true;
    case 48: workspace_bytes<T, 48>(max_iter, np, w); return true;
    case 96: workspace_bytes<T, 96>(max_iter, np, w); return true;
    default: return false;
  }
}

template <typename T>
static EngineBase* make_engine(int n) {
  switch (n) {
    case 16: return new (std::nothrow) Engine<T, 16>();
    case 32: return new (std::nothrow) Engine<T, 32>();
    case 64: return new (std::nothrow) Engine<T, 64>();
    case 128: return new (std::nothrow) Engine<T, 128>();
    case 256: return new (std::nothrow) Engine<T, 256>();
    case 512: return new (std::nothrow) Engine<T, 512>();
    case 48: return new (std::nothrow) Engine<T, 48>();
    case 96: return new (std::nothrow) Engine<T, 96>();
    default: return nullptr;
  }
}

}  // namespace dgp

struct dgp_ctx {
  dgp::EngineBase* eng;
};

extern "C" {

const char* dgp_strerror(int status) {
  switch (status) {
    case DGP_OK: return "ok";
    case DGP_E_INVALID: return "invalid argument";
    case DGP_E_CUDA: return "CUDA runtime error";
    case DGP_E_NOMEM: return "out of memory";
    case DGP_E_NONFINITE: return "non-finite value in input or solve";
    case DGP_E_NOT_CONVERGED: return "relaxation did not reach the tolerance (best iterate used)";
    case DGP_E_BAD_POINTS: return "discriminant clamped at some points";
    case DGP_E_TIMEOUT: return "device-side wait timed out";
    case DGP_E_STATE: return "invalid context state";
    default: return "unknown status";
  }
}

int dgp_background(const dgp_cosmology* cosmo, double rc_H0, double a, dgp_background_t* out) {
  if (!cosmo || !out || !(a > 0) || !(rc_H0 > 0) || !(cosmo->omega_m0 >= 0)) return DGP_E_INVALID;
  const dgp::Coef c = dgp::coefficients(a, cosmo->omega_m0, rc_H0);
  out->E = c.E; out->eta = c.eta; out->alpha = c.alpha; out->beta = c.beta; out->s = c.s;
  out->c2 = c.c2; out->c3 = c.c3; out->q = c.q; out->omega_m = c.omega_m;
  out->geff_local = dgp::geff_local(c);
  dgp::growth(a, cosmo->omega_m0, rc_H0, &out->growth_D, &out->growth_f);
  return DGP_OK;
}

int dgp_init(dgp_ctx** out, const dgp_params* p, const dgp_cosmology* cosmo, void* cuda_stream) {
  if (!out) return DGP_E_INVALID;
  *out = nullptr;
  if (!p || !cosmo) return DGP_E_INVALID;
  const int n = p->n;
  if (n != 16 && n != 32 && n != 48 && n != 64 && n != 96 && n != 128 && n != 256 && n != 512)
    return DGP_E_INVALID;
  if (!(p->box > 0) || !(p->rc_H0 > 0) || !(p->w >= 0 && p->w < 1) || p->max_iter < 0 || !(p->tol >= 0) ||
      !isfinite(p->tol) || p->sort_every < 0)
    return DGP_E_INVALID;
  if (p->precision < DGP_FP32 || p->precision > DGP_MIXED_F32R) return DGP_E_INVALID;
  if (p->gravity < DGP_GRAVITY_NL || p->gravity > DGP_GRAVITY_SPH) return DGP_E_INVALID;
  if (!(p->a_nonlinear >= 0.0) || !isfinite(p->a_nonlinear)) return DGP_E_INVALID;
  if (!(cosmo->omega_m0 > 0) || !(cosmo->c_over_H0 > 0)) return DGP_E_INVALID;
  dgp::EngineBase* e = p->precision == DGP_FP64 ? dgp::make_engine<double>(n) : dgp::make_engine<float>(n);
  if (!e) return DGP_E_NOMEM;
  e->p = *p;
  e->cosmo = *cosmo;
  e->stream = (cudaStream_t)cuda_stream;
  const int rc = e->init();
  if (rc != DGP_OK) {
    delete e;
    return rc;
  }
  dgp_ctx* c = new (std::nothrow) dgp_ctx;
  if (!c) {
    delete e;
    return DGP_E_NOMEM;
  }
  c->eng = e;
  *out = c;
  return DGP_OK;
}

void dgp_destroy(dgp_ctx* c) {
  if (!c) return;
  delete c->eng;
  delete c;
}

int dgp_reset(dgp_ctx* c) {
  if (!c) return DGP_E_INVALID;
  c->eng->reset();
  return DGP_OK;
}

int dgp_solve_phi(dgp_ctx* c, double a, const void* delta, void* phi, double tol, dgp_solve_info* info) {
  if (!c || !delta || !(a > 0) || !(tol >= 0)) return DGP_E_INVALID;
  return c->eng->solve(a, delta, phi, nullptr, nullptr, nullptr, tol, info);
}

int dgp_solve_forces(dgp_ctx* c, double a, const void* delta, void* phi, void* gx, void* gy, void* gz, double tol,
                     dgp_solve_info* info) {
  if (!c || !delta || !gx || !gy || !gz || !(a > 0) || !(tol >= 0)) return DGP_E_INVALID;
  return c->eng->solve(a, delta, phi, gx, gy, gz, tol, info);
}

int dgp_get_solution(dgp_ctx* c, void* D) {
  if (!c) return DGP_E_INVALID;
  return c->eng->get_solution(D);
}

int dgp_solve_history(dgp_ctx* c, double* out, int max_n) {
  if (!c || max_n < 0 || (max_n > 0 && !out)) return -DGP_E_INVALID;
  const std::vector<double>& h = c->eng->history;
  const int n = (int)h.size();
  for (int i = 0; i < n && i < max_n; ++i) out[i] = h[i];
  return n;
}

int dgp_profile(dgp_ctx* c, int timing) {
  if (!c) return DGP_E_INVALID;
  c->eng->prof.reset(timing != 0 ? (1u << dgp::KK_COUNT) - 1u : 0u);
  return DGP_OK;
}

int dgp_profile_kinds(dgp_ctx* c, unsigned kind_mask) {
  if (!c) return DGP_E_INVALID;
  c->eng->prof.reset(kind_mask & ((1u << dgp::KK_COUNT) - 1u));
  return DGP_OK;
}

}  // extern "C"

namespace dgp {
// One pm_step of a class of contexts (batch.cu): every context of the same mesh size,
// precision and stream, stepped with each kernel stage launched once for all of them.
int step_class(dgp_ctx* const* ctxs, int count, dgp_particles* parts, const double* a, const double* da,
               dgp_solve_info* info) {
  if (!ctxs || count < 1 || count > kBatchMax) return DGP_E_INVALID;
  EngineBase* m[kBatchMax];
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return DGP_E_INVALID;
    m[i] = ctxs[i]->eng;
  }
  return m[0]->step_class(m, count, parts, a, da, info);
}

void set_plane_pass(dgp_ctx* c, bool on) {
  if (c) c->eng->plane_pass = on;
}
}  // namespace dgp

extern "C" {

int dgp_set_wait_limit(dgp_ctx* c, double seconds, int withhold_first_copy) {
  if (!c || !(seconds > 0.0) || !(seconds <= 60.0)) return DGP_E_INVALID;
  c->eng->wait_ns = (unsigned long long)(seconds * 1e9);
  c->eng->withhold = withhold_first_copy ? 1 : 0;
  return DGP_OK;
}

int dgp_profile_sampled(dgp_ctx* c, unsigned kind_mask) {
  if (!c) return DGP_E_INVALID;
  c->eng->prof.reset(kind_mask & ((1u << dgp::KK_COUNT) - 1u), true);
  return DGP_OK;
}

int dgp_profile_read(dgp_ctx* c, int kind, int64_t* launches, double* bytes, int64_t* timed, double* ms,
                     double* timed_bytes) {
  if (!c || kind < 0 || kind >= dgp::KK_COUNT) return DGP_E_INVALID;
  dgp::Profiler& pr = c->eng->prof;
  const int rc = pr.resolve();
  if (rc != DGP_OK) return rc;
  if (launches) *launches = pr.launches[kind];
  if (bytes) *bytes = pr.bytes[kind];
  if (timed) *timed = pr.timed[kind];
  if (ms) *ms = pr.ms[kind];
  if (timed_bytes) *timed_bytes = pr.timed_bytes[kind];
  return DGP_OK;
}

const char* dgp_kernel_name(int kind) {
  if (kind < 0 || kind >= dgp::KK_COUNT) return nullptr;
  return dgp::kKernelNames[kind];
}

int dgp_deposit(dgp_ctx* c, const dgp_particles* parts, void* delta) {
  if (!c) return DGP_E_INVALID;
  return c->eng->deposit(parts, delta);
}

int dgp_zeldovich(dgp_ctx* c, const void* delta_l, double vel_factor, dgp_particles* out) {
  if (!c) return DGP_E_INVALID;
  return c->eng->zeldovich(delta_l, vel_factor, out);
}

int dgp_zeldovich_adjoint(dgp_ctx* c, const dgp_particles* cot, double vel_factor, void* delta_l_bar) {
  if (!c) return DGP_E_INVALID;
  return c->eng->zeldovich_adjoint(cot, vel_factor, delta_l_bar);
}

int dgp_power_spectrum_adjoint(dgp_ctx* c, const dgp_particles* parts, int nbins, const double* dl_dp,
                               dgp_particles* cot) {
  if (!c) return DGP_E_INVALID;
  return c->eng->pk_adjoint(parts, nbins, dl_dp, cot);
}

int pm_step_adjoint(dgp_ctx* c, const dgp_particles* start, double a, double da, dgp_particles* cot) {
  if (!c) return DGP_E_INVALID;
  return c->eng->step_adjoint(start, a, da, cot, nullptr);
}

int pm_step_adjoint_rc(dgp_ctx* c, const dgp_particles* start, double a, double da, dgp_particles* cot,
                       double* rc_bar) {
  if (!c || !rc_bar) return DGP_E_INVALID;
  return c->eng->step_adjoint(start, a, da, cot, rc_bar);
}

int dgp_zeldovich_vf_adjoint(dgp_ctx* c, const void* delta_l, const dgp_particles* cot, double* vf_bar) {
  if (!c) return DGP_E_INVALID;
  return c->eng->zeldovich_vf_adjoint(delta_l, cot, vf_bar);
}

int dgp_velocity_factor(const dgp_cosmology* cosmo, double rc_H0, double a, double* vf, double* dvf_drc) {
  if (!cosmo || !vf || !dvf_drc || !(a > 0) || !(rc_H0 > 0) || !(cosmo->omega_m0 >= 0)) return DGP_E_INVALID;
  dgp::velocity_factor(a, cosmo->omega_m0, rc_H0, vf, dvf_drc);
  return DGP_OK;
}

int dgp_solve_adjoint(dgp_ctx* c, const void* phibar, const void* gbar_x, const void* gbar_y, const void* gbar_z,
                      void* deltabar, double tol, dgp_solve_info* info) {
  if (!c) return DGP_E_INVALID;
  const void* g[3] = {gbar_x, gbar_y, gbar_z};
  return c->eng->adjoint(phibar, g, deltabar, tol, info, nullptr);
}

int dgp_solve_adjoint_rc(dgp_ctx* c, const void* phibar, const void* gbar_x, const void* gbar_y,
                         const void* gbar_z, void* deltabar, double tol, double* rc_bar, dgp_solve_info* info) {
  if (!c || !rc_bar) return DGP_E_INVALID;
  const void* g[3] = {gbar_x, gbar_y, gbar_z};
  return c->eng->adjoint(phibar, g, deltabar, tol, info, rc_bar);
}

int dgp_background_drc(const dgp_cosmology* cosmo, double rc_H0, double a, dgp_background_t* out) {
  if (!cosmo || !out || !(a > 0) || !(rc_H0 > 0) || !(cosmo->omega_m0 >= 0)) return DGP_E_INVALID;
  const double om = cosmo->omega_m0, h = dgp::cs_step(rc_H0);
  const dgp::Coef d = dgp::coefficients_drc(a, om, rc_H0);
  out->E = d.E; out->eta = d.eta; out->alpha = d.alpha; out->beta = d.beta; out->s = d.s;
  out->c2 = d.c2; out->c3 = d.c3; out->q = d.q; out->omega_m = d.omega_m;
  const dgp::CoefT<dgp::cplx> z = dgp::coefficients_t<dgp::cplx>(a, om, dgp::cplx(rc_H0, h));
  out->geff_local = dgp::geff_local_t<dgp::cplx>(z).imag() / h;
  dgp::cplx D, f;
  dgp::growth_t<dgp::cplx>(a, om, dgp::cplx(rc_H0, h), &D, &f);
  out->growth_D = D.imag() / h;
  out->growth_f = f.imag() / h;
  return DGP_OK;
}

int dgp_time_factors(const dgp_cosmology* cosmo, double rc_H0, double a0, double a1, double* out) {
  if (!cosmo || !out || !(a0 > 0) || !(a1 > 0) || !isfinite(a0) || !isfinite(a1) || !(rc_H0 > 0) ||
      !(cosmo->omega_m0 >= 0))
    return DGP_E_INVALID;
  const double om = cosmo->omega_m0;
  out[0] = dgp::time_integral(a0, a1, om, rc_H0, 0);
  out[1] = dgp::time_integral(a0, a1, om, rc_H0, 2);
  out[2] = dgp::time_integral_drc(a0, a1, om, rc_H0, 0);
  out[3] = dgp::time_integral_drc(a0, a1, om, rc_H0, 2);
  return DGP_OK;
}

int dgp_workspace_size(const dgp_params* p, int64_t np, dgp_workspace* out) {
  if (!p || !out || np < 0 || p->max_iter < 0) return DGP_E_INVALID;
  if (p->precision < DGP_FP32 || p->precision > DGP_MIXED_F32R) return DGP_E_INVALID;
  const bool ok = p->precision == DGP_FP64 ? dgp::workspace_for<double>(p->n, p->max_iter, np, out)
                                           : dgp::workspace_for<float>(p->n, p->max_iter, np, out);
  return ok ? DGP_OK : DGP_E_INVALID;
}

int dgp_tile_config(dgp_ctx* c, int* y_threads) {
  if (!c || !y_threads) return DGP_E_INVALID;
  *y_threads = c->eng->y_threads;
  return DGP_OK;
}

int dgp_set_tile_config(dgp_ctx* c, int y_threads) {
  if (!c || (y_threads != 128 && y_threads != 256 && y_threads != 512)) return DGP_E_INVALID;
  c->eng->y_threads = y_threads;
  return DGP_OK;
}

int dgp_set_hessian_fusion(dgp_ctx* c, int on) {
  if (!c) return DGP_E_INVALID;
  c->eng->xy_on = on != 0;
  return DGP_OK;
}

int dgp_hessian_fusion(dgp_ctx* c, int* active) {
  if (!c || !active) return DGP_E_INVALID;
  *active = (c->eng->xy_ok && c->eng->xy_on) ? 1 : 0;
  return DGP_OK;
}

int dgp_set_blocking_sync(dgp_ctx* c, int on) {
  if (!c) return DGP_E_INVALID;
  return c->eng->set_blocking(on != 0);
}

int dgp_brane_spectra(dgp_ctx* c, int nbins, double* k, double* pc, double* pC, double* delta_gradc,
                      int64_t* nmodes) {
  if (!c) return DGP_E_INVALID;
  return c->eng->brane(nbins, k, pc, pC, delta_gradc, nmodes);
}

int dgp_sort_particles(dgp_ctx* c, dgp_particles* parts, int32_t* cell_start) {
  if (!c) return DGP_E_INVALID;
  return c->eng->sort(parts, cell_start);
}

int pm_step(dgp_ctx* c, dgp_particles* parts, double a, double da, dgp_solve_info* info) {
  if (!c) return DGP_E_INVALID;
  return c->eng->step(parts, a, da, info);
}

int pm_step_host(dgp_ctx* c, dgp_particles* host_parts, double a, double da, dgp_solve_info* info) {
  if (!c) return DGP_E_INVALID;
  return c->eng->step_host(host_parts, a, da, info);
}

int power_spectrum(dgp_ctx* c, const void* delta, int nbins, double* k, double* pk, int64_t* nmodes) {
  if (!c) return DGP_E_INVALID;
  return c->eng->pk(delta, nbins, k, pk, nmodes);
}

int bispectrum(dgp_ctx* c, const void* delta, double k1, double k2, int ntheta, const double* theta, double dk,
               double* b, double* q) {
  if (!c) return DGP_E_INVALID;
  return c->eng->bispec(delta, k1, k2, ntheta, theta, dk, b, q);
}

}  // extern "C"
