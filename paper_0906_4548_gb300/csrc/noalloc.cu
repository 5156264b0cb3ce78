// power_spectrum without any device allocation (see dgp_power_spectrum_noalloc
// in include/dgp.h).
//
// Some callers cannot call cudaMalloc: a host framework that reserved the
// whole device for its own pooling allocator and refuses allocations made
// behind its back, or a long-running loop that is not allowed to allocate
// once it has started (allocation can block on the device and fragment the
// pool).  Creating a dgp context allocates its workspace, so such callers
// could not measure P(k) of a mesh field.  This file keeps every temporary of
// the P(k) path (the half spectrum, the twiddle tables, the per-block bin
// partials and the reduced bins) in one file-scope __device__ array of fixed
// size, enough for meshes up to 64^3.  The array is part of the loaded module:
// every GPU that loads the library holds it until the process exits.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/dgp.h"
#include "fft_core.cuh"
#include "kernels.cuh"

namespace dgp {
namespace {

constexpr int kMaxN = DGP_NOALLOC_MAX_N;
constexpr int kMaxBins = kMaxN / 2;
// x-pass blocks of the P(k) operation at the largest mesh (FP32)
constexpr int kMaxPkBlocks = (kMaxN / 16) * (kMaxN / 2 + 1);
constexpr size_t kSpecBytes = sizeof(float2) * (size_t)(kMaxN / 2 + 1) * kMaxN * kMaxN;
constexpr size_t kTwBytes = sizeof(float2) * 3 * kMaxN;  // one table set per mesh size
constexpr size_t kPartBytes = sizeof(double) * 3 * kMaxBins * (size_t)kMaxPkBlocks;
constexpr size_t kBinBytes = sizeof(double) * 3 * kMaxBins;
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// layout: [spectrum][twiddles N=16][twiddles N=32][twiddles N=64][partials][bins]
constexpr size_t kOffSpec = 0;
constexpr size_t kOffTw = align256(kOffSpec + kSpecBytes);
constexpr size_t kOffPart = align256(kOffTw + 3 * kTwBytes);
constexpr size_t kOffBins = align256(kOffPart + kPartBytes);
constexpr size_t kScratchBytes = align256(kOffBins + kBinBytes);
static_assert(kScratchBytes == DGP_NOALLOC_SCRATCH_BYTES, "scratch size in dgp.h is out of date");

static __device__ __align__(256) unsigned char g_pk_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};  // device address of g_pk_scratch, per device

// Twiddle tables of the four-step split, as the context engine builds them.
template <int N>
void twiddles(float2* out) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  auto w = [](int t) {
    const double ang = 2.0 * M_PI * (double)(t % N) / (double)N;
    return make_float2((float)cos(ang), (float)(-sin(ang)));
  };
  for (int t = 0; t < N; ++t) out[t] = w(t);
  for (int k1 = 0; k1 < N1; ++k1)
    for (int j2 = 0; j2 < N2; ++j2) out[N + k1 * N2 + j2] = w(j2 * k1);
  for (int m1 = 0; m1 < N2; ++m1)
    for (int k1 = 0; k1 < N1; ++k1) out[2 * N + m1 * N1 + k1] = w(k1 * m1);
}

// Once per device, with that device current: resolve the device address of
// the scratch array and write the twiddle tables into it.  The copy is ordered
// on the caller's stream and completed before the address is published, so no
// later call (on any stream) can read half-written tables.
int setup(int dev, cudaStream_t s, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev]) {
    *out = g_scratch_ptr[dev];
    return DGP_OK;
  }
  unsigned char* ptr = nullptr;
  if (cudaGetSymbolAddress((void**)&ptr, g_pk_scratch) != cudaSuccess || !ptr) return DGP_E_CUDA;
  std::vector<float2> tw(3 * 3 * kMaxN);
  twiddles<16>(tw.data());
  twiddles<32>(tw.data() + 3 * kMaxN);
  twiddles<64>(tw.data() + 6 * kMaxN);
  if (cudaMemcpyAsync(ptr + kOffTw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return DGP_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DGP_E_CUDA;
  g_scratch_ptr[dev] = ptr;
  *out = ptr;
  return DGP_OK;
}

template <int N>
int run(const float* delta, double box, int nbins, unsigned char* scratch, cudaStream_t s, double* host_bins) {
  float2* spec = reinterpret_cast<float2*>(scratch + kOffSpec);
  const int tsel = N == 16 ? 0 : (N == 32 ? 1 : 2);
  const float2* tw = reinterpret_cast<const float2*>(scratch + kOffTw + tsel * kTwBytes);
  double* parts = reinterpret_cast<double*>(scratch + kOffPart);
  double* bins = reinterpret_cast<double*>(scratch + kOffBins);
  launch_fft_z_r2c<float, N>(delta, 0, spec, 0, 1, ZPrologue{nullptr, 0.0, 0}, tw, s);
  FieldSet<float> f;
  for (int i = 0; i < kMaxFields; ++i) f.p[i] = i == 0 ? spec : nullptr;
  launch_fft_y<float, N>(f, 1, false, tw, s);
  KParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.box = box;
  kp.inv_m = 1.0 / ((double)N * N * N);
  kp.inv_m_f = (float)kp.inv_m;
  kp.kf_f = (float)(2.0 * M_PI / box);
  FieldSet<float> none;
  for (int i = 0; i < kMaxFields; ++i) none.p[i] = nullptr;
  launch_fft_x_op<float, N>(XOP_PK, spec, nullptr, none, 0, kp, parts, nbins, 0, 0, tw, s);
  launch_finalize(parts, x_pass_blocks<float, N>(), 3 * nbins, bins, s);
  if (cudaGetLastError() != cudaSuccess) return DGP_E_CUDA;
  if (cudaMemcpyAsync(host_bins, bins, sizeof(double) * 3 * nbins, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return DGP_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DGP_E_CUDA;
  return DGP_OK;
}

}  // namespace
}  // namespace dgp

extern "C" int dgp_power_spectrum_noalloc(const float* delta, int n, double box, int nbins, double* k, double* pk,
                                          int64_t* nmodes, void* cuda_stream) {
  using namespace dgp;
  if (n != 16 && n != 32 && n != 64) return DGP_E_INVALID;  // n > DGP_NOALLOC_MAX_N does not fit the scratch
  if (!delta || !k || !pk || !nmodes || !(box > 0) || nbins < 1 || nbins > n / 2) return DGP_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DGP_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DGP_E_INVALID;
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned char* scratch = nullptr;
  int rc = setup(dev, s, &scratch);
  if (rc != DGP_OK) return rc;
  double hb[3 * kMaxBins];
  if (n == 16) rc = run<16>(delta, box, nbins, scratch, s, hb);
  else if (n == 32) rc = run<32>(delta, box, nbins, scratch, s, hb);
  else rc = run<64>(delta, box, nbins, scratch, s, hb);
  if (rc != DGP_OK) return rc;
  for (int b = 0; b < nbins; ++b) {
    const double cnt = hb[b];
    nmodes[b] = (int64_t)llround(cnt);
    k[b] = cnt > 0 ? hb[nbins + b] / cnt : NAN;
    pk[b] = cnt > 0 ? hb[2 * nbins + b] / cnt : NAN;
  }
  return DGP_OK;
}
