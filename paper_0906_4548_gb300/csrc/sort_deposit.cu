// Counting sort of particles by CIC cell, and the CIC deposit that exploits it.
//
// Sort (locality support for the CIC assignment of Sec. III.A): key = cell of
// the lower CIC corner, (i0x N + i0y) N + i0z, computed by the same cic_axis as
// the deposit and the gather.  A histogram of keys, an exclusive scan of the
// histogram and a scatter through atomic cursors give the particles ordered by
// key; the order inside one cell is whatever the cursors hand out.
//
// Deposit (Eq. CIC) with warp-aggregated atomics: after a sort the particles
// of one cell sit in adjacent lanes, and a warp issues one set of eight
// atomics per cell it covers instead of one set per particle.  On unsorted
// input the kernel is the plain scatter of eight atomics per particle.
#include "cic.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace dgp {

template <typename T>
__global__ void __launch_bounds__(256) k_cell_hist(const T* __restrict__ x, const T* __restrict__ y,
                                                   const T* __restrict__ z, int64_t np, CicParams cp,
                                                   int* __restrict__ key, int* __restrict__ count) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const int c = cic_cell(x[p], y[p], z[p], cp);
    key[p] = c;
    atomicAdd(count + c, 1);
  }
}

// Exclusive scan of m ints in chunks of kScanChunk: chunk sums, a one-block
// scan of the sums, then each chunk scanned from its offset.
constexpr int kScanChunk = 2048;  // 256 threads x 8 elements

__global__ void __launch_bounds__(256) k_scan_sums(const int* __restrict__ in, int64_t m, int* __restrict__ sums) {
  __shared__ int s_w[8];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  int acc = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += 256)
    if (base + i < m) acc += in[base + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    sums[blockIdx.x] = t;
  }
}

__device__ __forceinline__ int warp_inclusive_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  return x;
}

// One block of 1024 threads: exclusive scan of the nb chunk sums, in place.
__global__ void __launch_bounds__(1024) k_scan_top(int* __restrict__ sums, int nb) {
  __shared__ int s_w[32];
  __shared__ int s_carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    __syncthreads();
    const int i = base + threadIdx.x;
    const int v = i < nb ? sums[i] : 0;
    const int x = warp_inclusive_scan(v, lane);
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) s_w[lane] = warp_inclusive_scan(s_w[lane], lane);
    __syncthreads();
    const int incl = x + (wid > 0 ? s_w[wid - 1] : 0) + s_carry;
    if (i < nb) sums[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
  }
}

__global__ void __launch_bounds__(256) k_scan_chunks(const int* __restrict__ in, int64_t m,
                                                     const int* __restrict__ sums, int* __restrict__ start,
                                                     int* __restrict__ cursor) {
  __shared__ int s_w[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * 8;
  int v[8], t = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v[j] = base + j < m ? in[base + j] : 0;
    t += v[j];
  }
  const int x = warp_inclusive_scan(t, lane);
  if (lane == 31) s_w[wid] = x;
  __syncthreads();
  int run = sums[blockIdx.x] + x - t;
  for (int w = 0; w < wid; ++w) run += s_w[w];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (base + j < m) {
      start[base + j] = run;
      cursor[base + j] = run;
    }
    run += v[j];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_scatter(const __grid_constant__ ParticleSet<T> in, int64_t np,
                                                 const int* __restrict__ key, int* __restrict__ cursor,
                                                 const __grid_constant__ ParticleSet<T> out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const int dst = atomicAdd(cursor + key[p], 1);
#pragma unroll
    for (int c = 0; c < 6; ++c) out.p[c][dst] = in.p[c][p];
  }
}

int sort_scan_blocks(int64_t m) { return (int)((m + kScanChunk - 1) / kScanChunk); }

template <typename T>
void launch_cell_sort(const ParticleSet<T>& parts, int64_t np, CicParams cp, const SortWork& w,
                      const ParticleSet<T>& tmp, cudaStream_t s) {
  const int64_t m = (int64_t)cp.n * cp.n * cp.n;
  cudaMemsetAsync(w.count, 0, sizeof(int) * m, s);
  int64_t blocks = (np + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (np > 0)
    k_cell_hist<T><<<(unsigned)blocks, 256, 0, s>>>(parts.p[0], parts.p[1], parts.p[2], np, cp, w.key, w.count);
  const int nb = sort_scan_blocks(m);
  k_scan_sums<<<nb, 256, 0, s>>>(w.count, m, w.sums);
  k_scan_top<<<1, 1024, 0, s>>>(w.sums, nb);
  k_scan_chunks<<<nb, 256, 0, s>>>(w.count, m, w.sums, w.start, w.cursor);
  if (np > 0) k_scatter<T><<<(unsigned)blocks, 256, 0, s>>>(parts, np, w.key, w.cursor, tmp);
}

// ---------------------------------------------------------------- deposit
// One particle per lane.  Lanes whose keys are equal and adjacent (a cell's
// particles, after a sort) form a segment, cut into pieces of at most 8 lanes: a
// segmented shuffle scan sums the eight corner weights over each piece and its
// last lane issues the eight global atomics.  A warp with no shared keys skips
// the scan.
template <typename T>
__device__ __forceinline__ void deposit_warp_body(const T* __restrict__ x, const T* __restrict__ y,
                                                  const T* __restrict__ z, int64_t np, T* __restrict__ rho,
                                                  const CicParams& cp, int64_t blk, int64_t nblk) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t n = cp.n;
  for (int64_t base = blk * blockDim.x; base < np; base += nblk * blockDim.x) {
    const int64_t p = base + threadIdx.x;
    const bool act = p < np;
    int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0};
    T f[3] = {(T)0, (T)0, (T)0};
    int key = -1 - lane;  // unique for lanes past the end
    if (act) {
      cic_axis(x[p], cp, i0[0], i1[0], f[0]);
      cic_axis(y[p], cp, i0[1], i1[1], f[1]);
      cic_axis(z[p], cp, i0[2], i1[2], f[2]);
      key = (int)((i0[0] * n + i0[1]) * n + i0[2]);
    }
    const T m = act ? (T)1 : (T)0;
    const T gx = m - m * f[0], fx = m * f[0];
    const T gy = (T)1 - f[1], gz = (T)1 - f[2];
    T w[8];
    w[0] = gx * gy * gz;
    w[1] = gx * gy * f[2];
    w[2] = gx * f[1] * gz;
    w[3] = gx * f[1] * f[2];
    w[4] = fx * gy * gz;
    w[5] = fx * gy * f[2];
    w[6] = fx * f[1] * gz;
    w[7] = fx * f[1] * f[2];
    const int prev = __shfl_up_sync(full, key, 1);
    unsigned heads = __ballot_sync(full, lane == 0 || prev != key);
    if (heads != full) {
      // segments of more than 8 lanes are cut into pieces of 8 (each piece issues its own
      // reductions), so three doubling rounds sum every piece
      const int seg_start = 31 - __clz(heads & (full >> (31 - lane)));
      heads = __ballot_sync(full, ((lane - seg_start) & 7) == 0);
      const int piece_start = 31 - __clz(heads & (full >> (31 - lane)));
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const bool take = lane - o >= piece_start;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const T v = __shfl_up_sync(full, w[t], o);
          if (take) w[t] += v;
        }
      }
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (act && tail) {
      const int64_t r00 = (i0[0] * n + i0[1]) * n, r01 = (i0[0] * n + i1[1]) * n;
      const int64_t r10 = (i1[0] * n + i0[1]) * n, r11 = (i1[0] * n + i1[1]) * n;
      atomicAdd(rho + r00 + i0[2], w[0]);
      atomicAdd(rho + r00 + i1[2], w[1]);
      atomicAdd(rho + r01 + i0[2], w[2]);
      atomicAdd(rho + r01 + i1[2], w[3]);
      atomicAdd(rho + r10 + i0[2], w[4]);
      atomicAdd(rho + r10 + i1[2], w[5]);
      atomicAdd(rho + r11 + i0[2], w[6]);
      atomicAdd(rho + r11 + i1[2], w[7]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_cic_deposit_warp(const T* __restrict__ x, const T* __restrict__ y,
                                                          const T* __restrict__ z, int64_t np, T* __restrict__ rho,
                                                          CicParams cp) {
  deposit_warp_body<T>(x, y, z, np, rho, cp, blockIdx.x, gridDim.x);
}

// Batched: realisation r = blockIdx.y
template <typename T> struct DepositBatch {
  DepositArgs<T> a[kBatchMax];
};
template <typename T>
__global__ void __launch_bounds__(256) k_cic_deposit_warp_batch(const __grid_constant__ DepositBatch<T> b) {
  const DepositArgs<T>& a = b.a[blockIdx.y];
  deposit_warp_body<T>(a.x, a.y, a.z, a.np, a.rho, a.cp, blockIdx.x, gridDim.x);
}

template <typename T>
void launch_cic_deposit_warp(const T* x, const T* y, const T* z, int64_t np, T* rho, CicParams cp, cudaStream_t s) {
  if (np <= 0) return;
  int64_t blocks = (np + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_cic_deposit_warp<T><<<(unsigned)blocks, 256, 0, s>>>(x, y, z, np, rho, cp);
}

template <typename T>
void launch_cic_deposit_batch(const DepositArgs<T>* a, int count, cudaStream_t s) {
  if (count < 1 || count > kBatchMax) return;
  DepositBatch<T> b;
  int64_t npmax = 0;
  for (int r = 0; r < count; ++r) {
    b.a[r] = a[r];
    npmax = a[r].np > npmax ? a[r].np : npmax;
  }
  if (npmax <= 0) return;
  int64_t blocks = (npmax + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16 / count + 1;
  if (blocks > cap) blocks = cap;
  k_cic_deposit_warp_batch<T><<<dim3((unsigned)blocks, (unsigned)count), 256, 0, s>>>(b);
}

#define DGP_INST_SORT(T)                                                                                   \
  template void launch_cell_sort<T>(const ParticleSet<T>&, int64_t, CicParams, const SortWork&,             \
                                    const ParticleSet<T>&, cudaStream_t);                                  \
  template void launch_cic_deposit_warp<T>(const T*, const T*, const T*, int64_t, T*, CicParams, cudaStream_t); \
  template void launch_cic_deposit_batch<T>(const DepositArgs<T>*, int, cudaStream_t);
DGP_INST_SORT(float)
DGP_INST_SORT(double)

}  // namespace dgp
