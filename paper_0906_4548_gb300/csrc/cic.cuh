// CIC geometry shared by the deposit, the force gather and the cell sort
// (Sec. III.A: mesh points at x = i d, d = box / N, periodic).
#pragma once
#include "kernels.cuh"

namespace dgp {

// Lower mesh index i0 = floor(x / d) mod N, its periodic neighbour i1 and the
// offset f = x / d - floor(x / d) in [0, 1).  FP32: x N / box is carried as an
// unevaluated pair (hi + lo), so the floor and f see ~48 bits of the product.
__device__ __forceinline__ void cic_axis(float x, const CicParams& cp, int& i0, int& i1, float& f) {
  const float hi = x * cp.inv_d_hi;
  const float lo = fmaf(x, cp.inv_d_hi, -hi) + x * cp.inv_d_lo;
  float fl = floorf(hi);
  f = (hi - fl) + lo;
  if (f < 0.f) { f += 1.f; fl -= 1.f; }
  else if (f >= 1.f) { f -= 1.f; fl += 1.f; }
  int i = (int)fl;
  // positions inside the box need at most one wrap; the division only for the rest
  if (i >= cp.n) i -= cp.n;
  else if (i < 0) i += cp.n;
  if ((unsigned)i >= (unsigned)cp.n) {
    i %= cp.n;
    if (i < 0) i += cp.n;
  }
  i0 = i;
  i1 = (i + 1 == cp.n) ? 0 : i + 1;
}

__device__ __forceinline__ void cic_axis(double x, const CicParams& cp, int& i0, int& i1, double& f) {
  const double u = x * cp.inv_d;
  const double fl = floor(u);
  f = u - fl;
  long long i = (long long)fl % cp.n;
  if (i < 0) i += cp.n;
  i0 = (int)i;
  i1 = (i0 + 1 == cp.n) ? 0 : i0 + 1;
}

// Cell of the lower CIC corner, (i0x N + i0y) N + i0z: the counting-sort key.
template <typename T>
__device__ __forceinline__ int cic_cell(T x, T y, T z, const CicParams& cp) {
  int ix0, ix1, iy0, iy1, iz0, iz1;
  T f;
  cic_axis(x, cp, ix0, ix1, f);
  cic_axis(y, cp, iy0, iy1, f);
  cic_axis(z, cp, iz0, iz1, f);
  return (ix0 * cp.n + iy0) * cp.n + iz0;
}

}  // namespace dgp
