// Unevaluated pairs of floats (hi + lo) with error-free transformations, the
// arithmetic of the relaxation's residual, split source and discriminant.
//   two_sum:  Knuth's TwoSum, a + b = s + e exactly (6 operations, any order);
//   fast:     the same when |a| >= |b| (3 operations; used to renormalise);
//   prod:     a b = p + e exactly, e = fma(a, b, -p) (the FMA form of Dekker's TwoProd).
// A sum of such pairs carried as (running TwoSum of the hi parts, plain sum of
// every error and lo part) keeps about 48 significant bits.
#pragma once

namespace dgp {

struct FP {
  float hi, lo;
};
__device__ __forceinline__ FP fp_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return FP{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FP fp_fast(float a, float b) {
  const float s = a + b;
  return FP{s, b - (s - a)};
}
__device__ __forceinline__ FP fp_prod(float a, float b) {
  const float p = a * b;
  return FP{p, fmaf(a, b, -p)};
}
// unnormalised accumulation: s.hi carries the running sum, s.lo the errors
__device__ __forceinline__ void fp_acc(FP& s, FP t) {
  const FP u = fp_two_sum(s.hi, t.hi);
  s.hi = u.hi;
  s.lo += u.lo + t.lo;
}
__device__ __forceinline__ FP pair_of(float x) { return FP{x, 0.f}; }
__device__ __forceinline__ FP pair_of(FP x) { return x; }

}  // namespace dgp
