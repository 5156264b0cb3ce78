// The Hessian x pass fused with the six-field inverse y pass (fft_x.cu).
#pragma once

#include "kernels.cuh"

namespace dgp {

// FP32 data, N = 128 or 256, one thread-block cluster of N / 16 CTAs per kz plane: from the
// y-transformed spectrum in (layout S[kz][x][ky]), the six relaxation inputs H_xx, H_yy, H_xy,
// H_xz, H_yz, N in out.p[0..5], transformed back along x and y (layout S[kz][x][y]), as the
// Hessian x pass followed by the six-field inverse y pass leaves them.  No-op for other T or N.
// skip as for the other passes (read at entry; set by an earlier launch).
// xy_hessian_available(n): n qualifies and the current device co-schedules the cluster.
bool xy_hessian_available(int n);
template <typename T, int N>
void launch_xy_hessian(const vec2_t<T>* in, const FieldSet<T>& out, const KParams& kp, const vec2_t<T>* tw,
                       cudaStream_t s, const int* skip);
template <typename T, int N>
void launch_xy_hessian_batch(const XReal<T>* r, int count, const vec2_t<T>* tw, cudaStream_t s);

}  // namespace dgp
