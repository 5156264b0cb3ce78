// Entry points shared between the library's translation units (not part of the C ABI).
#pragma once

#include "../../include/dgp.h"

namespace dgp {

// Most realisations one class step launches together (kernels.cuh: kBatchMax).
constexpr int kClassMax = 16;

// One pm_step of every context in ctxs (same mesh size, precision and stream;
// nonlinear mode, FP32 data, n <= 128), with each kernel stage launched once
// for the whole class.  DGP_E_INVALID when the class does not qualify or an
// argument is bad (nothing has been stepped then).
int step_class(dgp_ctx* const* ctxs, int count, dgp_particles* parts, const double* a, const double* da,
               dgp_solve_info* info);

// Class solves of the context use the plane-resident Hessian pass where the mesh allows it
// (on, the default) or the separate x and y passes (off).
void set_plane_pass(dgp_ctx* c, bool on);

}  // namespace dgp
