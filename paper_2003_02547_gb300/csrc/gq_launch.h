// Launch interface between the host entry points and the IPM kernels.
#pragma once
#include <cuda_runtime.h>

#include "gq_internal.h"

namespace gq {

enum class LaunchKind { Solve, Residuals, NewtonStep };

// Output of a single Newton direction (row-level entry point).
struct DirOut {
  double *dy, *dpi, *dlam, *dt;
};

// Extra sizes the kernels need for their shared-memory plan.
struct Shape {
  int nst_max;  // largest N + 1
  int ne_max;   // largest eliminated block (nu_n, or nu_0 + nx_0 at stage 0)
  int nside_max;  // largest side count of one QP
};

constexpr size_t kMaxSmem = 227 * 1024;

// Dynamic shared memory of the IPM kernel for this batch.
size_t ipm_smem_bytes(const Batch& b, const Shape& sh);

cudaError_t launch_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                       LaunchKind kind, double sigma_mu, const DirOut* out);

}  // namespace gq
