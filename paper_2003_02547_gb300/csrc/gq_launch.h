// Launch interface between the host entry points and the IPM kernels.
#pragma once
#include <cuda_runtime.h>

#include "gq_internal.h"

namespace gq {

enum class LaunchKind { Solve, Residuals, NewtonStep, Resume };

// Output of a single Newton direction (row-level entry point).
struct DirOut {
  double *dy, *dpi, *dlam, *dt;
};

// Largest sizes over the QPs of one launch (a bucket of the batch); the
// shared-memory plans are sized from these.
struct Shape {
  int nst_max;       // largest N + 1
  int ne_max;        // largest eliminated block (nu_n, or nu_0 + nx_0 at stage 0)
  int nside_max;     // largest side count of one QP
  int nvmax, nxmax, ngmax;
  int64_t data_max;  // largest stage data block (elements)
};

// QPs whose stages all have nu + nx <= 32 and nx <= 32 run one per warp.
constexpr int kWarpMaxNv = 32;

struct WarpPlan {
  size_t bars, stages, sL, sM, sP, sv, ring0, ring1, fac_off, bytes;
  int vmax;
};
WarpPlan warp_plan(const Batch& b, const Shape& sh, int elem);  // elem: factor element size
cudaError_t launch_warp_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                            LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count);

constexpr size_t kMaxSmem = 227 * 1024;

// Dynamic shared-memory plan of the IPM kernel (byte offsets).
struct SmemPlan {
  size_t bars, red, chunk, vec, mat, stages, ring0, ring1, ring_fac, bytes;
  int vmax;
  bool staged;  // stage blocks go through the bulk-copy ring
};
__host__ __device__ SmemPlan smem_plan(const Batch& b, const Shape& sh);

// Dynamic shared memory of the IPM kernel for this batch.
size_t ipm_smem_bytes(const Batch& b, const Shape& sh);

cudaError_t launch_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                       LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count);

}  // namespace gq
