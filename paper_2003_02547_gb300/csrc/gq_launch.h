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
  int32_t mat_global;  // block kernel: stage matrices in the global workspace (too large for shared memory)
  int32_t threads;     // block kernel: threads per block (0: 256)
  int32_t tc_off;      // block kernel: no tensor-core (tcgen05) products
};

// Column width of the block kernel's Cholesky panels.
constexpr int kBlockPanel = 8;

// Tensor-core (tcgen05) stage products of the block kernel's FP32 factor:
// stages with 128 <= nu + nx <= 256, nx_{n+1} <= 128 and no general rows.
// The operands pass through shared memory in K chunks of kTcK columns (TF32
// high and low parts of up to 256 rows), the accumulators live in
// kTcCols TMEM columns per block.
constexpr int kTcK = 16;
constexpr int kTcCols = 256;
__host__ __device__ inline bool tc_shape(const Shape& sh) {
  return !sh.tc_off && sh.nvmax >= 128 && sh.nvmax <= 256 && sh.nxmax <= 128 && sh.ngmax == 0;
}
__host__ __device__ inline size_t tc_tile_bytes() { return (size_t)256 * kTcK * 4; }

// Row stride of the block kernel's Phi and M' tiles: nv rounded up to 4.
__host__ __device__ inline int block_ld(int nv) { return (nv + 3) & ~3; }

// Elements (doubles) of the block kernel's stage-matrix scratch for a shape:
// L_{n+1} (nxmax^2), Phi (nvmax x block_ld), M' or X (wide x block_ld with
// wide = max(nxmax, ne_max)).
__host__ __device__ inline int64_t block_mat_elems(const Shape& sh) {
  const int wide = sh.nxmax > sh.ne_max ? sh.nxmax : sh.ne_max;
  const int64_t ld = block_ld(sh.nvmax);
  return ((int64_t)sh.nxmax * sh.nxmax + (int64_t)sh.nvmax * ld + ld * (wide > 0 ? wide : 1) + 15) & ~int64_t(15);
}

// QPs whose stages all have nu + nx <= 32 and nx <= 32 run one per warp.
constexpr int kWarpMaxNv = 32;

struct WarpPlan {
  size_t bars, stages, sL, sM, sP, sv, xb, ring0, ring1, fac_off, bytes;
  int vmax;
};
WarpPlan warp_plan(const Batch& b, const Shape& sh, int elem);  // elem: factor element size
cudaError_t launch_warp_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                            LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count);
// FP32 mirror of the stage data (values and their FP32 remainders), read by
// both kernels' FP32 factorisations and solves and the one-warp kernel's
// double-float residuals; launched before every mixed-precision launch pair
cudaError_t launch_mirror(const Batch& b, cudaStream_t stream);

constexpr size_t kMaxSmem = 227 * 1024;

// Dynamic shared-memory plan of the IPM kernel (byte offsets).
struct SmemPlan {
  size_t bars, red, chunk, vec, mat, panel, stages, tc, tcbar, ring0, ring1, ring_fac, bytes;
  int vmax;
  bool staged;  // stage blocks go through the bulk-copy ring
};
__host__ __device__ SmemPlan smem_plan(const Batch& b, const Shape& sh);

// Dynamic shared memory of the IPM kernel for this batch.
size_t ipm_smem_bytes(const Batch& b, const Shape& sh);

cudaError_t launch_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                       LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count);
// the same with the tensor-core products of large FP32 stages compiled in
size_t ipm_tc_smem_bytes(const Batch& b, const Shape& sh);
cudaError_t launch_ipm_tc(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                          LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count);
// the same with the slack elimination of soft constraints compiled in
cudaError_t launch_ipm_soft(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                       LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count);

}  // namespace gq
