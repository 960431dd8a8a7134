// Internal layout of a gq batch: descriptors, data blocks and vector offsets.
// Shared by the host planner (gq_host.cu) and the device code (gq_ipm.cu).
#pragma once
#include <cstdint>

#include "../../include/gq.h"

namespace gq {

// One stage of one QP.  Offsets index batch-wide arrays:
//   var  -> y / dy / r_g / ... (sum of nu+nx),  eq -> pi / r_b (sum of nx_{n+1}),
//   side -> lambda / t / r_d (sum of 2 nc),     idx -> int arena,
//   data -> FP64 stage data block (may be shared), fac -> factor arena element.
struct StageDesc {
  int32_t nx, nu, nx1, nbu, nbx, ng;
  int32_t var, eq, side, idx;
  int64_t data;
  int64_t fac;
};
static_assert(sizeof(StageDesc) == 56, "StageDesc layout");

struct QpDesc {
  int32_t N, stage0;          // stage count - 1, index of stage 0 in the stage table
  int32_t var0, eq0, side0;   // first batch-vector index of this QP
  int32_t nvt, neqt, nsidet;  // lengths of this QP's vectors
  int32_t nvmax, nxmax;       // largest stage sizes of this QP
  int32_t pad0, pad1;
  double cost;                // flop estimate of one Riccati factorisation
};
static_assert(sizeof(QpDesc) == 56, "QpDesc layout");

// Stage data block (doubles), for nv = nu + nx, nc = nbu + nbx + ng:
//   BAt  nv x nx1 row-major: row i holds column i of [B A]   (row-of-[u;x] order)
//   b    nx1
//   RSQ  nv x nv row-major, [[R, S], [S', Q]]
//   rq   nv, [r; q]
//   DC   ng x nv row-major, [D C]
//   lo   nc   (box u, box x, general), -inf masks the side
//   hi   nc
// padded to an even number of doubles (16-byte alignment of every block).
struct StageData {
  int64_t BAt, b, RSQ, rq, DC, lo, hi, size;
};
__host__ __device__ inline StageData stage_data_layout(int nx, int nu, int nx1, int nb, int ng) {
  StageData s;
  const int64_t nv = nx + nu, nc = nb + ng;
  s.BAt = 0;
  s.b = s.BAt + nv * nx1;
  s.RSQ = s.b + nx1;
  s.rq = s.RSQ + nv * nv;
  s.DC = s.rq + nv;
  s.lo = s.DC + (int64_t)ng * nv;
  s.hi = s.lo + nc;
  s.size = (s.hi + nc + 1) & ~int64_t(1);
  return s;
}

// Per-QP statistics at the head of the sol buffer (== gq_stats).
static_assert(sizeof(gq_stats) == 64, "gq_stats layout");

// Byte offsets of the regions of the three buffers.
struct Layout {
  // "in" buffer
  int64_t qpdesc, stagedesc, order, idx, data, in_bytes;
  // "sol" buffer
  int64_t stats, y, pi, lam, t, sol_bytes;
  // workspace: FP64 vectors then the factor arena
  int64_t rg, rb, rd, rm, gt, dy, dpi, dlam, dt, lp, rg2, rb2, dy2, dpi2, fac, ws_bytes;
};

// Kernel launch parameters (passed by value).
struct Batch {
  int32_t nqp, nvmax, nxmax, ngmax;
  const QpDesc* qp;
  const StageDesc* st;
  const int32_t* order;
  const int32_t* idx;
  const double* data;
  gq_stats* stats;
  double *y, *pi, *lam, *t;
  double *rg, *rb, *rd, *rm, *gt, *dy, *dpi, *dlam, *dt, *lp, *rg2, *rb2, *dy2, *dpi2;
  void* fac;
};

}  // namespace gq
