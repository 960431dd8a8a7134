// Internal layout of a gq batch: descriptors, data blocks and vector offsets.
// Shared by the host planner (gq_host.cu) and the device code (gq_ipm.cu).
#pragma once
#include <cstdint>

#include "../../include/gq.h"

namespace gq {

// One stage of one QP.  Offsets index batch-wide arrays:
//   var  -> y / dy / r_g / ... (sum of nu+nx+2ns: [u; x; s^l; s^u]),
//   eq   -> pi / r_b (sum of nx_{n+1}),
//   side -> lambda / t / r_d (sum of 2 nc + 2 ns: lower sides, upper sides,
//           bounds of s^l, bounds of s^u),
//   ns   -> soft constraints (slack pairs) of the stage (Sec. 2.2),
//   data -> FP64 stage data block (may be shared), fac -> factor arena element.
struct StageDesc {
  int32_t nx, nu, nx1, nbu, nbx, ng;
  int32_t var, eq, side, ns;
  int64_t data;
  int64_t fac;
};
static_assert(sizeof(StageDesc) == 56, "StageDesc layout");

struct QpDesc {
  int32_t N, stage0;          // stage count - 1, index of stage 0 in the stage table
  int32_t var0, eq0, side0;   // first batch-vector index of this QP
  int32_t nvt, neqt, nsidet;  // lengths of this QP's vectors
  int32_t nvmax, nxmax;       // largest stage sizes of this QP
  int32_t warm;               // 0: arg.warm_start applies; 1 + level: this QP's own warm-start level
  int32_t nsoft;              // slack pairs over all stages (soft constraints; block kernel only)
  double cost;                // flop estimate of one Riccati factorisation
};
static_assert(sizeof(QpDesc) == 56, "QpDesc layout");

// Stage data block (elements), for nv = nu + nx, nb = nbu + nbx, nc = nb + ng:
//   BAt  nv x ldb row-major (ldb = nx1 rounded up to odd): row i holds
//        column i of [B A]   (row-of-[u;x] order)
//   b    nx1
//   RSQ  nv x ldr row-major (ldr = nv rounded up to odd), [[R, S], [S', Q]]
//   rq   nv, [r; q]
//   DC   ng x nv row-major, [D C]
//   lo   nc   (box u, box x, general), -inf masks the side
//   hi   nc
//   Zs   2 ns, [Zl; Zu]  diagonal slack Hessians      (only when ns > 0)
//   zs   2 ns, [zl; zu]  slack gradients
//   ls   2 ns, [lls; lus] lower bounds of s^l, s^u
//   box  int32 region of nint element slots: bidx[nb] (variable index of
//        box c within [u;x]) then bmap[nv] (box index of variable i, or -1);
//        with slacks also sidx[ns] (constraint relaxed by slack k) and
//        smap[nc] (slack of constraint c, or -1)
// The same element layout serves the FP64 block and its FP32 mirror (the box
// region is sized so that its int32 entries fit at either element width).
// Odd row strides keep lane-per-row shared-memory reads free of bank
// conflicts; blocks are padded to a multiple of four elements, so every block
// is a multiple of 16 bytes at both widths and starts on a 16-byte boundary
// (one bulk copy per stage).
__host__ __device__ inline int odd_ld(int n) { return n | 1; }
struct StageData {
  int64_t BAt, b, RSQ, rq, DC, lo, hi, Zs, zs, ls, box, size;
  int ldb, ldr, nint;
};
__host__ __device__ inline StageData stage_data_layout(int nx, int nu, int nx1, int nb, int ng, int ns) {
  StageData s;
  const int64_t nv = nx + nu, nc = nb + ng;
  s.ldb = odd_ld(nx1);
  s.ldr = odd_ld((int)nv);
  s.BAt = 0;
  s.b = s.BAt + nv * s.ldb;
  s.RSQ = s.b + nx1;
  s.rq = s.RSQ + nv * s.ldr;
  s.DC = s.rq + nv;
  s.lo = s.DC + (int64_t)ng * nv;
  s.hi = s.lo + nc;
  s.Zs = s.hi + nc;
  s.zs = s.Zs + 2 * ns;
  s.ls = s.zs + 2 * ns;
  s.box = s.ls + 2 * ns;
  s.nint = (int)(nb + nv + (ns > 0 ? ns + nc : 0));
  s.size = (s.box + s.nint + 3) & ~int64_t(3);
  return s;
}
__host__ __device__ inline StageData stage_data_layout(const StageDesc& st) {
  return stage_data_layout(st.nx, st.nu, st.nx1, st.nbu + st.nbx, st.ng, st.ns);
}

// Factor block of a stage: nv x odd_ld(nv) row-major, padded to a multiple of
// four elements so that every block starts on a 16-byte boundary (bulk copies).
__host__ __device__ inline int64_t fac_block_elems(int nv) { return ((int64_t)nv * odd_ld(nv) + 3) & ~int64_t(3); }

// Per-QP statistics at the head of the sol buffer (== gq_stats).
static_assert(sizeof(gq_stats) == 64, "gq_stats layout");

// Byte offsets of the regions of the three buffers.
struct Layout {
  // "in" buffer
  int64_t qpdesc, stagedesc, order, slots, data, in_bytes;
  // "sol" buffer
  int64_t stats, y, pi, lam, t, sol_bytes;
  // workspace: FP64 vectors then the factor arena
  int64_t rg, rb, rd, rm, dy, dpi, dlam, dt, lp, rg2, rb2, dy2, dpi2, dlam2, dt2, tinv, fac, data32, data32lo, matg, queue,
      ws_bytes;
};

// Kernel launch parameters (passed by value).
struct Batch {
  int32_t nqp, nvmax, nxmax, ngmax;
  int32_t nslots, pad;
  const QpDesc* qp;
  const StageDesc* st;
  const int32_t* order;
  const int32_t* slots;   // one stage index per distinct data block
  const double* data;
  float* data32;          // FP32 mirror of `data` (same element layout)
  gq_stats* stats;
  double *y, *pi, *lam, *t;
  double *rg, *rb, *rd, *rm, *dy, *dpi, *dlam, *dt, *lp, *rg2, *rb2, *dy2, *dpi2, *dlam2, *dt2, *tinv;
  void* fac;
  double* matg;           // per-QP stage-matrix scratch of the block kernel (global mode only)
  int32_t* queue;         // work-queue counters of the persistent launches (kQueue* slots)
  float* data32lo;        // FP32 remainder of `data`: data = data32 + data32lo to about 48 bits
};

// slots of Batch::queue: next QP index of each persistent launch of a solve
constexpr int kQueueWarp = 0, kQueueResume = 1, kQueueBlock = 2, kQueueSlots = 4;

}  // namespace gq
