// Batched OCP-QP interior-point kernels for sm_103a.
//
// One thread block solves one QP: the whole Mehrotra predictor-corrector loop
// (Sec. 4.2) runs on the device, with
//   a1  residuals of eq. (delta)                                 FP64
//   a2  barrier terms and the reduced right-hand side, eq. (kkt)  FP64
//   a3  square-root Riccati factorisation (Sec. 3.3, variant b)   Tf
//   a4  Riccati solve: backward vector sweep, forward sweep        Tf
//   a5  affine step length and duality measure                    FP64
//   a6  Mehrotra corrector, conditional (Sec. 4.2)                 Tf solve
//   a7  iterative refinement on eq. (itref) (Sec. 3.4)             FP64 residual
//   a8  step, update, lower clamp of lambda and t (Sec. 4.2)       FP64
// Tf is double (plain path) or float (mixed path).
//
// Data movement.  Every phase walks the stages of its QP in order ("sweep").
// A sweep stages each stage's data block -- and in the solves its factor
// block -- into shared memory with one 1-D bulk copy (cp.async.bulk, the TMA
// unit) into a two-slot ring on mbarriers: stage n+-1 is in flight while
// stage n is computed, and every inner loop reads shared memory.  Stages too
// large for the ring are read from global memory by the same code.
//
// Riccati recursion used here.  The reduced system eq. (kkt) is the KKT system
// of an equality-constrained LQ problem with stage Hessians Ht_n = RSQ_n +
// C_n' W_n C_n and dynamics dx_{n+1} = A dx + B du + r_b,n.  With the
// cost-to-go Hessian P_{n+1} = L_{n+1} L_{n+1}' (Cholesky factor), each stage
// forms M = [B A]' L_{n+1}, Phi = Ht_n + M M' and its Cholesky factor
//   Lhat = [[L_ee, 0], [L_ke, L_kk]],
// where the leading "eliminated" block holds u_n (and also x_n at stage 0,
// which has no predecessor).  Then P_n = L_kk L_kk', so L_n = L_kk.  The
// leading block is inverted in place (X = L_ee^{-1}) so that every vector
// operation of the solves is a matrix-vector product:
//   backward: phi = gt_n + [B A]'(L_{n+1}(L_{n+1}' r_b,n) + p_{n+1}),
//             l = X phi_e,   p_n = phi_k - L_ke l
//   forward:  u_n = -X'(l + L_ke' x_n)   (stage 0: y_0 = -X' l),
//             x_{n+1} = [B A] y_n + r_b,n,
//             pi_{n+1} = L_{n+1}(L_{n+1}' x_{n+1}) + p_{n+1}.
#include <cuda_runtime.h>

#include <cstdint>

#include "gq_device.h"
#include "gq_internal.h"
#include "gq_launch.h"
#include "gq_mma.h"
#include "gq_soft.h"
#include "gq_tc.h"

// Soft constraints (Sec. 2.2): the slack elimination is compiled in only when
// GQ_IPM_SOFT is 1 (gq_ipm_soft.cu builds this file that way and exports
// launch_ipm_soft), so that the kernel for QPs without slacks keeps its
// register allocation; the host picks the variant per batch.
#ifndef GQ_IPM_SOFT
#define GQ_IPM_SOFT 0
#endif
// Tensor-core (tcgen05) stage products for large stages: compiled in only
// when GQ_IPM_TC is 1 (gq_ipm_tc.cu builds this file that way and exports
// launch_ipm_tc), so that the kernel for other batches keeps its register
// allocation; the host launches that variant for batches whose block bucket
// has large FP32 stages.
#ifndef GQ_IPM_TC
#define GQ_IPM_TC 0
#endif

namespace gq {

__host__ __device__ SmemPlan smem_plan(const Batch& b, const Shape& sh) {
  SmemPlan p;
  size_t o = 0;
  auto take = [&](size_t bytes, size_t align) {
    o = (o + align - 1) / align * align;
    const size_t at = o;
    o += bytes;
    return at;
  };
  p.vmax = sh.nvmax + sh.ngmax + 2;
  p.bars = take(2 * sizeof(uint64_t) + 16, 16);  // two mbarriers, then an int counter
  p.red = take(32 * sizeof(double), 16);
  p.chunk = take((size_t)((sh.nside_max + 31) / 32 + 1) * sizeof(double), 16);
  p.vec = take((size_t)8 * p.vmax * sizeof(double), 16);
  p.mat = sh.mat_global ? 0 : take((size_t)block_mat_elems(sh) * sizeof(double), 16);
  p.panel = take((size_t)(sh.nvmax > 0 ? sh.nvmax : 1) * kBlockPanel * sizeof(double), 16);
  p.stages = take((size_t)sh.nst_max * sizeof(StageDesc), 16);
  // tensor-core operand tiles (TF32 high and low parts of A and of B), the
  // MMA-completion mbarrier and the TMEM address
  if (GQ_IPM_TC && tc_shape(sh)) {
    p.tc = take(4 * tc_tile_bytes(), 1024);
    p.tcbar = take(16, 16);
  } else {
    p.tc = p.tcbar = 0;
  }
  // ring: two buffers of (data block + FP64-sized factor block)
  p.ring_fac = (size_t)((sh.data_max * 8 + 127) / 128 * 128);
  const size_t slot = p.ring_fac + (size_t)fac_block_elems(sh.nvmax) * sizeof(double);
  const size_t slot_al = (slot + 127) / 128 * 128;
  p.staged = ((o + 127) / 128 * 128) + 2 * slot_al <= kMaxSmem;
  if (p.staged) {
    p.ring0 = take(slot_al, 128);
    p.ring1 = take(slot_al, 128);
  } else {
    p.ring0 = p.ring1 = 0;
  }
  p.bytes = o;
  return p;
}

namespace {

constexpr double kLift = 1e-10;          // smallest floor of lambda, t after a lost FP64 pivot
constexpr double kLiftRel = 1e-2;        // ... relative to the stationarity residual
constexpr double kRegRetry = 1e-10;        // primal regularisation of an FP64 refactorisation after a lost pivot
constexpr double kInexact = 0.1;           // mixed path: direction residual allowed per unit of iterate residual

using namespace dev;

// ---------------------------------------------------------------------------
// block-wide reductions (max/min are exact, so their order does not matter)
// ---------------------------------------------------------------------------
struct OpMax {
  __device__ double operator()(double a, double b) const { return max_nan(a, b); }
};
struct OpMin {
  __device__ double operator()(double a, double b) const { return fmin(a, b); }
};

template <class Op>
__device__ double block_reduce(double v, double* red, Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = red[0];
  for (int i = 1; i < nw; ++i) r = op(r, red[i]);
  return r;
}

// ---------------------------------------------------------------------------
// per-block context
// ---------------------------------------------------------------------------
struct Ring {
  unsigned char* buf[2];
  uint64_t* bar;     // two mbarriers
  uint32_t parity;   // bit b: parity of the next phase of buffer b
  uint32_t fac_off;  // byte offset of the factor block within a buffer
  bool staged;       // false: read stages from global memory
  bool ok;           // every copy landed
};

struct Ctx {
  const Batch* B;
  const StageDesc* st;  // shared-memory copy of this QP's stage table
  int N;
  int nact;       // active (unmasked) sides
  int nside;      // all sides of this QP
  int v0, v1;     // this QP's range in the stage-variable vectors
  int e0, e1;     // ... in the dynamics vectors
  double* red;    // reduction scratch (32 doubles)
  double* chunk;  // per-32-side partial sums for fixed_sum
  double* vbuf;   // vector scratch (8 * vmax doubles)
  int vmax;
  void* panel;  // shared-memory copy of one Cholesky column panel (nv x kBlockPanel, Tf)
  void* mat;  // matrix scratch (Tf): L_{n+1}, Phi, M
  int nvmax, nxmax;
  bool classical;  // classical Riccati: explicit P_{n+1} in place of L_{n+1}
  bool array_qr;   // robust mode: chol(Ht + M M') by QR of [chol(Ht)'; M']
  Ring ring;
#if GQ_IPM_TC
  // tensor-core stage products (FP32 factor of large stages)
  bool tc;            // TMEM allocated and the shape qualifies
  uint32_t taddr;     // TMEM base address (kTcCols columns)
  uint64_t* tcbar;    // MMA-completion mbarrier
  uint32_t tcpar;     // its next phase parity
  float* tcA;         // A tile: high part, then the low part tc_tile_bytes() later
  float* tcB;         // B tile: high part, then the low part
#endif
};

// the tensor-core build updates the context inside the factorisation
#if GQ_IPM_TC
#define GQ_FCTX Ctx
#else
#define GQ_FCTX const Ctx
#endif

// Sum of f(i), i in [0, count), in an order fixed by `count` alone: 32-term
// chunks are reduced by a butterfly (bitwise identical in every lane), chunk
// sums are added by warp 0 in a fixed pattern.  The result does not depend on
// blockDim, so a QP gives the same bits alone or inside any batch.
template <class F>
__device__ double fixed_sum(const Ctx& C, int count, F f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nch = (count + 31) >> 5;
  for (int c = warp; c < nch; c += nw) {
    const int i = c * 32 + lane;
    double v = i < count ? f(i) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) C.chunk[c] = v;
  }
  __syncthreads();
  if (warp == 0) {
    double r = 0.0;
    for (int c = lane; c < nch; c += 32) r += C.chunk[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) C.red[0] = r;
  }
  __syncthreads();
  const double r = C.red[0];
  __syncthreads();
  return r;
}

// Sum of f(k) for k in [k0, k1) in four interleaved partial sums (a fixed
// order that depends on k0, k1 only): short dependent FMA chains.
template <typename Tf, class F>
__device__ __forceinline__ Tf dot4(int k0, int k1, F f) {
  Tf a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int k = k0;
  for (; k + 3 < k1; k += 4) {
    a0 += f(k);
    a1 += f(k + 1);
    a2 += f(k + 2);
    a3 += f(k + 3);
  }
  for (; k < k1; ++k) a0 += f(k);
  return (a0 + a1) + (a2 + a3);
}

// Row-parallel dot products: for every row r < nrows, out(r, sum of term(r, k)
// over k in [lo(r), hi(r))).  Each row gets tpr consecutive lanes (8, 4, 2 or 1
// so that all rows fit the block at once when they can); lane `sub` of a
// group sums k = lo + sub, lo + sub + tpr, ... in four interleaved partial
// sums, and the group combines by a butterfly.  The order depends on the
// row's range and tpr only (tpr on nrows and blockDim), and every warp runs
// the same number of rounds, so all shuffles are warp-uniform.
template <typename V, class Lo, class Hi, class Term, class Out>
__device__ __forceinline__ void rows_dot(int nrows, Lo lo, Hi hi, Term term, Out out) {
  const int NT = blockDim.x, tid = threadIdx.x;
  const int tpr = nrows * 8 <= NT ? 8 : (nrows * 4 <= NT ? 4 : (nrows * 2 <= NT ? 2 : 1));
  const int groups = NT / tpr, sub = tid & (tpr - 1);
  const int rounds = (nrows + groups - 1) / groups;
  for (int m = 0; m < rounds; ++m) {
    const int r = m * groups + tid / tpr;
    V a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if (r < nrows) {
      const int k1 = hi(r), st = 4 * tpr;
      int k = lo(r) + sub;
      for (; k + 3 * tpr < k1; k += st) {
        a0 += term(r, k);
        a1 += term(r, k + tpr);
        a2 += term(r, k + 2 * tpr);
        a3 += term(r, k + 3 * tpr);
      }
      for (; k < k1; k += tpr) a0 += term(r, k);
    }
    V acc = (a0 + a1) + (a2 + a3);
    for (int o = 1; o < tpr; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (r < nrows && sub == 0) out(r, acc);
  }
}

__device__ __forceinline__ StageData lay(const StageDesc& s) {
  return stage_data_layout(s);
}
__device__ __forceinline__ const int32_t* box_idx(const double* D, const StageData& L) {
  return reinterpret_cast<const int32_t*>(D + L.box);
}
__device__ __forceinline__ int elim_size(const StageDesc& s, int n) { return n == 0 ? s.nx + s.nu : s.nu; }

template <typename Tf>
__device__ __forceinline__ Tf* fac_global(const Batch& B, const StageDesc& s) {
  return reinterpret_cast<Tf*>(static_cast<double*>(B.fac) + s.fac);
}

// value of constraint c of stage s at the stage vector y (length nv)
__device__ __forceinline__ double cons_value(const StageDesc& s, const StageData& L, const double* D, int c,
                                             const double* y) {
  const int nb = s.nbu + s.nbx;
  if (c < nb) return y[box_idx(D, L)[c]];
  const int nv = s.nx + s.nu;
  const double* row = D + L.DC + (int64_t)(c - nb) * nv;
  double v = 0.0;
  for (int j = 0; j < nv; ++j) v = fma(row[j], y[j], v);
  return v;
}

// ---------------------------------------------------------------------------
// stage sweeps over the bulk-copy ring
// ---------------------------------------------------------------------------
// stage data of the precision data_elem selects: the FP64 block (8) or its
// FP32 mirror (4, the same element layout)
__device__ __forceinline__ const void* stage_data(const Batch& B, const StageDesc& s, int data_elem) {
  return data_elem == 4 ? static_cast<const void*>(B.data32 + s.data) : static_cast<const void*>(B.data + s.data);
}

__device__ __forceinline__ void ring_issue(Ctx& C, int n, int b, int fac_elem, int data_elem) {
  const Batch& B = *C.B;
  const StageDesc& s = C.st[n];
  if (threadIdx.x == 0) {
    const uint32_t dbytes = (uint32_t)(lay(s).size * data_elem);
    const uint32_t fbytes = fac_elem ? (uint32_t)(fac_block_elems(s.nx + s.nu) * fac_elem) : 0u;
    fence_async_shared();
    mbar_arrive_expect_tx(&C.ring.bar[b], dbytes + fbytes);
    bulk_g2s(C.ring.buf[b], stage_data(B, s, data_elem), dbytes, &C.ring.bar[b]);
    if (fbytes)
      bulk_g2s(C.ring.buf[b] + C.ring.fac_off, static_cast<const unsigned char*>(B.fac) + s.fac * 8, fbytes,
               &C.ring.bar[b]);
  }
}

__device__ __forceinline__ void ring_wait(Ctx& C, int b) {
  // once a copy is lost the QP's results are void: stop waiting
  const bool ok = C.ring.ok && mbar_wait(&C.ring.bar[b], (C.ring.parity >> b) & 1u);
  C.ring.parity ^= 1u << b;
  C.ring.ok = C.ring.ok && ok;
}

// Calls f(n, D, F) for every stage, forward or backward.  D is the stage data
// block (FP64, or with data_elem 4 its FP32 mirror: the callee reads it as
// its factor type) and F (when fac_elem > 0) the stage factor block, both in
// shared memory when the ring is on.  f may synchronise internally; the sweep
// adds a barrier after each stage before its buffer is refilled.
template <class F>
__device__ void sweep(Ctx& C, bool backward, int fac_elem, F f, int data_elem = 8) {
  const Batch& B = *C.B;
  const int N = C.N;
  if (!C.ring.staged) {
    for (int k = 0; k <= N; ++k) {
      const int n = backward ? N - k : k;
      const StageDesc& s = C.st[n];
      const unsigned char* fac = static_cast<const unsigned char*>(B.fac) + s.fac * 8;
      f(n, static_cast<const double*>(stage_data(B, s, data_elem)), static_cast<const void*>(fac));
      __syncthreads();
    }
    return;
  }
  ring_issue(C, backward ? N : 0, 0, fac_elem, data_elem);
  for (int k = 0; k <= N; ++k) {
    const int n = backward ? N - k : k, b = k & 1;
    if (k < N) ring_issue(C, backward ? n - 1 : n + 1, b ^ 1, fac_elem, data_elem);
    ring_wait(C, b);
    f(n, reinterpret_cast<const double*>(C.ring.buf[b]), static_cast<const void*>(C.ring.buf[b] + C.ring.fac_off));
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// a1: residual function of eq. (delta) for one stage.  With `lin` the constant
// terms (r, q, b and bounds) are dropped and (add_g, add_b) are added instead:
// that is the iterative-refinement residual of Sec. 3.4 for a direction.
// Updates the running max of |r_g|, |r_b| (and |r_d| when rd != nullptr).
// ---------------------------------------------------------------------------
struct Max3 {
  double g, b, d;
};

__device__ void stage_residual(const Ctx& C, int n, const double* D, const double* y, const double* pi,
                               const double* lam, const double* t, double* og, double* ob, double* rd, bool lin,
                               const double* add_g, const double* add_b, Max3& mx) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const StageDesc s = C.st[n];
  const StageData L = lay(s);
  const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
  const double* yn = y + s.var;
  const double* lm = lam + s.side;
  const int32_t* bmap = box_idx(D, L) + nb;
  // r_g rows: [RSQ row | [B A]' row] . [y_n | pi_{n+1}], then the rest
  {
    const double* pn1 = pi + s.eq;
    const int kend = n < C.N ? nv + nx1 : nv;
    rows_dot<double>(
        nv, [&](int) { return 0; }, [&](int) { return kend; },
        [&](int i, int k) {
          return k < nv ? D[L.RSQ + (int64_t)i * L.ldr + k] * yn[k] : D[L.BAt + (int64_t)i * L.ldb + (k - nv)] * pn1[k - nv];
        },
        [&](int i, double v) {
          double acc = (lin ? add_g[s.var + i] : D[L.rq + i]) + v;
          if (n > 0 && i >= s.nu) acc -= pi[C.st[n - 1].eq + (i - s.nu)];
          for (int g = 0; g < s.ng; ++g)
            acc = fma(-D[L.DC + (int64_t)g * nv + i], lm[nb + g] - lm[nc + nb + g], acc);
          if (nb > 0) {
            const int c = bmap[i];
            if (c >= 0) acc -= lm[c] - lm[nc + c];
          }
          og[s.var + i] = acc;
          mx.g = max_nan(mx.g, fabs(acc));
        });
  }
  if (n < C.N) {
    const double* yn1 = y + C.st[n + 1].var + C.st[n + 1].nu;
    rows_dot<double>(
        nx1, [&](int) { return 0; }, [&](int) { return nv; },
        [&](int k, int i) { return D[L.BAt + (int64_t)i * L.ldb + k] * yn[i]; },
        [&](int k, double v) {
          const double acc = (lin ? add_b[s.eq + k] : D[L.b + k]) + v - yn1[k];
          ob[s.eq + k] = acc;
          mx.b = max_nan(mx.b, fabs(acc));
        });
  }
  if (rd != nullptr) {
    for (int c = tid; c < nc; c += NT) {
      const double v = cons_value(s, L, D, c, yn);
      const double lo = D[L.lo + c], hi = D[L.hi + c];
      const int il = s.side + c, iu = s.side + nc + c;
      double a = 0.0, b = 0.0;
      if (lo != -INFINITY) a = lo - v + t[il];
      if (hi != INFINITY) b = v - hi + t[iu];
      if (GQ_IPM_SOFT && s.ns > 0) {
        // a relaxed side's row also holds its slack (Sec. 2.2)
        const int k = soft::soft_smap(box_idx(D, L), nb, nv, s.ns)[c];
        if (k >= 0) {
          if (lo != -INFINITY) a -= yn[nv + k];
          if (hi != INFINITY) b -= yn[nv + s.ns + k];
        }
      }
      rd[il] = a;
      rd[iu] = b;
      mx.d = max_nan(mx.d, max_nan(fabs(a), fabs(b)));
    }
  }
  if (GQ_IPM_SOFT && s.ns > 0) {
    // slack stationarity rows and the slack bound sides
    const int32_t* sidx = soft::soft_sidx(box_idx(D, L), nb, nv);
    for (int k = tid; k < s.ns; k += NT) {
      const soft::SoftSlot q = soft::soft_slot(s, nv, nc, k, sidx[k]);
      double sl, su, mg, md;
      soft::soft_residual(D, L, s.ns, k, q, y, lam, t, og, rd, lin, add_g, &sl, &su, &mg, &md);
      mx.g = max_nan(mx.g, mg);
      mx.d = max_nan(mx.d, md);
    }
  }
}

struct Norms {
  double g, b, d, mu;
};

__device__ Norms residuals(Ctx& C) {
  const Batch& B = *C.B;
  Max3 mx{0.0, 0.0, 0.0};
  sweep(C, false, 0, [&](int n, const double* D, const void*) {
    stage_residual(C, n, D, B.y, B.pi, B.lam, B.t, B.rg, B.rb, B.rd, false, nullptr, nullptr, mx);
  });
  // masked sides hold lambda = 0 and add nothing
  const int s0 = C.st[0].side;
  const double* lam = B.lam + s0;
  const double* tt = B.t + s0;
  const double sm = fixed_sum(C, C.nside, [&](int i) { return lam[i] * tt[i]; });
  Norms r;
  r.g = block_reduce(mx.g, C.red, OpMax());
  r.b = block_reduce(mx.b, C.red, OpMax());
  r.d = block_reduce(mx.d, C.red, OpMax());
  r.mu = C.nact ? sm / C.nact : 0.0;
  return r;
}

// ---------------------------------------------------------------------------
// a3: square-root Riccati factorisation, one stage (called for n = N..0)
// ---------------------------------------------------------------------------
// Register micro-tiles of kT x kT outputs per thread for the stage products,
// and a Cholesky panel width; tiles are dealt to threads round-robin, and each
// output's sum runs in a fixed order, so the result does not depend on
// blockDim.
constexpr int kT = 4;
constexpr int kPanel = kBlockPanel;

// lower-triangle tile index -> (I, J), J <= I
__device__ __forceinline__ void tri_tile(int t, int& I, int& J) {
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}

#if GQ_IPM_TC
// ---------------------------------------------------------------------------
// Tensor-core stage products of the FP32 factor (tcgen05, Blackwell):
//   M = [B A]' L_{n+1}          (nv x nx1, stored transposed as M')
//   Phi = RSQ + M M' + diag     (lower triangle)
// Each FP32 operand is split into a TF32 high part and a TF32 remainder and
// three kind::tf32 MMAs (lo*hi + hi*lo + hi*hi) accumulate in FP32 in TMEM,
// which keeps the products at FP32 accuracy.  Operand chunks of kTcK columns
// are staged in shared memory by all threads in the K-major layout of gq_tc.h;
// one thread issues the MMAs of a chunk and commits them to an mbarrier that
// every thread waits on (bounded) before the next chunk is staged.  Rows are
// padded to 128 (one M = 128 tile) or 256 (two tiles); zero padding.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tc_put(float* tile, int r, int k, float v) {
  const uint32_t o = tc::kmajor_off(r, k, kTcK) >> 2;
  const float hi = tc::tf32_round(v);
  tile[o] = hi;
  tile[o + (tc_tile_bytes() >> 2)] = tc::tf32_round(v - hi);
}

// one chunk: D[tile t] (+)= A[rows t*128..] B^T for every tile t in [t0, t1),
// B rows starting at brow, N columns; accumulate after the first chunk
__device__ __forceinline__ void tc_chunk_mma(Ctx& C, int t0, int t1, int brow, int N, uint32_t dcol, bool acc) {
  if (threadIdx.x == 0) {
    tc::fence_after();
    const uint32_t sbo = (kTcK / 4) * 128, lo = (uint32_t)tc_tile_bytes();
    const uint32_t a0 = tc::s32(C.tcA), b0 = tc::s32(C.tcB) + (uint32_t)(brow / 8) * sbo;
    const uint32_t id = tc::idesc_tf32(128, N);
    for (int t = t0; t < t1; ++t) {
      const uint32_t d = C.taddr + dcol + (uint32_t)((t - t0) * N);
      const uint32_t at = a0 + (uint32_t)(t * 16) * sbo;
#pragma unroll
      for (int s8 = 0; s8 < kTcK; s8 += 8) {
        const uint32_t ko = (uint32_t)s8 * 32;  // two core matrices along K per step
        const uint64_t ah = tc::sdesc(at + ko, 128, sbo), al = tc::sdesc(at + lo + ko, 128, sbo);
        const uint64_t bh = tc::sdesc(b0 + ko, 128, sbo), bl = tc::sdesc(b0 + lo + ko, 128, sbo);
        tc::mma_tf32(d, al, bh, id, acc || s8 > 0);
        tc::mma_tf32(d, ah, bl, id, true);
        tc::mma_tf32(d, ah, bh, id, true);
      }
    }
    tc::commit(C.tcbar);
  }
  // every thread waits for the chunk's MMAs (bounded; a lost completion
  // makes the QP time out like a lost bulk copy)
  const bool ok = C.ring.ok && mbar_wait(C.tcbar, C.tcpar);
  C.tcpar ^= 1u;
  C.ring.ok = C.ring.ok && ok;
  tc::fence_after();
}

__device__ __noinline__ void tc_products(Ctx& C, int n, const float* D, const StageData& L, const StageDesc& s, float* sL,
                            float* sPhi, float* sMt, int ldP, const float* sw, const int32_t* bmap, double reg) {
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, w = tid >> 5;
  const int nv = s.nx + s.nu, nx1 = s.nx1, nb = s.nbu + s.nbx;
  const int R = nv <= 128 ? 128 : 256, nt = R / 128;
  // ---- M = [B A]' L_{n+1}: rows i < R of [B A]', columns j < N1 of L
  const int N1 = (nx1 + 15) & ~15;
  for (int kc = 0; kc < nx1; kc += kTcK) {
    for (int e = tid; e < R * kTcK; e += NT) {
      const int r = e / kTcK, k = e - r * kTcK, kk = kc + k;
      tc_put(C.tcA, r, k, (r < nv && kk < nx1) ? (float)D[L.BAt + (int64_t)r * L.ldb + kk] : 0.f);
    }
    for (int e = tid; e < N1 * kTcK; e += NT) {
      const int j = e / kTcK, k = e - j * kTcK, kk = kc + k;
      // B[j][k] = L[k][j] (L lower triangular)
      tc_put(C.tcB, j, k, (j < nx1 && kk < nx1 && kk >= j) ? sL[kk * nx1 + j] : 0.f);
    }
    fence_async_shared();
    __syncthreads();
    tc_chunk_mma(C, 0, nt, 0, N1, 0, kc > 0);
  }
  // M' from TMEM: warp w reads rows 32 (w % 4) .. of tile w / 4
  if (w / 4 < nt) {
    const int t = w / 4, i = t * 128 + 32 * (w & 3) + lane;
    for (int c0 = 0; c0 < N1; c0 += 16) {
      float v[16];
      tc::ld16(C.taddr + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(t * N1 + c0), v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (i < nv && c0 + j < nx1) sMt[(c0 + j) * ldP + i] = v[j];
    }
  }
  tc::fence_before();
  __syncthreads();
  // ---- Phi = M M': column blocks of 128; block cb needs row tiles t >= cb
  for (int cb = 0; cb * 128 < nv; ++cb) {
    const int N2 = ((nv - cb * 128 < 128 ? nv - cb * 128 : 128) + 15) & ~15;
    for (int kc = 0; kc < nx1; kc += kTcK) {
      for (int e = tid; e < R * kTcK; e += NT) {
        const int r = e / kTcK, k = e - r * kTcK, kk = kc + k;
        tc_put(C.tcA, r, k, (r < nv && kk < nx1) ? sMt[kk * ldP + r] : 0.f);
      }
      fence_async_shared();
      __syncthreads();
      // B = rows cb*128.. of the same tile (M M' is symmetric in its operands)
      C.tcB = C.tcA;
      tc_chunk_mma(C, cb, nt, cb * 128, N2, 0, kc > 0);
      C.tcB = C.tcA + 2 * (tc_tile_bytes() >> 2);
    }
    if (w / 4 + cb < nt) {
      const int t = cb + w / 4, i = t * 128 + 32 * (w & 3) + lane;
      for (int c0 = 0; c0 < N2; c0 += 16) {
        float v[16];
        tc::ld16(C.taddr + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)((t - cb) * N2 + c0), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jj = cb * 128 + c0 + j;
          if (i < nv && jj <= i) {
            float x = (float)D[L.RSQ + (int64_t)i * L.ldr + jj] + v[j];
            if (i == jj) {
              x += (float)reg;
              if (nb > 0 && bmap[i] >= 0) x += sw[bmap[i]];
            }
            sPhi[i * ldP + jj] = x;
          }
        }
      }
    }
    tc::fence_before();
    __syncthreads();
  }
}

#endif  // GQ_IPM_TC

// D: the stage data in the factor's precision (the FP32 mirror for Tf = float)
template <typename Tf>
__device__ bool factor_stage(GQ_FCTX& C, int n, const Tf* D, double reg) {
  const Batch& B = *C.B;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ldP = block_ld(C.nvmax);
  Tf* sL = static_cast<Tf*>(C.mat);        // L_{n+1}: nx1 x nx1 (ld nx1), zero above the diagonal
  Tf* sPhi = sL + C.nxmax * C.nxmax;       // nv x nv (ld ldP)
  Tf* sMt = sPhi + C.nvmax * ldP;          // M': nx1 x nv (ld ldP), later X
  Tf* sw = reinterpret_cast<Tf*>(C.vbuf);  // per-constraint weight
  bool ok = true;
  const StageDesc s = C.st[n];
  const StageData L = lay(s);
  const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
  const int ne = elim_size(s, n), nk = nv - ne;
  const double* lm = B.lam + s.side;
  const double* tt = B.t + s.side;
  const double* D64 = B.data + s.data;  // FP64 stage data (global) where exact values are needed
  const int32_t* bmap = reinterpret_cast<const int32_t*>(D + L.box) + nb;
  // barrier weights W_lo + W_hi per constraint
  for (int c = tid; c < nc; c += NT) {
    double w = 0.0;
    if (D[L.lo + c] != -INFINITY) w += lm[c] / tt[c];
    if (D[L.hi + c] != INFINITY) w += lm[nc + c] / tt[nc + c];
    sw[c] = (Tf)w;
  }
  if (GQ_IPM_SOFT && s.ns > 0) {
    // relaxed constraints: their slacks eliminated into the weight (Sec. 2.2)
    __syncthreads();
    const int32_t* sidx = soft::soft_sidx(box_idx(D64, L), nb, nv);
    for (int k = tid; k < s.ns; k += NT) {
      const int c = sidx[k];
      const soft::SoftSlot q = soft::soft_slot(s, nv, nc, k, c);
      const soft::SoftElim e = soft::soft_elim(D64, L, s.ns, k, q, D[L.lo + c] != -INFINITY, D[L.hi + c] != INFINITY,
                                               B.lam, B.t, nullptr, nullptr, nullptr);
      sw[c] = (Tf)soft::soft_weight(e);
    }
    __syncthreads();
  }
  bool tc_done = false;
#if GQ_IPM_TC
  if constexpr (sizeof(Tf) == 4) {
    // large stages: both products on the Blackwell tensor cores (tcgen05,
    // operands in shared memory, accumulators in TMEM)
    if (C.tc && n < C.N && nv >= 128 && nv <= 256 && nx1 <= 128 && s.ng == 0 && !C.classical && !C.array_qr &&
        NT == 256) {
      __syncthreads();
      tc_products(C, n, D, L, s, reinterpret_cast<float*>(sL), reinterpret_cast<float*>(sPhi),
                  reinterpret_cast<float*>(sMt), ldP, reinterpret_cast<const float*>(sw), bmap, reg);
      tc_done = true;
    }
  }
#endif
  if constexpr (sizeof(Tf) == 4) {
    if (!tc_done) {
    // FP32 factor: both products on the tensor cores (3xTF32 mma.sync), each
    // warp owning 16-row strips of 4 n-tiles (16 x 32 outputs)
    const int lane = tid & 31, w = tid >> 5, NW = NT >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int nMT = (nv + 15) / 16;
    if (n < C.N) {
      // M = [B A]' L_{n+1} (L lower: k-steps left of an n-tile are zero), stored as M'
      const int nNT = (nx1 + 7) / 8, nNG = (nNT + 3) / 4;
      for (int u = w; u < nMT * nNG; u += NW) {
        const int mt = u / nNG, nt0 = (u - mt * nNG) * 4;
        float c[4][4] = {};
        for (int kt = C.classical ? 0 : nt0; kt * 8 < nx1; ++kt) {
          auto fa = [&](int r, int k) {
            const int ii = mt * 16 + r, kk = kt * 8 + k;
            return (ii < nv && kk < nx1) ? (float)D[L.BAt + (int64_t)ii * L.ldb + kk] : 0.f;
          };
          const Tf32Pair a0 = tf32_split(fa(g, q)), a1 = tf32_split(fa(g + 8, q));
          const Tf32Pair a2 = tf32_split(fa(g, q + 4)), a3 = tf32_split(fa(g + 8, q + 4));
          const uint32_t ahi[4] = {a0.hi, a1.hi, a2.hi, a3.hi}, alo[4] = {a0.lo, a1.lo, a2.lo, a3.lo};
#pragma unroll
          for (int jn = 0; jn < 4; ++jn) {
            const int nt = nt0 + jn;
            if (nt >= nNT || (kt < nt && !C.classical)) continue;
            auto fb = [&](int k, int j) {
              const int kk = kt * 8 + k, jj = nt * 8 + j;
              return (kk < nx1 && jj < nx1) ? (float)sL[kk * nx1 + jj] : 0.f;
            };
            const Tf32Pair b0 = tf32_split(fb(q, g)), b1 = tf32_split(fb(q + 4, g));
            const uint32_t bhi[2] = {b0.hi, b1.hi}, blo[2] = {b0.lo, b1.lo};
            mma_tf32(c[jn], alo, bhi);
            mma_tf32(c[jn], ahi, blo);
            mma_tf32(c[jn], ahi, bhi);
          }
        }
#pragma unroll
        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int ii = mt * 16 + g + (e >> 1) * 8, jj = (nt0 + jn) * 8 + 2 * q + (e & 1);
            if (ii < nv && jj < nx1) sMt[jj * ldP + ii] = (Tf)c[jn][e];
          }
      }
    }
    __syncthreads();
    // Phi = RSQ + M M' + [D C]' W [D C] + diagonal terms, lower strips
    {
      const int nNT = (nv + 7) / 8, nNG = (nNT + 3) / 4;
      const int kend = (n < C.N && !C.array_qr) ? nx1 : 0;
      for (int u = w; u < nMT * nNG; u += NW) {
        const int mt = u / nNG, nt0 = (u - mt * nNG) * 4;
        if (nt0 * 8 > mt * 16 + 15) continue;  // strip above the diagonal
        float c[4][4] = {};
        for (int kt = 0; kt * 8 < kend + s.ng; ++kt) {
          // k < kend: columns of M (rows of M'); then the general rows
          auto val = [&](int i, int k) -> float {
            if (i >= nv) return 0.f;
            if (k < kend) return (float)sMt[k * ldP + i];
            const int gg = k - kend;
            return gg < s.ng ? (float)D[L.DC + (int64_t)gg * nv + i] : 0.f;
          };
          auto fa = [&](int r, int k) {
            const int kk = kt * 8 + k, gg = kk - kend;
            const float v = val(mt * 16 + r, kk);
            return (kk >= kend && gg < s.ng) ? v * (float)sw[nb + gg] : v;
          };
          const Tf32Pair a0 = tf32_split(fa(g, q)), a1 = tf32_split(fa(g + 8, q));
          const Tf32Pair a2 = tf32_split(fa(g, q + 4)), a3 = tf32_split(fa(g + 8, q + 4));
          const uint32_t ahi[4] = {a0.hi, a1.hi, a2.hi, a3.hi}, alo[4] = {a0.lo, a1.lo, a2.lo, a3.lo};
#pragma unroll
          for (int jn = 0; jn < 4; ++jn) {
            const int nt = nt0 + jn;
            if (nt >= nNT || nt * 8 > mt * 16 + 15) continue;
            // B = M' (square-root: M M'), or [B A] rows (classical: M [B A]' = [B A]' P [B A])
            auto fbv = [&](int j, int k) -> float {
              if (C.classical && k < kend) return j < nv ? (float)D[L.BAt + (int64_t)j * L.ldb + k] : 0.f;
              return val(j, k);
            };
            const Tf32Pair b0 = tf32_split(fbv(nt * 8 + g, kt * 8 + q)), b1 = tf32_split(fbv(nt * 8 + g, kt * 8 + q + 4));
            const uint32_t bhi[2] = {b0.hi, b1.hi}, blo[2] = {b0.lo, b1.lo};
            mma_tf32(c[jn], alo, bhi);
            mma_tf32(c[jn], ahi, blo);
            mma_tf32(c[jn], ahi, bhi);
          }
        }
#pragma unroll
        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int ii = mt * 16 + g + (e >> 1) * 8, jj = (nt0 + jn) * 8 + 2 * q + (e & 1);
            if (ii < nv && jj <= ii) {
              Tf v = (Tf)D[L.RSQ + (int64_t)ii * L.ldr + jj] + (Tf)c[jn][e];
              if (ii == jj) {
                v += (Tf)reg;
                if (nb > 0 && bmap[ii] >= 0) v += sw[bmap[ii]];
              }
              sPhi[ii * ldP + jj] = v;
            }
          }
      }
    }
    __syncthreads();
    }
  } else {
  const int nI = (nv + kT - 1) / kT;
    // M' = ([B A]' L_{n+1})': Mt[j][i] = sum_{k >= j} BAt[i][k] L[k][j]
    if (n < C.N) {
      const int nJ = (nx1 + kT - 1) / kT;
      for (int t = tid; t < nI * nJ; t += NT) {
        const int I = t / nJ, J = t - I * nJ;
        Tf acc[kT][kT] = {};
        const Tf* ba[kT];
  #pragma unroll
        for (int r = 0; r < kT; ++r) ba[r] = D + L.BAt + (int64_t)min(I * kT + r, nv - 1) * L.ldb;
        for (int k = C.classical ? 0 : J * kT; k < nx1; ++k) {
          Tf a[kT], bb[kT];
  #pragma unroll
          for (int r = 0; r < kT; ++r) a[r] = (Tf)ba[r][k];
  #pragma unroll
          for (int c = 0; c < kT; ++c) bb[c] = J * kT + c < nx1 ? sL[k * nx1 + J * kT + c] : (Tf)0;
  #pragma unroll
          for (int r = 0; r < kT; ++r)
  #pragma unroll
            for (int c = 0; c < kT; ++c) acc[r][c] += a[r] * bb[c];
        }
  #pragma unroll
        for (int c = 0; c < kT; ++c) {
          const int j = J * kT + c;
          if (j < nx1) {
  #pragma unroll
            for (int r = 0; r < kT; ++r)
              if (I * kT + r < nv) sMt[j * ldP + I * kT + r] = acc[r][c];
          }
        }
      }
    }
    __syncthreads();
    // Phi = RSQ + reg I + W_box + [D C]' diag(w_g) [D C] + M M'   (lower tiles)
    for (int t = tid; t < nI * (nI + 1) / 2; t += NT) {
      int I, J;
      tri_tile(t, I, J);
      Tf acc[kT][kT];
  #pragma unroll
      for (int r = 0; r < kT; ++r) {
        const int i = min(I * kT + r, nv - 1);
  #pragma unroll
        for (int c = 0; c < kT; ++c) {
          const int j = min(J * kT + c, nv - 1);
          const int hi = i > j ? i : j, lo = i > j ? j : i;
          acc[r][c] = (Tf)D[L.RSQ + (int64_t)hi * L.ldr + lo];
        }
      }
      for (int g = 0; g < s.ng; ++g) {
        const Tf* row = D + L.DC + (int64_t)g * nv;
        const Tf wg = sw[nb + g];
        Tf a[kT], bb[kT];
  #pragma unroll
        for (int r = 0; r < kT; ++r) a[r] = (Tf)row[min(I * kT + r, nv - 1)] * wg;
  #pragma unroll
        for (int c = 0; c < kT; ++c) bb[c] = (Tf)row[min(J * kT + c, nv - 1)];
  #pragma unroll
        for (int r = 0; r < kT; ++r)
  #pragma unroll
          for (int c = 0; c < kT; ++c) acc[r][c] += a[r] * bb[c];
      }
      if (n < C.N && !C.array_qr) {
        for (int k = 0; k < nx1; ++k) {
          const Tf* mk = sMt + k * ldP;
          Tf a[kT], bb[kT];
  #pragma unroll
          for (int r = 0; r < kT; ++r) a[r] = mk[min(I * kT + r, nv - 1)];
  #pragma unroll
          for (int c = 0; c < kT; ++c)
            bb[c] = C.classical ? (Tf)D[L.BAt + (int64_t)min(J * kT + c, nv - 1) * L.ldb + k] : mk[min(J * kT + c, nv - 1)];
  #pragma unroll
          for (int r = 0; r < kT; ++r)
  #pragma unroll
            for (int c = 0; c < kT; ++c) acc[r][c] += a[r] * bb[c];
        }
      }
  #pragma unroll
      for (int r = 0; r < kT; ++r) {
        const int i = I * kT + r;
  #pragma unroll
        for (int c = 0; c < kT; ++c) {
          const int j = J * kT + c;
          if (i < nv && j <= i) {
            Tf v = acc[r][c];
            if (i == j) {
              v += (Tf)reg;
              if (nb > 0 && bmap[i] >= 0) v += sw[bmap[i]];
            }
            sPhi[i * ldP + j] = v;
          }
        }
      }
    }
    __syncthreads();
  }
  // blocked right-looking Cholesky: each kPanel-wide column panel is copied
  // to shared memory, factored there by one warp, written back, and its
  // rank-kPanel update is applied to the trailing lower triangle by all
  // threads in kT x kT tiles read from the shared copy
  const int lane = tid & 31;
  Tf* sPan = static_cast<Tf*>(C.panel);  // rows p0..nv-1 of the panel, ld kPanel
  // square-root: all nv columns; classical: the leading ne columns only, so
  // the trailing block becomes the Schur complement P_n = Phi_kk - L_ke L_ke'
  const int ncol = C.classical ? ne : nv;
  for (int p0 = 0; p0 < ncol; p0 += kPanel) {
    const int pw = min(kPanel, ncol - p0), pr = nv - p0;
    for (int e = tid; e < pr * kPanel; e += NT) {
      const int r = e / kPanel, c = e - r * kPanel;
      sPan[e] = c < pw ? sPhi[(p0 + r) * ldP + p0 + c] : (Tf)0;
    }
    __syncthreads();
    if (tid < 32) {
      for (int c = 0; c < pw; ++c) {
        Tf d = sPan[c * kPanel + c];
        if (!(d > (Tf)0)) {
          ok = false;
          d = (Tf)1;
        }
        const Tf lcc = sqrt(d);
        const Tf inv = (Tf)1 / lcc;
        for (int r = c + 1 + lane; r < pr; r += 32) sPan[r * kPanel + c] *= inv;
        __syncwarp();
        if (lane == 0) sPan[c * kPanel + c] = lcc;
        for (int r = c + 1 + lane; r < pr; r += 32) {
          const Tf lr = sPan[r * kPanel + c];
          const int cend = min(pw - 1, r);
          for (int c2 = c + 1; c2 <= cend; ++c2) sPan[r * kPanel + c2] -= lr * sPan[c2 * kPanel + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // write the factored panel back (lower part) ...
    for (int e = tid; e < pr * pw; e += NT) {
      const int r = e / pw, c = e - r * pw;
      if (c <= r) sPhi[(p0 + r) * ldP + p0 + c] = sPan[r * kPanel + c];
    }
    // ... and apply its update to the trailing lower triangle
    const int q0 = p0 + pw, m = nv - q0;
    if (m > 0) {
      const int nQ = (m + kT - 1) / kT;
      for (int t = tid; t < nQ * (nQ + 1) / 2; t += NT) {
        int I, J;
        tri_tile(t, I, J);
        Tf acc[kT][kT] = {};
        const Tf* ri[kT];
        const Tf* rj[kT];
#pragma unroll
        for (int r = 0; r < kT; ++r) {
          ri[r] = sPan + (min(q0 + I * kT + r, nv - 1) - p0) * kPanel;
          rj[r] = sPan + (min(q0 + J * kT + r, nv - 1) - p0) * kPanel;
        }
#pragma unroll
        for (int c = 0; c < kPanel; ++c) {
          Tf a[kT], bb[kT];
#pragma unroll
          for (int r = 0; r < kT; ++r) {
            a[r] = ri[r][c];
            bb[r] = rj[r][c];
          }
#pragma unroll
          for (int r = 0; r < kT; ++r)
#pragma unroll
            for (int c2 = 0; c2 < kT; ++c2) acc[r][c2] += a[r] * bb[c2];
        }
#pragma unroll
        for (int r = 0; r < kT; ++r) {
          const int i = q0 + I * kT + r;
#pragma unroll
          for (int c2 = 0; c2 < kT; ++c2) {
            const int j = q0 + J * kT + c2;
            if (i < nv && j <= i) sPhi[i * ldP + j] -= acc[r][c2];
          }
        }
      }
    }
    __syncthreads();
  }
  ok = __syncthreads_and(ok) != 0;
  if (C.array_qr && n < C.N && nx1 > 0) {
    // robust mode: Phi = Lh Lh' + M M' without forming M M'.  The factor of
    // Phi is the transposed triangle of the QR factorisation of the array
    // [Lh'; M']; column j's Householder reflector acts on row j of Lh' (the
    // stored column j of Lh) and on column j of M' (nx1 entries), and is
    // applied to the columns c > j of both.
    for (int j = 0; j < nv; ++j) {
      Tf* mj = sMt;  // M'[k][j] = sMt[k * ldP + j]
      const Tf alpha = sPhi[j * ldP + j];
      double ss = 0.0;
      for (int k = 0; k < nx1; ++k) ss += (double)mj[k * ldP + j] * (double)mj[k * ldP + j];
      const Tf sigma = (Tf)sqrt((double)alpha * (double)alpha + ss);
      // reflector u = [alpha - sigma; M'[:, j]] (alpha > 0, sigma >= alpha:
      // u0 <= 0 with no cancellation when ss is small relative to alpha^2
      // handled by the equivalent form u0 = -ss / (alpha + sigma))
      const Tf u0 = (Tf)(-ss / ((double)alpha + (double)sigma));
      const double utu = (double)u0 * (double)u0 + ss;
      const Tf beta = utu > 0.0 ? (Tf)(2.0 / utu) : (Tf)0;
      for (int c = j + 1 + tid; c < nv; c += NT) {
        // column c: top entry R[j][c] = Lh-stored (c, j); then M'[:, c]
        Tf wv = u0 * sPhi[c * ldP + j];
        for (int k = 0; k < nx1; ++k) wv += mj[k * ldP + j] * sMt[k * ldP + c];
        const Tf bw = beta * wv;
        sPhi[c * ldP + j] -= bw * u0;
        for (int k = 0; k < nx1; ++k) sMt[k * ldP + c] -= bw * mj[k * ldP + j];
      }
      __syncthreads();
      if (tid == 0) sPhi[j * ldP + j] = sigma;
      __syncthreads();
    }
  }
  // X = L_ee^{-1} (lower), column j by thread j, into the M' buffer (ld ne)
  for (int j = tid; j < ne; j += NT) {
    sMt[j * ne + j] = (Tf)1 / sPhi[j * ldP + j];
    for (int i = j + 1; i < ne; ++i) {
      Tf acc = 0;
      for (int k = j; k < i; ++k) acc += sPhi[i * ldP + k] * sMt[k * ne + j];
      sMt[i * ne + j] = -acc / sPhi[i * ldP + i];
    }
  }
  __syncthreads();
  // store the factor (ld nv), X in place of L_ee; keep L_n = L_kk for stage n-1
  Tf* F = fac_global<Tf>(B, s);
  for (int e = tid; e < nv * nv; e += NT) {
    const int i = e / nv, j = e - i * nv;
    F[e] = j > i ? (Tf)0 : (i < ne ? sMt[i * ne + j] : sPhi[i * ldP + j]);
  }
  // next stage: L_n = L_kk (lower, zeros above), or P_n (full symmetric)
  for (int e = tid; e < nk * nk; e += NT) {
    const int i = e / nk, j = e - i * nk;
    if (C.classical)
      sL[i * nk + j] = sPhi[(ne + max(i, j)) * ldP + ne + min(i, j)];
    else
      sL[i * nk + j] = (j <= i) ? sPhi[(ne + i) * ldP + ne + j] : (Tf)0;
  }
  return ok;
}

template <typename Tf>
__device__ bool factor(Ctx& C, double reg) {
  bool ok = true;
  sweep(
      C, true, 0,
      [&](int n, const double* D, const void*) { ok = factor_stage<Tf>(C, n, reinterpret_cast<const Tf*>(D), reg) && ok; },
      (int)sizeof(Tf));
  // factor blocks were written through the generic proxy; the solves read them
  // with bulk copies (async proxy)
  fence_async_global();
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------------------
// a2 + a4: Riccati solve of eq. (delta) for right-hand side (g, b) with the
// reduced gradient gt = g - C'(W r_d - T^{-1} r_m) formed per stage
// (rd = rm = nullptr: gt = g), -> (dy, dpi); then dt, dlam recovered in FP64.
// ---------------------------------------------------------------------------
template <typename Tf>
__device__ double riccati_solve(Ctx& C, const double* g, const double* rd, const double* rm, const double* rb,
                                double* dy, double* dpi, double* dlam, double* dt) {
  const Batch& B = *C.B;
  const int tid = threadIdx.x, NT = blockDim.x;
  Tf* va = reinterpret_cast<Tf*>(C.vbuf);
  Tf* vb = va + C.vmax;
  Tf* phi = vb + C.vmax;
  Tf* pn1 = phi + C.vmax;  // p_{n+1}
  Tf* ln = pn1 + C.vmax;
  Tf* sL = static_cast<Tf*>(C.mat);  // L_{n+1}
  double* vs = C.vbuf + 5 * C.vmax;  // per-constraint v_lo - v_hi, v = (lambda r_d - r_m) / t
  double* lp = B.lp;                 // per stage: l (ne entries) then p_n (nk entries)
  const int fe = (int)sizeof(Tf);
  double scale = 0.0;                // ||(gt, r_b)||inf of the reduced system
  // backward sweep; D is the stage data in the factor's precision (the FP32
  // mirror for Tf = float), D64 the FP64 data (global) where exact values
  // are needed
  sweep(C, true, fe, [&](int n, const double* Dv, const void* Fv) {
    const Tf* D = reinterpret_cast<const Tf*>(Dv);
    const Tf* F = static_cast<const Tf*>(Fv);
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D64 = B.data + s.data;
    const int nv = s.nx + s.nu, nx1 = s.nx1, nb = s.nbu + s.nbx, nc = nb + s.ng;
    const int ne = elim_size(s, n), nk = nv - ne;
    const int32_t* bmap = reinterpret_cast<const int32_t*>(D + L.box) + nb;
    if (rd != nullptr) {
      const double* lm = B.lam + s.side;
      const double* tt = B.t + s.side;
      for (int c = tid; c < nc; c += NT) {
        const int il = s.side + c, iu = s.side + nc + c;
        double v = 0.0;
        if (D[L.lo + c] != -INFINITY) v += (lm[c] * rd[il] - rm[il]) / tt[c];
        if (D[L.hi + c] != INFINITY) v -= (lm[nc + c] * rd[iu] - rm[iu]) / tt[nc + c];
        vs[c] = v;
      }
      if (GQ_IPM_SOFT && s.ns > 0) {
        // relaxed constraints: the eliminated slacks' gradient terms
        __syncthreads();
        const int32_t* sidx = soft::soft_sidx(box_idx(D64, L), nb, nv);
        for (int k = tid; k < s.ns; k += NT) {
          const int c = sidx[k];
          const soft::SoftSlot q = soft::soft_slot(s, nv, nc, k, c);
          const soft::SoftElim e = soft::soft_elim(D64, L, s.ns, k, q, D[L.lo + c] != -INFINITY,
                                                   D[L.hi + c] != INFINITY, B.lam, B.t, g, rd, rm);
          vs[c] += soft::soft_grad(e);
        }
      }
    }
    // rb_n in the factor's precision, converted once (a conversion from FP64
    // costs as much as an FP64 FMA on this GPU); phi is free until formed below
    Tf* rbf = phi;
    if (n < C.N)
      for (int j = tid; j < nx1; j += NT) rbf[j] = (Tf)rb[s.eq + j];
    __syncthreads();
    if (n < C.N && !C.classical) {
      // va = L_{n+1}' rb_n
      rows_dot<Tf>(
          nx1, [&](int k) { return k; }, [&](int) { return nx1; },
          [&](int k, int j) { return sL[j * nx1 + k] * rbf[j]; }, [&](int k, Tf v) { va[k] = v; });
    }
    __syncthreads();
    if (n < C.N) {
      if (C.classical) {
        // vb = P_{n+1} rb_n + p_{n+1}
        rows_dot<Tf>(
            nx1, [&](int) { return 0; }, [&](int) { return nx1; },
            [&](int k, int j) { return sL[k * nx1 + j] * rbf[j]; }, [&](int k, Tf v) { vb[k] = pn1[k] + v; });
      } else {
        // vb = L_{n+1} va + p_{n+1}
        rows_dot<Tf>(
            nx1, [&](int) { return 0; }, [&](int k) { return k + 1; },
            [&](int k, int j) { return sL[k * nx1 + j] * va[j]; }, [&](int k, Tf v) { vb[k] = pn1[k] + v; });
      }
    }
    __syncthreads();
    // phi = gt_n + [B A]' vb
    {
      const int kend = n < C.N ? nx1 : 0;
      rows_dot<Tf>(
          nv, [&](int) { return 0; }, [&](int) { return kend; },
          [&](int i, int k) { return (Tf)D[L.BAt + (int64_t)i * L.ldb + k] * vb[k]; },
          [&](int i, Tf v) {
            double gi = g[s.var + i];
            if (rd != nullptr) {
              for (int gg = 0; gg < s.ng; ++gg) gi = fma(-D64[L.DC + (int64_t)gg * nv + i], vs[nb + gg], gi);
              if (nb > 0 && bmap[i] >= 0) gi -= vs[bmap[i]];
            }
            scale = max_nan(scale, fabs(gi));
            phi[i] = (Tf)gi + v;
          });
    }
    if (n < C.N)
      for (int k = tid; k < nx1; k += NT) scale = max_nan(scale, fabs(rb[s.eq + k]));
    __syncthreads();
    // l = X phi_e
    rows_dot<Tf>(
        ne, [&](int) { return 0; }, [&](int i) { return i + 1; }, [&](int i, int j) { return F[i * nv + j] * phi[j]; },
        [&](int i, Tf v) {
          ln[i] = v;
          lp[s.var + i] = (double)v;
        });
    __syncthreads();
    // p_n = phi_k - L_ke l  -> p_{n+1} of stage n-1; L_n = L_kk -> L_{n+1} of stage n-1
    rows_dot<Tf>(
        nk, [&](int) { return 0; }, [&](int) { return ne; },
        [&](int i, int j) { return F[(ne + i) * nv + j] * ln[j]; },
        [&](int i, Tf v) {
          const Tf acc = phi[ne + i] - v;
          pn1[i] = acc;
          lp[s.var + ne + i] = (double)acc;
        });
    for (int e = tid; e < nk * nk; e += NT) {
      const int i = e / nk, j = e - i * nk;
      // L_n (lower, zeros above) or P_n (stored lower, used full)
      sL[i * nk + j] = C.classical ? F[(ne + max(i, j)) * nv + ne + min(i, j)] : F[(ne + i) * nv + ne + j];
    }
  }, fe);
  // forward sweep: pi_n at the start of stage n (needs L_n), then y_n and
  // x_{n+1}, then dt, dlam of stage n
  sweep(C, false, fe, [&](int n, const double* Dv, const void* Fv) {
    const Tf* D = reinterpret_cast<const Tf*>(Dv);
    const Tf* F = static_cast<const Tf*>(Fv);
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D64 = B.data + s.data;
    const int nv = s.nx + s.nu, nx1 = s.nx1, nb = s.nbu + s.nbx, nc = nb + s.ng;
    const int ne = elim_size(s, n), nk = nv - ne;
    double* yn = dy + s.var;
    // x_n (and below y_n) in the factor's precision, converted once into the
    // backward sweep's scratch (vb, phi are free here)
    Tf* xf = vb;
    Tf* yf = phi;
    for (int j = tid; j < nk; j += NT) xf[j] = (Tf)yn[ne + j];
    __syncthreads();
    if (n > 0) {
      const int eqp = C.st[n - 1].eq;
      if (C.classical) {
        // pi_n = P_n x_n + p_n, P_n stored in the lower kk block
        rows_dot<Tf>(
            nk, [&](int) { return 0; }, [&](int) { return nk; },
            [&](int k, int j) { return F[(ne + max(k, j)) * nv + ne + min(k, j)] * xf[j]; },
            [&](int k, Tf v) { dpi[eqp + k] = (double)((Tf)lp[s.var + ne + k] + v); });
      } else {
        // pi_n = L_n (L_n' x_n) + p_n,  L_n = L_kk of this stage
        rows_dot<Tf>(
            nk, [&](int k) { return k; }, [&](int) { return nk; },
            [&](int k, int j) { return F[(ne + j) * nv + ne + k] * xf[j]; }, [&](int k, Tf v) { va[k] = v; });
        __syncthreads();
        rows_dot<Tf>(
            nk, [&](int) { return 0; }, [&](int k) { return k + 1; },
            [&](int k, int j) { return F[(ne + k) * nv + ne + j] * va[j]; },
            [&](int k, Tf v) { dpi[eqp + k] = (double)((Tf)lp[s.var + ne + k] + v); });
      }
      __syncthreads();
    }
    // va = l + L_ke' x_n
    rows_dot<Tf>(
        ne, [&](int) { return 0; }, [&](int) { return nk; },
        [&](int j, int i) { return F[(ne + i) * nv + j] * xf[i]; },
        [&](int j, Tf v) { va[j] = (Tf)lp[s.var + j] + v; });
    __syncthreads();
    // y_e = -X' va
    rows_dot<Tf>(
        ne, [&](int i) { return i; }, [&](int) { return ne; }, [&](int i, int j) { return F[j * nv + i] * va[j]; },
        [&](int i, Tf v) { yn[i] = -(double)v; });
    __syncthreads();
    if (n < C.N) {
      // x_{n+1} = [B A] y_n + rb_n
      for (int i = tid; i < nv; i += NT) yf[i] = (Tf)yn[i];
      __syncthreads();
      double* x1 = dy + C.st[n + 1].var + C.st[n + 1].nu;
      rows_dot<Tf>(
          nx1, [&](int) { return 0; }, [&](int) { return nv; },
          [&](int k, int i) { return (Tf)D[L.BAt + (int64_t)i * L.ldb + k] * yf[i]; },
          [&](int k, Tf v) { x1[k] = (double)((Tf)rb[s.eq + k] + v); });
    }
    // dt = C dy - r_d, dlam = -T^{-1}(r_m + Lambda dt) on active sides
    for (int c = tid; c < nc; c += NT) {
      const double v = cons_value(s, L, D64, c, yn);
      const int il = s.side + c, iu = s.side + nc + c;
      const double dl = rd ? rd[il] : 0.0, du = rd ? rd[iu] : 0.0;
      const double ml = rm ? rm[il] : 0.0, mu = rm ? rm[iu] : 0.0;
      if (D[L.lo + c] != -INFINITY) {
        const double a = v - dl;
        dt[il] = a;
        dlam[il] = -(ml + B.lam[il] * a) / B.t[il];
      } else {
        dt[il] = 0.0;
        dlam[il] = 0.0;
      }
      if (D[L.hi + c] != INFINITY) {
        const double a = -v - du;
        dt[iu] = a;
        dlam[iu] = -(mu + B.lam[iu] * a) / B.t[iu];
      } else {
        dt[iu] = 0.0;
        dlam[iu] = 0.0;
      }
      if (GQ_IPM_SOFT && s.ns > 0) {
        // relaxed constraint: slack steps, then its sides' steps with them
        const int k = soft::soft_smap(box_idx(D64, L), nb, nv, s.ns)[c];
        if (k >= 0) {
          const soft::SoftSlot q = soft::soft_slot(s, nv, nc, k, c);
          const bool lo_on = D[L.lo + c] != -INFINITY, hi_on = D[L.hi + c] != INFINITY;
          const soft::SoftElim e = soft::soft_elim(D64, L, s.ns, k, q, lo_on, hi_on, B.lam, B.t, g, rd, rm);
          soft::soft_recover(e, q, lo_on, hi_on, v, B.lam, B.t, rd, rm, dy, dt, dlam);
        }
      }
    }
  }, fe);
  return block_reduce(scale, C.red, OpMax());
}

// elementwise pass over this QP's sides
template <class F>
__device__ void for_sides(const Ctx& C, F f) {
  const int s0 = C.st[0].side;
  for (int i = s0 + threadIdx.x; i < s0 + C.nside; i += blockDim.x) f(i);
}

// a5: largest alpha with lambda + alpha dlam >= 0 and t + alpha dt >= 0
__device__ double max_step(const Ctx& C, const double* dlam, const double* dt) {
  const Batch& B = *C.B;
  double a = INFINITY;
  for_sides(C, [&](int i) {
    if (dlam[i] < 0.0) a = fmin(a, -B.lam[i] / dlam[i]);
    if (dt[i] < 0.0) a = fmin(a, -B.t[i] / dt[i]);
  });
  return block_reduce(a, C.red, OpMin());
}

// (lambda + alpha dlam)'(t + alpha dt) / n_c over active sides
__device__ double mu_after(const Ctx& C, double alpha, const double* dlam, const double* dt) {
  const Batch& B = *C.B;
  const int s0 = C.st[0].side;
  // masked sides have lambda = 0 and dlam = 0: they add nothing
  const double s = fixed_sum(C, C.nside, [&](int k) {
    const int i = s0 + k;
    return (B.lam[i] + alpha * dlam[i]) * (B.t[i] + alpha * dt[i]);
  });
  return C.nact ? s / C.nact : 0.0;
}

struct Dir {
  double *dy, *dpi, *dlam, *dt;
};

// work counters reported in gq_stats (thread-uniform values)
struct Count {
  int ir = 0, fact = 0, fact64 = 0, solve = 0, res = 0;
  double m = 0.0;  // residual of the last refined direction (r_g, r_b rows)
};

// Newton direction of eq. (delta) for the current r_m with the factors in
// place; with ir > 0, iterative refinement on eq. (itref) (Sec. 3.4).
// Returns the final refinement residual ratio (0 without refinement).
template <typename Tf>
__device__ double newton_dir(Ctx& C, const Dir& d, int ir, double ir_tol, Count* cnt) {
  const Batch& B = *C.B;
  // mr: scale of the reduced right-hand side ||(gt, r_b)||inf
  const double mr = riccati_solve<Tf>(C, B.rg, B.rd, B.rm, B.rb, d.dy, d.dpi, d.dlam, d.dt);
  ++cnt->solve;
  if (ir <= 0) return 0.0;
  double ratio = 0.0;
  for (int k = 0; k <= ir; ++k) {
    // residual of eq. (delta) for the direction (the r_d and r_m rows vanish
    // because dt and dlam are recovered from dy in FP64)
    Max3 mx{0.0, 0.0, 0.0};
    sweep(C, false, 0, [&](int n, const double* D, const void*) {
      stage_residual(C, n, D, d.dy, d.dpi, d.dlam, nullptr, B.rg2, B.rb2, nullptr, true, B.rg, B.rb, mx);
    });
    ++cnt->res;
    const double m = block_reduce(max_nan(mx.g, mx.b), C.red, OpMax());
    ratio = mr > 0.0 ? m / mr : 0.0;
    cnt->m = m;
    if (k == ir || m <= ir_tol * mr) break;
    // correction: same factors, the refinement residual as right-hand side
    riccati_solve<Tf>(C, B.rg2, nullptr, nullptr, B.rb2, B.dy2, B.dpi2, B.dlam2, B.dt2);
    for (int i = C.v0 + threadIdx.x; i < C.v1; i += blockDim.x) d.dy[i] += B.dy2[i];
    for (int i = C.e0 + threadIdx.x; i < C.e1; i += blockDim.x) d.dpi[i] += B.dpi2[i];
    for_sides(C, [&](int i) {
      d.dlam[i] += B.dlam2[i];
      d.dt[i] += B.dt2[i];
    });
    __syncthreads();
    ++cnt->ir;
    ++cnt->solve;
  }
  return ratio;
}

// ---------------------------------------------------------------------------
// the kernel: one block per QP
// ---------------------------------------------------------------------------
// The slack build is held to 128 registers (two 256-thread or four
// 128-thread blocks per SM, as the other builds get from ptxas on their
// own): left free, ptxas gave it 230 registers and it ran 1.4x slower.
#if GQ_IPM_SOFT
#define GQ_IPM_BOUNDS __launch_bounds__(256, 2)
#else
#define GQ_IPM_BOUNDS __launch_bounds__(256)
#endif
__global__ void GQ_IPM_BOUNDS ipm_kernel(const __grid_constant__ Batch B, const Shape sh,
                                                  const __grid_constant__ gq_ipm_arg arg, int kind,
                                                  double sigma_mu, const DirOut out, const int32_t* order) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int q = order[blockIdx.x];
  const QpDesc qd = B.qp[q];
  const int tid = threadIdx.x;
  const SmemPlan P = smem_plan(B, sh);
  StageDesc* sst = reinterpret_cast<StageDesc*>(smem + P.stages);
  double* red = reinterpret_cast<double*>(smem + P.red);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P.bars);
  int& s_count = *reinterpret_cast<int*>(smem + P.bars + 2 * sizeof(uint64_t));

  for (int n = tid; n <= qd.N; n += blockDim.x) sst[n] = B.st[qd.stage0 + n];
  if (tid == 0) {
    s_count = 0;
    if (P.staged) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      fence_async_shared();
    }
  }
  __syncthreads();

  Ctx C;
  C.B = &B;
  C.st = sst;
  C.N = qd.N;
  C.red = red;
  C.chunk = reinterpret_cast<double*>(smem + P.chunk);
  C.nside = qd.nsidet;
  C.v0 = qd.var0;
  C.v1 = qd.var0 + qd.nvt;
  C.e0 = qd.eq0;
  C.e1 = qd.eq0 + qd.neqt;
  C.vbuf = reinterpret_cast<double*>(smem + P.vec);
  C.vmax = P.vmax;
  // stage matrices: shared memory, or this QP's slice of the global scratch
  // when the largest stage does not fit (one slice per block of the launch)
  C.mat = sh.mat_global ? static_cast<void*>(B.matg + (int64_t)blockIdx.x * block_mat_elems(sh))
                        : static_cast<void*>(smem + P.mat);
  C.nvmax = sh.nvmax;
  C.nxmax = sh.nxmax;
  C.panel = smem + P.panel;
  C.ring.buf[0] = smem + P.ring0;
  C.ring.buf[1] = smem + P.ring1;
  C.ring.bar = bars;
  C.ring.parity = 0;
  C.ring.fac_off = (uint32_t)P.ring_fac;
  C.ring.staged = P.staged;
  C.classical = arg.riccati == 1;
  C.array_qr = arg.mode == GQ_MODE_ROBUST;
  C.ring.ok = true;
  // tensor-core products for large stages in the FP32 factor: one TMEM
  // allocation per block
#if GQ_IPM_TC
  C.tc = tc_shape(sh) && arg.precision == GQ_PREC_MIXED && blockDim.x == 256 &&
         kind != (int)LaunchKind::Residuals;
  C.tcpar = 0;
  C.taddr = 0;
  if (C.tc) {
    C.tcbar = reinterpret_cast<uint64_t*>(smem + P.tcbar);
    C.tcA = reinterpret_cast<float*>(smem + P.tc);
    C.tcB = C.tcA + 2 * (tc_tile_bytes() >> 2);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + P.tcbar + 8);
    if (tid == 0) {
      mbar_init(C.tcbar, 1);
      fence_async_shared();
    }
    if (tid < 32) tc::alloc(tslot, kTcCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    C.taddr = *tslot;
  }
#endif

  // count active sides (integer count: exact in any order)
  {
    int cnt = 0;
    sweep(C, false, 0, [&](int n, const double* D, const void*) {
      const StageDesc s = sst[n];
      const StageData L = lay(s);
      const int nc = s.nbu + s.nbx + s.ng;
      for (int c = tid; c < nc; c += blockDim.x) cnt += (D[L.lo + c] != -INFINITY) + (D[L.hi + c] != INFINITY);
      if (tid == 0) cnt += 2 * s.ns;  // slack bound sides are always active
    });
    atomicAdd(&s_count, cnt);
    __syncthreads();
    C.nact = s_count;
    __syncthreads();
  }

  const bool mixed = arg.precision == GQ_PREC_MIXED;
  gq_stats* stats = B.stats + q;

  if (kind == (int)LaunchKind::Residuals) {
    Norms r = residuals(C);
    if (tid == 0) {
      stats->res[0] = r.g;
      stats->res[1] = r.b;
      stats->res[2] = r.d;
      stats->res[3] = r.mu;
      if (!C.ring.ok) stats->status = GQ_STATUS_TIMEOUT;
    }
    return;
  }

  if (kind == (int)LaunchKind::NewtonStep) {
    residuals(C);
    for_sides(C, [&](int i) { B.rm[i] = B.lam[i] * B.t[i] - (B.lam[i] != 0.0 ? sigma_mu : 0.0); });
    __syncthreads();
    Dir d{out.dy, out.dpi, out.dlam, out.dt};
    Count cnt;
    bool ok = mixed ? factor<float>(C, arg.reg_prim) : factor<double>(C, arg.reg_prim);
    if (mixed)
      newton_dir<float>(C, d, arg.ir_steps, arg.ir_tol, &cnt);
    else
      newton_dir<double>(C, d, arg.ir_steps, arg.ir_tol, &cnt);
    if (tid == 0) {
      stats->status = !C.ring.ok ? GQ_STATUS_TIMEOUT : (ok ? GQ_STATUS_CONVERGED : GQ_STATUS_NAN);
      stats->ir_total = cnt.ir;
    }
#if GQ_IPM_TC
    if (C.tc) {
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid < 32) tc::dealloc(C.taddr, kTcCols);
    }
#endif
    return;
  }

  // ---------------- full IPM (Sec. 4.2) ----------------
  const int64_t t_start = arg.timeout_ns > 0 ? globaltimer() : 0;
  // a0: start point
  {
    const int wlev = qd.warm > 0 ? qd.warm - 1 : arg.warm_start;
    const bool warm1 = wlev >= 1, warm2 = wlev >= 2;
    if (!warm1) {
      for (int i = C.v0 + tid; i < C.v1; i += blockDim.x) B.y[i] = 0.0;
      for (int i = C.e0 + tid; i < C.e1; i += blockDim.x) B.pi[i] = 0.0;
    }
    __syncthreads();
    sweep(C, false, 0, [&](int n, const double* D, const void*) {
      const StageDesc s = sst[n];
      const StageData L = lay(s);
      const int nb = s.nbu + s.nbx, nc = nb + s.ng, nv = s.nx + s.nu;
      for (int c = tid; c < nc; c += blockDim.x) {
        const double v = cons_value(s, L, D, c, B.y + s.var);
        const double lo = D[L.lo + c], hi = D[L.hi + c];
        const int il = s.side + c, iu = s.side + nc + c;
        double sl = 0.0, su = 0.0;  // slacks of a relaxed constraint (Sec. 2.2)
        if (GQ_IPM_SOFT && s.ns > 0) {
          const int k = soft::soft_smap(box_idx(D, L), nb, nv, s.ns)[c];
          if (k >= 0) {
            sl = B.y[s.var + nv + k];
            su = B.y[s.var + nv + s.ns + k];
          }
        }
        if (lo != -INFINITY) {
          if (warm2) {
            B.lam[il] = fmax(B.lam[il], arg.warm_min);
            B.t[il] = fmax(B.t[il], arg.warm_min);
          } else {
            B.lam[il] = 1.0;
            B.t[il] = fmax(1.0, v + sl - lo);
          }
        } else {
          B.lam[il] = 0.0;
          B.t[il] = 1.0;
        }
        if (hi != INFINITY) {
          if (warm2) {
            B.lam[iu] = fmax(B.lam[iu], arg.warm_min);
            B.t[iu] = fmax(B.t[iu], arg.warm_min);
          } else {
            B.lam[iu] = 1.0;
            B.t[iu] = fmax(1.0, hi - v + su);
          }
        } else {
          B.lam[iu] = 0.0;
          B.t[iu] = 1.0;
        }
      }
      // slack bound sides s - ls >= 0
      for (int k = tid; GQ_IPM_SOFT && k < s.ns; k += blockDim.x) {
        const int jl = s.side + 2 * nc + k, ju = jl + s.ns;
        if (warm2) {
          B.lam[jl] = fmax(B.lam[jl], arg.warm_min);
          B.t[jl] = fmax(B.t[jl], arg.warm_min);
          B.lam[ju] = fmax(B.lam[ju], arg.warm_min);
          B.t[ju] = fmax(B.t[ju], arg.warm_min);
        } else {
          B.lam[jl] = 1.0;
          B.t[jl] = fmax(1.0, B.y[s.var + nv + k] - D[L.ls + k]);
          B.lam[ju] = 1.0;
          B.t[ju] = fmax(1.0, B.y[s.var + nv + s.ns + k] - D[L.ls + s.ns + k]);
        }
      }
    });
  }

  int status = GQ_STATUS_MAX_ITER, it = 0, flags = 0;
  Count cnt;
  bool fp64 = !mixed;
  int lifted_at = -1;  // iteration whose lambda, t were lifted after a lost FP64 pivot
  double alpha = 1.0;
  Norms r{0, 0, 0, 0};
  const Dir d{B.dy, B.dpi, B.dlam, B.dt};
  while (true) {
    r = residuals(C);
    ++cnt.res;
    if (!C.ring.ok) {
      status = GQ_STATUS_TIMEOUT;
      break;
    }
    if (!(isfinite(r.g) && isfinite(r.b) && isfinite(r.d) && isfinite(r.mu))) {
      status = GQ_STATUS_NAN;
      break;
    }
    if (r.g <= arg.tol_stat && r.b <= arg.tol_eq && r.d <= arg.tol_ineq && r.mu <= arg.tol_comp) {
      status = GQ_STATUS_CONVERGED;
      break;
    }
    if (it >= arg.iter_max) {
      status = GQ_STATUS_MAX_ITER;
      break;
    }
    if (it > 0 && alpha < arg.alpha_min) {
      status = GQ_STATUS_MIN_STEP;
      break;
    }
    if (arg.timeout_ns > 0) {
      int64_t el = globaltimer() - t_start;
      // one clock for the block
      el = (int64_t)block_reduce((double)el, red, OpMax());
      if (el > arg.timeout_ns) {
        status = GQ_STATUS_TIMEOUT;
        break;
      }
    }
    // a2 + a3: predictor right-hand side and factorisation
    for_sides(C, [&](int i) { B.rm[i] = B.lam[i] * B.t[i]; });
    __syncthreads();
    const double reg = fp64 ? (mixed ? 0.0 : arg.reg_prim) : arg.reg_prim;
    bool ok = fp64 ? factor<double>(C, reg) : factor<float>(C, reg);
    ++cnt.fact;
    cnt.fact64 += fp64;
    int okall = (int)block_reduce(ok ? 1.0 : 0.0, red, OpMin());
    if (!okall && fp64 && reg < kRegRetry) {
      // an FP64 pivot lost positivity in the end game: regularise the primal
      // block (Sec. 4.2, regularisation) and factor once more
      ok = factor<double>(C, kRegRetry);
      ++cnt.fact;
      ++cnt.fact64;
      flags |= GQ_FLAG_REGULARIZED;
      okall = (int)block_reduce(ok ? 1.0 : 0.0, red, OpMin());
    }
    if (!okall && fp64 && lifted_at != it) {
      // still indefinite: complementarity ran far ahead of stationarity and
      // barrier weights lambda/t near 1/t_min swamp Phi.  Lift lambda and t
      // of active sides to a floor tied to the stationarity residual (moving
      // r_d by no more than that floor) and redo this iteration
      lifted_at = it;
      const double floor_lt = fmax(kLift, kLiftRel * fmax(r.g, r.b));
      flags |= GQ_FLAG_REGULARIZED;
      for_sides(C, [&](int i) {
        if (B.lam[i] != 0.0) {
          B.lam[i] = fmax(B.lam[i], floor_lt);
          B.t[i] = fmax(B.t[i], floor_lt);
        }
      });
      __syncthreads();
      continue;
    }
    if (!okall) {
      if (!fp64 && arg.fp64_fallback) {
        fp64 = true;
        flags |= GQ_FLAG_FP64_FALLBACK;
        continue;
      }
      status = GQ_STATUS_NAN;
      break;
    }
    // a4 + a5: affine predictor
    if (fp64)
      newton_dir<double>(C, d, 0, 0.0, &cnt);
    else
      newton_dir<float>(C, d, 0, 0.0, &cnt);
    const int ir = (mixed && !fp64) || arg.mode != GQ_MODE_SPEED ? arg.ir_steps : 0;
    // a refined FP32 direction must also be an inexact-Newton step for the
    // unscaled exit rule: its own residual well below the iterate's
    const double inexact = kInexact * fmax(fmax(r.g, r.b), arg.tol_stat);
    if (C.nact > 0) {
      const double a_aff = fmin(1.0, max_step(C, d.dlam, d.dt));
      const double mu_aff = mu_after(C, a_aff, d.dlam, d.dt);
      const double sigma = r.mu > 0.0 ? (mu_aff / r.mu) * (mu_aff / r.mu) * (mu_aff / r.mu) : 0.0;
      const double smu = sigma * r.mu;
      // a6: corrector r_m = lambda t + dlam_aff dt_aff - sigma mu
      for_sides(C, [&](int i) {
        B.rm[i] = B.lam[i] != 0.0 ? B.lam[i] * B.t[i] + d.dlam[i] * d.dt[i] - smu : 0.0;
      });
      __syncthreads();
      double ratio = fp64 ? newton_dir<double>(C, d, ir, arg.ir_tol, &cnt)
                          : newton_dir<float>(C, d, ir, arg.ir_tol, &cnt);
      if (arg.cond_corr) {
        const double a_c = fmin(1.0, max_step(C, d.dlam, d.dt));
        const double mu_c = mu_after(C, a_c, d.dlam, d.dt);
        if (mu_c > arg.corr_k * mu_aff) {
          for_sides(C, [&](int i) { B.rm[i] = B.lam[i] != 0.0 ? B.lam[i] * B.t[i] - smu : 0.0; });
          __syncthreads();
          ratio = fp64 ? newton_dir<double>(C, d, ir, arg.ir_tol, &cnt)
                       : newton_dir<float>(C, d, ir, arg.ir_tol, &cnt);
        }
      }
      if (ir > 0 && !(ratio <= arg.ir_fail_ratio && cnt.m <= inexact)) {
        // a7 failed to make the direction accurate: refactor in FP64 (mixed
        // path), else, in mode balance, with the array algorithm (Sec. 4.2),
        // and redo this iteration
        if (!fp64 && arg.fp64_fallback) {
          fp64 = true;
          flags |= GQ_FLAG_FP64_FALLBACK;
          continue;
        }
        if (arg.mode == GQ_MODE_BALANCE && !C.array_qr && !C.classical) {
          C.array_qr = true;
          flags |= GQ_FLAG_ARRAY_QR;
          continue;
        }
      }
      alpha = fmin(1.0, arg.tau_b * max_step(C, d.dlam, d.dt));
    } else {
      if (ir > 0) {
        // no inequalities: refine the single Newton step
        const double ratio = fp64 ? newton_dir<double>(C, d, ir, arg.ir_tol, &cnt)
                                  : newton_dir<float>(C, d, ir, arg.ir_tol, &cnt);
        if (!(ratio <= arg.ir_fail_ratio && cnt.m <= inexact)) {
          if (!fp64 && arg.fp64_fallback) {
            fp64 = true;
            flags |= GQ_FLAG_FP64_FALLBACK;
            continue;
          }
          if (arg.mode == GQ_MODE_BALANCE && !C.array_qr && !C.classical) {
            C.array_qr = true;
            flags |= GQ_FLAG_ARRAY_QR;
            continue;
          }
        }
      }
      alpha = 1.0;
    }
    // a8: step and clamp
    for (int i = C.v0 + tid; i < C.v1; i += blockDim.x) B.y[i] += alpha * d.dy[i];
    for (int i = C.e0 + tid; i < C.e1; i += blockDim.x) B.pi[i] += alpha * d.dpi[i];
    for_sides(C, [&](int i) {
      if (B.lam[i] != 0.0 || d.dlam[i] != 0.0) {
        B.lam[i] = fmax(B.lam[i] + alpha * d.dlam[i], arg.lam_min);
        B.t[i] = fmax(B.t[i] + alpha * d.dt[i], arg.t_min);
      }
    });
    __syncthreads();
    ++it;
  }
  if (tid == 0) {
    stats->status = status;
    stats->iters = it;
    stats->flags = flags;
    stats->ir_total = cnt.ir;
    stats->n_fact = cnt.fact;
    stats->n_fact64 = cnt.fact64;
    stats->n_solve = cnt.solve;
    stats->n_res = cnt.res;
    stats->res[0] = r.g;
    stats->res[1] = r.b;
    stats->res[2] = r.d;
    stats->res[3] = r.mu;
  }
#if GQ_IPM_TC
  if (C.tc) {
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::dealloc(C.taddr, kTcCols);
  }
#endif
}

}  // namespace

#if GQ_IPM_TC
size_t ipm_tc_smem_bytes(const Batch& b, const Shape& sh) { return smem_plan(b, sh).bytes; }

cudaError_t launch_ipm_tc(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                          LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count) {
#elif GQ_IPM_SOFT
cudaError_t launch_ipm_soft(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                            LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count) {
#else
size_t ipm_smem_bytes(const Batch& b, const Shape& sh) { return smem_plan(b, sh).bytes; }

cudaError_t launch_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                       LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count) {
#endif
  if (count <= 0) return cudaSuccess;
  const size_t smem = GQ_IPM_TC ? smem_plan(b, sh).bytes : ipm_smem_bytes(b, sh);
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  // opt in to the dynamic shared memory this launch needs (set on the current
  // device at every launch above the default: no cache shared between host
  // threads or devices)
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(ipm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // 256 threads by default whatever the stage size: the micro-tiled products
  // and the trailing Cholesky updates have work for all of them (measured
  // faster than one thread per stage row on the ragged and large-stage
  // workloads); the schedule may choose 64 or 128
  const int nt = sh.threads > 0 ? sh.threads : 256;
  DirOut o{};
  if (out) o = *out;
  ipm_kernel<<<count, nt, smem, stream>>>(b, sh, arg, (int)kind, sigma_mu, o, order);
  return cudaGetLastError();
}

}  // namespace gq
