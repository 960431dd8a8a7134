// Batched OCP-QP interior-point kernels for sm_103a.
//
// One thread block solves one QP: the whole Mehrotra predictor-corrector loop
// (Sec. 4.2) runs on the device, with
//   a1  residuals of eq. (delta)                              FP64
//   a2  barrier terms and the reduced right-hand side, eq. (kkt) FP64
//   a3  square-root Riccati factorisation (Sec. 3.3, variant b) Tf
//   a4  Riccati solve: backward vector sweep, forward sweep      Tf
//   a5  affine step length and duality measure                  FP64
//   a6  Mehrotra corrector, conditional (Sec. 4.2)               Tf solve
//   a7  iterative refinement on eq. (itref) (Sec. 3.4)           FP64 residual
//   a8  step, update, lower clamp of lambda and t (Sec. 4.2)     FP64
// Tf is double (plain path) or float (mixed path).
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

#include "gq_internal.h"
#include "gq_launch.h"

namespace gq {
namespace {

constexpr double kIrFailRatio = 1e-6;  // mixed path: IR residual ratio that triggers FP64 factors

__device__ __forceinline__ int64_t globaltimer() {
  int64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// block-wide reductions (fixed order: the result depends only on blockDim)
// ---------------------------------------------------------------------------
struct OpSum {
  __device__ double operator()(double a, double b) const { return a + b; }
};
struct OpMax {
  __device__ double operator()(double a, double b) const { return fmax(a, b); }
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
struct Ctx {
  const Batch* B;
  const StageDesc* st;  // shared-memory copy of this QP's stage table
  int N;
  int nact;             // active (unmasked) sides
  int nside;            // all sides of this QP
  double* red;          // reduction scratch (32 doubles)
  double* chunk;        // per-32-side partial sums for fixed_sum
  double* vbuf;         // vector scratch (6 * vmax doubles)
  int vmax;
  void* mat;            // matrix scratch (Tf): L_{n+1}, Phi, M
  int nvmax, nxmax, nemax;
};

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

__device__ __forceinline__ StageData lay(const StageDesc& s) {
  return stage_data_layout(s.nx, s.nu, s.nx1, s.nbu + s.nbx, s.ng);
}

// value of constraint c of stage s at the stage vector y (global, length nv)
__device__ __forceinline__ double cons_value(const Batch& B, const StageDesc& s, const StageData& L,
                                             const double* D, int c, const double* y) {
  const int nb = s.nbu + s.nbx;
  if (c < nb) return y[B.idx[s.idx + c]];
  const int nv = s.nx + s.nu;
  const double* row = D + L.DC + (int64_t)(c - nb) * nv;
  double v = 0.0;
  for (int j = 0; j < nv; ++j) v = fma(row[j], y[j], v);
  return v;
}

// ---------------------------------------------------------------------------
// a1: residual function of eq. (delta).  With `lin` the constant terms
// (r, q, b and bounds) are dropped and (add_g, add_b) are added instead:
// that is the iterative-refinement residual of Sec. 3.4 for a direction.
// ---------------------------------------------------------------------------
__device__ __noinline__ void residual_g_b(const Ctx& C, const double* y, const double* pi, const double* lam,
                             double* og, double* ob, bool lin, const double* add_g,
                             const double* add_b) {
  const Batch& B = *C.B;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int n = 0; n <= C.N; ++n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng;
    const double* yn = y + s.var;
    for (int i = tid; i < nv; i += NT) {
      const double* row = D + L.RSQ + (int64_t)i * nv;
      double acc = lin ? add_g[s.var + i] : D[L.rq + i];
      for (int j = 0; j < nv; ++j) acc = fma(row[j], yn[j], acc);
      if (n < C.N) {
        const double* ba = D + L.BAt + (int64_t)i * s.nx1;
        const double* pn1 = pi + s.eq;
        for (int k = 0; k < s.nx1; ++k) acc = fma(ba[k], pn1[k], acc);
      }
      if (n > 0 && i >= s.nu) acc -= pi[C.st[n - 1].eq + (i - s.nu)];
      const double* lm = lam + s.side;
      for (int g = 0; g < s.ng; ++g) {
        const double dc = D[L.DC + (int64_t)g * nv + i];
        acc = fma(-dc, lm[nb + g] - lm[nc + nb + g], acc);
      }
      og[s.var + i] = acc;
    }
    if (n < C.N) {
      const double* yn1 = y + C.st[n + 1].var + C.st[n + 1].nu;
      for (int k = tid; k < s.nx1; k += NT) {
        double acc = lin ? add_b[s.eq + k] : D[L.b + k];
        for (int i = 0; i < nv; ++i) acc = fma(D[L.BAt + (int64_t)i * s.nx1 + k], yn[i], acc);
        ob[s.eq + k] = acc - yn1[k];
      }
    }
  }
  __syncthreads();
  // box rows of -C' lambda (indices within a stage are distinct)
  for (int n = 0; n <= C.N; ++n) {
    const StageDesc s = C.st[n];
    const int nb = s.nbu + s.nbx, nc = nb + s.ng;
    const double* lm = lam + s.side;
    for (int c = tid; c < nb; c += NT) og[s.var + B.idx[s.idx + c]] -= lm[c] - lm[nc + c];
  }
  __syncthreads();
}

// r_d = -C y + d + t per side; returns max |r_d| over active sides.
__device__ __noinline__ double residual_d(const Ctx& C, const double* y, const double* t, double* rd) {
  const Batch& B = *C.B;
  double mx = 0.0;
  for (int n = 0; n <= C.N; ++n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nc = s.nbu + s.nbx + s.ng;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const double v = cons_value(B, s, L, D, c, y + s.var);
      const double lo = D[L.lo + c], hi = D[L.hi + c];
      const int il = s.side + c, iu = s.side + nc + c;
      double a = 0.0, b = 0.0;
      if (lo != -INFINITY) a = lo - v + t[il];
      if (hi != INFINITY) b = v - hi + t[iu];
      rd[il] = a;
      rd[iu] = b;
      mx = fmax(mx, fmax(fabs(a), fabs(b)));
    }
  }
  return mx;
}

struct Norms {
  double g, b, d, mu;
};

__device__ __noinline__ Norms residuals(const Ctx& C) {
  const Batch& B = *C.B;
  residual_g_b(C, B.y, B.pi, B.lam, B.rg, B.rb, false, nullptr, nullptr);
  double md = residual_d(C, B.y, B.t, B.rd);
  double mg = 0.0, mb = 0.0;
  const int q0v = C.st[0].var, q1v = C.st[C.N].var + C.st[C.N].nx + C.st[C.N].nu;
  for (int i = q0v + threadIdx.x; i < q1v; i += blockDim.x) mg = fmax(mg, fabs(B.rg[i]));
  const int q0e = C.st[0].eq, q1e = C.st[C.N].eq;
  for (int i = q0e + threadIdx.x; i < q1e; i += blockDim.x) mb = fmax(mb, fabs(B.rb[i]));
  // masked sides hold lambda = 0 and add nothing
  const int s0 = C.st[0].side;
  const double* lam = B.lam + s0;
  const double* tt = B.t + s0;
  const double sm = fixed_sum(C, C.nside, [&](int i) { return lam[i] * tt[i]; });
  Norms r;
  r.g = block_reduce(mg, C.red, OpMax());
  r.b = block_reduce(mb, C.red, OpMax());
  r.d = block_reduce(md, C.red, OpMax());
  r.mu = C.nact ? sm / C.nact : 0.0;
  return r;
}

// ---------------------------------------------------------------------------
// a2: reduced gradient gt = r_g - C'(W r_d - T^{-1} r_m), W = Lambda T^{-1}
// ---------------------------------------------------------------------------
__device__ __noinline__ void reduced_rhs(const Ctx& C, const double* rg, const double* rd, const double* rm,
                            double* gt) {
  const Batch& B = *C.B;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int n = 0; n <= C.N; ++n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng;
    const double* lm = B.lam + s.side;
    const double* tt = B.t + s.side;
    const double* d = rd + s.side;
    const double* m = rm + s.side;
    for (int i = tid; i < nv; i += NT) {
      double acc = rg[s.var + i];
      for (int g = 0; g < s.ng; ++g) {
        const int l = nb + g, u = nc + nb + g;
        double v = 0.0;
        if (D[L.lo + l] != -INFINITY) v += (lm[l] * d[l] - m[l]) / tt[l];
        if (D[L.hi + l] != INFINITY) v -= (lm[u] * d[u] - m[u]) / tt[u];
        acc = fma(-D[L.DC + (int64_t)g * nv + i], v, acc);
      }
      gt[s.var + i] = acc;
    }
  }
  __syncthreads();
  for (int n = 0; n <= C.N; ++n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nb = s.nbu + s.nbx, nc = nb + s.ng;
    const double* lm = B.lam + s.side;
    const double* tt = B.t + s.side;
    const double* d = rd + s.side;
    const double* m = rm + s.side;
    for (int c = tid; c < nb; c += NT) {
      double v = 0.0;
      if (D[L.lo + c] != -INFINITY) v += (lm[c] * d[c] - m[c]) / tt[c];
      if (D[L.hi + c] != INFINITY) v -= (lm[nc + c] * d[nc + c] - m[nc + c]) / tt[nc + c];
      gt[s.var + B.idx[s.idx + c]] -= v;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// a3: square-root Riccati factorisation, stages N..0
// ---------------------------------------------------------------------------
__device__ __forceinline__ int elim_size(const StageDesc& s, int n) { return n == 0 ? s.nx + s.nu : s.nu; }

template <typename Tf>
__device__ __forceinline__ Tf* fac_ptr(const Batch& B, const StageDesc& s) {
  return static_cast<Tf*>(B.fac) + s.fac;
}

// Returns false when a pivot is not positive (not positive definite).
template <typename Tf>
__device__ __noinline__ bool factor(const Ctx& C, double reg) {
  const Batch& B = *C.B;
  const int tid = threadIdx.x, NT = blockDim.x;
  Tf* sL = static_cast<Tf*>(C.mat);                      // L_{n+1}: nx1 x nx1
  Tf* sPhi = sL + C.nxmax * C.nxmax;                      // nv x nv
  Tf* sM = sPhi + C.nvmax * C.nvmax;                      // nv x nx1, also X temp
  Tf* sw = reinterpret_cast<Tf*>(C.vbuf);                 // per-constraint weight
  bool ok = true;
  for (int n = C.N; n >= 0; --n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
    const int ne = elim_size(s, n), nk = nv - ne;
    const double* lm = B.lam + s.side;
    const double* tt = B.t + s.side;
    // barrier weights W_lo + W_hi per constraint
    for (int c = tid; c < nc; c += NT) {
      double w = 0.0;
      if (D[L.lo + c] != -INFINITY) w += lm[c] / tt[c];
      if (D[L.hi + c] != INFINITY) w += lm[nc + c] / tt[nc + c];
      sw[c] = (Tf)w;
    }
    // M = [B A]' L_{n+1}
    if (n < C.N) {
      for (int e = tid; e < nv * nx1; e += NT) {
        const int i = e / nx1, j = e - i * nx1;
        const double* ba = D + L.BAt + (int64_t)i * nx1;
        Tf acc = 0;
        for (int k = j; k < nx1; ++k) acc += (Tf)ba[k] * sL[k * nx1 + j];
        sM[i * nx1 + j] = acc;
      }
    }
    __syncthreads();
    // Phi = RSQ + reg I + [D C]' diag(w_g) [D C] + M M'   (lower triangle)
    for (int e = tid; e < nv * nv; e += NT) {
      const int i = e / nv, j = e - i * nv;
      if (j > i) continue;
      Tf acc = (Tf)D[L.RSQ + (int64_t)i * nv + j];
      if (i == j) acc += (Tf)reg;
      for (int g = 0; g < s.ng; ++g)
        acc += (Tf)D[L.DC + (int64_t)g * nv + i] * sw[nb + g] * (Tf)D[L.DC + (int64_t)g * nv + j];
      if (n < C.N)
        for (int k = 0; k < nx1; ++k) acc += sM[i * nx1 + k] * sM[j * nx1 + k];
      sPhi[i * nv + j] = acc;
    }
    __syncthreads();
    for (int c = tid; c < nb; c += NT) {
      const int k = B.idx[s.idx + c];
      sPhi[k * nv + k] += sw[c];
    }
    __syncthreads();
    // right-looking Cholesky, outer-product form on the unscaled columns
    for (int k = 0; k < nv; ++k) {
      Tf d = sPhi[k * nv + k];
      if (!(d > (Tf)0)) {
        ok = false;
        d = (Tf)1;
      }
      const Tf inv = (Tf)1 / d;
      for (int i = k + 1 + tid; i < nv; i += NT) {
        const Tf lik = sPhi[i * nv + k] * inv;
        Tf* ri = sPhi + i * nv;
        for (int j = k + 1; j <= i; ++j) ri[j] -= lik * sPhi[j * nv + k];
      }
      __syncthreads();
    }
    // scale columns: L_jj = sqrt(d_j), L_ij = Phi_ij / sqrt(d_j)
    Tf* sdiag = sw;  // weights no longer needed
    for (int j = tid; j < nv; j += NT) {
      Tf d = sPhi[j * nv + j];
      sdiag[j] = d > (Tf)0 ? sqrt(d) : (Tf)1;
    }
    __syncthreads();
    for (int e = tid; e < nv * nv; e += NT) {
      const int i = e / nv, j = e - i * nv;
      if (j > i) continue;
      sPhi[i * nv + j] = (i == j) ? sdiag[j] : sPhi[i * nv + j] / sdiag[j];
    }
    __syncthreads();
    // X = L_ee^{-1} (lower), column j by thread j, into the M buffer
    for (int j = tid; j < ne; j += NT) {
      sM[j * ne + j] = (Tf)1 / sPhi[j * nv + j];
      for (int i = j + 1; i < ne; ++i) {
        Tf acc = 0;
        for (int k = j; k < i; ++k) acc += sPhi[i * nv + k] * sM[k * ne + j];
        sM[i * ne + j] = -acc / sPhi[i * nv + i];
      }
    }
    __syncthreads();
    for (int e = tid; e < ne * ne; e += NT) {
      const int i = e / ne, j = e - i * ne;
      if (j <= i) sPhi[i * nv + j] = sM[i * ne + j];
    }
    __syncthreads();
    // store the factor, keep L_n = L_kk for stage n-1
    Tf* F = fac_ptr<Tf>(B, s);
    for (int e = tid; e < nv * nv; e += NT) {
      const int i = e / nv, j = e - i * nv;
      F[e] = (j <= i) ? sPhi[e] : (Tf)0;
    }
    for (int e = tid; e < nk * nk; e += NT) {
      const int i = e / nk, j = e - i * nk;
      sL[i * nk + j] = (j <= i) ? sPhi[(ne + i) * nv + ne + j] : (Tf)0;
    }
    __syncthreads();
  }
  return ok;
}

// ---------------------------------------------------------------------------
// a4: Riccati solve of eq. (kkt) for right-hand side (gt, rb) -> (dy, dpi)
// ---------------------------------------------------------------------------
template <typename Tf>
__device__ __noinline__ void riccati_solve(const Ctx& C, const double* gt, const double* rb, double* dy, double* dpi) {
  const Batch& B = *C.B;
  const int tid = threadIdx.x, NT = blockDim.x;
  Tf* va = reinterpret_cast<Tf*>(C.vbuf);
  Tf* vb = va + C.vmax;
  Tf* phi = vb + C.vmax;
  Tf* pn1 = phi + C.vmax;  // p_{n+1}
  Tf* ln = pn1 + C.vmax;
  double* lp = B.lp;       // per stage: l (ne entries) then p_n (nk entries)
  // backward sweep
  for (int n = C.N; n >= 0; --n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nv = s.nx + s.nu, nx1 = s.nx1;
    const int ne = elim_size(s, n), nk = nv - ne;
    const Tf* F = fac_ptr<Tf>(B, s);
    if (n < C.N) {
      const StageDesc s1 = C.st[n + 1];
      const int nv1 = s1.nx + s1.nu, ne1 = s1.nu;
      const Tf* F1 = fac_ptr<Tf>(B, s1) + ne1 * nv1 + ne1;  // L_{n+1}, row stride nv1
      // va = L_{n+1}' rb_n
      for (int k = tid; k < nx1; k += NT) {
        Tf acc = 0;
        for (int j = k; j < nx1; ++j) acc += F1[j * nv1 + k] * (Tf)rb[s.eq + j];
        va[k] = acc;
      }
      __syncthreads();
      // vb = L_{n+1} va + p_{n+1}
      for (int k = tid; k < nx1; k += NT) {
        Tf acc = pn1[k];
        for (int j = 0; j <= k; ++j) acc += F1[k * nv1 + j] * va[j];
        vb[k] = acc;
      }
      __syncthreads();
    }
    // phi = gt_n + [B A]' vb
    for (int i = tid; i < nv; i += NT) {
      Tf acc = (Tf)gt[s.var + i];
      if (n < C.N) {
        const double* ba = D + L.BAt + (int64_t)i * nx1;
        for (int k = 0; k < nx1; ++k) acc += (Tf)ba[k] * vb[k];
      }
      phi[i] = acc;
    }
    __syncthreads();
    // l = X phi_e
    for (int i = tid; i < ne; i += NT) {
      Tf acc = 0;
      for (int j = 0; j <= i; ++j) acc += F[i * nv + j] * phi[j];
      ln[i] = acc;
      lp[s.var + i] = (double)acc;
    }
    __syncthreads();
    // p_n = phi_k - L_ke l  -> becomes p_{n+1} of stage n-1
    for (int i = tid; i < nk; i += NT) {
      Tf acc = phi[ne + i];
      for (int j = 0; j < ne; ++j) acc -= F[(ne + i) * nv + j] * ln[j];
      pn1[i] = acc;
      lp[s.var + ne + i] = (double)acc;
    }
    __syncthreads();
  }
  // forward sweep
  for (int n = 0; n <= C.N; ++n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nv = s.nx + s.nu, nx1 = s.nx1;
    const int ne = elim_size(s, n), nk = nv - ne;
    const Tf* F = fac_ptr<Tf>(B, s);
    double* yn = dy + s.var;
    // va = l + L_ke' x_n
    for (int j = tid; j < ne; j += NT) {
      Tf acc = (Tf)lp[s.var + j];
      for (int i = 0; i < nk; ++i) acc += F[(ne + i) * nv + j] * (Tf)yn[ne + i];
      va[j] = acc;
    }
    __syncthreads();
    // y_e = -X' va
    for (int i = tid; i < ne; i += NT) {
      Tf acc = 0;
      for (int j = i; j < ne; ++j) acc += F[j * nv + i] * va[j];
      yn[i] = -(double)acc;
    }
    __syncthreads();
    if (n < C.N) {
      const StageDesc s1 = C.st[n + 1];
      const int nv1 = s1.nx + s1.nu, ne1 = s1.nu;
      const Tf* F1 = fac_ptr<Tf>(B, s1) + ne1 * nv1 + ne1;
      double* x1 = dy + s1.var + s1.nu;
      // x_{n+1} = [B A] y_n + rb_n
      for (int k = tid; k < nx1; k += NT) {
        Tf acc = (Tf)rb[s.eq + k];
        for (int i = 0; i < nv; ++i) acc += (Tf)D[L.BAt + (int64_t)i * nx1 + k] * (Tf)yn[i];
        x1[k] = (double)acc;
        vb[k] = acc;
      }
      __syncthreads();
      // pi_{n+1} = L_{n+1}(L_{n+1}' x_{n+1}) + p_{n+1}
      for (int k = tid; k < nx1; k += NT) {
        Tf acc = 0;
        for (int j = k; j < nx1; ++j) acc += F1[j * nv1 + k] * vb[j];
        va[k] = acc;
      }
      __syncthreads();
      for (int k = tid; k < nx1; k += NT) {
        Tf acc = (Tf)lp[s1.var + ne1 + k];
        for (int j = 0; j <= k; ++j) acc += F1[k * nv1 + j] * va[j];
        dpi[s.eq + k] = (double)acc;
      }
      __syncthreads();
    }
  }
}

// dt = C dy - r_d, dlam = -T^{-1}(r_m + Lambda dt) on active sides (0 elsewhere)
__device__ __noinline__ void recover(const Ctx& C, const double* dy, double* dlam, double* dt) {
  const Batch& B = *C.B;
  for (int n = 0; n <= C.N; ++n) {
    const StageDesc s = C.st[n];
    const StageData L = lay(s);
    const double* D = B.data + s.data;
    const int nc = s.nbu + s.nbx + s.ng;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const double v = cons_value(B, s, L, D, c, dy + s.var);
      const int il = s.side + c, iu = s.side + nc + c;
      if (D[L.lo + c] != -INFINITY) {
        const double a = v - B.rd[il];
        dt[il] = a;
        dlam[il] = -(B.rm[il] + B.lam[il] * a) / B.t[il];
      } else {
        dt[il] = 0.0;
        dlam[il] = 0.0;
      }
      if (D[L.hi + c] != INFINITY) {
        const double a = -v - B.rd[iu];
        dt[iu] = a;
        dlam[iu] = -(B.rm[iu] + B.lam[iu] * a) / B.t[iu];
      } else {
        dt[iu] = 0.0;
        dlam[iu] = 0.0;
      }
    }
  }
  __syncthreads();
}

// elementwise pass over this QP's sides
template <class F>
__device__ void for_sides(const Ctx& C, F f) {
  const int s0 = C.st[0].side;
  const StageDesc& last = C.st[C.N];
  const int s1 = last.side + 2 * (last.nbu + last.nbx + last.ng);
  for (int i = s0 + threadIdx.x; i < s1; i += blockDim.x) f(i);
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
};

// factor-precision solve of eq. (delta) for the current r_m, then FP64
// recovery of (dlam, dt); with ir > 0, iterative refinement (Sec. 3.4).
// Returns the final refinement residual ratio (0 without refinement).
template <typename Tf>
__device__ __noinline__ double newton_dir(const Ctx& C, const Dir& d, int ir, double ir_tol, Count* cnt) {
  const Batch& B = *C.B;
  reduced_rhs(C, B.rg, B.rd, B.rm, B.gt);
  riccati_solve<Tf>(C, B.gt, B.rb, d.dy, d.dpi);
  ++cnt->solve;
  recover(C, d.dy, d.dlam, d.dt);
  if (ir <= 0) return 0.0;
  // ||rhs||inf of the reduced system
  double mr = 0.0;
  {
    const int v0 = C.st[0].var, v1 = C.st[C.N].var + C.st[C.N].nx + C.st[C.N].nu;
    for (int i = v0 + threadIdx.x; i < v1; i += blockDim.x) mr = fmax(mr, fabs(B.gt[i]));
    const int e0 = C.st[0].eq, e1 = C.st[C.N].eq;
    for (int i = e0 + threadIdx.x; i < e1; i += blockDim.x) mr = fmax(mr, fabs(B.rb[i]));
  }
  mr = block_reduce(mr, C.red, OpMax());
  double ratio = 0.0;
  for (int k = 0; k <= ir; ++k) {
    // residual of eq. (delta) for the direction (the r_d and r_m rows vanish
    // because dt and dlam are recovered from dy in FP64)
    residual_g_b(C, d.dy, d.dpi, d.dlam, B.rg2, B.rb2, true, B.rg, B.rb);
    ++cnt->res;
    double m = 0.0;
    const int v0 = C.st[0].var, v1 = C.st[C.N].var + C.st[C.N].nx + C.st[C.N].nu;
    for (int i = v0 + threadIdx.x; i < v1; i += blockDim.x) m = fmax(m, fabs(B.rg2[i]));
    const int e0 = C.st[0].eq, e1 = C.st[C.N].eq;
    for (int i = e0 + threadIdx.x; i < e1; i += blockDim.x) m = fmax(m, fabs(B.rb2[i]));
    m = block_reduce(m, C.red, OpMax());
    ratio = mr > 0.0 ? m / mr : 0.0;
    if (k == ir || m <= ir_tol * mr) break;
    // correction: same factors, the refinement residual as right-hand side
    // (reduced gradient = r_g^ir since the r_d and r_m rows are zero)
    riccati_solve<Tf>(C, B.rg2, B.rb2, B.dy2, B.dpi2);
    for (int i = v0 + threadIdx.x; i < v1; i += blockDim.x) d.dy[i] += B.dy2[i];
    for (int i = e0 + threadIdx.x; i < e1; i += blockDim.x) d.dpi[i] += B.dpi2[i];
    __syncthreads();
    recover(C, d.dy, d.dlam, d.dt);
    ++cnt->ir;
    ++cnt->solve;
  }
  return ratio;
}

template <typename Tf>
__device__ bool factor_dispatch(const Ctx& C, double reg) {
  return factor<Tf>(C, reg);
}

// ---------------------------------------------------------------------------
// the kernel: one block per QP
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ipm_kernel(const __grid_constant__ Batch B, const Shape sh,
                                                  const __grid_constant__ gq_ipm_arg arg, int kind,
                                                  double sigma_mu, const DirOut out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int q = B.order[blockIdx.x];
  const QpDesc qd = B.qp[q];
  const int tid = threadIdx.x;
  // shared-memory plan
  StageDesc* sst = reinterpret_cast<StageDesc*>(smem);
  size_t off = ((size_t)sh.nst_max * sizeof(StageDesc) + 15) & ~size_t(15);
  double* red = reinterpret_cast<double*>(smem + off);
  off += 32 * sizeof(double);
  double* chunk = reinterpret_cast<double*>(smem + off);
  off += (size_t)((sh.nside_max + 31) / 32 + 1) * sizeof(double);
  const int vmax = B.nvmax + B.ngmax + 2;
  double* vbuf = reinterpret_cast<double*>(smem + off);
  off += (size_t)6 * vmax * sizeof(double);
  void* mat = smem + off;

  for (int n = tid; n <= qd.N; n += blockDim.x) sst[n] = B.st[qd.stage0 + n];
  __syncthreads();

  Ctx C;
  C.B = &B;
  C.st = sst;
  C.N = qd.N;
  C.red = red;
  C.chunk = chunk;
  C.nside = qd.nsidet;
  C.vbuf = vbuf;
  C.vmax = vmax;
  C.mat = mat;
  C.nvmax = B.nvmax;
  C.nxmax = B.nxmax;
  C.nemax = sh.ne_max;

  // count active sides
  {
    double cnt = 0.0;
    for (int n = 0; n <= C.N; ++n) {
      const StageDesc s = sst[n];
      const StageData L = lay(s);
      const double* D = B.data + s.data;
      const int nc = s.nbu + s.nbx + s.ng;
      for (int c = tid; c < nc; c += blockDim.x)
        cnt += (D[L.lo + c] != -INFINITY) + (D[L.hi + c] != INFINITY);
    }
    C.nact = (int)block_reduce(cnt, red, OpSum());
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
      stats->status = ok ? GQ_STATUS_CONVERGED : GQ_STATUS_NAN;
      stats->ir_total = cnt.ir;
    }
    return;
  }

  // ---------------- full IPM (Sec. 4.2) ----------------
  const int64_t t_start = arg.timeout_ns > 0 ? globaltimer() : 0;
  // a0: start point
  {
    const bool warm1 = arg.warm_start >= 1, warm2 = arg.warm_start >= 2;
    if (!warm1) {
      for (int i = qd.var0 + tid; i < qd.var0 + qd.nvt; i += blockDim.x) B.y[i] = 0.0;
      for (int i = qd.eq0 + tid; i < qd.eq0 + qd.neqt; i += blockDim.x) B.pi[i] = 0.0;
    }
    __syncthreads();
    for (int n = 0; n <= C.N; ++n) {
      const StageDesc s = sst[n];
      const StageData L = lay(s);
      const double* D = B.data + s.data;
      const int nc = s.nbu + s.nbx + s.ng;
      for (int c = tid; c < nc; c += blockDim.x) {
        const double v = cons_value(B, s, L, D, c, B.y + s.var);
        const double lo = D[L.lo + c], hi = D[L.hi + c];
        const int il = s.side + c, iu = s.side + nc + c;
        if (lo != -INFINITY) {
          if (warm2) {
            B.lam[il] = fmax(B.lam[il], arg.warm_min);
            B.t[il] = fmax(B.t[il], arg.warm_min);
          } else {
            B.lam[il] = 1.0;
            B.t[il] = fmax(1.0, v - lo);
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
            B.t[iu] = fmax(1.0, hi - v);
          }
        } else {
          B.lam[iu] = 0.0;
          B.t[iu] = 1.0;
        }
      }
    }
    __syncthreads();
  }

  int status = GQ_STATUS_MAX_ITER, it = 0, flags = 0;
  Count cnt;
  bool fp64 = !mixed;
  double alpha = 1.0;
  Norms r{0, 0, 0, 0};
  const Dir d{B.dy, B.dpi, B.dlam, B.dt};
  while (true) {
    r = residuals(C);
    ++cnt.res;
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
      // one thread's clock decides for the block
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
    const bool ok = fp64 ? factor<double>(C, reg) : factor<float>(C, reg);
    ++cnt.fact;
    cnt.fact64 += fp64;
    const int okall = (int)block_reduce(ok ? 1.0 : 0.0, red, OpMin());
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
    const int ir = (mixed && !fp64) || arg.mode == GQ_MODE_BALANCE ? arg.ir_steps : 0;
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
      if (!fp64 && arg.fp64_fallback && ir > 0 && !(ratio <= kIrFailRatio)) {
        // a7 failed to recover the accuracy of the FP32 factors: refactor in FP64
        fp64 = true;
        flags |= GQ_FLAG_FP64_FALLBACK;
        continue;
      }
      alpha = fmin(1.0, arg.tau_b * max_step(C, d.dlam, d.dt));
    } else {
      if (ir > 0) {
        // no inequalities: refine the single Newton step
        double ratio = fp64 ? newton_dir<double>(C, d, ir, arg.ir_tol, &cnt)
                            : newton_dir<float>(C, d, ir, arg.ir_tol, &cnt);
        if (!fp64 && arg.fp64_fallback && !(ratio <= kIrFailRatio)) {
          fp64 = true;
          flags |= GQ_FLAG_FP64_FALLBACK;
          continue;
        }
      }
      alpha = 1.0;
    }
    // a8: step and clamp
    for (int i = qd.var0 + tid; i < qd.var0 + qd.nvt; i += blockDim.x) B.y[i] += alpha * d.dy[i];
    for (int i = qd.eq0 + tid; i < qd.eq0 + qd.neqt; i += blockDim.x) B.pi[i] += alpha * d.dpi[i];
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
}

}  // namespace

size_t ipm_smem_bytes(const Batch& b, const Shape& sh) {
  const int vmax = b.nvmax + b.ngmax + 2;
  size_t smem = ((size_t)sh.nst_max * sizeof(StageDesc) + 15) & ~size_t(15);
  smem += 32 * sizeof(double) + (size_t)6 * vmax * sizeof(double);
  smem += (size_t)((sh.nside_max + 31) / 32 + 1) * sizeof(double);
  const int wide = b.nxmax > sh.ne_max ? b.nxmax : sh.ne_max;
  const size_t mbuf = (size_t)b.nvmax * (wide > 0 ? wide : 1);
  smem += ((size_t)b.nxmax * b.nxmax + (size_t)b.nvmax * b.nvmax + mbuf) * sizeof(double);
  return smem;
}

cudaError_t launch_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                       LaunchKind kind, double sigma_mu, const DirOut* out) {
  const size_t smem = ipm_smem_bytes(b, sh);
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(ipm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int nt = ((b.nvmax + 31) / 32) * 32;
  nt = nt < 32 ? 32 : (nt > 256 ? 256 : nt);
  DirOut o{};
  if (out) o = *out;
  ipm_kernel<<<b.nqp, nt, smem, stream>>>(b, sh, arg, (int)kind, sigma_mu, o);
  return cudaGetLastError();
}

}  // namespace gq
