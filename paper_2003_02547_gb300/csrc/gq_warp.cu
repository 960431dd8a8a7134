// Warp-per-QP IPM kernel for QPs whose stages all have nu + nx <= 32 and
// nx <= 32 (the small stages of model predictive control).
//
// The algorithm is the one of gq_ipm.cu (Mehrotra predictor-corrector of
// Sec. 4.2, square-root Riccati factorisation of eq. (kkt), Sec. 3.3, with
// iterative refinement, Sec. 3.4), mapped onto one warp:
//   * lane i owns row i of the stage matrices: the Riccati stage matrix Phi,
//     the products M = [B A]' L_{n+1}, and element i of every stage vector;
//   * the Cholesky factorisation runs on register rows, with the pivot and
//     the factor column broadcast by warp shuffles -- no shared-memory
//     read-modify-write chains and no block barriers;
//   * shared-memory matrices use an odd row stride (33), so lane-per-row
//     reads are free of bank conflicts;
//   * each stage's data block (and in the solves its factor block) arrives
//     by one 1-D bulk copy into a two-slot ring, one stage ahead;
//   * the mixed-precision path reads an FP32 mirror of the data for the
//     factorisation and solves (no FP64->FP32 conversions in inner loops),
//     the FP64 data for residuals and refinement.
#include <cuda_runtime.h>

#include <cstdint>

#include "gq_device.h"
#include "gq_internal.h"
#include "gq_launch.h"
#include "gq_mma.h"

namespace gq {
namespace {

using namespace dev;

constexpr int LDS = 33;                 // shared-memory row stride
constexpr double kLift = 1e-10;          // smallest floor of lambda, t after a lost FP64 pivot
constexpr double kLiftRel = 1e-2;        // ... relative to the stationarity residual
constexpr double kRegRetry = 1e-10;     // primal regularisation of an FP64 refactorisation after a lost pivot
constexpr double kInexact = 0.1;        // mixed path: direction residual allowed per unit of iterate residual

__device__ __forceinline__ StageData wlay(const StageDesc& s) {
  return stage_data_layout(s);
}
__device__ __forceinline__ int welim(const StageDesc& s, int n) { return n == 0 ? s.nx + s.nu : s.nu; }

template <typename T>
__device__ __forceinline__ T wrsqrt(T x);
template <>
__device__ __forceinline__ float wrsqrt<float>(float x) {
  return rsqrtf(x);
}
template <>
__device__ __forceinline__ double wrsqrt<double>(double x) {
  return rsqrt(x);
}

struct WCtx {
  const Batch* B;
  const StageDesc* st;
  int N, nact, nside, side0, v0, v1, e0, e1, lane;
  unsigned char* ring0;  // two consecutive ring slots of `slot` bytes (no indexed
  uint32_t slot;         // array: keeps the context in registers)
  uint64_t* bar;
  uint32_t parity;
  uint32_t fac_off;
  bool ok;
  void* sL;    // L_{n+1}, 32 x LDS
  void* sM;    // M, then X = L_ee^{-1}, 32 x LDS
  void* sP;    // Phi and its factor, 32 x LDS
  double* sv;  // per-constraint scratch (vmax doubles)
  int vmax;
  bool qr;     // array algorithm: chol(Ht + M M') by QR of [chol(Ht)'; M']
  double* xb;  // two 32-entry broadcast buffers (stage vectors read by every lane)
};

// Stage vector held one element per lane, made readable by every lane from
// shared memory (buffer k of two): the dot-product loops then issue
// independent conflict-free loads instead of one dependent shuffle per term.
// Warp-wide; the barrier before the store keeps earlier readers of the buffer.
template <typename V>
__device__ __forceinline__ const V* wbcast(const WCtx& C, int k, V v) {
  V* buf = reinterpret_cast<V*>(C.xb) + 32 * k;
  __syncwarp();
  buf[C.lane] = v;
  __syncwarp();
  return buf;
}

// deterministic sum over this QP's sides: each lane sums its sides in index
// order, then one butterfly (every lane holds the same bits)
template <class F>
__device__ __forceinline__ double side_sum(const WCtx& C, F f) {
  double acc = 0.0;
#pragma unroll 4
  for (int k = C.lane; k < C.nside; k += 32) acc += f(C.side0 + k);
  return warp_sum(acc);
}

// largest of m (not negative) and |v| by the bit patterns on the integer pipe
// (for non-negative doubles the integer order is the numeric one, and a NaN
// orders above every number, so it propagates as in max_nan)
__device__ __forceinline__ double max_abs_bits(double m, double v) {
  const long long a = __double_as_longlong(m), b = __double_as_longlong(v) & 0x7fffffffffffffffLL;
  return __longlong_as_double(a > b ? a : b);
}

// bound tests on the integer pipe: lo is not -inf, hi is not +inf
__device__ __forceinline__ bool lo_on(double lo) { return __double_as_longlong(lo) != (long long)0xfff0000000000000ULL; }
__device__ __forceinline__ bool hi_on(double hi) { return __double_as_longlong(hi) != 0x7ff0000000000000LL; }
// x != 0 (either zero) on the integer pipe; NaN counts as non-zero, as in
// the FP64 test
__device__ __forceinline__ bool nonzero_bits(double x) { return (__double_as_longlong(x) << 1) != 0; }
// fmax(x, m) for m > 0 on the integer pipe: negative x (sign bit set, an
// integer below m's) and NaN give m, as fmax does
__device__ __forceinline__ double fmax_pos_bits(double x, double m) {
  const long long xi = __double_as_longlong(x), mi = __double_as_longlong(m);
  return (xi > mi && xi <= 0x7ff0000000000000LL) ? x : m;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic on the FP32 pipe: a value carried as the unevaluated
// sum h + l of two FP32 numbers, about 48 significant bits (Dekker's pair
// arithmetic: the product's error by one FMA, the sum's error by Knuth's
// two-sum).  On GB300 every FP64 instruction -- FMA, add, compare or a
// conversion to or from FP64 -- holds a sub-partition's FP64 pipe for about
// 70 cycles, an FP32 FMA for about 1.5, so the mixed path's refinement
// residual, whose mat-vecs need more than FP32 but not all of FP64, takes
// them here.  The _rn intrinsics keep the compiler from contracting the
// error-free steps into FMAs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_split(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}
// (sh, sl) += (ah + al)(xh + xl): the product to about 2^-46 (al xl dropped),
// the sum's rounding error and the product's low part gathered in sl
// (renormalised once, at the end)
__device__ __forceinline__ void df_acc(float ah, float al, float xh, float xl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, xh);
  float e = __fmaf_rn(ah, xh, -p);
  e = __fmaf_rn(ah, xl, e);
  e = __fmaf_rn(al, xh, e);
  const float t = __fadd_rn(sh, p);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}
// (h0 + l0) + (h1 + l1) as a double
__device__ __forceinline__ double df_join(float h0, float l0, float h1, float l1) {
  const float t = __fadd_rn(h0, h1);
  const float bp = __fsub_rn(t, h0);
  const float err = __fadd_rn(__fsub_rn(h0, __fsub_rn(t, bp)), __fsub_rn(h1, bp));
  return (double)t + (double)__fadd_rn(__fadd_rn(l0, l1), err);
}

// ---------------------------------------------------------------------------
// stage sweep over the bulk-copy ring
// ---------------------------------------------------------------------------
__device__ __forceinline__ void wissue(WCtx& C, int n, int b, const unsigned char* dbase, int delem,
                                       const unsigned char* fbase, int felem) {
  const StageDesc& s = C.st[n];
  if (C.lane == 0) {
    const uint32_t dbytes = (uint32_t)(wlay(s).size * delem);
    const uint32_t fbytes = felem ? (uint32_t)(fac_block_elems(s.nx + s.nu) * felem) : 0u;
    fence_async_shared();
    mbar_arrive_expect_tx(&C.bar[b], dbytes + fbytes);
    bulk_g2s((C.ring0 + b * C.slot), dbase + s.data * delem, dbytes, &C.bar[b]);
    if (fbytes) bulk_g2s(C.ring0 + b * C.slot + C.fac_off, fbase + s.fac * 8, fbytes, &C.bar[b]);
  }
}

// f(n, data block, factor block) for every stage, forward or backward
template <class F>
__device__ void wsweep(WCtx& C, bool backward, const void* dbase, int delem, const void* fbase, int felem, F f) {
  const unsigned char* db = static_cast<const unsigned char*>(dbase);
  const unsigned char* fb = static_cast<const unsigned char*>(fbase);
  const int N = C.N;
  wissue(C, backward ? N : 0, 0, db, delem, fb, felem);
  for (int k = 0; k <= N; ++k) {
    const int n = backward ? N - k : k, b = k & 1;
    if (k < N) wissue(C, backward ? n - 1 : n + 1, b ^ 1, db, delem, fb, felem);
    // once a copy is lost the QP's results are void: stop waiting
    const bool ok = C.ok && mbar_wait(&C.bar[b], (C.parity >> b) & 1u);
    C.parity ^= 1u << b;
    C.ok = C.ok && ok;
    f(n, static_cast<const void*>((C.ring0 + b * C.slot)), static_cast<const void*>(C.ring0 + b * C.slot + C.fac_off));
    __syncwarp();
  }
}

// f(n, hi block, lo block) for every stage, forward: the FP32 mirror and its
// remainder of each stage's data block, one after the other in a ring slot
// (a slot holds an FP64 block, the same bytes)
template <class F>
__device__ void wsweep_df(WCtx& C, F f) {
  const Batch& B = *C.B;
  const int N = C.N;
  auto issue = [&](int n, int b) {
    const StageDesc& s = C.st[n];
    if (C.lane == 0) {
      const uint32_t bytes = (uint32_t)(wlay(s).size * 4);
      fence_async_shared();
      mbar_arrive_expect_tx(&C.bar[b], 2 * bytes);
      bulk_g2s(C.ring0 + b * C.slot, B.data32 + s.data, bytes, &C.bar[b]);
      bulk_g2s(C.ring0 + b * C.slot + bytes, B.data32lo + s.data, bytes, &C.bar[b]);
    }
  };
  issue(0, 0);
  for (int n = 0; n <= N; ++n) {
    const int b = n & 1;
    if (n < N) issue(n + 1, b ^ 1);
    const bool ok = C.ok && mbar_wait(&C.bar[b], (C.parity >> b) & 1u);
    C.parity ^= 1u << b;
    C.ok = C.ok && ok;
    const float* hi = reinterpret_cast<const float*>(C.ring0 + b * C.slot);
    f(n, hi, hi + wlay(C.st[n]).size);
    __syncwarp();
  }
}

// value of general constraint g (row of [D C]) at the stage vector held one
// element per lane
template <typename T>
__device__ __forceinline__ double gen_value(const WCtx& C, const T* D, const StageData& L, int nv, int g,
                                            double yl) {
  const double part = C.lane < nv ? (double)D[L.DC + (int64_t)g * nv + C.lane] * yl : 0.0;
  return warp_sum(part);
}

// ---------------------------------------------------------------------------
// a1: residuals of eq. (delta) for one stage, FP64 (lin: refinement residual)
// ---------------------------------------------------------------------------
struct WMax {
  double g, b, d;
};

__device__ __forceinline__ void wres_stage(WCtx& C, int n, const double* D, const double* y, const double* pi, const double* lam,
                           const double* t, double* og, double* ob, double* rd, bool lin, const double* add_g,
                           const double* add_b, WMax& mx) {
  const Batch& B = *C.B;
  const int lane = C.lane;
  const StageDesc s = C.st[n];
  const StageData L = wlay(s);
  const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
  const int32_t* bidx = reinterpret_cast<const int32_t*>(D + L.box);
  const int32_t* bmap = bidx + nb;
  const double yl = lane < nv ? y[s.var + lane] : 0.0;
  const double pl = (n < C.N && lane < nx1) ? pi[s.eq + lane] : 0.0;
  const double* lm = lam + s.side;
  // the other global terms of rows r_g and r_b, loaded before the mat-vecs
  // (their loads would otherwise wait behind the broadcast barriers)
  const double g0 = lane < nv ? (lin ? add_g[s.var + lane] : D[L.rq + lane]) : 0.0;
  const double pprev = (n > 0 && lane >= s.nu && lane < nv) ? pi[C.st[n - 1].eq + (lane - s.nu)] : 0.0;
  const int cbox = (nb > 0 && lane < nv) ? bmap[lane] : -1;
  const double lbox = cbox >= 0 ? lm[cbox] - lm[nc + cbox] : 0.0;
  const bool brow = n < C.N && lane < nx1;
  const double b0 = brow ? (lin ? add_b[s.eq + lane] : D[L.b + lane]) : 0.0;
  const double x1 = brow ? y[C.st[n + 1].var + C.st[n + 1].nu + lane] : 0.0;
  const bool side0 = rd != nullptr && lane < nc;
  const double tl0 = side0 ? t[s.side + lane] : 0.0, tu0 = side0 ? t[s.side + nc + lane] : 0.0;
  const double* yv = wbcast<double>(C, 0, yl);
  // r_g, row `lane`
  {
    const double* row = D + L.RSQ + (int64_t)(lane < nv ? lane : 0) * L.ldr;
    double a0 = 0.0, a1 = 0.0;
    int j = 0;
#pragma unroll 4
    for (; j + 1 < nv; j += 2) {
      a0 = fma(row[j], yv[j], a0);
      a1 = fma(row[j + 1], yv[j + 1], a1);
    }
    if (j < nv) a0 = fma(row[j], yv[j], a0);
    if (n < C.N) {
      const double* pv = wbcast<double>(C, 1, pl);
      const double* ba = D + L.BAt + (int64_t)(lane < nv ? lane : 0) * L.ldb;
      int k = 0;
#pragma unroll 4
      for (; k + 1 < nx1; k += 2) {
        a0 = fma(ba[k], pv[k], a0);
        a1 = fma(ba[k + 1], pv[k + 1], a1);
      }
      if (k < nx1) a0 = fma(ba[k], pv[k], a0);
    }
    if (lane < nv) {
      double acc = g0 + (a0 + a1);
      if (n > 0 && lane >= s.nu) acc -= pprev;
      for (int g = 0; g < s.ng; ++g) acc = fma(-D[L.DC + (int64_t)g * nv + lane], lm[nb + g] - lm[nc + nb + g], acc);
      if (cbox >= 0) acc -= lbox;
      og[s.var + lane] = acc;
      mx.g = max_abs_bits(mx.g, acc);
    }
  }
  // r_b, row `lane`
  if (n < C.N) {
    double a0 = 0.0, a1 = 0.0;
    const int kk = lane < nx1 ? lane : 0;
    int i = 0;
#pragma unroll 4
    for (; i + 1 < nv; i += 2) {
      a0 = fma(D[L.BAt + (int64_t)i * L.ldb + kk], yv[i], a0);
      a1 = fma(D[L.BAt + (int64_t)(i + 1) * L.ldb + kk], yv[i + 1], a1);
    }
    if (i < nv) a0 = fma(D[L.BAt + (int64_t)i * L.ldb + kk], yv[i], a0);
    if (lane < nx1) {
      const double acc = b0 + (a0 + a1) - x1;
      ob[s.eq + lane] = acc;
      mx.b = max_abs_bits(mx.b, acc);
    }
  }
  // r_d per side
  if (rd != nullptr) {
    for (int g = 0; g < s.ng; ++g) {
      const double v = gen_value<double>(C, D, L, nv, g, yl);
      if (lane == 0) C.sv[g] = v;
    }
    __syncwarp();
    for (int c0 = 0; c0 < nc; c0 += 32) {
      const int c = c0 + lane;
      const int src = (c < nb) ? bidx[c] : 0;
      const double yb = yv[src];
      if (c < nc) {
        const double v = c < nb ? yb : C.sv[c - nb];
        const double lo = D[L.lo + c], hi = D[L.hi + c];
        const int il = s.side + c, iu = s.side + nc + c;
        double a = 0.0, bb = 0.0;
        if (lo_on(lo)) a = lo - v + (c0 == 0 ? tl0 : t[il]);
        if (hi_on(hi)) bb = v - hi + (c0 == 0 ? tu0 : t[iu]);
        rd[il] = a;
        rd[iu] = bb;
        mx.d = max_abs_bits(max_abs_bits(mx.d, a), bb);
      }
    }
    __syncwarp();
  }
  (void)B;
}

// sum over lanes < nv of (Dh + Dl)[k0 + lane] (yh + ylo) in double-float, by
// a butterfly whose two-sum errors are exact, so every lane ends with the
// same bits
__device__ __forceinline__ double gen_value_df(const float* Dh, const float* Dl, int64_t k0, int nv, int lane,
                                               float yh, float ylo) {
  float h = 0.0f, l = 0.0f;
  if (lane < nv) {
    const float ah = Dh[k0 + lane], al = Dl[k0 + lane];
    h = __fmul_rn(ah, yh);
    l = __fmaf_rn(ah, yh, -h);
    l = __fmaf_rn(ah, ylo, l);
    l = __fmaf_rn(al, yh, l);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(kFull, h, o), l2 = __shfl_xor_sync(kFull, l, o);
    const float t = __fadd_rn(h, h2);
    const float bp = __fsub_rn(t, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(h2, bp));
    h = t;
    l = __fadd_rn(__fadd_rn(l, l2), err);
  }
  return (double)h + (double)l;
}

// the residuals of eq. (delta) for one stage (wres_stage) with the mat-vecs
// in double-float from the FP32 data mirror and its remainder, two
// independent chains per row; the other terms in FP64.  kFull: the iterate's
// residual, r_d included (the linear terms, bounds and general rows read
// from the FP64 data block in global memory); else the refinement residual
// of a direction (r_g and r_b rows, add_g and add_b in place of q and b).
template <bool kFull>
__device__ __forceinline__ void wres_stage_df(WCtx& C, int n, const float* Dh, const float* Dl, const double* y,
                                              const double* pi, const double* lam, const double* t, double* og,
                                              double* ob, double* rd, const double* add_g, const double* add_b,
                                              WMax& mx) {
  const int lane = C.lane;
  const StageDesc s = C.st[n];
  const StageData L = wlay(s);
  const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
  const int32_t* bidx = reinterpret_cast<const int32_t*>(Dh + L.box);
  const int32_t* bmap = bidx + nb;
  const double* D64 = C.B->data + s.data;
  const double* lm = lam + s.side;
  // global loads of the stage, issued before the mat-vecs
  const double yl = lane < nv ? y[s.var + lane] : 0.0;
  const double pl = (n < C.N && lane < nx1) ? pi[s.eq + lane] : 0.0;
  const double g0 = lane < nv ? (kFull ? D64[L.rq + lane] : add_g[s.var + lane]) : 0.0;
  const double pprev = (n > 0 && lane >= s.nu && lane < nv) ? pi[C.st[n - 1].eq + (lane - s.nu)] : 0.0;
  const int cbox = (nb > 0 && lane < nv) ? bmap[lane] : -1;
  const double lbox = cbox >= 0 ? lm[cbox] - lm[nc + cbox] : 0.0;
  const bool brow = n < C.N && lane < nx1;
  const double b0 = brow ? (kFull ? D64[L.b + lane] : add_b[s.eq + lane]) : 0.0;
  const double x1 = brow ? y[C.st[n + 1].var + C.st[n + 1].nu + lane] : 0.0;
  const bool side0 = kFull && lane < nc;
  const double tl0 = side0 ? t[s.side + lane] : 0.0, tu0 = side0 ? t[s.side + nc + lane] : 0.0;
  const double lo0 = side0 ? D64[L.lo + lane] : 0.0, hi0 = side0 ? D64[L.hi + lane] : 0.0;
  float yh, ylo, ph, plo;
  df_split(yl, yh, ylo);
  df_split(pl, ph, plo);
  // y_n and pi_n, high and low parts, readable by every lane
  float* xb = reinterpret_cast<float*>(C.xb);
  __syncwarp();
  xb[lane] = yh;
  xb[32 + lane] = ylo;
  xb[64 + lane] = ph;
  xb[96 + lane] = plo;
  __syncwarp();
  // r_g, row `lane`
  {
    const int64_t r = lane < nv ? lane : 0;
    const float* rh = Dh + L.RSQ + r * L.ldr;
    const float* rl = Dl + L.RSQ + r * L.ldr;
    float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
    int j = 0;
#pragma unroll 2
    for (; j + 1 < nv; j += 2) {
      df_acc(rh[j], rl[j], xb[j], xb[32 + j], h0, l0);
      df_acc(rh[j + 1], rl[j + 1], xb[j + 1], xb[33 + j], h1, l1);
    }
    if (j < nv) df_acc(rh[j], rl[j], xb[j], xb[32 + j], h0, l0);
    if (n < C.N) {
      const float* bh = Dh + L.BAt + r * L.ldb;
      const float* bl = Dl + L.BAt + r * L.ldb;
      int k = 0;
#pragma unroll 2
      for (; k + 1 < nx1; k += 2) {
        df_acc(bh[k], bl[k], xb[64 + k], xb[96 + k], h0, l0);
        df_acc(bh[k + 1], bl[k + 1], xb[65 + k], xb[97 + k], h1, l1);
      }
      if (k < nx1) df_acc(bh[k], bl[k], xb[64 + k], xb[96 + k], h0, l0);
    }
    if (lane < nv) {
      double acc = g0 + df_join(h0, l0, h1, l1);
      if (n > 0 && lane >= s.nu) acc -= pprev;
      for (int g = 0; g < s.ng; ++g) acc = fma(-D64[L.DC + (int64_t)g * nv + lane], lm[nb + g] - lm[nc + nb + g], acc);
      if (cbox >= 0) acc -= lbox;
      og[s.var + lane] = acc;
      mx.g = max_abs_bits(mx.g, acc);
    }
  }
  // r_b, row `lane`
  if (n < C.N) {
    const int kk = lane < nx1 ? lane : 0;
    float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
    int i = 0;
#pragma unroll 2
    for (; i + 1 < nv; i += 2) {
      const int64_t k = L.BAt + (int64_t)i * L.ldb + kk;
      df_acc(Dh[k], Dl[k], xb[i], xb[32 + i], h0, l0);
      df_acc(Dh[k + L.ldb], Dl[k + L.ldb], xb[i + 1], xb[33 + i], h1, l1);
    }
    if (i < nv) {
      const int64_t k = L.BAt + (int64_t)i * L.ldb + kk;
      df_acc(Dh[k], Dl[k], xb[i], xb[32 + i], h0, l0);
    }
    if (lane < nx1) {
      const double acc = b0 + df_join(h0, l0, h1, l1) - x1;
      ob[s.eq + lane] = acc;
      mx.b = max_abs_bits(mx.b, acc);
    }
  }
  // r_d per side
  if constexpr (kFull) {
    for (int g = 0; g < s.ng; ++g) {
      const double v = gen_value_df(Dh, Dl, L.DC + (int64_t)g * nv, nv, lane, yh, ylo);
      if (lane == 0) C.sv[g] = v;
    }
    __syncwarp();
    for (int c0 = 0; c0 < nc; c0 += 32) {
      const int c = c0 + lane;
      const int src = (c < nb) ? bidx[c] : 0;
      const double yb = __shfl_sync(dev::kFull, yl, src);
      if (c < nc) {
        const double v = c < nb ? yb : C.sv[c - nb];
        const bool first = c0 == 0;
        const double lo = first ? lo0 : D64[L.lo + c], hi = first ? hi0 : D64[L.hi + c];
        const int il = s.side + c, iu = s.side + nc + c;
        double a = 0.0, bb = 0.0;
        if (lo_on(lo)) a = lo - v + (first ? tl0 : t[il]);
        if (hi_on(hi)) bb = v - hi + (first ? tu0 : t[iu]);
        rd[il] = a;
        rd[iu] = bb;
        mx.d = max_abs_bits(max_abs_bits(mx.d, a), bb);
      }
    }
    __syncwarp();
  }
}

struct WNorms {
  double g, b, d, mu;
};

// the iterate's residuals; with T = float (the mixed path) the mat-vecs in
// double-float
template <typename T>
__device__ WNorms wresiduals(WCtx& C) {
  const Batch& B = *C.B;
  WMax mx{0.0, 0.0, 0.0};
  if constexpr (sizeof(T) == 4) {
    wsweep_df(C, [&](int n, const float* Dh, const float* Dl) {
      wres_stage_df<true>(C, n, Dh, Dl, B.y, B.pi, B.lam, B.t, B.rg, B.rb, B.rd, nullptr, nullptr, mx);
    });
  } else {
    wsweep(C, false, B.data, 8, nullptr, 0, [&](int n, const void* Dv, const void*) {
      wres_stage(C, n, static_cast<const double*>(Dv), B.y, B.pi, B.lam, B.t, B.rg, B.rb, B.rd, false, nullptr,
                 nullptr, mx);
    });
  }
  WNorms r;
  r.g = warp_max(mx.g);
  r.b = warp_max(mx.b);
  r.d = warp_max(mx.d);
  const double s = side_sum(C, [&](int i) { return B.lam[i] * B.t[i]; });
  r.mu = C.nact ? s / C.nact : 0.0;
  return r;
}

// ---------------------------------------------------------------------------
// Warp-level tensor-core products for the FP32 factor: mma.sync m16n8k8 with
// TF32 operands and FP32 accumulation, each FP32 operand split into a TF32
// high part and a TF32 remainder ("3xTF32": hi*hi + hi*lo + lo*hi), which
// keeps the products at FP32 accuracy.  A stage product is at most 32 x 32
// with k <= 32 here, a handful of 16 x 8 tiles per warp; the CTA-wide tcgen05
// path needs M >= 64 tiles from shared-memory descriptors and does not fit a
// warp that owns one QP.
// Fragment layout (PTX ISA, mma.m16n8k8, .tf32): with g = lane / 4 and
// q = lane % 4, A holds (g, q), (g + 8, q), (g, q + 4), (g + 8, q + 4); B holds
// (k = q, n = g), (k = q + 4, n = g); C holds (g, 2q), (g, 2q + 1), (g + 8, 2q),
// (g + 8, 2q + 1).
// ---------------------------------------------------------------------------
// (tf32_split, mma_tf32 and mma3_tile live in gq_mma.h)

// ---------------------------------------------------------------------------
// a3: square-root Riccati factorisation of one stage, lane i <-> row i.
// Compact loops over shared-memory matrices (odd stride, conflict-free): the
// code stays small enough for the instruction cache, which a fully unrolled
// register version does not.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ bool wfactor_stage(WCtx& C, int n, const T* D, double reg) {
  const Batch& B = *C.B;
  const int lane = C.lane;
  const StageDesc s = C.st[n];
  const StageData L = wlay(s);
  const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
  const int ne = welim(s, n), nk = nv - ne;
  T* sL = static_cast<T*>(C.sL);  // L_{n+1}
  T* sM = static_cast<T*>(C.sM);  // M rows, later X = L_ee^{-1}
  T* sP = static_cast<T*>(C.sP);  // Phi, factorised in place
  T* sw = reinterpret_cast<T*>(C.sv);
  const int32_t* bmap = reinterpret_cast<const int32_t*>(D + L.box) + nb;
  const bool act = lane < nv;
  const int i = act ? lane : 0;
  // barrier weights W_lo + W_hi per constraint; the first 32 are loaded here
  // and stored after the products, so that their global loads overlap them
  auto weight = [&](int c) {
    double w = 0.0;
    if (D[L.lo + c] != -INFINITY) w += B.lam[s.side + c] * B.tinv[s.side + c];
    if (D[L.hi + c] != INFINITY) w += B.lam[s.side + nc + c] * B.tinv[s.side + nc + c];
    return w;
  };
  const double w0 = lane < nc ? weight(lane) : 0.0;
  constexpr bool kMma = sizeof(T) == 4;
  // M row i: M[i][j] = sum_{k >= j} [B A]'[i][k] L_{n+1}[k][j]
  if constexpr (kMma) {
    if (n < C.N) {
    // tensor-core tiles: rows of [B A]' by columns of L_{n+1} (lower
    // triangular, so k-steps left of the diagonal block are skipped)
    const float* ba = reinterpret_cast<const float*>(D) + L.BAt;
    const float* lf = reinterpret_cast<const float*>(sL);
    const int ldb = L.ldb;
    const int g = lane >> 2, q = lane & 3;
    for (int mt = 0; mt * 16 < nv; ++mt) {
      for (int nt = 0; nt * 8 < nx1; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kt = nt; kt * 8 < nx1; ++kt) {
          mma3_tile(
              c, lane,
              [&](int r, int k) {
                const int ii = mt * 16 + r, kk = kt * 8 + k;
                return (ii < nv && kk < nx1) ? ba[ii * ldb + kk] : 0.f;
              },
              [&](int k, int j) {
                const int kk = kt * 8 + k, jj = nt * 8 + j;
                return (kk < nx1 && jj < nx1) ? lf[kk * LDS + jj] : 0.f;
              });
        }
        float* mf = reinterpret_cast<float*>(sM);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int ii = mt * 16 + g + (e >> 1) * 8, jj = nt * 8 + 2 * q + (e & 1);
          if (ii < nv && jj < nx1) mf[ii * LDS + jj] = c[e];
        }
      }
    }
    }
  } else if (n < C.N && act) {
    const T* ba = D + L.BAt + (int64_t)i * L.ldb;
    for (int j = 0; j < nx1; ++j) {
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int k = j;
      for (; k + 3 < nx1; k += 4) {
        a0 += ba[k] * sL[k * LDS + j];
        a1 += ba[k + 1] * sL[(k + 1) * LDS + j];
        a2 += ba[k + 2] * sL[(k + 2) * LDS + j];
        a3 += ba[k + 3] * sL[(k + 3) * LDS + j];
      }
      for (; k < nx1; ++k) a0 += ba[k] * sL[k * LDS + j];
      sM[i * LDS + j] = (a0 + a1) + (a2 + a3);
    }
  }
  if (lane < nc) sw[lane] = (T)w0;
  for (int c = lane + 32; c < nc; c += 32) sw[c] = (T)weight(c);
  __syncwarp();
  // Phi row i (lower part): RSQ + M M' + [D C]' diag(w_g) [D C] + diagonal terms
  if constexpr (kMma) {
    // tensor-core tiles of the lower triangle: M M' over k < nx1, then the
    // general rows' [D C]' W [D C] over k < ng
    const float* mf = reinterpret_cast<const float*>(sM);
    const float* dcf = reinterpret_cast<const float*>(D) + L.DC;
    const float* rsf = reinterpret_cast<const float*>(D) + L.RSQ;
    const float* swf = reinterpret_cast<const float*>(sw);
    float* pf = reinterpret_cast<float*>(sP);
    const int ldr = L.ldr, ng = s.ng;
    const bool prod = n < C.N && !C.qr;
    const int g = lane >> 2, q = lane & 3;
    for (int mt = 0; mt * 16 < nv; ++mt) {
      for (int nt = 0; nt * 8 < nv && nt * 8 <= mt * 16 + 15; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        if (prod) {
          for (int kt = 0; kt * 8 < nx1; ++kt) {
            mma3_tile(
                c, lane,
                [&](int r, int k) {
                  const int ii = mt * 16 + r, kk = kt * 8 + k;
                  return (ii < nv && kk < nx1) ? mf[ii * LDS + kk] : 0.f;
                },
                [&](int k, int j) {
                  const int kk = kt * 8 + k, jj = nt * 8 + j;
                  return (kk < nx1 && jj < nv) ? mf[jj * LDS + kk] : 0.f;
                });
          }
        }
        for (int kt = 0; kt * 8 < ng; ++kt) {
          mma3_tile(
              c, lane,
              [&](int r, int k) {
                const int ii = mt * 16 + r, kk = kt * 8 + k;
                return (ii < nv && kk < ng) ? dcf[kk * nv + ii] * swf[nb + kk] : 0.f;
              },
              [&](int k, int j) {
                const int kk = kt * 8 + k, jj = nt * 8 + j;
                return (kk < ng && jj < nv) ? dcf[kk * nv + jj] : 0.f;
              });
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int ii = mt * 16 + g + (e >> 1) * 8, jj = nt * 8 + 2 * q + (e & 1);
          if (ii < nv && jj <= ii) pf[ii * LDS + jj] = rsf[ii * ldr + jj] + c[e];
        }
      }
    }
    __syncwarp();
    if (act) {
      T dadd = (T)reg;
      if (nb > 0 && bmap[i] >= 0) dadd += sw[bmap[i]];
      sP[i * LDS + i] += dadd;
    }
  } else if (act) {
    const T* rs = D + L.RSQ + (int64_t)i * L.ldr;
    const T* mi = sM + i * LDS;
    const bool prod = n < C.N && !C.qr;
    for (int j = 0; j <= i; ++j) {
      const T* mj = sM + j * LDS;
      T a0 = rs[j], a1 = T(0), a2 = T(0), a3 = T(0);
      if (prod) {
        int k = 0;
        for (; k + 3 < nx1; k += 4) {
          a0 += mi[k] * mj[k];
          a1 += mi[k + 1] * mj[k + 1];
          a2 += mi[k + 2] * mj[k + 2];
          a3 += mi[k + 3] * mj[k + 3];
        }
        for (; k < nx1; ++k) a0 += mi[k] * mj[k];
      }
      a0 = (a0 + a1) + (a2 + a3);
      a1 = T(0);
      for (int g = 0; g < s.ng; ++g) {
        const T* dc = D + L.DC + (int64_t)g * nv;
        a1 += dc[i] * sw[nb + g] * dc[j];
      }
      sP[i * LDS + j] = a0 + a1;
    }
    T dadd = (T)reg;
    if (nb > 0 && bmap[i] >= 0) dadd += sw[bmap[i]];
    sP[i * LDS + i] += dadd;
  }
  __syncwarp();
  // left-looking Cholesky in place: column k from the finished columns < k
  bool ok = true;
  for (int k = 0; k < nv; ++k) {
    T sk = T(0);
    if (act && i >= k) {
      const T* pi_ = sP + i * LDS;
      const T* pk = sP + k * LDS;
      T a0 = pi_[k], a1 = T(0), a2 = T(0), a3 = T(0);
      int p = 0;
      for (; p + 3 < k; p += 4) {
        a0 -= pi_[p] * pk[p];
        a1 -= pi_[p + 1] * pk[p + 1];
        a2 -= pi_[p + 2] * pk[p + 2];
        a3 -= pi_[p + 3] * pk[p + 3];
      }
      for (; p < k; ++p) a0 -= pi_[p] * pk[p];
      sk = (a0 + a1) + (a2 + a3);
    }
    const T d = __shfl_sync(kFull, sk, k);
    const bool good = d > T(0);
    ok = ok && good;
    const T r = good ? wrsqrt<T>(d) : T(1);
    if (act && i >= k) sP[i * LDS + k] = sk * r;  // i == k: d / sqrt(d)
    __syncwarp();
  }
  if (C.qr && n < C.N) {
    // array algorithm (Sec. 4.2): sP holds Lh = chol(Ht) and sM the rows of
    // M; the factor of Ht + M M' is the transposed R of the QR factorisation
    // of [Lh'; M'].  Reflector j zeroes column j of M' (row j of sM) against
    // the pivot Lh[j][j] and acts on row j of Lh' and on M' only; lane c > j
    // applies it to its own column (row c of Lh and of sM).
    for (int j = 0; j < nv; ++j) {
      const T* mj = sM + j * LDS;
      const T alpha = sP[j * LDS + j];
      T ss = T(0);
      for (int k = 0; k < nx1; ++k) ss += mj[k] * mj[k];
      const T sigma = sqrt(alpha * alpha + ss);
      const T u0 = -ss / (alpha + sigma);  // alpha - sigma without cancellation
      const T utu = u0 * u0 + ss;
      const T beta = utu > T(0) ? T(2) / utu : T(0);
      __syncwarp();
      if (act && i > j) {
        T* mi = sM + i * LDS;
        T wv = u0 * sP[i * LDS + j];
        for (int k = 0; k < nx1; ++k) wv += mj[k] * mi[k];
        const T bw = beta * wv;
        sP[i * LDS + j] -= bw * u0;
        for (int k = 0; k < nx1; ++k) mi[k] -= bw * mj[k];
      }
      if (lane == j) sP[j * LDS + j] = sigma;
      __syncwarp();
    }
  }
  // X = L_ee^{-1}: lane j computes column j (entries i >= j) into sM
  if (lane < ne) {
    const int j = lane;
    for (int r = j; r < ne; ++r) {
      T acc = (r == j) ? T(1) : T(0);
      for (int k = j; k < r; ++k) acc -= sP[r * LDS + k] * sM[k * LDS + j];
      sM[r * LDS + j] = acc / sP[r * LDS + r];
    }
  }
  __syncwarp();
  // store the factor block (ld odd_ld(nv)): X in the leading block, L elsewhere;
  // keep L_n = L_kk in sL
  T* F = reinterpret_cast<T*>(static_cast<double*>(B.fac) + s.fac);
  const int ldf = odd_ld(nv);
  for (int r = 0; r < nv; ++r) {
    if (act) {
      T v = T(0);
      if (lane <= r) v = (r < ne) ? sM[r * LDS + lane] : sP[r * LDS + lane];
      F[(int64_t)r * ldf + lane] = v;
    }
  }
  for (int a = 0; a < nk; ++a)
    if (lane < nk) sL[a * LDS + lane] = lane <= a ? sP[(ne + a) * LDS + ne + lane] : T(0);
  __syncwarp();
  return ok;
}

template <typename T>
__device__ bool wfactor(WCtx& C, double reg) {
  const Batch& B = *C.B;
  bool ok = true;
  const void* dbase = sizeof(T) == 8 ? static_cast<const void*>(B.data) : static_cast<const void*>(B.data32);
  wsweep(C, true, dbase, (int)sizeof(T), nullptr, 0, [&](int n, const void* Dv, const void*) {
    ok = wfactor_stage<T>(C, n, static_cast<const T*>(Dv), reg) && ok;
  });
  fence_async_global();
  __syncwarp();
  return ok;
}

// ---------------------------------------------------------------------------
// a2 + a4: Riccati solve of eq. (delta) (reduced gradient per stage), then
// dt, dlam recovered in FP64.  Returns ||(gt, r_b)||inf.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double wsolve(WCtx& C, const double* g, const double* rd, const double* rm, const double* rb, double* dy,
                         double* dpi, double* dlam, double* dt) {
  const Batch& B = *C.B;
  const int lane = C.lane;
  T* sL = static_cast<T*>(C.sL);
  // l and p of each stage, from the backward sweep to the forward one, kept
  // in the factor's precision (the FP64 workspace vector holds them)
  T* lp = reinterpret_cast<T*>(B.lp);
  const void* dbase = sizeof(T) == 8 ? static_cast<const void*>(B.data) : static_cast<const void*>(B.data32);
  double scale = 0.0;
  T p1 = T(0);  // p_{n+1}, element `lane`
  wsweep(C, true, dbase, (int)sizeof(T), B.fac, (int)sizeof(T), [&](int n, const void* Dv, const void* Fv) {
    const T* D = static_cast<const T*>(Dv);
    const T* F = static_cast<const T*>(Fv);
    const StageDesc s = C.st[n];
    const StageData L = wlay(s);
    const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
    const int ne = welim(s, n), nk = nv - ne;
    const int ldf = odd_ld(nv);
    const int32_t* bmap = reinterpret_cast<const int32_t*>(D + L.box) + nb;
    // global loads of this stage's rows, issued before the per-side pass
    const double g0 = lane < nv ? g[s.var + lane] : 0.0;
    const double rb0 = (n < C.N && lane < nx1) ? rb[s.eq + lane] : 0.0;
    // per-constraint v_lo - v_hi, v = (lambda r_d - r_m) / t
    if (rd != nullptr) {
      for (int c0 = 0; c0 < nc; c0 += 32) {
        const int c = c0 + lane;
        if (c < nc) {
          const int il = s.side + c, iu = s.side + nc + c;
          double v = 0.0;
          if (D[L.lo + c] != (T)-INFINITY) v += (B.lam[il] * rd[il] - rm[il]) * B.tinv[il];
          if (D[L.hi + c] != (T)INFINITY) v -= (B.lam[iu] * rd[iu] - rm[iu]) * B.tinv[iu];
          C.sv[c] = v;
        }
      }
      __syncwarp();
    }
    // reduced gradient element `lane`
    double gi = 0.0;
    if (lane < nv) {
      gi = g0;
      if (rd != nullptr) {
        for (int gg = 0; gg < s.ng; ++gg) gi = fma(-(double)D[L.DC + (int64_t)gg * nv + lane], C.sv[nb + gg], gi);
        if (nb > 0 && bmap[lane] >= 0) gi -= C.sv[bmap[lane]];
      }
      scale = max_abs_bits(scale, gi);
    }
    T vb = T(0);
    if (n < C.N) {
      const double rbd = rb0;
      scale = max_abs_bits(scale, rbd);
      const T rbl = (T)rbd;
      // va = L_{n+1}' rb
      const T* rbv = wbcast<T>(C, 0, rbl);
      T va = T(0);
      #pragma unroll 4
      for (int j = 0; j < nx1; ++j) {
        if (j >= lane) va += sL[j * LDS + (lane < nx1 ? lane : 0)] * rbv[j];
      }
      // vb = L_{n+1} va + p_{n+1}
      const T* vav = wbcast<T>(C, 1, va);
      vb = p1;
      #pragma unroll 4
      for (int j = 0; j < nx1; ++j) {
        if (j <= lane && lane < nx1) vb += sL[lane * LDS + j] * vav[j];
      }
    }
    // phi = gt + [B A]' vb
    T phi = (T)gi;
    if (n < C.N) {
      const T* vbv = wbcast<T>(C, 0, vb);
      const T* ba = D + L.BAt + (int64_t)(lane < nv ? lane : 0) * L.ldb;
      T ph2 = T(0);
      int k = 0;
#pragma unroll 4
      for (; k + 1 < nx1; k += 2) {
        phi += ba[k] * vbv[k];
        ph2 += ba[k + 1] * vbv[k + 1];
      }
      if (k < nx1) phi += ba[k] * vbv[k];
      phi += ph2;
    }
    // l = X phi_e (lanes < ne)
    const T* phv = wbcast<T>(C, 1, phi);
    T l = T(0);
    {
      const T* xr = F + (int64_t)(lane < ne ? lane : 0) * ldf;
      #pragma unroll 4
      for (int j = 0; j < ne; ++j) {
        if (j <= lane) l += xr[j] * phv[j];
      }
    }
    // p_n = phi_k - L_ke l (lanes < nk)
    T p = phv[(ne + lane) & 31];
    {
      const T* lv = wbcast<T>(C, 0, l);
      const T* lr = F + (int64_t)(lane < nk ? ne + lane : 0) * ldf;
      #pragma unroll 4
      for (int j = 0; j < ne; ++j) p -= lr[j] * lv[j];
    }
    if (lane < ne) lp[s.var + lane] = l;
    if (lane < nk) lp[s.var + ne + lane] = p;
    p1 = lane < nk ? p : T(0);
    for (int a = 0; a < nk; ++a)
      if (lane < nk) sL[a * LDS + lane] = lane <= a ? F[(int64_t)(ne + a) * ldf + ne + lane] : T(0);
    __syncwarp();
  });
  // forward sweep; x_{n+1} passes to the next stage in a register (lane k
  // holds element k), besides its store into dy
  T xn = T(0);
  wsweep(C, false, dbase, (int)sizeof(T), B.fac, (int)sizeof(T), [&](int n, const void* Dv, const void* Fv) {
    const T* D = static_cast<const T*>(Dv);
    const T* F = static_cast<const T*>(Fv);
    const StageDesc s = C.st[n];
    const StageData L = wlay(s);
    const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng, nx1 = s.nx1;
    const int ne = welim(s, n), nk = nv - ne;
    const int ldf = odd_ld(nv);
    const int32_t* bidx = reinterpret_cast<const int32_t*>(D + L.box);
    // global loads of this stage, issued before the recursion's dependent
    // steps: l and p of the backward sweep, rb, and the per-side terms of the
    // recovery for the first 32 constraints
    const T lpk = (n > 0 && lane < nk) ? lp[s.var + ne + lane] : T(0);
    const T lpe = lane < ne ? lp[s.var + lane] : T(0);
    const T rbn = (n < C.N && lane < nx1) ? (T)rb[s.eq + lane] : T(0);
    const int c0l = lane, il0 = s.side + c0l, iu0 = s.side + nc + c0l;
    const bool side0 = lane < nc;
    const double dl0 = (side0 && rd) ? rd[il0] : 0.0, du0 = (side0 && rd) ? rd[iu0] : 0.0;
    const double ml0 = (side0 && rm) ? rm[il0] : 0.0, mu0 = (side0 && rm) ? rm[iu0] : 0.0;
    const double la0 = side0 ? B.lam[il0] : 0.0, lb0 = side0 ? B.lam[iu0] : 0.0;
    const double ta0 = side0 ? B.tinv[il0] : 0.0, tb0 = side0 ? B.tinv[iu0] : 0.0;
    // x_n (lanes ne..nv-1 of the stage vector), from the previous stage
    const T xsh = __shfl_sync(kFull, xn, (lane - ne) & 31);
    const bool xlane = lane >= ne && lane < nv;
    const double xd = xlane ? (double)xsh : 0.0;
    const T xl = xlane ? xsh : T(0);  // (T)xd, without the conversion
    const T* xv = wbcast<T>(C, 0, xl);
    if (n > 0) {
      // pi_n = L_n (L_n' x_n) + p_n, L_n = L_kk
      T w = T(0);
      #pragma unroll 4
      for (int j = 0; j < nk; ++j) {
        if (j >= lane && lane < nk) w += F[(int64_t)(ne + j) * ldf + ne + lane] * xv[ne + j];
      }
      const T* wv = wbcast<T>(C, 1, w);
      T pk = lpk;
      #pragma unroll 4
      for (int j = 0; j < nk; ++j) {
        if (j <= lane && lane < nk) pk += F[(int64_t)(ne + lane) * ldf + ne + j] * wv[j];
      }
      if (lane < nk) dpi[C.st[n - 1].eq + lane] = (double)pk;
    }
    // va = l + L_ke' x_n (lanes < ne)
    T va = lpe;
    #pragma unroll 4
    for (int i = 0; i < nk; ++i) {
      if (lane < ne) va += F[(int64_t)(ne + i) * ldf + lane] * xv[ne + i];
    }
    // u = -X' va
    const T* vav = wbcast<T>(C, 1, va);
    T u = T(0);
    #pragma unroll 4
    for (int j = 0; j < ne; ++j) {
      if (j >= lane && lane < ne) u -= F[(int64_t)j * ldf + lane] * vav[j];
    }
    const double yd = lane < ne ? (double)u : xd;
    if (lane < ne) dy[s.var + lane] = yd;
    const T yl = lane < ne ? u : xl;  // (T)yd, without the conversion
    if (n < C.N) {
      // x_{n+1} = [B A] y_n + rb_n
      const T* yv = wbcast<T>(C, 0, yl);
      T acc = rbn;
      const int kk = lane < nx1 ? lane : 0;
      T acc2 = T(0);
      int i = 0;
#pragma unroll 4
      for (; i + 1 < nv; i += 2) {
        acc += D[L.BAt + (int64_t)i * L.ldb + kk] * yv[i];
        acc2 += D[L.BAt + (int64_t)(i + 1) * L.ldb + kk] * yv[i + 1];
      }
      if (i < nv) acc += D[L.BAt + (int64_t)i * L.ldb + kk] * yv[i];
      acc += acc2;
      if (lane < nx1) dy[C.st[n + 1].var + C.st[n + 1].nu + lane] = (double)acc;
      xn = acc;
    }
    // dt = C dy - r_d, dlam = -T^{-1}(r_m + Lambda dt), FP64
    for (int gg = 0; gg < s.ng; ++gg) {
      const double v = gen_value<double>(C, B.data + s.data, L, nv, gg, yd);
      if (lane == 0) C.sv[gg] = v;
    }
    __syncwarp();
    for (int c0 = 0; c0 < nc; c0 += 32) {
      const int c = c0 + lane;
      const int src = (c < nb) ? bidx[c] : 0;
      const double yb = __shfl_sync(kFull, yd, src);
      if (c < nc) {
        const double v = c < nb ? yb : C.sv[c - nb];
        const int il = s.side + c, iu = s.side + nc + c;
        const bool first = c0 == 0;
        const double dl = first ? dl0 : (rd ? rd[il] : 0.0), du = first ? du0 : (rd ? rd[iu] : 0.0);
        const double ml = first ? ml0 : (rm ? rm[il] : 0.0), mu = first ? mu0 : (rm ? rm[iu] : 0.0);
        if (D[L.lo + c] != (T)-INFINITY) {
          const double a = v - dl;
          dt[il] = a;
          dlam[il] = -(ml + (first ? la0 : B.lam[il]) * a) * (first ? ta0 : B.tinv[il]);
        } else {
          dt[il] = 0.0;
          dlam[il] = 0.0;
        }
        if (D[L.hi + c] != (T)INFINITY) {
          const double a = -v - du;
          dt[iu] = a;
          dlam[iu] = -(mu + (first ? lb0 : B.lam[iu]) * a) * (first ? tb0 : B.tinv[iu]);
        } else {
          dt[iu] = 0.0;
          dlam[iu] = 0.0;
        }
      }
    }
    __syncwarp();
  });
  return warp_max(scale);
}

struct WDir {
  double *dy, *dpi, *dlam, *dt;
};
struct WCount {
  int ir = 0, fact = 0, fact64 = 0, solve = 0, res = 0;
  double m = 0.0;  // residual of the last refined direction (r_g, r_b rows)
};

template <typename T>
__device__ double wnewton(WCtx& C, const WDir& d, int ir, double ir_tol, WCount* cnt) {
  const Batch& B = *C.B;
  const double mr = wsolve<T>(C, B.rg, B.rd, B.rm, B.rb, d.dy, d.dpi, d.dlam, d.dt);
  ++cnt->solve;
  if (ir <= 0) return 0.0;
  double ratio = 0.0;
  for (int k = 0; k <= ir; ++k) {
    WMax mx{0.0, 0.0, 0.0};
    if constexpr (sizeof(T) == 4) {
      wsweep_df(C, [&](int n, const float* Dh, const float* Dl) {
        wres_stage_df<false>(C, n, Dh, Dl, d.dy, d.dpi, d.dlam, nullptr, B.rg2, B.rb2, nullptr, B.rg, B.rb, mx);
      });
    } else {
      wsweep(C, false, B.data, 8, nullptr, 0, [&](int n, const void* Dv, const void*) {
        wres_stage(C, n, static_cast<const double*>(Dv), d.dy, d.dpi, d.dlam, nullptr, B.rg2, B.rb2, nullptr, true,
                   B.rg, B.rb, mx);
      });
    }
    ++cnt->res;
    const double m = warp_max(max_nan(mx.g, mx.b));
    ratio = mr > 0.0 ? m / mr : 0.0;
    cnt->m = m;
    if (k == ir || m <= ir_tol * mr) break;
    wsolve<T>(C, B.rg2, nullptr, nullptr, B.rb2, B.dy2, B.dpi2, B.dlam2, B.dt2);
    #pragma unroll 4
    for (int i = C.v0 + C.lane; i < C.v1; i += 32) d.dy[i] += B.dy2[i];
    #pragma unroll 4
    for (int i = C.e0 + C.lane; i < C.e1; i += 32) d.dpi[i] += B.dpi2[i];
    #pragma unroll 4
    for (int i = C.side0 + C.lane; i < C.side0 + C.nside; i += 32) {
      d.dlam[i] += B.dlam2[i];
      d.dt[i] += B.dt2[i];
    }
    __syncwarp();
    ++cnt->ir;
    ++cnt->solve;
  }
  return ratio;
}

// largest step to the boundary: the minimum over sides of lambda / -dlambda
// and t / -dt where the direction decreases them.  Each lane keeps its
// running minimum as a fraction num / den (den > 0 once set; 1 / 0 = +inf
// stands for no blocking side) and compares candidates by cross-
// multiplication, so it divides once, for its own winner, instead of once
// per side (an FP64 division is a long sequence on the FP64 pipe).
// The sign tests read the sign bit on the integer pipe (an FP64 compare
// costs as much as an FMA here): -0 and negative NaNs pass them but then
// fail the comparison, as they fail the FP64 test.
__device__ double wmax_step(const WCtx& C, const double* dlam, const double* dt) {
  const Batch& B = *C.B;
  double num = 1.0, den = 0.0;
  #pragma unroll 4
  for (int i = C.side0 + C.lane; i < C.side0 + C.nside; i += 32) {
    const double dl = dlam[i], dd = dt[i];
    if (__double_as_longlong(dl) < 0) {
      const double a = B.lam[i];
      if (a * den < num * -dl) {
        num = a;
        den = -dl;
      }
    }
    if (__double_as_longlong(dd) < 0) {
      const double a = B.t[i];
      if (a * den < num * -dd) {
        num = a;
        den = -dd;
      }
    }
  }
  return warp_min(num / den);
}

__device__ double wmu_after(const WCtx& C, double alpha, const double* dlam, const double* dt) {
  const Batch& B = *C.B;
  const double s =
      side_sum(C, [&](int i) { return (B.lam[i] + alpha * dlam[i]) * (B.t[i] + alpha * dt[i]); });
  return C.nact ? s / C.nact : 0.0;
}

// ---------------------------------------------------------------------------
// the kernel: one warp (one block of 32 threads) per QP
// ---------------------------------------------------------------------------
// QP status while a mixed-precision solve hands over to the FP64 resume launch
constexpr int kStatusResumeFp64 = 100;

template <typename T>
// one warp per block; the register limit (in place of launch bounds, which cap
// a 32-thread kernel's registers low enough to spill) keeps the whole solver
// context in registers, and 12 blocks still fit an SM
__global__ void __maxnreg__(200) warp_ipm_kernel(const __grid_constant__ Batch B, const WarpPlan P,
                                                      const __grid_constant__ gq_ipm_arg arg, int kind,
                                                      double sigma_mu, const DirOut out, const int32_t* order,
                                                      int count, int qslot) {
  extern __shared__ __align__(128) unsigned char smem[];
  const bool resume = kind == (int)LaunchKind::Resume;
  const int lane = threadIdx.x;
  StageDesc* sst = reinterpret_cast<StageDesc*>(smem + P.stages);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P.bars);
  if (lane == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_async_shared();
  }
  WCtx C;
  C.parity = 0;  // mbarrier phases carry over from one QP to the next
  C.ok = true;
  // persistent warps: the next QP of the launch from an atomic counter over
  // `order` (longest first)
  for (;;) {
  __syncwarp();
  int idx = 0;
  if (lane == 0) idx = atomicAdd(B.queue + qslot, 1);
  idx = __shfl_sync(kFull, idx, 0);
  if (idx >= count) break;
  const int q = order[idx];
  gq_stats* stats = B.stats + q;
  if (resume && stats->status != kStatusResumeFp64) continue;  // uniform across the warp
  if (!C.ok) {
    // a lost bulk copy left this warp's ring in an unknown phase: the QPs it
    // still takes are reported as timed out instead of solved
    if (lane == 0) {
      stats->status = GQ_STATUS_TIMEOUT;
      stats->iters = 0;
    }
    continue;
  }
  const QpDesc qd = B.qp[q];
  for (int n = lane; n <= qd.N; n += 32) sst[n] = B.st[qd.stage0 + n];
  __syncwarp();

  C.B = &B;
  C.st = sst;
  C.N = qd.N;
  C.nside = qd.nsidet;
  C.side0 = qd.side0;
  C.v0 = qd.var0;
  C.v1 = qd.var0 + qd.nvt;
  C.e0 = qd.eq0;
  C.e1 = qd.eq0 + qd.neqt;
  C.lane = lane;
  C.ring0 = smem + P.ring0;
  C.slot = (uint32_t)(P.ring1 - P.ring0);
  C.bar = bars;
  C.fac_off = (uint32_t)P.fac_off;
  C.sL = smem + P.sL;
  C.sM = smem + P.sM;
  C.sP = smem + P.sP;
  C.sv = reinterpret_cast<double*>(smem + P.sv);
  C.vmax = P.vmax;
  C.qr = arg.mode == GQ_MODE_ROBUST;
  C.xb = reinterpret_cast<double*>(smem + P.xb);

  // active sides (integer count, exact)
  {
    int cnt = 0;
    wsweep(C, false, B.data, 8, nullptr, 0, [&](int n, const void* Dv, const void*) {
      const double* D = static_cast<const double*>(Dv);
      const StageDesc s = sst[n];
      const StageData L = wlay(s);
      const int nc = s.nbu + s.nbx + s.ng;
      for (int c = lane; c < nc; c += 32) cnt += (D[L.lo + c] != -INFINITY) + (D[L.hi + c] != INFINITY);
    });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    C.nact = cnt;
  }

  const bool mixed = arg.precision == GQ_PREC_MIXED;
  // 1/t on every side (masked sides: t = 1)
  auto set_tinv = [&]() {
    #pragma unroll 4
    for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32) B.tinv[i] = 1.0 / B.t[i];
    __syncwarp();
  };

  if (kind == (int)LaunchKind::Residuals) {
    const WNorms r = wresiduals<T>(C);
    if (lane == 0) {
      stats->res[0] = r.g;
      stats->res[1] = r.b;
      stats->res[2] = r.d;
      stats->res[3] = r.mu;
      if (!C.ok) stats->status = GQ_STATUS_TIMEOUT;
    }
    continue;
  }
  if (kind == (int)LaunchKind::NewtonStep) {
    wresiduals<T>(C);
    #pragma unroll 4
    for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32)
      B.rm[i] = B.lam[i] * B.t[i] - (B.lam[i] != 0.0 ? sigma_mu : 0.0);
    set_tinv();
    WDir d{out.dy, out.dpi, out.dlam, out.dt};
    WCount cnt;
    const bool ok = wfactor<T>(C, arg.reg_prim);
    wnewton<T>(C, d, arg.ir_steps, arg.ir_tol, &cnt);
    if (lane == 0) {
      stats->status = !C.ok ? GQ_STATUS_TIMEOUT : (ok ? GQ_STATUS_CONVERGED : GQ_STATUS_NAN);
      stats->ir_total = cnt.ir;
    }
    continue;
  }

  // ---------------- full IPM (Sec. 4.2) ----------------
  const int64_t t_start = arg.timeout_ns > 0 ? globaltimer() : 0;
  if (!resume) {
    const int wlev = qd.warm > 0 ? qd.warm - 1 : arg.warm_start;
    const bool warm1 = wlev >= 1, warm2 = wlev >= 2;
    if (!warm1) {
      #pragma unroll 4
      for (int i = C.v0 + lane; i < C.v1; i += 32) B.y[i] = 0.0;
      #pragma unroll 4
      for (int i = C.e0 + lane; i < C.e1; i += 32) B.pi[i] = 0.0;
    }
    __syncwarp();
    wsweep(C, false, B.data, 8, nullptr, 0, [&](int n, const void* Dv, const void*) {
      const double* D = static_cast<const double*>(Dv);
      const StageDesc s = sst[n];
      const StageData L = wlay(s);
      const int nv = s.nx + s.nu, nb = s.nbu + s.nbx, nc = nb + s.ng;
      const int32_t* bidx = reinterpret_cast<const int32_t*>(D + L.box);
      const double yl = lane < nv ? B.y[s.var + lane] : 0.0;
      for (int g = 0; g < s.ng; ++g) {
        const double v = gen_value<double>(C, D, L, nv, g, yl);
        if (lane == 0) C.sv[g] = v;
      }
      __syncwarp();
      for (int c0 = 0; c0 < nc; c0 += 32) {
        const int c = c0 + lane;
        const int src = c < nb ? bidx[c] : 0;
        const double yb = __shfl_sync(kFull, yl, src);
        if (c < nc) {
          const double v = c < nb ? yb : C.sv[c - nb];
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
      __syncwarp();
    });
  }

  // a mixed solve runs with T = float; T = double is the plain FP64 solve or
  // the FP64 continuation of mixed QPs whose refinement stagnated
  const bool fp64 = sizeof(T) == 8;
  int status = GQ_STATUS_MAX_ITER, it = 0, flags = 0;
  WCount cnt;
  if (resume) {
    it = stats->iters;
    flags = stats->flags | GQ_FLAG_FP64_FALLBACK;
    cnt.ir = stats->ir_total;
    cnt.fact = stats->n_fact;
    cnt.fact64 = stats->n_fact64;
    cnt.solve = stats->n_solve;
    cnt.res = stats->n_res;
  }
  int lifted_at = -1;  // iteration whose lambda, t were lifted after a lost FP64 pivot
  const bool pos_min = arg.lam_min > 0.0 && arg.t_min > 0.0;  // the clamps can run on the integer pipe
  double alpha = 1.0;
  WNorms r{0, 0, 0, 0};
  const WDir d{B.dy, B.dpi, B.dlam, B.dt};
  while (true) {
    r = wresiduals<T>(C);
    ++cnt.res;
    if (!C.ok) {
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
      const int64_t el = __shfl_sync(kFull, globaltimer() - t_start, 0);
      if (el > arg.timeout_ns) {
        status = GQ_STATUS_TIMEOUT;
        break;
      }
    }
    #pragma unroll 4
    for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32) {
      const double ti = B.t[i];
      B.rm[i] = B.lam[i] * ti;
      B.tinv[i] = 1.0 / ti;
    }
    __syncwarp();
    const double reg = fp64 ? (mixed ? 0.0 : arg.reg_prim) : arg.reg_prim;
    bool ok = wfactor<T>(C, reg);
    ++cnt.fact;
    cnt.fact64 += fp64;
    bool okall = __all_sync(kFull, ok);
    if (!okall && fp64 && reg < kRegRetry) {
      // an FP64 pivot lost positivity in the end game: regularise the primal
      // block (Sec. 4.2, regularisation) and factor once more
      ok = wfactor<T>(C, kRegRetry);
      ++cnt.fact;
      ++cnt.fact64;
      flags |= GQ_FLAG_REGULARIZED;
      okall = __all_sync(kFull, ok);
    }
    if (!okall && fp64 && lifted_at != it) {
      // still indefinite: complementarity ran far ahead of stationarity and
      // barrier weights lambda/t near 1/t_min swamp Phi.  Lift lambda and t
      // of active sides to a floor tied to the stationarity residual (moving
      // r_d by no more than that floor) and redo this iteration
      lifted_at = it;
      const double floor_lt = fmax(kLift, kLiftRel * fmax(r.g, r.b));
      flags |= GQ_FLAG_REGULARIZED;
      #pragma unroll 4
      for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32) {
        if (B.lam[i] != 0.0) {
          B.lam[i] = fmax(B.lam[i], floor_lt);
          B.t[i] = fmax(B.t[i], floor_lt);
        }
      }
      __syncwarp();
      continue;
    }
    if (!okall) {
      if (!fp64 && arg.fp64_fallback) {
        status = kStatusResumeFp64;
        break;
      }
      status = GQ_STATUS_NAN;
      break;
    }
    wnewton<T>(C, d, 0, 0.0, &cnt);
    const int ir = (mixed && !fp64) || arg.mode != GQ_MODE_SPEED ? arg.ir_steps : 0;
    // a refined FP32 direction must also be an inexact-Newton step for the
    // unscaled exit rule: its own residual well below the iterate's
    const double inexact = kInexact * fmax(fmax(r.g, r.b), arg.tol_stat);
    if (C.nact > 0) {
      const double a_aff = fmin(1.0, wmax_step(C, d.dlam, d.dt));
      const double mu_aff = wmu_after(C, a_aff, d.dlam, d.dt);
      const double sigma = r.mu > 0.0 ? (mu_aff / r.mu) * (mu_aff / r.mu) * (mu_aff / r.mu) : 0.0;
      const double smu = sigma * r.mu;
      #pragma unroll 4
      for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32)
        B.rm[i] = nonzero_bits(B.lam[i]) ? B.lam[i] * B.t[i] + d.dlam[i] * d.dt[i] - smu : 0.0;
      __syncwarp();
      double ratio = wnewton<T>(C, d, ir, arg.ir_tol, &cnt);
      double amax = -1.0;  // step to the boundary of the current direction, once known
      if (arg.cond_corr) {
        amax = wmax_step(C, d.dlam, d.dt);
        const double a_c = fmin(1.0, amax);
        const double mu_c = wmu_after(C, a_c, d.dlam, d.dt);
        if (mu_c > arg.corr_k * mu_aff) {
          #pragma unroll 4
          for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32)
            B.rm[i] = nonzero_bits(B.lam[i]) ? B.lam[i] * B.t[i] - smu : 0.0;
          __syncwarp();
          ratio = wnewton<T>(C, d, ir, arg.ir_tol, &cnt);
          amax = -1.0;
        }
      }
      if (ir > 0 && !(ratio <= arg.ir_fail_ratio && cnt.m <= inexact)) {
        // refinement could not make the direction accurate: the FP64 launch
        // continues this QP from the current iterate (mixed path), else, in
        // mode balance, this iteration is redone with the array algorithm
        if (!fp64 && arg.fp64_fallback) {
          status = kStatusResumeFp64;
          break;
        }
        if (arg.mode == GQ_MODE_BALANCE && !C.qr) {
          C.qr = true;
          flags |= GQ_FLAG_ARRAY_QR;
          continue;
        }
      }
      alpha = fmin(1.0, arg.tau_b * (amax >= 0.0 ? amax : wmax_step(C, d.dlam, d.dt)));
    } else {
      if (ir > 0) {
        const double ratio = wnewton<T>(C, d, ir, arg.ir_tol, &cnt);
        if (!(ratio <= arg.ir_fail_ratio && cnt.m <= inexact)) {
          if (!fp64 && arg.fp64_fallback) {
            status = kStatusResumeFp64;
            break;
          }
          if (arg.mode == GQ_MODE_BALANCE && !C.qr) {
            C.qr = true;
            flags |= GQ_FLAG_ARRAY_QR;
            continue;
          }
        }
      }
      alpha = 1.0;
    }
    #pragma unroll 4
    for (int i = C.v0 + lane; i < C.v1; i += 32) B.y[i] += alpha * d.dy[i];
    #pragma unroll 4
    for (int i = C.e0 + lane; i < C.e1; i += 32) B.pi[i] += alpha * d.dpi[i];
    if (pos_min) {
      #pragma unroll 4
      for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32) {
        if (nonzero_bits(B.lam[i]) || nonzero_bits(d.dlam[i])) {
          B.lam[i] = fmax_pos_bits(B.lam[i] + alpha * d.dlam[i], arg.lam_min);
          B.t[i] = fmax_pos_bits(B.t[i] + alpha * d.dt[i], arg.t_min);
        }
      }
    } else {
      #pragma unroll 4
      for (int i = C.side0 + lane; i < C.side0 + C.nside; i += 32) {
        if (B.lam[i] != 0.0 || d.dlam[i] != 0.0) {
          B.lam[i] = fmax(B.lam[i] + alpha * d.dlam[i], arg.lam_min);
          B.t[i] = fmax(B.t[i] + alpha * d.dt[i], arg.t_min);
        }
      }
    }
    __syncwarp();
    ++it;
  }
  if (lane == 0) {
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
  }  // next QP
}

// FP32 mirror of the stage data blocks: values rounded to FP32 (data32) and
// the FP32 rounding of what that leaves (data32lo), so that hi + lo carries a
// value to about 48 bits; box indices copied into both
__global__ void mirror_kernel(const __grid_constant__ Batch B) {
  for (int sl = blockIdx.x; sl < B.nslots; sl += gridDim.x) {
    const StageDesc s = B.st[B.slots[sl]];
    const StageData L = wlay(s);
    const double* src = B.data + s.data;
    float* dst = B.data32 + s.data;
    float* dlo = B.data32lo + s.data;
    for (int64_t i = threadIdx.x; i < L.box; i += blockDim.x) {
      const double v = src[i];
      const float h = (float)v;
      dst[i] = h;
      // v - h is exact in FP64; an infinite value (or one beyond the FP32
      // range) leaves 0
      dlo[i] = isfinite(h) ? (float)(v - (double)h) : 0.0f;
    }
    const int32_t* si = reinterpret_cast<const int32_t*>(src + L.box);
    int32_t* di = reinterpret_cast<int32_t*>(dst + L.box);
    int32_t* dli = reinterpret_cast<int32_t*>(dlo + L.box);
    for (int i = threadIdx.x; i < L.nint; i += blockDim.x) {
      di[i] = si[i];
      dli[i] = si[i];
    }
  }
}

}  // namespace

WarpPlan warp_plan(const Batch& b, const Shape& sh, int elem) {
  (void)b;
  WarpPlan p;
  size_t o = 0;
  auto take = [&](size_t bytes, size_t align) {
    o = (o + align - 1) / align * align;
    const size_t at = o;
    o += bytes;
    return at;
  };
  const size_t te = (size_t)elem;  // factor precision: 4 (mixed) or 8 (FP64)
  const int nv = sh.nvmax > 0 ? sh.nvmax : 1, nx = sh.nxmax > 0 ? sh.nxmax : 1;
  p.vmax = sh.nvmax + sh.ngmax + 2 > 32 ? sh.nvmax + sh.ngmax + 2 : 32;
  p.bars = take(2 * sizeof(uint64_t), 16);
  p.stages = take((size_t)sh.nst_max * sizeof(StageDesc), 16);
  p.sL = take((size_t)nx * LDS * te, 16);
  p.sM = take((size_t)nv * LDS * te, 16);
  p.sP = take((size_t)nv * LDS * te, 16);
  p.sv = take((size_t)p.vmax * 8, 16);
  p.xb = take(64 * sizeof(double), 16);
  // ring slot: the FP64 data block (residual sweeps), or a factor-precision
  // data block followed by a factor block (factorisation and solves)
  p.fac_off = ((size_t)sh.data_max * te + 127) / 128 * 128;
  size_t slot = p.fac_off + (size_t)fac_block_elems(sh.nvmax) * te;
  const size_t d64 = (size_t)sh.data_max * 8;
  if (slot < d64) slot = d64;
  slot = (slot + 127) / 128 * 128;
  p.ring0 = take(slot, 128);
  p.ring1 = take(slot, 128);
  p.bytes = o;
  return p;
}

template <typename T>
static cudaError_t launch_one(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                              LaunchKind kind, double sigma_mu, const DirOut& o, const int32_t* order, int count) {
  const WarpPlan P = warp_plan(b, sh, (int)sizeof(T));
  // opt in to more than the default dynamic shared memory on the current
  // device (no cache shared between host threads or devices)
  if (P.bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(warp_ipm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.bytes);
    if (e != cudaSuccess) return e;
  }
  // persistent grid: as many one-warp blocks as fit the device at once
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, warp_ipm_kernel<T>, 32, P.bytes);
  if (e != cudaSuccess) return e;
  const int64_t resident = (int64_t)(per_sm > 0 ? per_sm : 1) * (nsm > 0 ? nsm : 1);
  const int grid = (int)(count < resident ? count : resident);
  const int qslot = kind == LaunchKind::Resume ? kQueueResume : kQueueWarp;
  e = cudaMemsetAsync(b.queue + qslot, 0, sizeof(int32_t), stream);
  if (e != cudaSuccess) return e;
  warp_ipm_kernel<T><<<grid, 32, P.bytes, stream>>>(b, P, arg, (int)kind, sigma_mu, o, order, count, qslot);
  return cudaGetLastError();
}

cudaError_t launch_mirror(const Batch& b, cudaStream_t stream) {
  int grid = b.nslots < 4096 ? b.nslots : 4096;
  if (grid < 1) grid = 1;
  mirror_kernel<<<grid, 128, 0, stream>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_warp_ipm(const Batch& b, const Shape& sh, const gq_ipm_arg& arg, cudaStream_t stream,
                            LaunchKind kind, double sigma_mu, const DirOut* out, const int32_t* order, int count) {
  if (count <= 0) return cudaSuccess;
  DirOut o{};
  if (out) o = *out;
  if (arg.precision != GQ_PREC_MIXED || kind == LaunchKind::Residuals)
    return launch_one<double>(b, sh, arg, stream, kind, sigma_mu, o, order, count);
  cudaError_t e = launch_one<float>(b, sh, arg, stream, kind, sigma_mu, o, order, count);
  if (e != cudaSuccess || kind != LaunchKind::Solve || !arg.fp64_fallback) return e;
  // FP64 continuation of the QPs whose FP32 factors were not accurate enough
  return launch_one<double>(b, sh, arg, stream, LaunchKind::Resume, sigma_mu, o, order, count);
}

}  // namespace gq
