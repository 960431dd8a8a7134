// Soft constraints (Sec. 2.2): the slack variables of a stage are eliminated
// from the Newton system at linear cost, one slack at a time, and folded into
// the barrier terms of the constraint they relax.  FP64 per-slack arithmetic
// of the block kernel (QPs with slacks are scheduled there).
//
// Slack pair k of a stage relaxes constraint c = sidx[k] of the stage's list
// [box u; box x; general]: lower side  c(y) + s^l - lo >= 0  (row +1 on s^l),
// upper side  hi - c(y) + s^u >= 0  (row +1 on s^u), and has two sides of
// its own, s^l - lls >= 0 and s^u - lus >= 0, with the diagonal cost
// 1/2 Zl (s^l)^2 + zl s^l + 1/2 Zu (s^u)^2 + zu s^u.
//
// With w = lambda / t and q = (lambda r_d - r_m) / t per side, the Newton
// rows of s^l are  (Zl + w_lo + w_bl) ds^l + w_lo (a' dy) = -gt_l,
// gt_l = r_g(s^l) - q_lo - q_bl  (a the relaxed constraint's row in y), so
//   ds^l = -(gt_l + w_lo a'dy) / Dl,   Dl = Zl + w_lo + w_bl,
// and eliminating it leaves the lower side with the weight
// w_lo - w_lo^2 / Dl and the gradient term q_lo + w_lo gt_l / Dl; the upper
// side is the same with the sign of a' dy reversed.
#pragma once
#include "gq_device.h"
#include "gq_internal.h"

namespace gq {
namespace soft {
using dev::max_nan;

// int maps of a stage data block with slacks: sidx[ns] then smap[nc]
__host__ __device__ inline const int32_t* soft_sidx(const int32_t* ints, int nb, int nv) { return ints + nb + nv; }
__host__ __device__ inline const int32_t* soft_smap(const int32_t* ints, int nb, int nv, int ns) {
  return ints + nb + nv + ns;
}

// positions of slack k in the batch vectors
struct SoftSlot {
  int il, iu;  // lower / upper side of the relaxed constraint
  int jl, ju;  // sides s^l >= lls, s^u >= lus
  int rl, ru;  // rows of s^l, s^u in the var vectors (y, dy, r_g)
};
__host__ __device__ inline SoftSlot soft_slot(const StageDesc& s, int nv, int nc, int k, int c) {
  SoftSlot q;
  q.il = s.side + c;
  q.iu = s.side + nc + c;
  q.jl = s.side + 2 * nc + k;
  q.ju = q.jl + s.ns;
  q.rl = s.var + nv + k;
  q.ru = q.rl + s.ns;
  return q;
}

struct SoftElim {
  double wl, wu;  // barrier weights of the relaxed sides (0 where masked)
  double Dl, Du;  // Z + w_side + w_bound
  double gl, gu;  // reduced slack gradients gt (0 for a refinement right-hand side)
};

// Elimination terms of slack k (FP64 data block Dd).  g: the r_g vector
// holding the slack rows; rd == nullptr marks a refinement right-hand side,
// whose slack rows and side rows are met exactly by construction.
__device__ __forceinline__ SoftElim soft_elim(const double* Dd, const StageData& L, int ns, int k, const SoftSlot& q,
                                              bool lo_on, bool hi_on, const double* lam, const double* t,
                                              const double* g, const double* rd, const double* rm) {
  SoftElim e;
  e.wl = lo_on ? lam[q.il] / t[q.il] : 0.0;
  e.wu = hi_on ? lam[q.iu] / t[q.iu] : 0.0;
  e.Dl = Dd[L.Zs + k] + e.wl + lam[q.jl] / t[q.jl];
  e.Du = Dd[L.Zs + ns + k] + e.wu + lam[q.ju] / t[q.ju];
  e.gl = 0.0;
  e.gu = 0.0;
  if (rd != nullptr) {
    const double ql = lo_on ? (lam[q.il] * rd[q.il] - rm[q.il]) / t[q.il] : 0.0;
    const double qu = hi_on ? (lam[q.iu] * rd[q.iu] - rm[q.iu]) / t[q.iu] : 0.0;
    e.gl = g[q.rl] - ql - (lam[q.jl] * rd[q.jl] - rm[q.jl]) / t[q.jl];
    e.gu = g[q.ru] - qu - (lam[q.ju] * rd[q.ju] - rm[q.ju]) / t[q.ju];
  }
  return e;
}

// weight of the relaxed constraint in the reduced Hessian (both sides)
__device__ __forceinline__ double soft_weight(const SoftElim& e) {
  return (e.wl - e.wl * e.wl / e.Dl) + (e.wu - e.wu * e.wu / e.Du);
}

// addition to the constraint's reduced-gradient term q_lo - q_hi
__device__ __forceinline__ double soft_grad(const SoftElim& e) { return e.wl * e.gl / e.Dl - e.wu * e.gu / e.Du; }

// Slack steps and the steps of the four sides of slack k, given a = a'dy,
// the relaxed constraint's value on the direction: dt = row . d - r_d and
// dlam = -(r_m + lambda dt) / t on every side (masked sides keep dt = dlam = 0).
__device__ __forceinline__ void soft_recover(const SoftElim& e, const SoftSlot& q, bool lo_on, bool hi_on, double a,
                                             const double* lam, const double* t, const double* rd, const double* rm,
                                             double* dy, double* dt, double* dlam) {
  const double dsl = -(e.gl + e.wl * a) / e.Dl;
  const double dsu = -(e.gu - e.wu * a) / e.Du;
  dy[q.rl] = dsl;
  dy[q.ru] = dsu;
  auto side = [&](int i, double v) {
    const double x = v - (rd ? rd[i] : 0.0);
    dt[i] = x;
    dlam[i] = -((rm ? rm[i] : 0.0) + lam[i] * x) / t[i];
  };
  if (lo_on) side(q.il, a + dsl);
  if (hi_on) side(q.iu, -a + dsu);
  side(q.jl, dsl);
  side(q.ju, dsu);
}

// Slack parts of the residuals of slack k at (y, lam, t): the stationarity
// rows of s^l, s^u, and (rd != nullptr) the r_d of the two bound sides; the
// caller subtracts s^l, s^u from the relaxed sides' r_d (*sl, *su).  lin:
// the Newton-system residual of a direction (y = dy, lam = dlam, add_g the
// right-hand side's r_g).  Returns the largest |r_g| and |r_d| written.
__device__ __forceinline__ void soft_residual(const double* Dd, const StageData& L, int ns, int k, const SoftSlot& q,
                                              const double* y, const double* lam, const double* t, double* og,
                                              double* rd, bool lin, const double* add_g, double* sl, double* su,
                                              double* mg, double* md) {
  *sl = y[q.rl];
  *su = y[q.ru];
  const double gl = (lin ? add_g[q.rl] : Dd[L.zs + k]) + Dd[L.Zs + k] * *sl - lam[q.il] - lam[q.jl];
  const double gu = (lin ? add_g[q.ru] : Dd[L.zs + ns + k]) + Dd[L.Zs + ns + k] * *su - lam[q.iu] - lam[q.ju];
  og[q.rl] = gl;
  og[q.ru] = gu;
  *mg = max_nan(fabs(gl), fabs(gu));
  *md = 0.0;
  if (rd != nullptr) {
    const double bl = Dd[L.ls + k] - *sl + t[q.jl];
    const double bu = Dd[L.ls + ns + k] - *su + t[q.ju];
    rd[q.jl] = bl;
    rd[q.ju] = bu;
    *md = max_nan(fabs(bl), fabs(bu));
  }
}

}  // namespace soft
}  // namespace gq
