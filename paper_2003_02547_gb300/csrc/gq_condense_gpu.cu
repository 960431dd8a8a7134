// Partial (block) condensing on the device (Sec. 3.5).
//
// One thread block per condensed stage (QP q, block k of stages n0..n1,
// m = n1 - n0 + 1) reads the stage data blocks of the source batch in device
// memory and writes the condensed stage's data block of the destination batch
// in place, in the solver's own layout, so a condensed batch goes from
// uploaded source data to a solvable batch without a host round trip.  The
// arithmetic is FP64 and follows the host implementation (gq_condense.cu):
//   * forward maps x_{n0+j} = Phi_j x' + Gam_j u' + c_j of the block's states
//     in terms of x' = x_{n0} and u' = [u_{n0}; ...; u_{n1}] (the condensed
//     stage's dynamics are (Phi_m, Gam_m, c_m); state bounds inside the block
//     become general rows through the same maps);
//   * the Hessian and gradient by the backward recursion of Sec. 3.5, the
//     condensing analogue of the classical Riccati recursion, quadratic in m
//     and cubic in the state size: with the tail cost 1/2 v' W v + w' v over
//     v_j = [u_j; u_{j+1..}; x_j], W_m = 0 and W_{j+1} = [[Wuu, Wux], [Wxu, Wxx]],
//       W_j = [[R + B'Wxx B, B'Wxu, S + B'Wxx A], [., Wuu, Wux A], [., ., Q + A'Wxx A]]
//       w_j = [r + B'(Wxx b + wx); wu + Wux b; q + A'(Wxx b + wx)].
// The terminal stage is copied unchanged.  Every loop is parallel over the
// block's threads, with a barrier between dependent steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gq_batch.h"
#include "gq_internal.h"

namespace gq {
namespace {

constexpr int kCondThreads = 256;

// per-block scratch (doubles), sized on the host from the source dims
struct CondScratch {
  int64_t phi, gam, cvec, W, W2, w, w2, PB, KB, e, total;
};

__host__ __device__ inline CondScratch cond_scratch(int m, int nxmax, int nup, int nxp, int numax) {
  CondScratch c;
  const int64_t nvp = nup + nxp, nvs = numax + nxmax;
  int64_t o = 0;
  c.phi = o;
  o += (int64_t)(m + 1) * nxmax * (nxp > 0 ? nxp : 1);
  c.gam = o;
  o += (int64_t)(m + 1) * nxmax * (nup > 0 ? nup : 1);
  c.cvec = o;
  o += (int64_t)(m + 1) * nxmax;
  const int64_t wn = nup + nxmax > nvp ? nup + nxmax : nvp;  // the tail's [u; x] never exceeds this
  c.W = o;
  o += wn * wn;
  c.W2 = o;
  o += wn * wn;
  c.w = o;
  o += wn;
  c.w2 = o;
  o += wn;
  c.PB = o;
  o += (int64_t)nxmax * nvs;
  c.KB = o;
  o += (int64_t)nup * nvs;
  c.e = o;
  o += nxmax;
  c.total = (o + 31) & ~int64_t(31);
  return c;
}

struct CondArgs {
  const QpDesc* sqp;
  const StageDesc* sst;
  const double* sdata;
  const QpDesc* dqp;
  const StageDesc* dst;
  double* ddata;
  int nqp, block, n2max;   // n2max: largest condensed horizon + 1 (stages per QP)
  int m_max, nxmax, numax, nup_max, nxp_max;
  int64_t slice;           // scratch doubles per thread block
  double* ws;
};

// [B A] of source stage s: BA(k, c) for row k < nx1, column c < nu + nx
__device__ __forceinline__ double ba_at(const double* D, const StageData& L, int k, int c) {
  return D[L.BAt + (int64_t)c * L.ldb + k];
}

__global__ void __launch_bounds__(kCondThreads) condense_kernel(const CondArgs a) {
  const int tid = threadIdx.x, NT = blockDim.x;
  double* S = a.ws + (int64_t)blockIdx.x * a.slice;
  const int64_t items = (int64_t)a.nqp * a.n2max;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int q = (int)(item / a.n2max), k = (int)(item - (int64_t)q * a.n2max);
    const QpDesc sq = a.sqp[q], dq = a.dqp[q];
    const int N = sq.N, N2 = dq.N;
    if (k > N2) continue;  // uniform across the block
    const StageDesc& dsd = a.dst[dq.stage0 + k];
    const StageData DL = stage_data_layout(dsd);
    double* Dd = a.ddata + dsd.data;
    if (k == N2) {
      // terminal stage: the source block unchanged (identical sizes and layout)
      const StageDesc& ssd = a.sst[sq.stage0 + N];
      const double* Ds = a.sdata + ssd.data;
      for (int64_t e = tid; e < DL.size; e += NT) Dd[e] = Ds[e];
      continue;
    }
    const int n0 = k * a.block, n1 = min(N, (k + 1) * a.block) - 1, m = n1 - n0 + 1;
    const StageDesc* ss = a.sst + sq.stage0 + n0;
    int nup = 0;
    for (int j = 0; j < m; ++j) nup += ss[j].nu;
    const int nxp = ss[0].nx, nvp = nup + nxp;
    const CondScratch cs = cond_scratch(m, a.nxmax, nup, nxp, a.numax);
    double* Phi = S + cs.phi;  // Phi_j: nx_j x nxp, stride nxmax * nxp per j
    double* Gam = S + cs.gam;  // Gam_j: nx_j x nup
    double* cv = S + cs.cvec;  // c_j: nx_j
    const int64_t sp = (int64_t)a.nxmax * (nxp > 0 ? nxp : 1), sg = (int64_t)a.nxmax * (nup > 0 ? nup : 1);
    // ---- forward maps
    for (int e = tid; e < nxp * nxp; e += NT) Phi[e] = (e / nxp == e % nxp) ? 1.0 : 0.0;
    for (int e = tid; e < nxp * nup; e += NT) Gam[e] = 0.0;
    for (int e = tid; e < nxp; e += NT) cv[e] = 0.0;
    __syncthreads();
    int uoff = 0;
    for (int j = 0; j < m; ++j) {
      const StageDesc& s = ss[j];
      const StageData L = stage_data_layout(s);
      const double* D = a.sdata + s.data;
      const int nx = s.nx, nu = s.nu, nx1 = s.nx1;
      const double* P0 = Phi + j * sp;
      const double* G0 = Gam + j * sg;
      const double* c0 = cv + (int64_t)j * a.nxmax;
      double* P1 = Phi + (j + 1) * sp;
      double* G1 = Gam + (j + 1) * sg;
      double* c1 = cv + (int64_t)(j + 1) * a.nxmax;
      for (int e = tid; e < nx1 * (nxp + nup + 1); e += NT) {
        const int r = e / (nxp + nup + 1), c = e - r * (nxp + nup + 1);
        double v = 0.0;
        if (c < nxp) {
          for (int t = 0; t < nx; ++t) v = fma(ba_at(D, L, r, nu + t), P0[t * nxp + c], v);
          P1[r * nxp + c] = v;
        } else if (c < nxp + nup) {
          const int cu = c - nxp;
          for (int t = 0; t < nx; ++t) v = fma(ba_at(D, L, r, nu + t), G0[t * nup + cu], v);
          if (cu >= uoff && cu < uoff + nu) v += ba_at(D, L, r, cu - uoff);
          G1[r * nup + cu] = v;
        } else {
          for (int t = 0; t < nx; ++t) v = fma(ba_at(D, L, r, nu + t), c0[t], v);
          c1[r] = v + D[L.b + r];
        }
      }
      uoff += nu;
      __syncthreads();
    }
    // ---- backward recursion for the Hessian and gradient
    double* W = S + cs.W;
    double* W2 = S + cs.W2;
    double* w = S + cs.w;
    double* w2 = S + cs.w2;
    double* PB = S + cs.PB;
    double* KB = S + cs.KB;
    double* ev = S + cs.e;
    int U = 0, X = ss[m - 1].nx1;
    for (int e = tid; e < X * X; e += NT) W[e] = 0.0;
    for (int e = tid; e < X; e += NT) w[e] = 0.0;
    __syncthreads();
    for (int j = m - 1; j >= 0; --j) {
      const StageDesc& s = ss[j];
      const StageData L = stage_data_layout(s);
      const double* D = a.sdata + s.data;
      const int nu = s.nu, nx = s.nx, nx1 = s.nx1, nvj = nu + nx, n1w = U + X;
      // e = Wxx b + wx; PB = Wxx [B A]; KB = Wux [B A]
      for (int i = tid; i < nx1; i += NT) {
        double v = w[U + i];
        for (int t = 0; t < nx1; ++t) v = fma(W[(int64_t)(U + i) * n1w + U + t], D[L.b + t], v);
        ev[i] = v;
      }
      for (int e = tid; e < (nx1 + U) * nvj; e += NT) {
        const int r = e / nvj, c = e - r * nvj;
        const int row = r < nx1 ? U + r : r - nx1;  // Wxx rows, then Wux rows
        double v = 0.0;
        for (int t = 0; t < nx1; ++t) v = fma(W[(int64_t)row * n1w + U + t], ba_at(D, L, t, c), v);
        if (r < nx1)
          PB[(int64_t)r * nvj + c] = v;
        else
          KB[(int64_t)(r - nx1) * nvj + c] = v;
      }
      __syncthreads();
      // W_j over [u_j (nu); u_{j+1..} (U); x_j (nx)]
      const int U2 = nu + U, n2 = U2 + nx;
      for (int e = tid; e < n2 * n2; e += NT) {
        const int r = e / n2, c = e - r * n2;
        // position -> index into [u_j; x_j] (or -1 for the later inputs)
        const int ar = r < nu ? r : (r >= U2 ? nu + (r - U2) : -1);
        const int ac = c < nu ? c : (c >= U2 ? nu + (c - U2) : -1);
        double v;
        if (ar >= 0 && ac >= 0) {
          const double h = D[L.RSQ + (int64_t)ar * L.ldr + ac];  // [[R, S], [S', Q]]
          double t2 = 0.0;
          for (int t = 0; t < nx1; ++t) t2 = fma(ba_at(D, L, t, ar), PB[(int64_t)t * nvj + ac], t2);
          v = h + t2;
        } else if (ar >= 0) {
          v = KB[(int64_t)(c - nu) * nvj + ar];
        } else if (ac >= 0) {
          v = KB[(int64_t)(r - nu) * nvj + ac];
        } else {
          v = W[(int64_t)(r - nu) * n1w + (c - nu)];
        }
        W2[e] = v;
      }
      for (int c = tid; c < n2; c += NT) {
        const int ac = c < nu ? c : (c >= U2 ? nu + (c - U2) : -1);
        double v;
        if (ac >= 0) {
          v = D[L.rq + ac];
          for (int t = 0; t < nx1; ++t) v = fma(ba_at(D, L, t, ac), ev[t], v);
        } else {
          v = w[c - nu];
          for (int t = 0; t < nx1; ++t) v = fma(W[(int64_t)(c - nu) * n1w + U + t], D[L.b + t], v);
        }
        w2[c] = v;
      }
      __syncthreads();
      double* tmp = W;
      W = W2;
      W2 = tmp;
      tmp = w;
      w = w2;
      w2 = tmp;
      U = U2;
      X = nx;
    }
    // ---- write the condensed stage's data block
    // dynamics (Phi_m, Gam_m, c_m): BAt row i = column i of [Gam_m Phi_m]
    const int nx1p = ss[m - 1].nx1;
    const double* Pm = Phi + m * sp;
    const double* Gm = Gam + m * sg;
    const double* cm = cv + (int64_t)m * a.nxmax;
    for (int e = tid; e < nvp * nx1p; e += NT) {
      const int i = e / nx1p, r = e - i * nx1p;
      Dd[DL.BAt + (int64_t)i * DL.ldb + r] = i < nup ? Gm[r * nup + i] : Pm[r * nxp + (i - nup)];
    }
    for (int r = tid; r < nx1p; r += NT) Dd[DL.b + r] = cm[r];
    // cost (symmetrised, as the host condensing does)
    for (int e = tid; e < nvp * nvp; e += NT) {
      const int i = e / nvp, j = e - i * nvp;
      Dd[DL.RSQ + (int64_t)i * DL.ldr + j] = 0.5 * (W[(int64_t)i * nvp + j] + W[(int64_t)j * nvp + i]);
    }
    for (int i = tid; i < nvp; i += NT) Dd[DL.rq + i] = w[i];
    // boxes (u of every stage, x of the first) and general rows (per stage its
    // own rows, then from the second stage on its state boxes); one thread
    // per constraint of the condensed stage
    const int nbp = dsd.nbu + dsd.nbx, ngp = dsd.ng;
    int32_t* I = reinterpret_cast<int32_t*>(Dd + DL.box);
    for (int i = tid; i < nvp; i += NT) I[nbp + i] = -1;
    __syncthreads();
    if (tid == 0) {
      int cb = 0, uo = 0;
      for (int j = 0; j < m; ++j) {
        const StageDesc& s = ss[j];
        const StageData L = stage_data_layout(s);
        const double* D = a.sdata + s.data;
        const int32_t* bi = reinterpret_cast<const int32_t*>(D + L.box);
        for (int t = 0; t < s.nbu; ++t) {
          I[cb] = uo + bi[t];
          Dd[DL.lo + cb] = D[L.lo + t];
          Dd[DL.hi + cb] = D[L.hi + t];
          ++cb;
        }
        uo += s.nu;
      }
      {
        const StageDesc& s = ss[0];
        const StageData L = stage_data_layout(s);
        const double* D = a.sdata + s.data;
        const int32_t* bi = reinterpret_cast<const int32_t*>(D + L.box);
        for (int t = 0; t < s.nbx; ++t) {
          I[cb] = nup + (bi[s.nbu + t] - s.nu);
          Dd[DL.lo + cb] = D[L.lo + s.nbu + t];
          Dd[DL.hi + cb] = D[L.hi + s.nbu + t];
          ++cb;
        }
      }
      for (int c = 0; c < cb; ++c) I[nbp + I[c]] = c;
    }
    // general rows: the coefficient rows are filled in parallel below; the
    // bounds need the shift of each row and are filled here per row
    __syncthreads();
    {
      // row r of the condensed general block -> (stage j, kind, index)
      // enumerated in the same order by every thread
      int r0 = 0, uo = 0;
      for (int j = 0; j < m; ++j) {
        const StageDesc& s = ss[j];
        const StageData L = stage_data_layout(s);
        const double* D = a.sdata + s.data;
        const int nu = s.nu, nx = s.nx, nv = nu + nx, nb = s.nbu + s.nbx;
        const int32_t* bi = reinterpret_cast<const int32_t*>(D + L.box);
        const double* Pj = Phi + j * sp;
        const double* Gj = Gam + j * sg;
        const double* cj = cv + (int64_t)j * a.nxmax;
        const int nrows = s.ng + (j > 0 ? s.nbx : 0);
        // coefficients over [u'; x']: row = coef T_j, coef over [u_j; x_j]
        for (int e = tid; e < nrows * nvp; e += NT) {
          const int rr = e / nvp, p = e - rr * nvp;
          double v = 0.0;
          if (rr < s.ng) {
            const double* dc = D + L.DC + (int64_t)rr * nv;
            if (p < nup) {
              if (p >= uo && p < uo + nu) v = dc[p - uo];
              for (int t = 0; t < nx; ++t) v = fma(dc[nu + t], Gj[t * nup + p], v);
            } else {
              for (int t = 0; t < nx; ++t) v = fma(dc[nu + t], Pj[t * nxp + (p - nup)], v);
            }
          } else {
            const int xi = bi[s.nbu + (rr - s.ng)] - nu;  // state index of the box
            v = p < nup ? Gj[xi * nup + p] : Pj[xi * nxp + (p - nup)];
          }
          Dd[DL.DC + (int64_t)(r0 + rr) * nvp + p] = v;
        }
        for (int rr = tid; rr < nrows; rr += NT) {
          double shift = 0.0, lo, hi;
          if (rr < s.ng) {
            const double* dc = D + L.DC + (int64_t)rr * nv;
            for (int t = 0; t < nx; ++t) shift = fma(dc[nu + t], cj[t], shift);
            lo = D[L.lo + nb + rr];
            hi = D[L.hi + nb + rr];
          } else {
            const int bx = s.nbu + (rr - s.ng);
            shift = cj[bi[bx] - nu];
            lo = D[L.lo + bx];
            hi = D[L.hi + bx];
          }
          // an infinite bound stays infinite
          Dd[DL.lo + nbp + r0 + rr] = lo - shift;
          Dd[DL.hi + nbp + r0 + rr] = hi - shift;
        }
        r0 += nrows;
        uo += nu;
      }
      (void)ngp;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace gq

using namespace gq;

namespace {

struct CondPlan {
  int n2max, m_max, nxmax, numax, nup_max, nxp_max;
  int64_t slice;
};

int cond_plan(const gq_batch* src, int block, CondPlan* p) {
  p->n2max = p->m_max = p->nxmax = p->numax = p->nup_max = p->nxp_max = 0;
  int64_t slice = 0;
  for (int q = 0; q < src->nqp; ++q) {
    const QpDesc& d = src->qp[q];
    const int N = d.N, N2 = (N + block - 1) / block;
    p->n2max = std::max(p->n2max, N2 + 1);
    for (int n = 0; n <= N; ++n) {
      const StageDesc& s = src->st[d.stage0 + n];
      if (s.ns > 0) return set_error(GQ_ERR_ARG, "condensing of QPs with soft constraints is not supported");
      p->nxmax = std::max(p->nxmax, std::max(s.nx, s.nx1));
      p->numax = std::max(p->numax, s.nu);
    }
  }
  for (int q = 0; q < src->nqp; ++q) {
    const QpDesc& d = src->qp[q];
    const int N = d.N, N2 = (N + block - 1) / block;
    for (int k = 0; k < N2; ++k) {
      const int n0 = k * block, n1 = std::min(N, (k + 1) * block) - 1, m = n1 - n0 + 1;
      int nup = 0;
      for (int n = n0; n <= n1; ++n) nup += src->st[d.stage0 + n].nu;
      const int nxp = src->st[d.stage0 + n0].nx;
      p->m_max = std::max(p->m_max, m);
      p->nup_max = std::max(p->nup_max, nup);
      p->nxp_max = std::max(p->nxp_max, nxp);
      slice = std::max(slice, cond_scratch(m, p->nxmax, nup, nxp, p->numax).total);
    }
  }
  p->slice = slice;
  return GQ_OK;
}

int cond_grid() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    nsm = 1;
  return 4 * std::max(1, nsm);
}

}  // namespace

extern "C" {

size_t gq_condense_ws_bytes(const gq_batch* src, int block) {
  if (src == nullptr || block < 1) return 0;
  CondPlan p;
  if (cond_plan(src, block, &p)) return 0;
  const int64_t items = (int64_t)src->nqp * p.n2max;
  const int64_t grid = std::min<int64_t>(items, cond_grid());
  return (size_t)(grid * p.slice * 8);
}

int gq_condense_device(const gq_batch* src, int block, gq_batch* dst, void* dev_ws, size_t ws_bytes, void* stream) {
  if (src == nullptr || dst == nullptr || dev_ws == nullptr) return set_error(GQ_ERR_ARG, "NULL argument");
  if (block < 1) return set_error(GQ_ERR_ARG, "block must be >= 1");
  if (dst->nqp != src->nqp) return set_error(GQ_ERR_DIMS, "destination holds %d QPs, source %d", dst->nqp, src->nqp);
  if (!src->dev_in || !dst->dev_in) return set_error(GQ_ERR_STATE, "device buffers not attached");
  CondPlan p;
  int rc = cond_plan(src, block, &p);
  if (rc) return rc;
  // the destination must hold, QP by QP, the condensed QP's sizes
  for (int q = 0; q < src->nqp; ++q) {
    const QpDesc& s = src->qp[q];
    const QpDesc& d = dst->qp[q];
    const int N = s.N, N2 = (N + block - 1) / block;
    if (d.N != N2) return set_error(GQ_ERR_DIMS, "QP %d: destination horizon %d != %d", q, d.N, N2);
    for (int k = 0; k <= N2; ++k) {
      const StageDesc& ds = dst->st[d.stage0 + k];
      int nu = 0, nbu = 0, ng = 0, nx, nbx, nx1;
      if (k < N2) {
        const int n0 = k * block, n1 = std::min(N, (k + 1) * block) - 1;
        for (int n = n0; n <= n1; ++n) {
          const StageDesc& ss = src->st[s.stage0 + n];
          nu += ss.nu;
          nbu += ss.nbu;
          ng += ss.ng + (n > n0 ? ss.nbx : 0);
        }
        nx = src->st[s.stage0 + n0].nx;
        nbx = src->st[s.stage0 + n0].nbx;
        nx1 = src->st[s.stage0 + n1].nx1;
      } else {
        const StageDesc& ss = src->st[s.stage0 + N];
        nu = ss.nu;
        nbu = ss.nbu;
        ng = ss.ng;
        nx = ss.nx;
        nbx = ss.nbx;
        nx1 = 0;
      }
      if (ds.nx != nx || ds.nu != nu || ds.nbu != nbu || ds.nbx != nbx || ds.ng != ng || ds.nx1 != nx1 || ds.ns != 0)
        return set_error(GQ_ERR_DIMS, "QP %d: destination stage %d does not have the condensed sizes", q, k);
    }
    for (int k = 0; k <= N2; ++k)
      for (int k2 = 0; k2 < k; ++k2)
        if (dst->st[d.stage0 + k].data == dst->st[d.stage0 + k2].data)
          return set_error(GQ_ERR_ARG, "QP %d: destination stages must have private data blocks", q);
  }
  const int64_t items = (int64_t)src->nqp * p.n2max;
  const int grid = (int)std::min<int64_t>(items, cond_grid());
  if (ws_bytes < (size_t)(grid * p.slice * 8))
    return set_error(GQ_ERR_SIZE, "workspace %zu < %zu bytes (gq_condense_ws_bytes)", ws_bytes,
                     (size_t)(grid * p.slice * 8));
  if (reinterpret_cast<uintptr_t>(dev_ws) % 256) return set_error(GQ_ERR_ARG, "workspace must be 256-byte aligned");
  const char* sin = static_cast<const char*>(src->dev_in);
  char* din = static_cast<char*>(dst->dev_in);
  CondArgs a;
  a.sqp = reinterpret_cast<const QpDesc*>(sin + src->L.qpdesc);
  a.sst = reinterpret_cast<const StageDesc*>(sin + src->L.stagedesc);
  a.sdata = reinterpret_cast<const double*>(sin + src->L.data);
  a.dqp = reinterpret_cast<const QpDesc*>(din + dst->L.qpdesc);
  a.dst = reinterpret_cast<const StageDesc*>(din + dst->L.stagedesc);
  a.ddata = reinterpret_cast<double*>(din + dst->L.data);
  a.nqp = src->nqp;
  a.block = block;
  a.n2max = p.n2max;
  a.m_max = p.m_max;
  a.nxmax = p.nxmax;
  a.numax = p.numax;
  a.nup_max = p.nup_max;
  a.nxp_max = p.nxp_max;
  a.slice = p.slice;
  a.ws = static_cast<double*>(dev_ws);
  condense_kernel<<<grid, kCondThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GQ_ERR_CUDA, "condense launch: %s", cudaGetErrorString(e));
  return GQ_OK;
}

}  // extern "C"
