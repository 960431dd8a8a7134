// Partial (block) condensing of OCP QPs on the host (Sec. 3.5): blocks of
// `block` consecutive stages become one stage by eliminating the states
// inside the block through the dynamics, so the recursion that the solver
// runs has fewer, larger stages.  For a block of stages n0..n1 the new stage
// keeps x_{n0} and stacks u_{n0..n1}; with
//   x_{n0+j} = Phi_j x_{n0} + Gam_j u' + c_j  (Phi_0 = I, Gam_0 = 0, c_0 = 0)
// each original stage's variables are [u_n; x_n] = T_j [u'; x'] + [0; c_j],
// its cost and general rows are mapped through T_j, the box bounds on the
// eliminated states become general rows, and the block's dynamics are
// (Phi_m, Gam_m, c_m).  The terminal stage is kept as it is.  The solution
// of the condensed QP is expanded back: states from the recursion above,
// lambda and t by the constraint correspondence, and the multipliers of the
// eliminated dynamics from the stationarity rows of the eliminated states,
// solved backward from the block's last one.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/gq.h"
#include "gq_batch.h"

namespace {

using gq::set_error;
using Mat = std::vector<double>;  // row-major

struct StageDims {
  int nx, nu, nbx, nbu, ng, nx1;
};

StageDims dims_of(const gq_batch* b, int qp, int n) {
  const gq::StageDesc& s = b->st[b->qp[qp].stage0 + n];
  return StageDims{s.nx, s.nu, s.nbx, s.nbu, s.ng, s.nx1};
}

// first and last original stage of condensed stage k (k < N2)
void block_range(int N, int block, int k, int* n0, int* n1) {
  *n0 = k * block;
  *n1 = std::min(N, (k + 1) * block) - 1;
}

int condensed_horizon(int N, int block) { return (N + block - 1) / block; }

// Column-major getter outputs into row-major matrices.
Mat get_colmajor(int rows, int cols, const std::vector<double>& cm, int ld) {
  Mat m((size_t)rows * cols);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) m[(size_t)i * cols + j] = cm[i + (size_t)j * ld];
  return m;
}

struct StageData {
  StageDims d;
  Mat A, B, Q, S, R, C, D;  // row-major
  std::vector<double> b, q, r, lg, ug, lbu, ubu, lbx, ubx;
  std::vector<int> idxbu, idxbx;
};

int read_stage(gq_batch* src, int qp, int n, int N, StageData* o) {
  o->d = dims_of(src, qp, n);
  const StageDims& d = o->d;
  const int nx1 = n < N ? d.nx1 : 0;
  std::vector<double> a((size_t)std::max(1, nx1 * d.nx)), bb((size_t)std::max(1, nx1 * d.nu));
  o->b.assign(nx1, 0.0);
  if (n < N) {
    int rc = gq_get_dynamics(src, qp, n, a.data(), std::max(1, nx1), bb.data(), std::max(1, nx1), o->b.data());
    if (rc) return rc;
  }
  o->A = get_colmajor(nx1, d.nx, a, std::max(1, nx1));
  o->B = get_colmajor(nx1, d.nu, bb, std::max(1, nx1));
  std::vector<double> Q((size_t)std::max(1, d.nx * d.nx)), S((size_t)std::max(1, d.nu * d.nx)),
      R((size_t)std::max(1, d.nu * d.nu));
  o->q.assign(d.nx, 0.0);
  o->r.assign(d.nu, 0.0);
  int rc = gq_get_cost(src, qp, n, Q.data(), std::max(1, d.nx), S.data(), std::max(1, d.nu), R.data(),
                       std::max(1, d.nu), o->q.data(), o->r.data());
  if (rc) return rc;
  o->Q = get_colmajor(d.nx, d.nx, Q, std::max(1, d.nx));
  o->S = get_colmajor(d.nu, d.nx, S, std::max(1, d.nu));
  o->R = get_colmajor(d.nu, d.nu, R, std::max(1, d.nu));
  o->idxbu.assign(d.nbu, 0);
  o->idxbx.assign(d.nbx, 0);
  o->lbu.assign(d.nbu, 0.0);
  o->ubu.assign(d.nbu, 0.0);
  o->lbx.assign(d.nbx, 0.0);
  o->ubx.assign(d.nbx, 0.0);
  rc = gq_get_box(src, qp, n, o->idxbu.data(), o->lbu.data(), o->ubu.data(), o->idxbx.data(), o->lbx.data(),
                  o->ubx.data());
  if (rc) return rc;
  std::vector<double> C((size_t)std::max(1, d.ng * d.nx)), Dm((size_t)std::max(1, d.ng * d.nu));
  o->lg.assign(d.ng, 0.0);
  o->ug.assign(d.ng, 0.0);
  rc = gq_get_general(src, qp, n, C.data(), std::max(1, d.ng), Dm.data(), std::max(1, d.ng), o->lg.data(),
                      o->ug.data());
  if (rc) return rc;
  o->C = get_colmajor(d.ng, d.nx, C, std::max(1, d.ng));
  o->D = get_colmajor(d.ng, d.nu, Dm, std::max(1, d.ng));
  return GQ_OK;
}

// The block recursion x_{n0+j} = Phi_j x' + Gam_j u' + c_j, j = 0..m.
struct BlockMaps {
  int nxp, nup;                 // x' and u' sizes
  std::vector<int> uoff;        // offset of u_{n0+j} in u'
  std::vector<Mat> Phi, Gam;    // nx_{n0+j} x nxp, nx_{n0+j} x nup
  std::vector<std::vector<double>> c;
};

BlockMaps block_maps(const std::vector<StageData>& st) {
  BlockMaps m;
  const int mlen = (int)st.size();
  m.nxp = st[0].d.nx;
  m.nup = 0;
  for (int j = 0; j < mlen; ++j) {
    m.uoff.push_back(m.nup);
    m.nup += st[j].d.nu;
  }
  Mat phi((size_t)m.nxp * m.nxp, 0.0);
  for (int i = 0; i < m.nxp; ++i) phi[(size_t)i * m.nxp + i] = 1.0;
  m.Phi.push_back(phi);
  m.Gam.push_back(Mat((size_t)m.nxp * m.nup, 0.0));
  m.c.push_back(std::vector<double>(m.nxp, 0.0));
  for (int j = 0; j < mlen; ++j) {
    const StageData& s = st[j];
    const int nx = s.d.nx, nx1 = s.d.nx1, nu = s.d.nu;
    Mat P1((size_t)nx1 * m.nxp, 0.0), G1((size_t)nx1 * m.nup, 0.0);
    std::vector<double> c1(nx1, 0.0);
    for (int k = 0; k < nx1; ++k) {
      for (int a = 0; a < nx; ++a) {
        const double akl = s.A[(size_t)k * nx + a];
        if (akl == 0.0) continue;
        for (int col = 0; col < m.nxp; ++col) P1[(size_t)k * m.nxp + col] += akl * m.Phi[j][(size_t)a * m.nxp + col];
        for (int col = 0; col < m.nup; ++col) G1[(size_t)k * m.nup + col] += akl * m.Gam[j][(size_t)a * m.nup + col];
        c1[k] += akl * m.c[j][a];
      }
      for (int a = 0; a < nu; ++a) G1[(size_t)k * m.nup + m.uoff[j] + a] += s.B[(size_t)k * nu + a];
      c1[k] += s.b[k];
    }
    m.Phi.push_back(P1);
    m.Gam.push_back(G1);
    m.c.push_back(c1);
  }
  return m;
}

// Row r of the map from [u'; x'] to [u_n; x_n] (nu_n + nx_n rows).
void t_row(const BlockMaps& m, int j, int nu, int r, std::vector<double>* row) {
  row->assign((size_t)m.nup + m.nxp, 0.0);
  if (r < nu) {
    (*row)[(size_t)m.uoff[j] + r] = 1.0;
  } else {
    const int i = r - nu;
    for (int col = 0; col < m.nup; ++col) (*row)[col] = m.Gam[j][(size_t)i * m.nup + col];
    for (int col = 0; col < m.nxp; ++col) (*row)[(size_t)m.nup + col] = m.Phi[j][(size_t)i * m.nxp + col];
  }
}

bool has_slacks(const gq_batch* b, int qp) {
  const gq::QpDesc& d = b->qp[qp];
  for (int n = 0; n <= d.N; ++n)
    if (b->st[d.stage0 + n].ns > 0) return true;
  return false;
}

int read_block(gq_batch* src, int qp, int N, int n0, int n1, std::vector<StageData>* st) {
  st->resize((size_t)(n1 - n0 + 1));
  for (int n = n0; n <= n1; ++n) {
    int rc = read_stage(src, qp, n, N, &(*st)[(size_t)(n - n0)]);
    if (rc) return rc;
  }
  return GQ_OK;
}

}  // namespace

extern "C" {

int gq_condense_dims(const gq_batch* src, int qp, int block, int* dims, size_t cap, size_t* len) {
  if (src == nullptr || len == nullptr) return set_error(GQ_ERR_ARG, "NULL argument");
  if (qp < 0 || qp >= src->nqp) return set_error(GQ_ERR_ARG, "qp out of range");
  if (block < 1) return set_error(GQ_ERR_ARG, "block must be >= 1");
  if (has_slacks(src, qp)) return set_error(GQ_ERR_ARG, "condensing of QPs with soft constraints is not supported");
  const int N = src->qp[qp].N;
  const int N2 = condensed_horizon(N, block);
  const size_t need = 1 + 5 * (size_t)(N2 + 1);
  *len = need;
  if (dims == nullptr) return GQ_OK;
  if (cap < need) return set_error(GQ_ERR_SIZE, "dims capacity %zu < %zu", cap, need);
  size_t p = 0;
  dims[p++] = N2;
  for (int k = 0; k < N2; ++k) {
    int n0, n1;
    block_range(N, block, k, &n0, &n1);
    int nu = 0, nbu = 0, ng = 0;
    for (int n = n0; n <= n1; ++n) {
      const StageDims d = dims_of(src, qp, n);
      nu += d.nu;
      nbu += d.nbu;
      ng += d.ng + (n > n0 ? d.nbx : 0);
    }
    const StageDims d0 = dims_of(src, qp, n0);
    dims[p++] = d0.nx;
    dims[p++] = nu;
    dims[p++] = d0.nbx;
    dims[p++] = nbu;
    dims[p++] = ng;
  }
  const StageDims dN = dims_of(src, qp, N);
  dims[p++] = dN.nx;
  dims[p++] = dN.nu;
  dims[p++] = dN.nbx;
  dims[p++] = dN.nbu;
  dims[p++] = dN.ng;
  return GQ_OK;
}

int gq_condense(gq_batch* src, int src_qp, int block, gq_batch* dst, int dst_qp) {
  if (src == nullptr || dst == nullptr) return set_error(GQ_ERR_ARG, "NULL batch");
  if (src_qp < 0 || src_qp >= src->nqp || dst_qp < 0 || dst_qp >= dst->nqp)
    return set_error(GQ_ERR_ARG, "QP index out of range");
  if (block < 1) return set_error(GQ_ERR_ARG, "block must be >= 1");
  if (has_slacks(src, src_qp))
    return set_error(GQ_ERR_ARG, "condensing of QPs with soft constraints is not supported");
  const int N = src->qp[src_qp].N;
  const int N2 = condensed_horizon(N, block);
  if (dst->qp[dst_qp].N != N2) return set_error(GQ_ERR_DIMS, "destination horizon %d != %d", dst->qp[dst_qp].N, N2);
  for (int k = 0; k < N2; ++k) {
    int n0, n1;
    block_range(N, block, k, &n0, &n1);
    std::vector<StageData> st;
    int rc = read_block(src, src_qp, N, n0, n1, &st);
    if (rc) return rc;
    const BlockMaps m = block_maps(st);
    const int nup = m.nup, nxp = m.nxp, nvp = nup + nxp, mlen = (int)st.size();
    const int nx1p = st.back().d.nx1;
    const StageDims dd = dims_of(dst, dst_qp, k);
    if (dd.nx != nxp || dd.nu != nup || dd.nx1 != nx1p)
      return set_error(GQ_ERR_DIMS, "destination stage %d has other sizes than the condensed block", k);
    // cost: the backward recursion of Sec. 3.5 (condensing analogous to the
    // classical Riccati recursion), quadratic in the block length and cubic
    // in the state size.  The cost of stages j..m-1 as a function of
    // v_j = [u_j; u_{j+1..}; x_j] is 1/2 v_j' W_j v_j + w_j' v_j; W_m = 0 on x_m,
    // and with x_{j+1} = A x_j + B u_j + b and W_{j+1} = [[Wuu, Wux], [Wxu, Wxx]]:
    //   W_j = [[R + B'Wxx B,  B'Wxu,  S + B'Wxx A],
    //          [Wux' B,       Wuu,    Wux A      ],
    //          [.,            .,      Q + A'Wxx A]]   (symmetric)
    //   w_j = [r + B'(Wxx b + wx); wu + Wux b; q + A'(Wxx b + wx)].
    // W_0 is the condensed Hessian over [u'; x'] and w_0 its gradient.
    Mat H;
    std::vector<double> g;
    {
      int U = 0, X = st.back().d.nx1;  // sizes of the tail's inputs and of its state
      Mat W((size_t)X * X, 0.0);       // (U + X) x (U + X), row-major
      std::vector<double> w((size_t)X, 0.0);
      for (int j = mlen - 1; j >= 0; --j) {
        const StageData& s = st[j];
        const int nu = s.d.nu, nx = s.d.nx, nx1 = s.d.nx1, n1 = U + X;
        auto Wv = [&](int a, int c2) { return W[(size_t)a * n1 + c2]; };
        // P = Wxx (X x X), K = Wux (U x X), e = Wxx b + wx
        std::vector<double> e((size_t)nx1, 0.0);
        for (int i = 0; i < nx1; ++i) {
          double v = w[(size_t)U + i];
          for (int k = 0; k < nx1; ++k) v += Wv(U + i, U + k) * s.b[k];
          e[i] = v;
        }
        // PB = Wxx [B A] (X x (nu + nx)), KB = Wux [B A] (U x (nu + nx))
        const int nvj = nu + nx;
        auto BA = [&](int k, int c2) { return c2 < nu ? s.B[(size_t)k * nu + c2] : s.A[(size_t)k * nx + (c2 - nu)]; };
        Mat PB((size_t)nx1 * nvj, 0.0), KB((size_t)U * nvj, 0.0);
        for (int i = 0; i < nx1; ++i)
          for (int k = 0; k < nx1; ++k) {
            const double p = Wv(U + i, U + k);
            if (p == 0.0) continue;
            for (int c2 = 0; c2 < nvj; ++c2) PB[(size_t)i * nvj + c2] += p * BA(k, c2);
          }
        for (int i = 0; i < U; ++i)
          for (int k = 0; k < nx1; ++k) {
            const double p = Wv(i, U + k);
            if (p == 0.0) continue;
            for (int c2 = 0; c2 < nvj; ++c2) KB[(size_t)i * nvj + c2] += p * BA(k, c2);
          }
        // new ordering [u_j (nu); u_{j+1..} (U); x_j (nx)]
        const int U2 = nu + U, n2 = U2 + nx;
        Mat W2((size_t)n2 * n2, 0.0);
        std::vector<double> w2((size_t)n2, 0.0);
        auto idx = [&](int c2) { return c2 < nu ? c2 : U2 + (c2 - nu); };  // [u_j; x_j] -> position
        // [B A]' Wxx [B A] + stage Hessian
        for (int a2 = 0; a2 < nvj; ++a2)
          for (int c2 = 0; c2 < nvj; ++c2) {
            double v = 0.0;
            for (int k = 0; k < nx1; ++k) v += BA(k, a2) * PB[(size_t)k * nvj + c2];
            double h;
            if (a2 < nu && c2 < nu) h = s.R[(size_t)a2 * nu + c2];
            else if (a2 < nu) h = s.S[(size_t)a2 * nx + (c2 - nu)];
            else if (c2 < nu) h = s.S[(size_t)c2 * nx + (a2 - nu)];
            else h = s.Q[(size_t)(a2 - nu) * nx + (c2 - nu)];
            W2[(size_t)idx(a2) * n2 + idx(c2)] = h + v;
          }
        // Wux [B A] couples the later inputs with [u_j; x_j]
        for (int i = 0; i < U; ++i)
          for (int c2 = 0; c2 < nvj; ++c2) {
            const double v = KB[(size_t)i * nvj + c2];
            W2[(size_t)(nu + i) * n2 + idx(c2)] = v;
            W2[(size_t)idx(c2) * n2 + nu + i] = v;
          }
        for (int i = 0; i < U; ++i)
          for (int k = 0; k < U; ++k) W2[(size_t)(nu + i) * n2 + nu + k] = Wv(i, k);
        // gradient
        for (int c2 = 0; c2 < nvj; ++c2) {
          double v = c2 < nu ? s.r[c2] : s.q[c2 - nu];
          for (int k = 0; k < nx1; ++k) v += BA(k, c2) * e[k];
          w2[idx(c2)] = v;
        }
        for (int i = 0; i < U; ++i) {
          double v = w[i];
          for (int k = 0; k < nx1; ++k) v += Wv(i, U + k) * s.b[k];
          w2[(size_t)nu + i] = v;
        }
        W.swap(W2);
        w.swap(w2);
        U = U2;
        X = nx;
      }
      H.swap(W);
      g.swap(w);
    }
    for (int p = 0; p < nvp; ++p)
      for (int q2 = 0; q2 < p; ++q2) {
        const double v = 0.5 * (H[(size_t)p * nvp + q2] + H[(size_t)q2 * nvp + p]);
        H[(size_t)p * nvp + q2] = H[(size_t)q2 * nvp + p] = v;
      }
    // setters take column-major arrays
    std::vector<double> Qc((size_t)std::max(1, nxp * nxp)), Sc((size_t)std::max(1, nup * nxp)),
        Rc((size_t)std::max(1, nup * nup)), qv(nxp), rv(nup);
    for (int i = 0; i < nup; ++i)
      for (int j2 = 0; j2 < nup; ++j2) Rc[i + (size_t)j2 * nup] = H[(size_t)i * nvp + j2];
    for (int i = 0; i < nup; ++i)
      for (int j2 = 0; j2 < nxp; ++j2) Sc[i + (size_t)j2 * nup] = H[(size_t)i * nvp + nup + j2];
    for (int i = 0; i < nxp; ++i)
      for (int j2 = 0; j2 < nxp; ++j2) Qc[i + (size_t)j2 * nxp] = H[(size_t)(nup + i) * nvp + nup + j2];
    for (int i = 0; i < nup; ++i) rv[i] = g[i];
    for (int i = 0; i < nxp; ++i) qv[i] = g[nup + i];
    rc = gq_set_cost(dst, dst_qp, k, Qc.data(), std::max(1, nxp), Sc.data(), std::max(1, nup), Rc.data(),
                     std::max(1, nup), qv.data(), rv.data());
    if (rc) return rc;
    // dynamics (Phi_m, Gam_m, c_m)
    std::vector<double> Ac((size_t)std::max(1, nx1p * nxp)), Bc((size_t)std::max(1, nx1p * nup));
    for (int i = 0; i < nx1p; ++i) {
      for (int j2 = 0; j2 < nxp; ++j2) Ac[i + (size_t)j2 * nx1p] = m.Phi[mlen][(size_t)i * nxp + j2];
      for (int j2 = 0; j2 < nup; ++j2) Bc[i + (size_t)j2 * nx1p] = m.Gam[mlen][(size_t)i * nup + j2];
    }
    rc = gq_set_dynamics(dst, dst_qp, k, Ac.data(), std::max(1, nx1p), Bc.data(), std::max(1, nx1p),
                         m.c[mlen].data());
    if (rc) return rc;
    // boxes: u of every stage, x of the first
    std::vector<int> ibu, ibx;
    std::vector<double> lbu, ubu, lbx, ubx;
    for (int j = 0; j < mlen; ++j)
      for (int a = 0; a < st[j].d.nbu; ++a) {
        ibu.push_back(m.uoff[j] + st[j].idxbu[a]);
        lbu.push_back(st[j].lbu[a]);
        ubu.push_back(st[j].ubu[a]);
      }
    ibx = st[0].idxbx;
    lbx = st[0].lbx;
    ubx = st[0].ubx;
    rc = gq_set_box(dst, dst_qp, k, ibu.data(), lbu.data(), ubu.data(), ibx.data(), lbx.data(), ubx.data());
    if (rc) return rc;
    // general rows: per stage its own rows, then (after the first stage) its
    // state boxes, both mapped through T_j
    const int ngp = dd.ng;
    std::vector<double> Cc((size_t)std::max(1, ngp * nxp), 0.0), Dc((size_t)std::max(1, ngp * nup), 0.0),
        lg(ngp), ug(ngp);
    int gr = 0;
    std::vector<double> row;
    for (int j = 0; j < mlen; ++j) {
      const StageData& s = st[j];
      const int nu = s.d.nu, nx = s.d.nx;
      std::vector<Mat> Trows(nu + nx);
      for (int r = 0; r < nu + nx; ++r) t_row(m, j, nu, r, &Trows[r]);
      auto put = [&](const std::vector<double>& coef, double shift, double lo, double hi) {
        // coef over [u_n; x_n]; row over [u'; x'] = coef T_j; bounds minus coef [0; c_j]
        for (int a = 0; a < nu + nx; ++a) {
          if (coef[a] == 0.0) continue;
          for (int p = 0; p < nup; ++p) Dc[gr + (size_t)p * ngp] += coef[a] * Trows[a][p];
          for (int p = 0; p < nxp; ++p) Cc[gr + (size_t)p * ngp] += coef[a] * Trows[a][nup + p];
        }
        lg[gr] = lo - shift;  // an infinite bound stays infinite
        ug[gr] = hi - shift;
        ++gr;
      };
      for (int gg = 0; gg < s.d.ng; ++gg) {
        std::vector<double> coef(nu + nx, 0.0);
        double shift = 0.0;
        for (int a = 0; a < nu; ++a) coef[a] = s.D[(size_t)gg * nu + a];
        for (int a = 0; a < nx; ++a) {
          coef[nu + a] = s.C[(size_t)gg * nx + a];
          shift += coef[nu + a] * m.c[j][a];
        }
        put(coef, shift, s.lg[gg], s.ug[gg]);
      }
      if (j > 0)
        for (int a = 0; a < s.d.nbx; ++a) {
          std::vector<double> coef(nu + nx, 0.0);
          coef[nu + s.idxbx[a]] = 1.0;
          put(coef, m.c[j][s.idxbx[a]], s.lbx[a], s.ubx[a]);
        }
    }
    if (gr != ngp) return set_error(GQ_ERR_DIMS, "condensed stage %d: %d general rows, expected %d", k, gr, ngp);
    if (ngp) {
      rc = gq_set_general(dst, dst_qp, k, Cc.data(), ngp, Dc.data(), ngp, lg.data(), ug.data());
      if (rc) return rc;
    }
  }
  // terminal stage unchanged
  StageData t;
  int rc = read_stage(src, src_qp, N, N, &t);
  if (rc) return rc;
  const int nx = t.d.nx, nu = t.d.nu;
  std::vector<double> Qc((size_t)std::max(1, nx * nx)), Sc((size_t)std::max(1, nu * nx)), Rc((size_t)std::max(1, nu * nu));
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < nx; ++j) Qc[i + (size_t)j * nx] = t.Q[(size_t)i * nx + j];
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nx; ++j) Sc[i + (size_t)j * std::max(1, nu)] = t.S[(size_t)i * nx + j];
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j) Rc[i + (size_t)j * nu] = t.R[(size_t)i * nu + j];
  rc = gq_set_cost(dst, dst_qp, N2, Qc.data(), std::max(1, nx), Sc.data(), std::max(1, nu), Rc.data(),
                   std::max(1, nu), t.q.data(), t.r.data());
  if (rc) return rc;
  rc = gq_set_box(dst, dst_qp, N2, t.idxbu.data(), t.lbu.data(), t.ubu.data(), t.idxbx.data(), t.lbx.data(),
                  t.ubx.data());
  if (rc) return rc;
  if (t.d.ng) {
    std::vector<double> Cc((size_t)t.d.ng * std::max(1, nx)), Dc((size_t)t.d.ng * std::max(1, nu));
    for (int gg = 0; gg < t.d.ng; ++gg) {
      for (int a = 0; a < nx; ++a) Cc[gg + (size_t)a * t.d.ng] = t.C[(size_t)gg * nx + a];
      for (int a = 0; a < nu; ++a) Dc[gg + (size_t)a * t.d.ng] = t.D[(size_t)gg * nu + a];
    }
    rc = gq_set_general(dst, dst_qp, N2, Cc.data(), t.d.ng, Dc.data(), t.d.ng, t.lg.data(), t.ug.data());
    if (rc) return rc;
  }
  return GQ_OK;
}

int gq_expand(gq_batch* src, int src_qp, int block, const gq_batch* dst, int dst_qp, const double* y2,
              const double* pi2, const double* lam2, const double* t2, double* y, double* pi, double* lam, double* t) {
  if (src == nullptr || dst == nullptr || y2 == nullptr || pi2 == nullptr || lam2 == nullptr || t2 == nullptr ||
      y == nullptr || pi == nullptr || lam == nullptr || t == nullptr)
    return set_error(GQ_ERR_ARG, "NULL argument");
  if (src_qp < 0 || src_qp >= src->nqp || dst_qp < 0 || dst_qp >= dst->nqp)
    return set_error(GQ_ERR_ARG, "QP index out of range");
  if (block < 1) return set_error(GQ_ERR_ARG, "block must be >= 1");
  const int N = src->qp[src_qp].N;
  const int N2 = condensed_horizon(N, block);
  if (dst->qp[dst_qp].N != N2) return set_error(GQ_ERR_DIMS, "condensed horizon mismatch");
  const gq::QpDesc& qs = src->qp[src_qp];
  const gq::QpDesc& qd = dst->qp[dst_qp];
  auto sst = [&](int n) -> const gq::StageDesc& { return src->st[qs.stage0 + n]; };
  auto dst_st = [&](int k) -> const gq::StageDesc& { return dst->st[qd.stage0 + k]; };
  for (int k = 0; k <= N2; ++k) {
    const gq::StageDesc& ds = dst_st(k);
    const int dvar = ds.var - qd.var0, dside = ds.side - qd.side0;
    const int ncd = ds.nbu + ds.nbx + ds.ng;
    if (k == N2) {
      // terminal stage: identity
      const gq::StageDesc& s = sst(N);
      const int nv = s.nx + s.nu, nc = s.nbu + s.nbx + s.ng;
      std::memcpy(y + (s.var - qs.var0), y2 + dvar, 8 * (size_t)nv);
      std::memcpy(lam + (s.side - qs.side0), lam2 + dside, 8 * (size_t)(2 * nc));
      std::memcpy(t + (s.side - qs.side0), t2 + dside, 8 * (size_t)(2 * nc));
      break;
    }
    int n0, n1;
    block_range(N, block, k, &n0, &n1);
    std::vector<StageData> st;
    int rc = read_block(src, src_qp, N, n0, n1, &st);
    if (rc) return rc;
    const BlockMaps m = block_maps(st);
    const int nup = m.nup, mlen = (int)st.size();
    const double* up = y2 + dvar;
    const double* xp = y2 + dvar + nup;
    // primal: u_n from u', x_n = Phi_j x' + Gam_j u' + c_j
    for (int j = 0; j < mlen; ++j) {
      const gq::StageDesc& s = sst(n0 + j);
      double* yn = y + (s.var - qs.var0);
      for (int a = 0; a < s.nu; ++a) yn[a] = up[m.uoff[j] + a];
      for (int i = 0; i < s.nx; ++i) {
        double v = m.c[j][i];
        for (int p = 0; p < m.nxp; ++p) v += m.Phi[j][(size_t)i * m.nxp + p] * xp[p];
        for (int p = 0; p < nup; ++p) v += m.Gam[j][(size_t)i * nup + p] * up[p];
        yn[s.nu + i] = v;
      }
    }
    // lambda, t: condensed constraint list [box u'; box x'; general], lower
    // sides then upper sides
    int bu = 0, gr = 0;
    for (int j = 0; j < mlen; ++j) {
      const gq::StageDesc& s = sst(n0 + j);
      const int nc = s.nbu + s.nbx + s.ng, side = s.side - qs.side0;
      auto copy_side = [&](int c, int cd) {
        lam[side + c] = lam2[dside + cd];
        lam[side + nc + c] = lam2[dside + ncd + cd];
        t[side + c] = t2[dside + cd];
        t[side + nc + c] = t2[dside + ncd + cd];
      };
      for (int a = 0; a < s.nbu; ++a) copy_side(a, bu++);
      const int gstart = ds.nbu + ds.nbx;
      for (int a = 0; a < s.ng; ++a) copy_side(s.nbu + s.nbx + a, gstart + gr++);
      for (int a = 0; a < s.nbx; ++a) {
        if (j == 0)
          copy_side(s.nbu + a, ds.nbu + a);
        else
          copy_side(s.nbu + a, gstart + gr++);
      }
    }
    // pi: the block's last dynamics keep the condensed multiplier; the
    // eliminated states' stationarity rows give the others, backward:
    // pi_n = Q x + S' u + q + A' pi_{n+1} - C'(lam_gl - lam_gu) - box terms
    const gq::StageDesc& slast = sst(n1);
    std::memcpy(pi + (slast.eq - qs.eq0), pi2 + (ds.eq - qd.eq0), 8 * (size_t)slast.nx1);
    for (int n = n1; n > n0; --n) {
      const StageData& s = st[(size_t)(n - n0)];
      const gq::StageDesc& sd = sst(n);
      const int nx = s.d.nx, nu = s.d.nu, nb = s.d.nbu + s.d.nbx, nc = nb + s.d.ng;
      const double* yn = y + (sd.var - qs.var0);
      const double* pn1 = pi + (sd.eq - qs.eq0);
      const double* ln = lam + (sd.side - qs.side0);
      double* pn = pi + (sst(n - 1).eq - qs.eq0);
      for (int i = 0; i < nx; ++i) {
        double v = s.q[i];
        for (int a = 0; a < nx; ++a) v += s.Q[(size_t)i * nx + a] * yn[nu + a];
        for (int a = 0; a < nu; ++a) v += s.S[(size_t)a * nx + i] * yn[a];
        for (int a = 0; a < s.d.nx1; ++a) v += s.A[(size_t)a * nx + i] * pn1[a];
        for (int gg = 0; gg < s.d.ng; ++gg) v -= s.C[(size_t)gg * nx + i] * (ln[nb + gg] - ln[nc + nb + gg]);
        for (int a = 0; a < s.d.nbx; ++a)
          if (s.idxbx[a] == i) v -= ln[s.d.nbu + a] - ln[nc + s.d.nbu + a];
        pn[i] = v;
      }
    }
  }
  return GQ_OK;
}

}  // extern "C"
