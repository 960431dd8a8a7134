// Host side of the gq C ABI: batch layout planning, validated setters and
// getters, transfers and the solve entry point.  Nothing here allocates: all
// memory comes from the caller (Sec. 1 of the HPIPM paper: the solver works on
// externally provided chunks of memory).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "gq_internal.h"
#include "gq_launch.h"
#include "gq_batch.h"

using namespace gq;

namespace {

thread_local char g_err[512] = "no error";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(GQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr uint32_t kMagic = 0x67716231u;  // "gqb1"

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace

namespace gq {
int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}
}  // namespace gq


namespace {

struct Counts {
  int64_t n_stages = 0;
  bool ok = false;
};

// Parses dims and checks their consistency; returns the stage count.
Counts count_stages(int nqp, const int* dims, size_t dims_len) {
  Counts c;
  if (nqp <= 0 || dims == nullptr) {
    fail(GQ_ERR_ARG, "nqp must be positive and dims non-NULL");
    return c;
  }
  size_t pos = 0;
  for (int q = 0; q < nqp; ++q) {
    if (pos >= dims_len) {
      fail(GQ_ERR_DIMS, "dims too short at QP %d", q);
      return c;
    }
    const int N = dims[pos++];
    if (N < 0 || N > (1 << 20)) {
      fail(GQ_ERR_DIMS, "QP %d: horizon N=%d out of range", q, N);
      return c;
    }
    if (pos + 5 * (size_t)(N + 1) > dims_len) {
      fail(GQ_ERR_DIMS, "dims too short for QP %d (N=%d)", q, N);
      return c;
    }
    for (int n = 0; n <= N; ++n) {
      const int* d = dims + pos + 5 * n;
      const int nx = d[0], nu = d[1], nbx = d[2], nbu = d[3], ng = d[4];
      if (nx < 0 || nu < 0 || nbx < 0 || nbu < 0 || ng < 0 || nbx > nx || nbu > nu ||
          nx > 4096 || nu > 4096 || ng > 65536) {
        fail(GQ_ERR_DIMS, "QP %d stage %d: invalid sizes nx=%d nu=%d nbx=%d nbu=%d ng=%d", q, n,
             nx, nu, nbx, nbu, ng);
        return c;
      }
      if (nx + nu == 0) {
        fail(GQ_ERR_DIMS, "QP %d stage %d: stage without variables", q, n);
        return c;
      }
    }
    pos += 5 * (size_t)(N + 1);
    c.n_stages += N + 1;
  }
  if (pos != dims_len) {
    fail(GQ_ERR_DIMS, "dims has %zu trailing entries", dims_len - pos);
    return c;
  }
  c.ok = true;
  return c;
}

int64_t hash_capacity(int64_t n) {
  int64_t cap = 16;
  while (cap < 2 * n) cap <<= 1;
  return cap;
}

size_t handle_bytes(int nqp, int64_t n_stages, int64_t cap) {
  int64_t b = align_up(sizeof(gq_batch), 64);
  b += align_up((int64_t)nqp * sizeof(QpDesc), 64);
  b += align_up(n_stages * sizeof(StageDesc), 64);
  b += align_up((int64_t)nqp * sizeof(int32_t), 64);
  b += align_up(n_stages * sizeof(int32_t), 64);
  b += align_up(cap * sizeof(SlotEntry), 64);
  return (size_t)b;
}

inline double* host_data(gq_batch* b) {
  return reinterpret_cast<double*>(static_cast<char*>(b->host_in) + b->L.data);
}

int check_batch(const gq_batch* b) {
  if (b == nullptr || b->magic != kMagic) return fail(GQ_ERR_ARG, "invalid batch handle");
  return GQ_OK;
}

int stage_of(gq_batch* b, int qp, int n, StageDesc** out) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (qp < 0 || qp >= b->nqp) return fail(GQ_ERR_ARG, "qp %d out of range [0,%d)", qp, b->nqp);
  const QpDesc& d = b->qp[qp];
  if (n < 0 || n > d.N) return fail(GQ_ERR_ARG, "stage %d out of range [0,%d] for QP %d", n, d.N, qp);
  if (b->host_in == nullptr) return fail(GQ_ERR_STATE, "host_in buffer not attached");
  *out = &b->st[d.stage0 + n];
  return GQ_OK;
}

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

}  // namespace

extern "C" {

const char* gq_last_error(void) { return g_err; }

int gq_ipm_arg_default(gq_ipm_arg* arg, int mode, int precision) {
  if (arg == nullptr) return fail(GQ_ERR_ARG, "arg is NULL");
  if (mode != GQ_MODE_SPEED && mode != GQ_MODE_BALANCE && mode != GQ_MODE_ROBUST)
    return fail(GQ_ERR_ARG, "unknown mode %d", mode);
  if (precision != GQ_PREC_FP64 && precision != GQ_PREC_MIXED)
    return fail(GQ_ERR_ARG, "unknown precision %d", precision);
  std::memset(arg, 0, sizeof(*arg));
  arg->mode = mode;
  arg->precision = precision;
  arg->iter_max = 100;
  arg->warm_start = 0;
  arg->cond_corr = 1;
  arg->fp64_fallback = 1;
  arg->tol_stat = arg->tol_eq = arg->tol_ineq = arg->tol_comp = 1e-8;
  arg->alpha_min = 1e-12;
  const bool mixed = precision == GQ_PREC_MIXED;
  arg->lam_min = arg->t_min = mixed ? 1e-12 : 1e-16;
  arg->tau_b = 0.995;
  arg->corr_k = 2.0;
  arg->reg_prim = mixed ? 1e-9 : 0.0;
  arg->ir_steps = (mixed || mode != GQ_MODE_SPEED) ? 3 : 0;
  // refine to 1e-12 relative: a looser inexact-Newton tolerance (1e-4) was
  // measured to skip refinement but raise the mass-spring iteration count
  // from 7.0 to 10.6, a net loss
  arg->ir_tol = 1e-12;
  arg->warm_min = 1e-2;
  arg->timeout_ns = 0;
  arg->ir_fail_ratio = 1e-6;
  return GQ_OK;
}

}  // extern "C"

namespace {

// Shape of the QPs at positions [lo, hi) of the order array (all QPs when
// `all`, whatever the order).
// largest nu + nx of the block bucket for which the automatic block size is 128
constexpr int kAutoThreadsNv = 96;

// SMs of the current device; 0 without one (the automatic block size then
// stays at 256)
int device_sms() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nsm;
}

Shape bucket_shape(const gq_batch* b, int lo, int hi, bool all) {
  Shape sh;
  std::memset(&sh, 0, sizeof(sh));
  for (int k = lo; k < hi; ++k) {
    const QpDesc& d = b->qp[all ? k : b->order[k]];
    sh.nst_max = std::max(sh.nst_max, d.N + 1);
    sh.nside_max = std::max(sh.nside_max, d.nsidet);
    for (int n = 0; n <= d.N; ++n) {
      const StageDesc& st = b->st[d.stage0 + n];
      const int nv = st.nx + st.nu;
      sh.nvmax = std::max(sh.nvmax, nv);
      sh.nxmax = std::max(sh.nxmax, st.nx);
      sh.ngmax = std::max(sh.ngmax, st.ng);
      sh.ne_max = std::max(sh.ne_max, n == 0 ? nv : st.nu);
      sh.data_max = std::max(sh.data_max, stage_data_layout(st).size);
    }
  }
  return sh;
}

// Buckets under the batch's schedule: QPs whose stages fit one warp
// (nu + nx and nx at most warp_max_nv) first, then the rest; each bucket in
// longest-processing-time order (most expensive QPs launch first).
void plan_buckets(gq_batch* b) {
  const int nqp = b->nqp;
  const QpDesc* qd = b->qp;
  const int wmax = b->warp_max_nv;
  // the one-warp kernel has no slack elimination: QPs with soft constraints
  // run in the block kernel
  auto warp_ok = [&](int q) { return qd[q].nvmax <= wmax && qd[q].nxmax <= wmax && qd[q].nsoft == 0; };
  int nw = 0;
  for (int q = 0; q < nqp; ++q)
    if (warp_ok(q)) b->order[nw++] = q;
  int nb = nw;
  for (int q = 0; q < nqp; ++q)
    if (!warp_ok(q)) b->order[nb++] = q;
  auto by_cost = [qd](int32_t a, int32_t c2) { return qd[a].cost > qd[c2].cost; };
  std::stable_sort(b->order, b->order + nw, by_cost);
  std::stable_sort(b->order + nw, b->order + nqp, by_cost);
  b->nwarp = nw;
  b->soft_block = 0;
  for (int i = nw; i < nqp; ++i) b->soft_block |= qd[b->order[i]].nsoft > 0;
  b->shape_w = bucket_shape(b, 0, nw, false);
  b->shape_b = bucket_shape(b, nw, nqp, false);
  if (nqp > nw) b->shape_b.mat_global = 1;
  // automatic block size (0): 128 threads (four QPs per SM) when the block
  // bucket's stages have nu + nx <= 96 and it holds more QPs than two per SM
  // take at once, else 256 (measured: ragged batch of 4096 QPs 1.17x mixed,
  // 1.26x FP64 at 128 threads; large stages of nu + nx = 192 1.6x slower at
  // 128; a bucket that fits the GPU at 256 threads finishes sooner with them,
  // as the server's micro-batches do)
  const int nsm = b->block_threads > 0 ? 0 : device_sms();
  b->shape_b.threads = b->block_threads > 0 ? b->block_threads
                       : (b->shape_b.nvmax <= kAutoThreadsNv && nsm > 0 && nqp - nw > 2 * nsm) ? 128
                                                                                               : 256;
  b->shape_b.tc_off = b->tensor_cores ? 0 : 1;
}

}  // namespace

extern "C" {

size_t gq_batch_memsize(int nqp, const int* dims, size_t dims_len, const int* stage_slot) {
  (void)stage_slot;
  Counts c = count_stages(nqp, dims, dims_len);
  if (!c.ok) return 0;
  return handle_bytes(nqp, c.n_stages, hash_capacity(c.n_stages));
}

int gq_batch_create(int nqp, const int* dims, size_t dims_len, const int* stage_slot, void* mem,
                    size_t mem_bytes, gq_batch** out) {
  return gq_batch_create_soft(nqp, dims, dims_len, stage_slot, nullptr, mem, mem_bytes, out);
}

int gq_batch_create_soft(int nqp, const int* dims, size_t dims_len, const int* stage_slot, const int* stage_ns,
                         void* mem, size_t mem_bytes, gq_batch** out) {
  if (out == nullptr || mem == nullptr) return fail(GQ_ERR_ARG, "mem and out must be non-NULL");
  *out = nullptr;
  if (reinterpret_cast<uintptr_t>(mem) % 16) return fail(GQ_ERR_ARG, "mem must be 16-byte aligned");
  Counts c = count_stages(nqp, dims, dims_len);
  if (!c.ok) return GQ_ERR_DIMS;
  const int64_t cap = hash_capacity(c.n_stages);
  const size_t need = handle_bytes(nqp, c.n_stages, cap);
  if (mem_bytes < need) return fail(GQ_ERR_SIZE, "handle memory %zu < %zu bytes", mem_bytes, need);

  char* p = static_cast<char*>(mem);
  gq_batch* b = reinterpret_cast<gq_batch*>(p);
  std::memset(b, 0, sizeof(gq_batch));
  p += align_up(sizeof(gq_batch), 64);
  b->qp = reinterpret_cast<QpDesc*>(p);
  p += align_up((int64_t)nqp * sizeof(QpDesc), 64);
  b->st = reinterpret_cast<StageDesc*>(p);
  p += align_up(c.n_stages * sizeof(StageDesc), 64);
  b->order = reinterpret_cast<int32_t*>(p);
  p += align_up((int64_t)nqp * sizeof(int32_t), 64);
  b->slot_stage = reinterpret_cast<int32_t*>(p);
  p += align_up(c.n_stages * sizeof(int32_t), 64);
  b->hash = reinterpret_cast<SlotEntry*>(p);
  b->hash_cap = cap;
  for (int64_t i = 0; i < cap; ++i) b->hash[i].key = -1;
  b->nqp = nqp;
  b->n_stages = c.n_stages;

  // walk the dims: stage descriptors, vector offsets, data blocks
  int64_t var = 0, eq = 0, side = 0, data = 0, fac = 0, slots = 0;
  int nvmax = 0, nxmax = 0, ngmax = 0, nstmax = 0, nemax = 0, nsidemax = 0;
  int64_t datamax = 0;
  size_t pos = 0;
  int64_t si = 0;
  for (int q = 0; q < nqp; ++q) {
    const int N = dims[pos++];
    QpDesc& d = b->qp[q];
    std::memset(&d, 0, sizeof(d));
    d.N = N;
    d.stage0 = (int32_t)si;
    d.var0 = (int32_t)var;
    d.eq0 = (int32_t)eq;
    d.side0 = (int32_t)side;
    nstmax = std::max(nstmax, N + 1);
    double cost = 0.0;
    for (int n = 0; n <= N; ++n, ++si) {
      const int* dn = dims + pos + 5 * n;
      StageDesc& s = b->st[si];
      s.nx = dn[0];
      s.nu = dn[1];
      s.nbx = dn[2];
      s.nbu = dn[3];
      s.ng = dn[4];
      s.nx1 = (n < N) ? dims[pos + 5 * (n + 1)] : 0;
      const int nv = s.nx + s.nu, nb = s.nbx + s.nbu, nc = nb + s.ng;
      s.ns = stage_ns ? stage_ns[si] : 0;
      if (s.ns < 0 || s.ns > nc)
        return fail(GQ_ERR_DIMS, "QP %d stage %d: %d slacks for %d constraints", q, n, s.ns, nc);
      s.var = (int32_t)var;
      s.eq = (int32_t)eq;
      s.side = (int32_t)side;
      s.fac = fac;
      var += nv + 2 * s.ns;
      d.nsoft += s.ns;
      eq += s.nx1;
      side += 2 * nc + 2 * s.ns;
      fac += fac_block_elems(nv);
      nvmax = std::max(nvmax, nv);
      nxmax = std::max(nxmax, s.nx);
      nemax = std::max(nemax, n == 0 ? nv : s.nu);
      ngmax = std::max(ngmax, s.ng);
      d.nvmax = std::max(d.nvmax, nv);
      d.nxmax = std::max(d.nxmax, s.nx);
      cost += (double)s.nx1 * s.nx1 * nv + (double)s.nx1 * nv * nv + (double)nv * nv * nv / 3.0 +
              (double)s.ng * nv * nv;
      const StageData lay = stage_data_layout(s);
      datamax = std::max(datamax, lay.size);
      const int slot = stage_slot ? stage_slot[si] : -1;
      if (slot < 0) {
        s.data = data;
        data += lay.size;
        b->slot_stage[slots++] = (int32_t)si;
      } else {
        int64_t h = ((uint64_t)slot * 0x9E3779B97F4A7C15ull) & (cap - 1);
        while (b->hash[h].key != -1 && b->hash[h].key != slot) h = (h + 1) & (cap - 1);
        if (b->hash[h].key == -1) {
          b->hash[h].key = slot;
          b->hash[h].block = data;
          b->hash[h].stage = (int32_t)si;
          s.data = data;
          data += lay.size;
          b->slot_stage[slots++] = (int32_t)si;
        } else {
          const StageDesc& f = b->st[b->hash[h].stage];
          if (f.nx != s.nx || f.nu != s.nu || f.nx1 != s.nx1 || f.nbx != s.nbx || f.nbu != s.nbu ||
              f.ng != s.ng || f.ns != s.ns)
            return fail(GQ_ERR_DIMS, "QP %d stage %d shares slot %d with a stage of other sizes", q, n,
                        slot);
          s.data = b->hash[h].block;
        }
      }
    }
    pos += 5 * (size_t)(N + 1);
    d.nvt = (int32_t)(var - d.var0);
    d.neqt = (int32_t)(eq - d.eq0);
    d.nsidet = (int32_t)(side - d.side0);
    d.cost = cost;
    nsidemax = std::max(nsidemax, d.nsidet);
  }
  if (var >= INT32_MAX || eq >= INT32_MAX || side >= INT32_MAX)
    return fail(GQ_ERR_DIMS, "batch too large for 32-bit vector offsets");

  b->warp_max_nv = kWarpMaxNv;
  b->block_threads = 0;
  b->tensor_cores = 1;
  plan_buckets(b);
  // the block kernel keeps its stage matrices in a per-QP slice of a global
  // scratch region (read through L1/L2): shared memory then holds only
  // vectors and the stage ring, so two blocks of 256 threads fit an SM.  On
  // the ragged workload this ran 1.5x faster than matrices in shared memory
  // at one block per SM (measured), and it is the only layout for stages
  // whose matrices exceed shared memory.  The scratch is sized for every QP
  // in the block bucket, so that any schedule (gq_set_schedule) fits it.
  const int64_t matg_elems = (int64_t)nqp * block_mat_elems(bucket_shape(b, 0, nqp, true));

  Layout& L = b->L;
  int64_t o = 0;
  L.qpdesc = o;
  o = align_up(o + (int64_t)nqp * sizeof(QpDesc), 256);
  L.stagedesc = o;
  o = align_up(o + c.n_stages * sizeof(StageDesc), 256);
  L.order = o;
  o = align_up(o + (int64_t)nqp * 4, 256);
  L.slots = o;
  o = align_up(o + slots * 4, 256);
  L.data = o;
  o = align_up(o + data * 8, 256);
  L.in_bytes = o;

  o = 0;
  L.stats = o;
  o = align_up(o + (int64_t)nqp * sizeof(gq_stats), 256);
  L.y = o;
  o = align_up(o + var * 8, 256);
  L.pi = o;
  o = align_up(o + eq * 8, 256);
  L.lam = o;
  o = align_up(o + side * 8, 256);
  L.t = o;
  o = align_up(o + side * 8, 256);
  L.sol_bytes = o;

  o = 0;
  int64_t* vecs[] = {&L.rg, &L.rb, &L.rd, &L.rm, &L.dy, &L.dpi, &L.dlam, &L.dt, &L.lp,
                     &L.rg2, &L.rb2, &L.dy2, &L.dpi2, &L.dlam2, &L.dt2, &L.tinv};
  const int64_t lens[] = {var, eq, side, side, var, eq, side, side, var, var, eq, var, eq, side, side, side};
  for (int i = 0; i < 16; ++i) {
    *vecs[i] = o;
    o = align_up(o + lens[i] * 8, 256);
  }
  L.fac = o;
  o = align_up(o + fac * 8, 256);
  L.data32 = o;
  o = align_up(o + data * 4, 256);
  L.data32lo = o;
  o = align_up(o + data * 4, 256);
  L.matg = o;
  o = align_up(o + matg_elems * 8, 256);
  L.queue = o;
  o = align_up(o + kQueueSlots * 4, 256);
  L.ws_bytes = o;

  gq_sizes& z = b->sizes;
  z.in_bytes = (size_t)L.in_bytes;
  z.sol_bytes = (size_t)L.sol_bytes;
  z.ws_bytes = (size_t)L.ws_bytes;
  z.n_stages = c.n_stages;
  z.n_slots = slots;
  z.nv_total = var;
  z.neq_total = eq;
  z.nside_total = side;
  z.nv_max = nvmax;
  z.nx_max = nxmax;
  b->ngmax = ngmax;
  (void)nstmax;
  (void)nemax;
  (void)nsidemax;
  (void)datamax;
  b->n_slots = slots;
  b->magic = kMagic;
  *out = b;
  return GQ_OK;
}

int gq_batch_sizes(const gq_batch* b, gq_sizes* out) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (out == nullptr) return fail(GQ_ERR_ARG, "out is NULL");
  *out = b->sizes;
  return GQ_OK;
}

int gq_batch_attach(gq_batch* b, void* host_in, void* host_sol, void* dev_in, void* dev_sol,
                    void* dev_ws) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (dev_in == nullptr || dev_sol == nullptr || dev_ws == nullptr)
    return fail(GQ_ERR_ARG, "device buffers must be non-NULL");
  for (void* p : {dev_in, dev_sol, dev_ws})
    if (reinterpret_cast<uintptr_t>(p) % 256) return fail(GQ_ERR_ARG, "device buffers must be 256-byte aligned");
  for (void* p : {host_in, host_sol})
    if (p && reinterpret_cast<uintptr_t>(p) % 16) return fail(GQ_ERR_ARG, "host buffers must be 16-byte aligned");
  b->host_in = host_in;
  b->host_sol = host_sol;
  b->dev_in = dev_in;
  b->dev_sol = dev_sol;
  b->dev_ws = dev_ws;
  if (host_in) {
    char* h = static_cast<char*>(host_in);
    std::memset(h + b->L.data, 0, (size_t)(b->L.in_bytes - b->L.data));
    // stages with slacks start from a consistent default until gq_set_soft:
    // slack k relaxes constraint k at zero cost with zero lower bounds
    for (int64_t i = 0; i < b->n_slots; ++i) {
      const StageDesc& st = b->st[b->slot_stage[i]];
      if (st.ns == 0) continue;
      const StageData lay = stage_data_layout(st);
      const int nb = st.nbu + st.nbx, nc = nb + st.ng, nv = st.nx + st.nu;
      int32_t* sidx = reinterpret_cast<int32_t*>(host_data(b) + st.data + lay.box) + nb + nv;
      int32_t* smap = sidx + st.ns;
      for (int k = 0; k < st.ns; ++k) sidx[k] = k;
      for (int c = 0; c < nc; ++c) smap[c] = c < st.ns ? c : -1;
    }
    std::memcpy(h + b->L.qpdesc, b->qp, (size_t)b->nqp * sizeof(QpDesc));
    std::memcpy(h + b->L.stagedesc, b->st, (size_t)b->n_stages * sizeof(StageDesc));
    std::memcpy(h + b->L.order, b->order, (size_t)b->nqp * sizeof(int32_t));
    std::memcpy(h + b->L.slots, b->slot_stage, (size_t)b->n_slots * sizeof(int32_t));
  }
  return GQ_OK;
}

int gq_set_dynamics(gq_batch* b, int qp, int n, const double* A, int lda, const double* B, int ldb,
                    const double* bvec) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  if (n == b->qp[qp].N) return fail(GQ_ERR_ARG, "stage %d is terminal: no dynamics", n);
  const int nx = s->nx, nu = s->nu, nx1 = s->nx1;
  if ((nx && A == nullptr) || (nu && B == nullptr) || bvec == nullptr)
    return fail(GQ_ERR_ARG, "dynamics pointers must be non-NULL");
  if ((nx && lda < nx1) || (nu && ldb < nx1)) return fail(GQ_ERR_ARG, "leading dimension too small");
  const StageData lay = stage_data_layout(*s);
  double* D = host_data(b) + s->data;
  for (int i = 0; i < nu; ++i)
    for (int k = 0; k < nx1; ++k) D[lay.BAt + (int64_t)i * lay.ldb + k] = B[k + (int64_t)i * ldb];
  for (int i = 0; i < nx; ++i)
    for (int k = 0; k < nx1; ++k) D[lay.BAt + (int64_t)(nu + i) * lay.ldb + k] = A[k + (int64_t)i * lda];
  for (int k = 0; k < nx1; ++k) D[lay.b + k] = bvec[k];
  if (!finite_all(D + lay.BAt, (nu + nx) * lay.ldb + nx1)) return fail(GQ_ERR_DATA, "non-finite dynamics data");
  return GQ_OK;
}

int gq_set_cost(gq_batch* b, int qp, int n, const double* Q, int ldq, const double* S, int lds,
                const double* R, int ldr, const double* q, const double* r) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int nx = s->nx, nu = s->nu, nv = nx + nu;
  if ((nx && (Q == nullptr || q == nullptr)) || (nu && (R == nullptr || r == nullptr)) ||
      (nx && nu && S == nullptr))
    return fail(GQ_ERR_ARG, "cost pointers must be non-NULL");
  if ((nx && ldq < nx) || (nu && ldr < nu) || (nx && nu && lds < nu))
    return fail(GQ_ERR_ARG, "leading dimension too small");
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < i; ++j) {
      const double a = Q[i + (int64_t)j * ldq], c = Q[j + (int64_t)i * ldq];
      if (!(std::fabs(a - c) <= 1e-12 * (1.0 + std::fabs(a)))) return fail(GQ_ERR_DATA, "Q not symmetric");
    }
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < i; ++j) {
      const double a = R[i + (int64_t)j * ldr], c = R[j + (int64_t)i * ldr];
      if (!(std::fabs(a - c) <= 1e-12 * (1.0 + std::fabs(a)))) return fail(GQ_ERR_DATA, "R not symmetric");
    }
  const StageData lay = stage_data_layout(*s);
  double* D = host_data(b) + s->data;
  double* RSQ = D + lay.RSQ;
  const int64_t lr = lay.ldr;
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j) RSQ[i * lr + j] = R[i + (int64_t)j * ldr];
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nx; ++j) {
      const double v = S[i + (int64_t)j * lds];
      RSQ[i * lr + nu + j] = v;
      RSQ[(int64_t)(nu + j) * lr + i] = v;
    }
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < nx; ++j) RSQ[(int64_t)(nu + i) * lr + nu + j] = Q[i + (int64_t)j * ldq];
  for (int i = 0; i < nu; ++i) D[lay.rq + i] = r[i];
  for (int i = 0; i < nx; ++i) D[lay.rq + nu + i] = q[i];
  if (!finite_all(RSQ, (int)(nv * lr + nv))) return fail(GQ_ERR_DATA, "non-finite cost data");
  return GQ_OK;
}

int gq_set_box(gq_batch* b, int qp, int n, const int* idxbu, const double* lbu, const double* ubu,
               const int* idxbx, const double* lbx, const double* ubx) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int nbu = s->nbu, nbx = s->nbx, nb = nbu + nbx, nc = nb + s->ng;
  if ((nbu && (idxbu == nullptr || lbu == nullptr || ubu == nullptr)) ||
      (nbx && (idxbx == nullptr || lbx == nullptr || ubx == nullptr)))
    return fail(GQ_ERR_ARG, "box pointers must be non-NULL");
  const StageData lay = stage_data_layout(*s);
  double* D = host_data(b) + s->data;
  int32_t* I = reinterpret_cast<int32_t*>(D + lay.box);   // bidx[nb], then bmap[nv]
  for (int k = 0; k < nbu; ++k) {
    if (idxbu[k] < 0 || idxbu[k] >= s->nu) return fail(GQ_ERR_ARG, "idxbu[%d]=%d out of range", k, idxbu[k]);
    for (int j = 0; j < k; ++j)
      if (idxbu[j] == idxbu[k]) return fail(GQ_ERR_ARG, "idxbu has a repeated index %d", idxbu[k]);
    I[k] = idxbu[k];
    D[lay.lo + k] = lbu[k];
    D[lay.hi + k] = ubu[k];
  }
  for (int k = 0; k < nbx; ++k) {
    if (idxbx[k] < 0 || idxbx[k] >= s->nx) return fail(GQ_ERR_ARG, "idxbx[%d]=%d out of range", k, idxbx[k]);
    for (int j = 0; j < k; ++j)
      if (idxbx[j] == idxbx[k]) return fail(GQ_ERR_ARG, "idxbx has a repeated index %d", idxbx[k]);
    I[nbu + k] = s->nu + idxbx[k];
    D[lay.lo + nbu + k] = lbx[k];
    D[lay.hi + nbu + k] = ubx[k];
  }
  for (int k = 0; k < nb; ++k) {
    const double lo = D[lay.lo + k], hi = D[lay.hi + k];
    if (std::isnan(lo) || std::isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY)
      return fail(GQ_ERR_DATA, "box bound %d invalid (lo=%g hi=%g)", k, lo, hi);
  }
  int32_t* M = I + nb;
  const int nv = s->nx + s->nu;
  for (int i = 0; i < nv; ++i) M[i] = -1;
  for (int k = 0; k < nb; ++k) M[I[k]] = k;
  (void)nc;
  return GQ_OK;
}

int gq_set_general(gq_batch* b, int qp, int n, const double* C, int ldc, const double* Dm, int ldd,
                   const double* lg, const double* ug) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int ng = s->ng, nx = s->nx, nu = s->nu, nv = nx + nu, nb = s->nbu + s->nbx;
  if (ng == 0) return GQ_OK;
  if ((nx && C == nullptr) || (nu && Dm == nullptr) || lg == nullptr || ug == nullptr)
    return fail(GQ_ERR_ARG, "general-constraint pointers must be non-NULL");
  if ((nx && ldc < ng) || (nu && ldd < ng)) return fail(GQ_ERR_ARG, "leading dimension too small");
  const StageData lay = stage_data_layout(*s);
  double* D = host_data(b) + s->data;
  for (int g = 0; g < ng; ++g) {
    for (int i = 0; i < nu; ++i) D[lay.DC + (int64_t)g * nv + i] = Dm[g + (int64_t)i * ldd];
    for (int i = 0; i < nx; ++i) D[lay.DC + (int64_t)g * nv + nu + i] = C[g + (int64_t)i * ldc];
    const double lo = lg[g], hi = ug[g];
    if (std::isnan(lo) || std::isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY)
      return fail(GQ_ERR_DATA, "general bound %d invalid (lo=%g hi=%g)", g, lo, hi);
    D[lay.lo + nb + g] = lo;
    D[lay.hi + nb + g] = hi;
  }
  if (!finite_all(D + lay.DC, ng * nv)) return fail(GQ_ERR_DATA, "non-finite general-constraint data");
  return GQ_OK;
}

int gq_set_soft(gq_batch* b, int qp, int n, const int* idxs, const double* Zl, const double* Zu,
                const double* zl, const double* zu, const double* lls, const double* lus) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int ns = s->ns, nb = s->nbu + s->nbx, nc = nb + s->ng, nv = s->nx + s->nu;
  if (ns == 0) return GQ_OK;
  if (!idxs || !Zl || !Zu || !zl || !zu || !lls || !lus) return fail(GQ_ERR_ARG, "slack pointers must be non-NULL");
  const StageData lay = stage_data_layout(*s);
  double* D = host_data(b) + s->data;
  int32_t* I = reinterpret_cast<int32_t*>(D + lay.box);
  int32_t* sidx = I + nb + nv;
  int32_t* smap = sidx + ns;
  for (int c = 0; c < nc; ++c) smap[c] = -1;
  for (int k = 0; k < ns; ++k) {
    if (idxs[k] < 0 || idxs[k] >= nc) return fail(GQ_ERR_ARG, "idxs[%d]=%d out of range", k, idxs[k]);
    if (smap[idxs[k]] >= 0) return fail(GQ_ERR_ARG, "idxs has a repeated index %d", idxs[k]);
    if (!(Zl[k] >= 0.0 && Zu[k] >= 0.0) || !std::isfinite(Zl[k]) || !std::isfinite(Zu[k]) ||
        !std::isfinite(zl[k]) || !std::isfinite(zu[k]) || !std::isfinite(lls[k]) || !std::isfinite(lus[k]))
      return fail(GQ_ERR_DATA, "slack %d: Z must be finite and >= 0, z and the slack bounds finite", k);
    sidx[k] = idxs[k];
    smap[idxs[k]] = k;
    D[lay.Zs + k] = Zl[k];
    D[lay.Zs + ns + k] = Zu[k];
    D[lay.zs + k] = zl[k];
    D[lay.zs + ns + k] = zu[k];
    D[lay.ls + k] = lls[k];
    D[lay.ls + ns + k] = lus[k];
  }
  return GQ_OK;
}

int gq_set_initial_state(gq_batch* b, int qp, const double* x0, int nx0, const double* A0, int lda,
                         const double* b0, const double* S0, int lds, const double* r0, const double* C0, int ldc,
                         const double* lg0, const double* ug0) {
  StageDesc* s;
  int rc = stage_of(b, qp, 0, &s);
  if (rc) return rc;
  if (s->nx != 0) return fail(GQ_ERR_DIMS, "stage 0 of QP %d keeps x_0 (nx_0 = %d): nothing to eliminate", qp, s->nx);
  if (b->qp[qp].N == 0) return fail(GQ_ERR_DIMS, "QP %d has no dynamics to fold x0 into", qp);
  const int nu = s->nu, nx1 = s->nx1, ng = s->ng, nb = s->nbu + s->nbx;
  if (nx0 < 0 || (nx0 > 0 && (x0 == nullptr || A0 == nullptr || (nu && S0 == nullptr) || (ng && C0 == nullptr))))
    return fail(GQ_ERR_ARG, "x0 and its stage-0 matrices must be non-NULL");
  if (b0 == nullptr || (nu && r0 == nullptr) || (ng && (lg0 == nullptr || ug0 == nullptr)))
    return fail(GQ_ERR_ARG, "b0, r0, lg0, ug0 must be non-NULL");
  if (nx0 > 0 && (lda < nx1 || (nu && lds < nu) || (ng && ldc < ng)))
    return fail(GQ_ERR_ARG, "leading dimension too small");
  const StageData lay = stage_data_layout(*s);
  double* D = host_data(b) + s->data;
  // b_0 + A_0 x0, r_0 + S_0 x0, and the general bounds minus C_0 x0
  for (int k = 0; k < nx1; ++k) {
    double v = b0[k];
    for (int j = 0; j < nx0; ++j) v += A0[k + (int64_t)j * lda] * x0[j];
    D[lay.b + k] = v;
  }
  for (int i = 0; i < nu; ++i) {
    double v = r0[i];
    for (int j = 0; j < nx0; ++j) v += S0[i + (int64_t)j * lds] * x0[j];
    D[lay.rq + i] = v;
  }
  for (int g = 0; g < ng; ++g) {
    double cx = 0.0;
    for (int j = 0; j < nx0; ++j) cx += C0[g + (int64_t)j * ldc] * x0[j];
    const double lo = lg0[g] - cx, hi = ug0[g] - cx;  // an infinite bound stays infinite (masked)
    if (std::isnan(lo) || std::isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY)
      return fail(GQ_ERR_DATA, "general bound %d invalid after folding x0 (lo=%g hi=%g)", g, lo, hi);
    D[lay.lo + nb + g] = lo;
    D[lay.hi + nb + g] = hi;
  }
  if (!finite_all(D + lay.b, nx1) || !finite_all(D + lay.rq, nu))
    return fail(GQ_ERR_DATA, "non-finite data after folding x0");
  return GQ_OK;
}

// ---- getters of the staged problem data (inverse of the setters; any
// output pointer may be NULL; column-major outputs with leading dimensions) ----
int gq_get_dynamics(gq_batch* b, int qp, int n, double* A, int lda, double* B, int ldb, double* bvec) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  if (n == b->qp[qp].N) return fail(GQ_ERR_ARG, "stage %d is terminal: no dynamics", n);
  const int nx = s->nx, nu = s->nu, nx1 = s->nx1;
  if ((A && nx && lda < nx1) || (B && nu && ldb < nx1)) return fail(GQ_ERR_ARG, "leading dimension too small");
  const StageData lay = stage_data_layout(*s);
  const double* D = host_data(b) + s->data;
  for (int i = 0; i < nu && B; ++i)
    for (int k = 0; k < nx1; ++k) B[k + (int64_t)i * ldb] = D[lay.BAt + (int64_t)i * lay.ldb + k];
  for (int i = 0; i < nx && A; ++i)
    for (int k = 0; k < nx1; ++k) A[k + (int64_t)i * lda] = D[lay.BAt + (int64_t)(nu + i) * lay.ldb + k];
  for (int k = 0; k < nx1 && bvec; ++k) bvec[k] = D[lay.b + k];
  return GQ_OK;
}

int gq_get_cost(gq_batch* b, int qp, int n, double* Q, int ldq, double* S, int lds, double* R, int ldr, double* q,
                double* r) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int nx = s->nx, nu = s->nu;
  if ((Q && nx && ldq < nx) || (R && nu && ldr < nu) || (S && nu && nx && lds < nu))
    return fail(GQ_ERR_ARG, "leading dimension too small");
  const StageData lay = stage_data_layout(*s);
  const double* D = host_data(b) + s->data;
  const double* RSQ = D + lay.RSQ;
  const int64_t lr = lay.ldr;
  for (int i = 0; i < nu && R; ++i)
    for (int j = 0; j < nu; ++j) R[i + (int64_t)j * ldr] = RSQ[i * lr + j];
  for (int i = 0; i < nu && S; ++i)
    for (int j = 0; j < nx; ++j) S[i + (int64_t)j * lds] = RSQ[i * lr + nu + j];
  for (int i = 0; i < nx && Q; ++i)
    for (int j = 0; j < nx; ++j) Q[i + (int64_t)j * ldq] = RSQ[(int64_t)(nu + i) * lr + nu + j];
  for (int i = 0; i < nu && r; ++i) r[i] = D[lay.rq + i];
  for (int i = 0; i < nx && q; ++i) q[i] = D[lay.rq + nu + i];
  return GQ_OK;
}

int gq_get_box(gq_batch* b, int qp, int n, int* idxbu, double* lbu, double* ubu, int* idxbx, double* lbx,
               double* ubx) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int nbu = s->nbu, nbx = s->nbx;
  const StageData lay = stage_data_layout(*s);
  const double* D = host_data(b) + s->data;
  const int32_t* I = reinterpret_cast<const int32_t*>(D + lay.box);
  for (int k = 0; k < nbu; ++k) {
    if (idxbu) idxbu[k] = I[k];
    if (lbu) lbu[k] = D[lay.lo + k];
    if (ubu) ubu[k] = D[lay.hi + k];
  }
  for (int k = 0; k < nbx; ++k) {
    if (idxbx) idxbx[k] = I[nbu + k] - s->nu;
    if (lbx) lbx[k] = D[lay.lo + nbu + k];
    if (ubx) ubx[k] = D[lay.hi + nbu + k];
  }
  return GQ_OK;
}

int gq_get_general(gq_batch* b, int qp, int n, double* C, int ldc, double* Dm, int ldd, double* lg, double* ug) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int ng = s->ng, nx = s->nx, nu = s->nu, nv = nx + nu, nb = s->nbu + s->nbx;
  if ((C && nx && ng && ldc < ng) || (Dm && nu && ng && ldd < ng)) return fail(GQ_ERR_ARG, "leading dimension too small");
  const StageData lay = stage_data_layout(*s);
  const double* D = host_data(b) + s->data;
  for (int g = 0; g < ng; ++g) {
    for (int i = 0; i < nu && Dm; ++i) Dm[g + (int64_t)i * ldd] = D[lay.DC + (int64_t)g * nv + i];
    for (int i = 0; i < nx && C; ++i) C[g + (int64_t)i * ldc] = D[lay.DC + (int64_t)g * nv + nu + i];
    if (lg) lg[g] = D[lay.lo + nb + g];
    if (ug) ug[g] = D[lay.hi + nb + g];
  }
  return GQ_OK;
}

int gq_get_soft(gq_batch* b, int qp, int n, int* ns_out, int* idxs, double* Zl, double* Zu, double* zl, double* zu,
                double* lls, double* lus) {
  StageDesc* s;
  int rc = stage_of(b, qp, n, &s);
  if (rc) return rc;
  const int ns = s->ns, nb = s->nbu + s->nbx, nv = s->nx + s->nu;
  if (ns_out) *ns_out = ns;
  if (ns == 0) return GQ_OK;
  const StageData lay = stage_data_layout(*s);
  const double* D = host_data(b) + s->data;
  const int32_t* sidx = reinterpret_cast<const int32_t*>(D + lay.box) + nb + nv;
  for (int k = 0; k < ns; ++k) {
    if (idxs) idxs[k] = sidx[k];
    if (Zl) Zl[k] = D[lay.Zs + k];
    if (Zu) Zu[k] = D[lay.Zs + ns + k];
    if (zl) zl[k] = D[lay.zs + k];
    if (zu) zu[k] = D[lay.zs + ns + k];
    if (lls) lls[k] = D[lay.ls + k];
    if (lus) lus[k] = D[lay.ls + ns + k];
  }
  return GQ_OK;
}

int gq_set_guess(gq_batch* b, int qp, const double* y, const double* pi, const double* lam,
                 const double* t) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (qp < 0 || qp >= b->nqp) return fail(GQ_ERR_ARG, "qp out of range");
  if (b->host_sol == nullptr) return fail(GQ_ERR_STATE, "host_sol not attached");
  const QpDesc& d = b->qp[qp];
  char* h = static_cast<char*>(b->host_sol);
  if (y) std::memcpy(h + b->L.y + 8 * (int64_t)d.var0, y, 8 * (size_t)d.nvt);
  if (pi) std::memcpy(h + b->L.pi + 8 * (int64_t)d.eq0, pi, 8 * (size_t)d.neqt);
  if (lam) std::memcpy(h + b->L.lam + 8 * (int64_t)d.side0, lam, 8 * (size_t)d.nsidet);
  if (t) std::memcpy(h + b->L.t + 8 * (int64_t)d.side0, t, 8 * (size_t)d.nsidet);
  return GQ_OK;
}

static int copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, void* stream,
                const char* what) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, what);
  return GQ_OK;
}

int gq_upload(gq_batch* b, void* stream) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (!b->host_in || !b->dev_in) return fail(GQ_ERR_STATE, "buffers not attached");
  return copy(b->dev_in, b->host_in, b->sizes.in_bytes, cudaMemcpyHostToDevice, stream, "upload");
}

int gq_upload_sol(gq_batch* b, void* stream) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (!b->host_sol || !b->dev_sol) return fail(GQ_ERR_STATE, "buffers not attached");
  return copy(b->dev_sol, b->host_sol, b->sizes.sol_bytes, cudaMemcpyHostToDevice, stream, "upload_sol");
}

int gq_download(gq_batch* b, void* stream) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (!b->host_sol || !b->dev_sol) return fail(GQ_ERR_STATE, "buffers not attached");
  return copy(b->host_sol, b->dev_sol, b->sizes.sol_bytes, cudaMemcpyDeviceToHost, stream, "download");
}

// the classical Riccati variant is implemented in the block kernel only
static int check_variant(const gq_batch* b, const gq_ipm_arg* a) {
  if (a->riccati == 1 && b->nwarp > 0)
    return fail(GQ_ERR_ARG,
                "classical Riccati runs in the block kernel: set the schedule's warp_max_nv to 0 "
                "(%d QPs are in the warp bucket)",
                b->nwarp);
  if (a->riccati == 1 && a->mode == GQ_MODE_ROBUST)
    return fail(GQ_ERR_ARG, "the robust mode's array algorithm is the square-root Riccati variant");
  return GQ_OK;
}

// Kernel arguments for the batch's layout over the given device buffers (the
// attached ones for gq_solve; the caller's and the static scratch for
// gq_solve_noalloc, which leaves the handle untouched).
static int make_kernel_batch_on(const gq_batch* b, void* dev_in, void* dev_sol, void* dev_ws, Batch* k) {
  if (!dev_in || !dev_sol || !dev_ws) return fail(GQ_ERR_STATE, "device buffers not attached");
  char* in = static_cast<char*>(dev_in);
  char* so = static_cast<char*>(dev_sol);
  char* ws = static_cast<char*>(dev_ws);
  const Layout& L = b->L;
  k->nqp = b->nqp;
  k->nvmax = b->sizes.nv_max;
  k->nxmax = b->sizes.nx_max;
  k->ngmax = b->ngmax;
  k->qp = reinterpret_cast<const QpDesc*>(in + L.qpdesc);
  k->st = reinterpret_cast<const StageDesc*>(in + L.stagedesc);
  k->order = reinterpret_cast<const int32_t*>(in + L.order);
  k->slots = reinterpret_cast<const int32_t*>(in + L.slots);
  k->nslots = (int32_t)b->n_slots;
  k->data = reinterpret_cast<const double*>(in + L.data);
  k->data32 = reinterpret_cast<float*>(ws + L.data32);
  k->data32lo = reinterpret_cast<float*>(ws + L.data32lo);
  k->stats = reinterpret_cast<gq_stats*>(so + L.stats);
  k->y = reinterpret_cast<double*>(so + L.y);
  k->pi = reinterpret_cast<double*>(so + L.pi);
  k->lam = reinterpret_cast<double*>(so + L.lam);
  k->t = reinterpret_cast<double*>(so + L.t);
  double** w[] = {&k->rg, &k->rb, &k->rd, &k->rm, &k->dy, &k->dpi, &k->dlam, &k->dt, &k->lp,
                  &k->rg2, &k->rb2, &k->dy2, &k->dpi2, &k->dlam2, &k->dt2, &k->tinv};
  const int64_t off[] = {L.rg, L.rb, L.rd, L.rm, L.dy, L.dpi, L.dlam, L.dt, L.lp,
                         L.rg2, L.rb2, L.dy2, L.dpi2, L.dlam2, L.dt2, L.tinv};
  for (int i = 0; i < 16; ++i) *w[i] = reinterpret_cast<double*>(ws + off[i]);
  k->fac = ws + L.fac;
  k->matg = reinterpret_cast<double*>(ws + L.matg);
  k->queue = reinterpret_cast<int32_t*>(ws + L.queue);
  if (b->nwarp < b->nqp) {
    const size_t smem = tc_shape(b->shape_b) ? ipm_tc_smem_bytes(*k, b->shape_b) : ipm_smem_bytes(*k, b->shape_b);
    if (smem > kMaxSmem)
      return fail(GQ_ERR_DIMS,
                  "largest stage (nu+nx=%d, nx=%d) needs %zu bytes of shared memory per block (limit %zu)",
                  b->shape_b.nvmax, b->shape_b.nxmax, smem, kMaxSmem);
  }
  if (b->nwarp > 0) {
    const size_t smem = warp_plan(*k, b->shape_w, 8).bytes;
    if (smem > kMaxSmem)
      return fail(GQ_ERR_DIMS, "warp bucket needs %zu bytes of shared memory per block (limit %zu)", smem, kMaxSmem);
  }
  return GQ_OK;
}

static int make_kernel_batch(const gq_batch* b, Batch* k) {
  return make_kernel_batch_on(b, b->dev_in, b->dev_sol, b->dev_ws, k);
}

// both buckets of the batch, in order, on one stream
static cudaError_t launch_all(gq_batch* b, const Batch& k, const gq_ipm_arg& arg, cudaStream_t st, LaunchKind kind,
                              double sigma_mu, const DirOut* out) {
  const int32_t* ord = k.order;
  cudaError_t e = cudaSuccess;
  if (arg.precision == GQ_PREC_MIXED && kind != LaunchKind::Residuals) e = launch_mirror(k, st);
  if (e != cudaSuccess) return e;
  e = launch_warp_ipm(k, b->shape_w, arg, st, kind, sigma_mu, out, ord, b->nwarp);
  if (e != cudaSuccess) return e;
  // block-kernel variant: slack elimination, tensor-core products of large
  // FP32 stages, or neither
  bool tc = !b->soft_block && tc_shape(b->shape_b) && arg.precision == GQ_PREC_MIXED &&
            (b->shape_b.threads == 256);
  if (tc && b->tensor_cores == 1) {
    // automatic: only while the block bucket leaves at least every other SM
    // idle (measured on the large-stage batch: 1.5 % faster at 76 QPs on 152
    // SMs, 1.6 % slower at 152, 10 % slower at 256)
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
      nsm = 0;
    tc = 2 * (b->nqp - b->nwarp) <= nsm;
  }
  return (b->soft_block ? launch_ipm_soft : (tc ? launch_ipm_tc : launch_ipm))(k, b->shape_b, arg, st, kind,
                                                                            sigma_mu, out, ord + b->nwarp,
                                                                            b->nqp - b->nwarp);
}

static int check_arg(const gq_ipm_arg* a) {
  if (a == nullptr) return fail(GQ_ERR_ARG, "arg is NULL");
  if (a->mode != GQ_MODE_SPEED && a->mode != GQ_MODE_BALANCE && a->mode != GQ_MODE_ROBUST)
    return fail(GQ_ERR_ARG, "unknown mode");
  if (a->precision != GQ_PREC_FP64 && a->precision != GQ_PREC_MIXED) return fail(GQ_ERR_ARG, "unknown precision");
  if (a->iter_max < 0 || a->ir_steps < 0 || a->ir_steps > 64) return fail(GQ_ERR_ARG, "iter_max/ir_steps out of range");
  if (a->warm_start < 0 || a->warm_start > 2) return fail(GQ_ERR_ARG, "warm_start must be 0, 1 or 2");
  if (a->riccati != 0 && a->riccati != 1) return fail(GQ_ERR_ARG, "riccati must be 0 (square-root) or 1 (classical)");
  if (!(a->tau_b > 0.0 && a->tau_b <= 1.0)) return fail(GQ_ERR_ARG, "tau_b must be in (0, 1]");
  if (!(a->lam_min > 0.0 && a->t_min > 0.0)) return fail(GQ_ERR_ARG, "lam_min and t_min must be positive");
  if (!(a->reg_prim >= 0.0)) return fail(GQ_ERR_ARG, "reg_prim must be >= 0");
  if (a->timeout_ns < 0) return fail(GQ_ERR_ARG, "timeout_ns must be >= 0");
  if (!(a->ir_fail_ratio >= 0.0)) return fail(GQ_ERR_ARG, "ir_fail_ratio must be >= 0");
  return GQ_OK;
}

int gq_solve(gq_batch* b, const gq_ipm_arg* arg, void* stream) {
  int rc = check_batch(b);
  if (rc) return rc;
  rc = check_arg(arg);
  if (rc) return rc;
  rc = check_variant(b, arg);
  if (rc) return rc;
  Batch k;
  rc = make_kernel_batch(b, &k);
  if (rc) return rc;
  cudaError_t e = launch_all(b, k, *arg, static_cast<cudaStream_t>(stream), LaunchKind::Solve, 0.0, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "solve launch");
  return GQ_OK;
}

int gq_get_schedule(const gq_batch* b, gq_schedule* out) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (out == nullptr) return fail(GQ_ERR_ARG, "out is NULL");
  out->warp_max_nv = b->warp_max_nv;
  out->block_threads = b->block_threads;
  out->tensor_cores = b->tensor_cores;
  out->warp_qps = b->nwarp;
  out->block_qps = b->nqp - b->nwarp;
  return GQ_OK;
}

int gq_set_schedule(gq_batch* b, const gq_schedule* sch) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (sch == nullptr) return fail(GQ_ERR_ARG, "schedule is NULL");
  if (sch->warp_max_nv < 0 || sch->warp_max_nv > kWarpMaxNv)
    return fail(GQ_ERR_ARG, "warp_max_nv must be in 0..%d", kWarpMaxNv);
  if (sch->block_threads != 0 && sch->block_threads != 64 && sch->block_threads != 128 && sch->block_threads != 256)
    return fail(GQ_ERR_ARG, "block_threads must be 0 (automatic), 64, 128 or 256");
  if (sch->tensor_cores < 0 || sch->tensor_cores > 2) return fail(GQ_ERR_ARG, "tensor_cores must be 0, 1 or 2");
  b->warp_max_nv = sch->warp_max_nv;
  b->block_threads = sch->block_threads;
  b->tensor_cores = sch->tensor_cores;
  plan_buckets(b);
  if (b->host_in)
    std::memcpy(static_cast<char*>(b->host_in) + b->L.order, b->order, (size_t)b->nqp * sizeof(int32_t));
  return GQ_OK;
}

int gq_autotune(gq_batch* b, const gq_ipm_arg* arg, void* stream, int reps, gq_schedule* best, double* best_ms) {
  int rc = check_batch(b);
  if (rc) return rc;
  rc = check_arg(arg);
  if (rc) return rc;
  if (reps < 1 || reps > 100) return fail(GQ_ERR_ARG, "reps must be in 1..100");
  if (!b->host_in) return fail(GQ_ERR_STATE, "host_in not attached");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // warp threshold x block threads x tensor-core products
  gq_schedule cands[4 * 3 * 2];
  int ncand = 0;
  for (int wm : {kWarpMaxNv, 24, 16, 0})
    for (int th : {256, 128, 64})
      for (int tcs : {2, 0}) cands[ncand++] = gq_schedule{wm, th, 0, 0, tcs};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double tbest = -1.0;
  gq_schedule sbest = cands[0];
  int seen_nwarp[4 * 3 * 2], seen_threads[4 * 3 * 2], seen_tc[4 * 3 * 2], nseen = 0;
  for (int ci = 0; ci < ncand; ++ci) {
    const gq_schedule& c = cands[ci];
    if (e != cudaSuccess) break;
    gq_schedule probe = c;
    rc = gq_set_schedule(b, &probe);
    if (rc) break;
    // a candidate that runs the same kernels as an earlier one is skipped
    // (block size without block-bucket QPs; tensor cores where no stage uses them)
    const int thr = b->nqp > b->nwarp ? b->shape_b.threads : 0;
    const int tcu = (b->nqp > b->nwarp && thr == 256 && arg->precision == GQ_PREC_MIXED) ? c.tensor_cores : 0;
    bool dup = false;
    for (int k = 0; k < nseen; ++k)
      dup = dup || (seen_nwarp[k] == b->nwarp && seen_threads[k] == thr && seen_tc[k] == tcu);
    if (dup) continue;
    seen_nwarp[nseen] = b->nwarp;
    seen_threads[nseen] = thr;
    seen_tc[nseen++] = tcu;
    rc = gq_upload(b, stream);
    if (rc) break;
    rc = gq_solve(b, arg, stream);  // warm-up
    if (rc) break;
    e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess && rc == GQ_OK; ++r) rc = gq_solve(b, arg, stream);
    if (rc) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    const double per = (double)ms / reps;
    if (tbest < 0.0 || per < tbest) {
      tbest = per;
      sbest = c;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  if (rc) return rc;
  rc = gq_set_schedule(b, &sbest);
  if (rc) return rc;
  rc = gq_upload(b, stream);
  if (rc) return rc;
  if (best) gq_get_schedule(b, best);
  if (best_ms) *best_ms = tbest;
  return GQ_OK;
}

int gq_residuals(gq_batch* b, void* stream) {
  int rc = check_batch(b);
  if (rc) return rc;
  Batch k;
  rc = make_kernel_batch(b, &k);
  if (rc) return rc;
  gq_ipm_arg a;
  gq_ipm_arg_default(&a, GQ_MODE_SPEED, GQ_PREC_FP64);
  cudaError_t e = launch_all(b, k, a, static_cast<cudaStream_t>(stream), LaunchKind::Residuals, 0.0, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "residual launch");
  return GQ_OK;
}

int gq_newton_step(gq_batch* b, const gq_ipm_arg* arg, double sigma_mu, void* dev_dir, void* stream) {
  int rc = check_batch(b);
  if (rc) return rc;
  rc = check_arg(arg);
  if (rc) return rc;
  rc = check_variant(b, arg);
  if (rc) return rc;
  if (dev_dir == nullptr || reinterpret_cast<uintptr_t>(dev_dir) % 256)
    return fail(GQ_ERR_ARG, "dev_dir must be non-NULL and 256-byte aligned");
  if (!std::isfinite(sigma_mu) || sigma_mu < 0) return fail(GQ_ERR_ARG, "sigma_mu must be finite and >= 0");
  Batch k;
  rc = make_kernel_batch(b, &k);
  if (rc) return rc;
  char* d = static_cast<char*>(dev_dir);
  DirOut out;
  out.dy = reinterpret_cast<double*>(d + b->L.y);
  out.dpi = reinterpret_cast<double*>(d + b->L.pi);
  out.dlam = reinterpret_cast<double*>(d + b->L.lam);
  out.dt = reinterpret_cast<double*>(d + b->L.t);
  cudaError_t e = launch_all(b, k, *arg, static_cast<cudaStream_t>(stream), LaunchKind::NewtonStep, sigma_mu, &out);
  if (e != cudaSuccess) return cuda_fail(e, "newton-step launch");
  return GQ_OK;
}

int gq_get_stage_sol(const gq_batch* b, int qp, int n, double* u, double* x, double* pi, double* lam,
                     double* t) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (qp < 0 || qp >= b->nqp) return fail(GQ_ERR_ARG, "qp out of range");
  const QpDesc& d = b->qp[qp];
  if (n < 0 || n > d.N) return fail(GQ_ERR_ARG, "stage out of range");
  if (b->host_sol == nullptr) return fail(GQ_ERR_STATE, "host_sol not attached");
  const StageDesc& s = b->st[d.stage0 + n];
  const char* h = static_cast<const char*>(b->host_sol);
  const double* Y = reinterpret_cast<const double*>(h + b->L.y) + s.var;
  if (u) std::memcpy(u, Y, 8 * (size_t)s.nu);
  if (x) std::memcpy(x, Y + s.nu, 8 * (size_t)s.nx);
  if (pi && n < d.N) std::memcpy(pi, reinterpret_cast<const double*>(h + b->L.pi) + s.eq, 8 * (size_t)s.nx1);
  const int nside = 2 * (s.nbu + s.nbx + s.ng + s.ns);
  if (lam) std::memcpy(lam, reinterpret_cast<const double*>(h + b->L.lam) + s.side, 8 * (size_t)nside);
  if (t) std::memcpy(t, reinterpret_cast<const double*>(h + b->L.t) + s.side, 8 * (size_t)nside);
  return GQ_OK;
}

int gq_get_stage_slacks(const gq_batch* b, int qp, int n, double* sl, double* su) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (qp < 0 || qp >= b->nqp) return fail(GQ_ERR_ARG, "qp out of range");
  const QpDesc& d = b->qp[qp];
  if (n < 0 || n > d.N) return fail(GQ_ERR_ARG, "stage out of range");
  if (b->host_sol == nullptr) return fail(GQ_ERR_STATE, "host_sol not attached");
  const StageDesc& s = b->st[d.stage0 + n];
  const double* Y = reinterpret_cast<const double*>(static_cast<const char*>(b->host_sol) + b->L.y) + s.var;
  if (sl) std::memcpy(sl, Y + s.nu + s.nx, 8 * (size_t)s.ns);
  if (su) std::memcpy(su, Y + s.nu + s.nx + s.ns, 8 * (size_t)s.ns);
  return GQ_OK;
}

int gq_get_stats(const gq_batch* b, int qp, gq_stats* out) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (qp < 0 || qp >= b->nqp || out == nullptr) return fail(GQ_ERR_ARG, "qp out of range or out NULL");
  if (b->host_sol == nullptr) return fail(GQ_ERR_STATE, "host_sol not attached");
  const char* h = static_cast<const char*>(b->host_sol);
  std::memcpy(out, h + b->L.stats + (int64_t)qp * sizeof(gq_stats), sizeof(gq_stats));
  return GQ_OK;
}

int gq_get_statuses(const gq_batch* b, int32_t* status, int32_t* iters) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (status == nullptr) return fail(GQ_ERR_ARG, "status is NULL");
  if (b->host_sol == nullptr) return fail(GQ_ERR_STATE, "host_sol not attached");
  const gq_stats* st = reinterpret_cast<const gq_stats*>(static_cast<const char*>(b->host_sol) + b->L.stats);
  for (int q = 0; q < b->nqp; ++q) {
    status[q] = st[q].status;
    if (iters) iters[q] = st[q].iters;
  }
  return GQ_OK;
}

int gq_get_sol_offsets(const gq_batch* b, int qp, int64_t off[8]) {
  int rc = check_batch(b);
  if (rc) return rc;
  if (qp < 0 || qp >= b->nqp || off == nullptr) return fail(GQ_ERR_ARG, "qp out of range or off NULL");
  const QpDesc& d = b->qp[qp];
  off[0] = b->L.y / 8 + d.var0;
  off[1] = b->L.pi / 8 + d.eq0;
  off[2] = b->L.lam / 8 + d.side0;
  off[3] = b->L.t / 8 + d.side0;
  off[4] = d.nvt;
  off[5] = d.neqt;
  off[6] = d.nsidet;
  off[7] = d.nsidet;
  return GQ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve without any device allocation by the caller or the library.
//
// For callers that cannot allocate device memory at solve time: code running
// under a fixed memory budget that forbids runtime allocation (safety-critical
// embedded controllers), plug-ins whose host application owns the allocator,
// or solves issued from inside a region where allocation would synchronise or
// fail.  They still pass the input and solution buffers; the workspace comes
// from one file-scope device array of GQ_NOALLOC_SCRATCH_BYTES, which every
// GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) unsigned char g_noalloc_scratch[GQ_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (set-up on the
// first call per device; the host-side name is only a stand-in)
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(GQ_ERR_ARG, "noalloc: device index %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GQ_OK;
}

}  // namespace

extern "C" size_t gq_noalloc_scratch_bytes(void) { return (size_t)GQ_NOALLOC_SCRATCH_BYTES; }

extern "C" int gq_solve_noalloc(gq_batch* b, const gq_ipm_arg* arg, void* dev_in, void* dev_sol, void* stream) {
  int rc = check_batch(b);
  if (rc) return rc;
  rc = check_arg(arg);
  if (rc) return rc;
  rc = check_variant(b, arg);
  if (rc) return rc;
  if (dev_in == nullptr || dev_sol == nullptr) return fail(GQ_ERR_ARG, "noalloc: dev_in and dev_sol must be non-NULL");
  if (reinterpret_cast<uintptr_t>(dev_in) % 256 || reinterpret_cast<uintptr_t>(dev_sol) % 256)
    return fail(GQ_ERR_ARG, "noalloc: device buffers must be 256-byte aligned");
  if (b->sizes.ws_bytes > (size_t)GQ_NOALLOC_SCRATCH_BYTES)
    return fail(GQ_ERR_SIZE, "noalloc: batch needs %zu workspace bytes, the static scratch holds %zu (use gq_solve)",
                b->sizes.ws_bytes, (size_t)GQ_NOALLOC_SCRATCH_BYTES);
  void* ws = nullptr;
  rc = noalloc_scratch(&ws);
  if (rc) return rc;
  // the same kernel arguments as gq_solve, built over the caller's buffers and
  // the static scratch; the handle's attached pointers are not touched, so
  // other threads using the handle meanwhile see no change
  Batch k;
  rc = make_kernel_batch_on(b, dev_in, dev_sol, ws, &k);
  if (rc) return rc;
  cudaError_t e = launch_all(b, k, *arg, static_cast<cudaStream_t>(stream), LaunchKind::Solve, 0.0, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "noalloc solve launch");
  return GQ_OK;
}

// ---------------------------------------------------------------------------
// Copy the problem data of QP src_qp of batch src into QP dst_qp of batch dst
// (host staging to host staging; both QPs must have identical stage sizes).
// Used by the serving loop to assemble micro-batches from packed requests.
// ---------------------------------------------------------------------------
extern "C" int gq_copy_qp(gq_batch* dst, int dst_qp, const gq_batch* src, int src_qp) {
  int rc = check_batch(dst);
  if (rc) return rc;
  rc = check_batch(src);
  if (rc) return rc;
  if (dst_qp < 0 || dst_qp >= dst->nqp || src_qp < 0 || src_qp >= src->nqp)
    return fail(GQ_ERR_ARG, "copy_qp: QP index out of range");
  if (dst->host_in == nullptr || src->host_in == nullptr) return fail(GQ_ERR_STATE, "copy_qp: host_in not attached");
  const QpDesc& a = dst->qp[dst_qp];
  const QpDesc& c = src->qp[src_qp];
  if (a.N != c.N) return fail(GQ_ERR_DIMS, "copy_qp: horizons differ (%d vs %d)", a.N, c.N);
  for (int n = 0; n <= a.N; ++n) {
    const StageDesc& sa = dst->st[a.stage0 + n];
    const StageDesc& sc = src->st[c.stage0 + n];
    if (sa.nx != sc.nx || sa.nu != sc.nu || sa.nbx != sc.nbx || sa.nbu != sc.nbu || sa.ng != sc.ng || sa.ns != sc.ns)
      return fail(GQ_ERR_DIMS, "copy_qp: stage %d sizes differ", n);
  }
  const char* sb = static_cast<const char*>(src->host_in) + src->L.data;
  char* db = static_cast<char*>(dst->host_in) + dst->L.data;
  for (int n = 0; n <= a.N; ++n) {
    const StageDesc& sa = dst->st[a.stage0 + n];
    const StageDesc& sc = src->st[c.stage0 + n];
    const StageData lay = stage_data_layout(sa);
    std::memcpy(db + 8 * sa.data, sb + 8 * sc.data, 8 * (size_t)lay.size);
  }
  return GQ_OK;
}
