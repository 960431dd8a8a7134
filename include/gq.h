/*
 * gq.h -- C ABI of the batched OCP-QP interior-point solver for GB300 (sm_103a).
 *
 * The library solves batches of optimal-control QPs (the OCP QP of Sec. 2.2 of
 * the HPIPM paper, arXiv 2003.02547) with the primal-dual Mehrotra
 * predictor-corrector interior-point method of Sec. 3.1-3.4 and 4.2.  The
 * Newton system eq. (delta) is reduced to eq. (kkt) by eliminating dt and
 * dlambda (Sec. 3.3) and factorised by the square-root backward Riccati
 * recursion (Sec. 3.3, variant (b); variant (a), the classical recursion, on
 * request; the QR array algorithm in modes balance and robust); the whole
 * IPM loop of every QP runs inside CUDA kernels, one warp or one thread
 * block per QP.
 *
 * Problem statement (Sec. 2.2).  For stages n = 0..N, y_n = [u_n; x_n]:
 *   min  sum_n 1/2 [u;x;1]' [[R, S, r], [S', Q, q], [r', q', 0]] [u;x;1]
 *   s.t. x_{n+1} = A_n x_n + B_n u_n + b_n                 n = 0..N-1
 *        lbu_n <= u_n[idxbu_n] <= ubu_n,  lbx_n <= x_n[idxbx_n] <= ubx_n
 *        lg_n  <= D_n u_n + C_n x_n <= ug_n                 n = 0..N
 * S_n has shape nu_n x nx_n.  Sizes may vary per stage and per QP.  A bound
 * of -INFINITY (lower) or +INFINITY (upper) masks that single side (Sec. 2.1).
 * An initial-state constraint is expressed either by eliminating x_0
 * (nx_0 = 0, x0 folded into b_0, r_0 and the stage-0 general bounds) or, as
 * in the paper, by a box on x_0 with equal bounds.  Any box or general
 * constraint may be made soft by a slack pair with diagonal L2 and linear
 * L1 costs (Sec. 2.2; gq_batch_create_soft, gq_set_soft).
 *
 * Sign conventions of the outputs (Lagrangian of Sec. 3.1):
 *   equality rows -B_n u_n - A_n x_n + x_{n+1} = b_n with multiplier pi_{n+1}
 *   (pi_{n+1} is the cost-to-go gradient at x_{n+1});
 *   each constraint lo <= c(y) <= hi gives the sides c(y) - lo >= 0 and
 *   hi - c(y) >= 0; per stage the constraint list is [box u (idxbu order);
 *   box x (idxbx order); general rows], nc_n = nbu_n + nbx_n + ng_n, and
 *   lambda/t hold the nc_n lower sides followed by the nc_n upper sides.
 *   Masked sides report lambda = 0, t = 1.
 *
 * Memory (Sec. 1: no internal allocation, externally provided chunks).
 *   The library never allocates.  The caller provides
 *     - the host memory of the batch handle            (gq_batch_memsize)
 *     - a host "in" staging buffer and a device "in" buffer of equal size
 *       holding descriptors, indices and FP64 problem data (sizes.in_bytes)
 *     - a host and a device "sol" buffer of equal size holding per-QP
 *       statistics and the iterates y, pi, lambda, t  (sizes.sol_bytes)
 *     - a device workspace                             (sizes.ws_bytes)
 *   Device buffers must be 256-byte aligned (cudaMalloc / PyTorch storage).
 *   Host buffers should be pinned for asynchronous copies.
 *
 * Errors.  Every call returns 0 (GQ_OK) or a negative GQ_ERR_* code and never
 * aborts, throws or traps; gq_last_error() gives a per-thread message.  Solve
 * results carry a per-QP status (GQ_STATUS_*); a failing QP never affects its
 * batch neighbours.
 */
#ifndef GQ_H
#define GQ_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GQ_API __attribute__((visibility("default")))
#else
#define GQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define GQ_OK 0
#define GQ_ERR_ARG -1     /* null pointer, index out of range, bad enum        */
#define GQ_ERR_DIMS -2    /* inconsistent or unsupported dimensions            */
#define GQ_ERR_SIZE -3    /* caller buffer smaller than required               */
#define GQ_ERR_CUDA -4    /* a CUDA runtime call failed                        */
#define GQ_ERR_DATA -5    /* NaN in data, lo > hi, non-symmetric Q/R, ...      */
#define GQ_ERR_STATE -6   /* call made before the buffers it needs are attached */

/* ---- per-QP solve status ---- */
#define GQ_STATUS_CONVERGED 0
#define GQ_STATUS_MAX_ITER 1
#define GQ_STATUS_MIN_STEP 2
#define GQ_STATUS_NAN 3      /* non-finite residual or non-positive pivot     */
#define GQ_STATUS_TIMEOUT 4  /* arg.timeout_ns elapsed on the device          */
/* flag bits in gq_stats.flags */
#define GQ_FLAG_FP64_FALLBACK 1  /* mixed path switched this QP to FP64 factors */
#define GQ_FLAG_REGULARIZED 2    /* an FP64 factorisation lost a pivot: it was
                                    redone with a 1e-10 primal regularisation
                                    and, if still indefinite, the iteration
                                    was redone with lambda, t lifted to
                                    max(1e-10, 1e-2 max(|r_g|, |r_b|))       */
#define GQ_FLAG_ARRAY_QR 4       /* mode balance: refinement fell short of the accuracy
                                    rule, so the rest of the solve factors with the QR
                                    array algorithm */

/* ---- solver arguments (Sec. 4.2) ---- */
#define GQ_MODE_SPEED 0     /* delta formulation, residual-based exit (Sec. 4.2) */
#define GQ_MODE_BALANCE 1   /* speed + iterative refinement of every direction;
                               a direction that refinement cannot make accurate
                               (ir_fail_ratio) switches the QP's factorisations
                               to the array algorithm below (Sec. 4.2)          */
#define GQ_MODE_ROBUST 2    /* balance + every Riccati factorisation by the array
                               algorithm: chol(Ht + M M') taken from the QR
                               factorisation of [chol(Ht)'; M'] without forming
                               M M' (Sec. 4.2, mode robust)                     */
#define GQ_PREC_FP64 0      /* Riccati factor/solve in FP64                       */
#define GQ_PREC_MIXED 1     /* Riccati factor/solve in FP32, residuals, IR,
                               step length and duality measure in FP64          */

typedef struct gq_ipm_arg {
    int32_t mode;          /* GQ_MODE_*                                            */
    int32_t precision;     /* GQ_PREC_*                                            */
    int32_t iter_max;      /* maximum IPM iterations                               */
    int32_t warm_start;    /* 0 cold, 1 primal (y, pi), 2 primal + dual (Sec. 4.2) */
    int32_t ir_steps;      /* max iterative-refinement steps per direction (3.4)   */
    int32_t cond_corr;     /* 1: conditional Mehrotra corrector (Sec. 4.2)         */
    int32_t fp64_fallback; /* mixed path: 1 = refactor in FP64 when IR stagnates   */
    int32_t riccati;       /* 0 square-root Riccati (Sec. 3.3, variant b: needs every
                              stage Hessian plus barrier terms positive definite);
                              1 classical Riccati (variant a: only the reduced
                              Hessians R + B'PB positive definite, so an indefinite
                              Q is allowed); the classical form runs in the block
                              kernel only (schedule warp_max_nv = 0)                */
    double tol_stat;       /* exit: ||r_g||inf <= tol_stat                          */
    double tol_eq;         /*       ||r_b||inf <= tol_eq                            */
    double tol_ineq;       /*       ||r_d||inf <= tol_ineq                          */
    double tol_comp;       /*       mu = lambda't / n_c <= tol_comp                 */
    double alpha_min;      /* exit when the step length drops below this           */
    double lam_min;        /* lower clamp of lambda after each step (Sec. 4.2)     */
    double t_min;          /* lower clamp of t after each step                     */
    double tau_b;          /* fraction to the boundary, alpha = min(1, tau_b a_max) */
    double corr_k;         /* keep corrector if mu_corr <= corr_k * mu_aff          */
    double reg_prim;       /* primal regularisation added to the factored Hessian
                              only (Sec. 4.2); offset by IR                         */
    double ir_tol;         /* IR stops when ||res||inf <= ir_tol ||rhs||inf          */
    double warm_min;       /* warm start 2: lambda, t clamped below by this         */
    int64_t timeout_ns;    /* per-QP device wall-clock limit, 0 = none             */
    double ir_fail_ratio;  /* a refined direction whose residual ratio exceeds this
                              (or whose residual is not an inexact-Newton step)
                              counts as inaccurate: the mixed path then refactors
                              in FP64 (fp64_fallback), and mode balance then
                              refactors with the QR array algorithm (Sec. 4.2) */
} gq_ipm_arg;

/* Defaults for a mode and precision: iter_max 100, tolerances 1e-8,
 * alpha_min 1e-12, lam_min = t_min = 1e-16 (FP64) or 1e-12 (mixed),
 * tau_b 0.995, corr_k 2, reg_prim 0 (FP64) or 1e-9 (mixed), ir_steps 0
 * (FP64 speed) or 3 (mixed, balance or robust), ir_tol 1e-12, warm_min 1e-2,
 * ir_fail_ratio 1e-6.
 * Returns GQ_ERR_ARG on a null pointer or unknown mode/precision. */
GQ_API int gq_ipm_arg_default(gq_ipm_arg* arg, int mode, int precision);

/* ---- per-QP results ---- */
typedef struct gq_stats {
    int32_t status;        /* GQ_STATUS_*                                          */
    int32_t iters;         /* IPM iterations taken                                 */
    int32_t flags;         /* GQ_FLAG_* bits                                       */
    int32_t ir_total;      /* iterative-refinement solves performed                */
    int32_t n_fact;        /* Riccati factorisations (all precisions)              */
    int32_t n_fact64;      /*   of which in FP64                                   */
    int32_t n_solve;       /* Riccati solves (all right-hand sides)                */
    int32_t n_res;         /* residual evaluations (IPM and refinement)            */
    double res[4];         /* ||r_g||inf, ||r_b||inf, ||r_d||inf, mu at exit        */
} gq_stats;

/* ---- batch layout ---- */
typedef struct gq_batch gq_batch;

typedef struct gq_sizes {
    size_t in_bytes;       /* host staging == device "in" buffer                   */
    size_t sol_bytes;      /* host == device solution buffer                       */
    size_t ws_bytes;       /* device workspace                                     */
    int64_t n_stages;      /* total stages over the batch                          */
    int64_t n_slots;       /* distinct stage data blocks                           */
    int64_t nv_total;      /* sum of nu_n + nx_n + 2 ns_n over the batch           */
    int64_t neq_total;     /* sum of nx_{n+1}                                      */
    int64_t nside_total;   /* sum of 2 (nbu_n + nbx_n + ng_n + ns_n)               */
    int32_t nv_max;        /* largest stage nu_n + nx_n                            */
    int32_t nx_max;        /* largest stage nx_n                                   */
} gq_sizes;

/* dims: for QP q in order, N_q followed by (N_q + 1) groups of five ints
 * (nx_n, nu_n, nbx_n, nbu_n, ng_n), n = 0..N_q.  Requires nx_n >= 0,
 * nu_n >= 0, 0 <= nbu_n <= nu_n, 0 <= nbx_n <= nx_n, ng_n >= 0, N_q >= 0.
 * stage_slot (may be NULL): one int per stage in the same order; stages with
 * equal non-negative slot ids share one problem-data block (they must have
 * identical sizes, including nx_{n+1}); NULL or -1 gives a private block.
 * Returns the host bytes the batch handle needs, or 0 on invalid input. */
GQ_API size_t gq_batch_memsize(int nqp, const int* dims, size_t dims_len, const int* stage_slot);

/* Lays the batch out in the caller's host memory `mem` (>= memsize bytes,
 * 16-byte aligned) and returns the handle in *out.  The handle stays valid
 * while `mem` does; there is no destroy call. */
GQ_API int gq_batch_create(int nqp, const int* dims, size_t dims_len, const int* stage_slot,
                    void* mem, size_t mem_bytes, gq_batch** out);

/* Soft constraints (Sec. 2.2).  As gq_batch_create, plus stage_ns (may be
 * NULL: no slacks): one int per stage in the order of stage_slot, the number
 * ns_n (0 <= ns_n <= nc_n) of constraints of that stage made soft.  Slack
 * pair k of stage n relaxes constraint idxs_n[k] of the stage's list [box
 * on u; box on x; general rows]: its lower side becomes c + s^l_k >= lo and
 * its upper side c - s^u_k <= hi, with s^l_k >= lls_k, s^u_k >= lus_k and
 * the cost 1/2 Zl_k (s^l_k)^2 + zl_k s^l_k + 1/2 Zu_k (s^u_k)^2 + zu_k s^u_k.
 * With slacks, a stage's block of the y vector is [u; x; s^l; s^u] and its
 * block of lambda and t is [lower sides (nc); upper sides (nc); bounds of
 * s^l (ns); bounds of s^u (ns)].  Stages sharing a slot must have equal ns.
 * The slacks are eliminated inside the solver (a diagonal elimination at
 * linear cost folded into the barrier terms).  Partial condensing rejects
 * QPs with slacks (GQ_ERR_ARG).  Errors: those of gq_batch_create, and
 * GQ_ERR_DIMS for ns_n outside [0, nc_n]. */
GQ_API int gq_batch_create_soft(int nqp, const int* dims, size_t dims_len, const int* stage_slot,
                                const int* stage_ns, void* mem, size_t mem_bytes, gq_batch** out);

GQ_API int gq_batch_sizes(const gq_batch* b, gq_sizes* out);

/* Attaches the caller-owned buffers.  host_in/host_sol may be NULL when
 * setters/getters are not used; dev_* must be non-NULL, 256-byte aligned.
 * Writes the layout descriptors into host_in (if given). */
GQ_API int gq_batch_attach(gq_batch* b, void* host_in, void* host_sol,
                    void* dev_in, void* dev_sol, void* dev_ws);

/* ---- data setters: write FP64 data of stage n of QP qp into host_in ----
 * Matrices are column-major with leading dimension >= their row count.
 * A: nx_{n+1} x nx_n, B: nx_{n+1} x nu_n, b: nx_{n+1} (Sec. 2.2 dynamics). */
GQ_API int gq_set_dynamics(gq_batch* b, int qp, int n, const double* A, int lda,
                    const double* B, int ldb, const double* bvec);
/* Q: nx_n x nx_n, S: nu_n x nx_n, R: nu_n x nu_n (Q, R symmetric), q, r. */
GQ_API int gq_set_cost(gq_batch* b, int qp, int n, const double* Q, int ldq, const double* S, int lds,
                const double* R, int ldr, const double* q, const double* r);
/* idxbu: nbu_n distinct indices into u_n; idxbx: nbx_n distinct into x_n;
 * bounds with lo <= hi, +-INFINITY masks a side. */
GQ_API int gq_set_box(gq_batch* b, int qp, int n, const int* idxbu, const double* lbu, const double* ubu,
               const int* idxbx, const double* lbx, const double* ubx);
/* C: ng_n x nx_n, D: ng_n x nu_n, lg, ug: ng_n. */
GQ_API int gq_set_general(gq_batch* b, int qp, int n, const double* C, int ldc, const double* D, int ldd,
                   const double* lg, const double* ug);
/* Slack data of stage n (ns_n entries each; nothing to do when ns_n = 0;
 * until it is called, gq_batch_attach leaves slack k relaxing constraint k
 * at zero cost with zero slack bounds):
 * idxs distinct constraint indices in [0, nc_n), Zl, Zu >= 0 and finite,
 * zl, zu, lls, lus finite.  Errors: GQ_ERR_ARG (NULL pointer, index out of
 * range or repeated), GQ_ERR_DATA (invalid values). */
GQ_API int gq_set_soft(gq_batch* b, int qp, int n, const int* idxs, const double* Zl, const double* Zu,
                       const double* zl, const double* zu, const double* lls, const double* lus);

/* Writes an initial guess for QP qp into host_sol (y: sum nv + 2 ns entries in
 * stage order [u_0; x_0; s^l_0; s^u_0; u_1; ...], pi: sum nx_{n+1}, lam/t:
 * sum 2 (nc_n + ns_n); any may be
 * NULL to leave that part unchanged).  Used with arg.warm_start after
 * gq_upload_sol. */
GQ_API int gq_set_guess(gq_batch* b, int qp, const double* y, const double* pi,
                 const double* lam, const double* t);

/* ---- partial condensing (Sec. 3.5), host side ----
 * Blocks of `block` consecutive stages of QP `qp` (stages kb..kb+block-1,
 * the last block possibly shorter) become one stage: the states inside a
 * block are eliminated through the dynamics, the new stage keeps the block's
 * first state and stacks its controls; state bounds inside a block become
 * general rows (after the stage's own general rows, stage by stage); the
 * terminal stage is kept.  The condensed horizon is ceil(N / block).
 * gq_condense_dims writes the condensed QP's dims (the format of
 * gq_batch_memsize; dims may be NULL to query *len).  gq_condense fills
 * QP dst_qp of `dst` (created with those dims and attached) through the
 * setters.  gq_expand maps a condensed solution (y2, pi2, lam2, t2 in the
 * layout of gq_get_sol_offsets for dst_qp) back to the original QP's (y,
 * pi, lam, t): states by the block recursion, lambda and t by the
 * constraint correspondence, the eliminated dynamics' multipliers from the
 * eliminated states' stationarity rows.  Errors: GQ_ERR_ARG, GQ_ERR_DIMS,
 * GQ_ERR_SIZE, and the setters' errors. */
GQ_API int gq_condense_dims(const gq_batch* src, int qp, int block, int* dims, size_t cap, size_t* len);
GQ_API int gq_condense(gq_batch* src, int src_qp, int block, gq_batch* dst, int dst_qp);
GQ_API int gq_expand(gq_batch* src, int src_qp, int block, const gq_batch* dst, int dst_qp, const double* y2,
                     const double* pi2, const double* lam2, const double* t2, double* y, double* pi, double* lam,
                     double* t);

/* Partial condensing on the device (Sec. 3.5), every QP of a batch at once.
 * QP q of `src` (uploaded: its device "in" buffer holds the data) is condensed
 * into QP q of `dst`, which must hold exactly the condensed sizes of
 * gq_condense_dims for every QP, with private (unshared) stage blocks, and be
 * attached with its descriptors on the device (gq_upload once after
 * gq_batch_attach; its data need not be set).  The kernel writes dst's
 * device data blocks directly (dst's host staging is not updated).  The
 * arithmetic is that of gq_condense: the Hessian by the backward recursion of
 * Sec. 3.5 (quadratic in the block length, cubic in the state size), the block
 * dynamics and the general rows through the forward maps of the block.
 * dev_ws: caller device memory of at least gq_condense_ws_bytes(src, block)
 * bytes, 256-byte aligned.  Asynchronous on `stream`.
 * Errors: GQ_ERR_ARG (NULL, block < 1, soft constraints, shared dst blocks),
 * GQ_ERR_DIMS (dst sizes), GQ_ERR_SIZE (workspace), GQ_ERR_STATE, GQ_ERR_CUDA.
 * gq_condense_ws_bytes returns 0 on invalid input. */
GQ_API size_t gq_condense_ws_bytes(const gq_batch* src, int block);
GQ_API int gq_condense_device(const gq_batch* src, int block, gq_batch* dst, void* dev_ws, size_t ws_bytes,
                              void* stream);

/* Getters of the staged problem data, the inverse of the four setters above
 * (same argument meaning and column-major layouts; any output may be NULL;
 * the box getter returns idxbx relative to x).  Errors: GQ_ERR_ARG. */
GQ_API int gq_get_dynamics(gq_batch* b, int qp, int n, double* A, int lda, double* B, int ldb, double* bvec);
GQ_API int gq_get_cost(gq_batch* b, int qp, int n, double* Q, int ldq, double* S, int lds, double* R, int ldr,
                       double* q, double* r);
GQ_API int gq_get_box(gq_batch* b, int qp, int n, int* idxbu, double* lbu, double* ubu, int* idxbx, double* lbx,
                      double* ubx);
GQ_API int gq_get_general(gq_batch* b, int qp, int n, double* C, int ldc, double* D, int ldd, double* lg,
                          double* ug);
/* The slack data of gq_set_soft (ns_out receives ns_n; arrays ns_n long). */
GQ_API int gq_get_soft(gq_batch* b, int qp, int n, int* ns_out, int* idxs, double* Zl, double* Zu, double* zl,
                       double* zu, double* lls, double* lus);

/* Initial state by elimination (Sec. 2.2 allows stage-wise sizes, so x_0 can
 * be removed: nx_0 = 0).  Stage 0 of QP `qp` must have nx_0 = 0; given the
 * measured state x0 (nx0 entries) and the stage-0 data that multiply it --
 * A0 (nx_1 x nx0, column-major, lda), S0 (nu_0 x nx0, lds), C0 (ng_0 x nx0,
 * ldc) -- and the unfolded b0, r0, lg0, ug0, this writes
 *   b_0 = b0 + A0 x0,  r_0 = r0 + S0 x0,  lg_0 = lg0 - C0 x0,  ug_0 = ug0 - C0 x0
 * into the host staging (an infinite bound stays infinite).  Idempotent:
 * call it again with a new x0 for the next MPC solve (then gq_upload).
 * The other stage-0 data (B_0, R_0, boxes on u_0, D_0) come from the usual
 * setters.  Errors: GQ_ERR_DIMS (nx_0 != 0), GQ_ERR_ARG, GQ_ERR_DATA. */
GQ_API int gq_set_initial_state(gq_batch* b, int qp, const double* x0, int nx0, const double* A0, int lda,
                                const double* b0, const double* S0, int lds, const double* r0, const double* C0,
                                int ldc, const double* lg0, const double* ug0);

/* Copies all stage data of QP src_qp of batch `src` into QP dst_qp of batch
 * `dst` (host staging buffers; identical stage sizes required, else
 * GQ_ERR_DIMS).  Lets a server pack each request once and assemble
 * micro-batches by copying blocks (Sec. 1: data in solver layout, filled by
 * setters once). */
GQ_API int gq_copy_qp(gq_batch* dst, int dst_qp, const gq_batch* src, int src_qp);

/* ---- schedule: which QPs run one per warp, block size of the rest ---- */
typedef struct gq_schedule {
    int32_t warp_max_nv;   /* QPs whose stages all have nu + nx and nx at most this run
                              one per warp (0..32; 0: every QP in the block kernel);
                              QPs with soft constraints always run in the block
                              kernel                                                   */
    int32_t block_threads; /* threads per block of the block kernel: 64, 128 or 256;
                              0 (default): automatic, 128 when every block-bucket
                              stage has nu + nx <= 96 and the bucket holds more
                              QPs than two per SM, else 256 (measured: more QPs per
                              SM pay for full buckets of small stages, more threads
                              per QP for large stages and for buckets that fit the
                              GPU at once)                                             */
    int32_t warp_qps;      /* out: QPs in the warp bucket                             */
    int32_t block_qps;     /* out: QPs in the block bucket                            */
    int32_t tensor_cores;  /* FP32 factors of large stages (128 <= nu + nx <= 256,
                              nx <= 128, no general rows, 256 threads) form their
                              products on the tcgen05 tensor cores (TF32 operands in
                              shared memory, accumulators in tensor memory) when this
                              is 2, or when it is 1 and the block bucket holds at most
                              one QP per two SMs (measured: once blocks share SMs the
                              operand tiles' shared memory costs more than the
                              products gain); 0: always the warp-level mma.sync
                              products                                                  */
} gq_schedule;

/* Defaults: warp_max_nv 32, block_threads 0 (automatic), tensor_cores 1
 * (automatic). */
GQ_API int gq_get_schedule(const gq_batch* b, gq_schedule* out);

/* Re-plans the buckets (host handle and host "in" staging); gq_upload before
 * the next solve.  A different schedule may change the last bits of a QP's
 * result (another summation split), never its accuracy.  Errors: GQ_ERR_ARG. */
GQ_API int gq_set_schedule(gq_batch* b, const gq_schedule* sch);

/* Autotuner: times `reps` solves of the batch (inputs attached, solution
 * buffers overwritten) under each distinct candidate schedule -- warp
 * threshold 32, 24, 16 or 0 (one QP per warp for stages up to that size,
 * one block per QP for the rest), 256, 128 or 64 threads per block, tensor-
 * core products on (2) or off (0) -- keeps the fastest, uploads it and returns it
 * (and its mean solve time in ms).  Candidates that run the same kernels as
 * an earlier one are skipped.  Blocks until the timing solves finish (it synchronises `stream`).
 * Errors: as gq_solve, GQ_ERR_CUDA for event failures. */
GQ_API int gq_autotune(gq_batch* b, const gq_ipm_arg* arg, void* stream, int reps, gq_schedule* best,
                       double* best_ms);

/* ---- transfers (asynchronous on `stream`, a cudaStream_t; NULL = legacy) ---- */
GQ_API int gq_upload(gq_batch* b, void* stream);       /* host_in  -> dev_in  */
GQ_API int gq_upload_sol(gq_batch* b, void* stream);   /* host_sol -> dev_sol */
GQ_API int gq_download(gq_batch* b, void* stream);     /* dev_sol  -> host_sol */

/* ---- solve (Sec. 4.2): enqueue the IPM for every QP of the batch ----
 * Asynchronous: one kernel launch on `stream`; results appear in dev_sol.
 * Errors in the arguments are reported before anything is enqueued. */
GQ_API int gq_solve(gq_batch* b, const gq_ipm_arg* arg, void* stream);

/* Row-level entry points, used to check the solver step by step.
 * gq_residuals: residual function of eq. (delta) at the iterate in dev_sol;
 *   writes per-QP norms into the stats res[] fields (status left as is).
 * gq_newton_step: one Newton direction of eq. (delta) at the iterate in dev_sol
 *   with r_m = lambda t - sigma_mu, through the Riccati factorisation of
 *   eq. (kkt) in the precision of arg; writes (dy, dpi, dlambda, dt) into
 *   dev_dir, a device buffer laid out like the iterate part of the sol buffer
 *   (sizes.sol_bytes bytes; its stats part is left untouched). */
GQ_API int gq_residuals(gq_batch* b, void* stream);
GQ_API int gq_newton_step(gq_batch* b, const gq_ipm_arg* arg, double sigma_mu, void* dev_dir, void* stream);

/* ---- solve without allocation (no counterpart in the paper) ----
 * For callers that cannot allocate device memory when they solve (a fixed
 * memory budget, an allocator owned by a host application, or a region where
 * allocation would synchronise).  Same arguments and results as gq_solve, but
 * the input and solution buffers are passed here and the workspace is a
 * file-scope device array of GQ_NOALLOC_SCRATCH_BYTES inside the library,
 * held by every GPU that loads the library until the process exits.
 *   - dev_in / dev_sol: 256-byte aligned device buffers of sizes.in_bytes and
 *     sizes.sol_bytes laid out as for gq_solve (gq_upload / gq_download use the
 *     attached buffers; copy into these with cudaMemcpyAsync when they differ).
 *   - Returns GQ_ERR_SIZE, before any GPU work, when sizes.ws_bytes exceeds
 *     GQ_NOALLOC_SCRATCH_BYTES.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.  The first
 *     call on each device looks up the array's device address (with that
 *     device current); make that first call before any stream capture.
 *   - Every call shares the one array and leaves its contents behind; the
 *     solver writes every workspace entry before reading it, so nothing needs
 *     clearing.  Calls whose GPU work overlaps (other streams, other threads)
 *     race on the array: serialise them. */
#define GQ_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
/* The size of that array in this build of the library (GQ_NOALLOC_SCRATCH_BYTES
 * as compiled in), for bindings that cannot read the macro. */
GQ_API size_t gq_noalloc_scratch_bytes(void);
GQ_API int gq_solve_noalloc(gq_batch* b, const gq_ipm_arg* arg, void* dev_in, void* dev_sol, void* stream);

/* ---- getters (read host_sol after gq_download + stream sync) ---- */
/* u: nu_n, x: nx_n, pi: nx_{n+1} (n < N; multiplier of dynamics block n),
 * lam, t: 2 (nc_n + ns_n).  Any pointer may be NULL. */
GQ_API int gq_get_stage_sol(const gq_batch* b, int qp, int n, double* u, double* x, double* pi,
                     double* lam, double* t);
/* sl, su: the ns_n slacks s^l, s^u of stage n (either may be NULL). */
GQ_API int gq_get_stage_slacks(const gq_batch* b, int qp, int n, double* sl, double* su);
GQ_API int gq_get_stats(const gq_batch* b, int qp, gq_stats* out);
/* Offsets (in doubles) of QP qp's vectors inside the sol buffer:
 * off[0] y, off[1] pi, off[2] lam, off[3] t, and their lengths off[4..7]. */
/* Status (GQ_STATUS_*) and, if iters is non-NULL, iteration count of every
 * QP, from the host "sol" buffer after gq_download (arrays of nqp entries). */
GQ_API int gq_get_statuses(const gq_batch* b, int32_t* status, int32_t* iters);

GQ_API int gq_get_sol_offsets(const gq_batch* b, int qp, int64_t off[8]);

/* ---- measurement helper (no counterpart in the paper) ----
 * FP32 (fp64 = 0) or FP64 (fp64 = 1) fused multiply-add throughput of the
 * current device in flop/s, measured by a probe kernel on `stream` with
 * CUDA events (best of three timed launches after one warm-up).  Benchmarks
 * use it as the ALU roofline denominator.  Synchronises `stream`.
 * Errors: GQ_ERR_ARG, GQ_ERR_CUDA. */
GQ_API int gq_probe_fma_rate(int fp64, void* stream, double* flops_per_s);

/* Per-thread description of the last error, never NULL. */
GQ_API const char* gq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GQ_H */
