/*
 * gq_server.h -- continuous-batching request loop over the gq solver.
 *
 * The paper (arXiv 2003.02547) solves one QP per call; a model-predictive
 * controller calls it again at every sampling instant with a new initial
 * state and warm-starts from the previous solution (Sec. 4.2, warm start of
 * the IPM; Sec. 5.1, MPC use).  The server runs many such callers at once on
 * one GPU: requests for OCP QPs of any sizes arrive at any time, are admitted
 * into micro-batches as lanes and device memory free up, and the
 * micro-batches of several lanes run concurrently, each on its own CUDA
 * stream.  The iterates of every solved key stay resident in device memory so
 * that a repeat request for the same key starts from them (primal + dual warm
 * start, Sec. 4.2) without a host round trip.
 *
 * Threads.  gq_server_create starts one native worker thread that forms
 * micro-batches, launches them and retires finished ones; submit / poll /
 * drain may be called from any thread.
 *
 * Memory.  The caller provides one device arena (the budget) and one pinned
 * host arena.  The device arena holds the resident warm-start cache
 * (cfg.cache_bytes) followed by `lanes` equal partitions, each holding one
 * micro-batch's input, solution and workspace; the pinned arena is split into
 * `lanes` equal staging partitions.  A micro-batch is admitted only if it fits
 * its lane's partitions, so the device memory used never exceeds the arena.
 * The server's own control structures (queues, ticket table, key map) are the
 * one place this library allocates host memory; it never allocates device
 * memory.
 *
 * Warm starts.  A warm-started request that does not converge is solved once
 * more from a cold start (its resident iterate is dropped; latency counts
 * both attempts); gq_ticket_info.warm_used then reads 0.
 *
 * Ordering.  Requests with the same non-zero key are solved in submission
 * order, one at a time: a request whose key is still being solved waits in
 * the queue (other requests pass it), so a warm start always reads the
 * solution of the previous request of that key.
 */
#ifndef GQ_SERVER_H
#define GQ_SERVER_H

#include "gq.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gq_server gq_server;

typedef struct gq_server_cfg {
    int32_t lanes;        /* micro-batches in flight at once, one stream each (1..64)   */
    int32_t max_batch;    /* most QPs in one micro-batch (>= 1)                          */
    int32_t max_wait_us;  /* a free lane waits at most this long for max_batch requests
                             before launching fewer (0: launch at once)                  */
    int32_t device;       /* CUDA device ordinal of the arena                            */
    size_t cache_bytes;   /* leading part of the device arena kept for resident
                             warm-start iterates (0: no warm starts)                    */
    gq_ipm_arg arg;       /* solver arguments of every micro-batch (warm_start is set
                             per request)                                                */
    double class_ratio;   /* size classes: a micro-batch takes only requests whose
                             factorisation cost estimate lies in the same power of
                             class_ratio as the oldest eligible request's, so small
                             QPs do not wait for the largest (<= 1: no classes)      */
} gq_server_cfg;

typedef struct gq_request {
    const gq_batch* src;  /* host-staged source batch holding the QP (filled by the
                             setters; only its host "in" buffer is read, at admission) */
    int32_t src_qp;       /* QP index in src                                          */
    int32_t warm;         /* 1: start from the resident iterate of `key` (primal+dual);
                             0 or no resident iterate: cold start                     */
    uint64_t key;         /* problem identity across re-solves; 0 = none (not cached) */
    int64_t t_arrival_ns; /* CLOCK_MONOTONIC arrival time; 0 = time of submission      */
    /* caller-owned outputs written before the ticket reports done (NULL: skip);
       lengths as gq_get_sol_offsets reports for the source QP                */
    double* y;
    double* pi;
    double* lam;
    double* t;
} gq_request;

typedef struct gq_ticket_info {
    int32_t done;         /* 1 once outputs are written                                 */
    int32_t code;         /* GQ_OK, or GQ_ERR_SIZE (QP larger than a lane partition),
                             GQ_ERR_CUDA (launch failed) for this request              */
    int32_t warm_used;    /* 1 if it started from a resident iterate                     */
    int32_t batch_size;   /* QPs in its micro-batch                                      */
    int64_t latency_ns;   /* arrival -> outputs visible on the host                      */
    int64_t wait_ns;      /* arrival -> admission into a micro-batch                     */
    gq_stats stats;       /* per-QP solver statistics                                    */
} gq_ticket_info;

typedef struct gq_server_report {
    int64_t submitted, completed, rejected, failed;
    int64_t batches, batched_qps;      /* micro-batches launched, QPs in them            */
    int64_t warm_hits, warm_misses;    /* warm requests with / without a resident iterate */
    int64_t cache_entries;             /* live resident iterates                         */
    int64_t cache_evictions;           /* iterates overwritten by newer ones             */
    int64_t cache_skips;               /* results not cached (cache region busy)         */
    int64_t deferrals;                 /* requests passed over while their key was busy  */
    int64_t max_lanes_busy;
    int64_t max_queue;
    int64_t cold_retries;              /* warm starts that did not converge, re-solved cold */
} gq_server_report;

/* Default configuration: 4 lanes, max_batch 256, max_wait_us 0, device 0,
 * cache_bytes 0, arg = gq_ipm_arg_default(SPEED, MIXED), class_ratio 4. */
GQ_API int gq_server_cfg_default(gq_server_cfg* cfg);

/* Creates the server and starts its worker thread.  dev_arena (256-byte
 * aligned, dev_bytes long, on cfg->device) and pinned (16-byte aligned,
 * pinned_bytes long) stay owned by the caller and must outlive the server.
 * Errors: GQ_ERR_ARG (bad cfg or pointers), GQ_ERR_SIZE (arena smaller than
 * the cache plus one byte per lane), GQ_ERR_CUDA (stream or event creation). */
GQ_API int gq_server_create(const gq_server_cfg* cfg, void* dev_arena, size_t dev_bytes, void* pinned,
                            size_t pinned_bytes, gq_server** out);

/* Queues one request; *ticket identifies it (tickets count up from 0).  The
 * source QP's host data must stay unchanged until the ticket is done.
 * Errors: GQ_ERR_ARG (NULL pointers, QP index out of range), GQ_ERR_STATE
 * (server stopped after a CUDA error). */
GQ_API int gq_server_submit(gq_server* s, const gq_request* req, int64_t* ticket);

/* Non-blocking status of a ticket. */
GQ_API int gq_server_poll(gq_server* s, int64_t ticket, gq_ticket_info* info);

/* Blocks until every submitted request is done or timeout_ns (> 0) elapses;
 * returns GQ_OK, or GQ_ERR_STATE on timeout or after a CUDA error. */
GQ_API int gq_server_drain(gq_server* s, int64_t timeout_ns);

/* Counters since creation. */
GQ_API int gq_server_report_get(gq_server* s, gq_server_report* out);

/* Stops the worker after the micro-batches in flight finish and frees the
 * server's host structures (queued requests not yet admitted are dropped and
 * reported failed).  The arenas are the caller's to free afterwards. */
GQ_API int gq_server_destroy(gq_server* s);

#ifdef __cplusplus
}
#endif

#endif /* GQ_SERVER_H */
