/* fftu_serve.h - a serving loop over the fftu transforms: many independent requests of mixed shapes,
 * dtypes and directions, each a whole d-dimensional DFT (eq. dftd) computed by the cyclic method of
 * Algorithm 2.3 with plans of fftu.h.
 *
 * A server owns one host thread and a few CUDA streams on the device that was current when it was
 * created: half of them, at the device's highest stream priority, carry batched requests, the other
 * half, at the lowest, requests that run alone; request buffers come from the device's stream-ordered
 * memory pool, so creating or evicting them never synchronises the device.  Submitted requests queue
 * per key (shape, dtype, direction).  The thread
 *   - admits work against a device-memory budget (request buffers, resident plans and twiddle
 *     tables); a request that cannot fit even alone completes at once with FFTU_ERR_NOMEM,
 *     otherwise it waits until completed work frees memory;
 *   - keeps at most max_inflight launches in flight, of them at most max_inflight_solo solo ones;
 *     while that many run, new requests queue;
 *   - batches queued requests of one key, largest power of two first (at most max_batch), into one
 *     persistent launch (fftu_batch_*), or runs a request with N >= large_elems alone through its
 *     own plan's kernels (fftu_exec);
 *   - replays a CUDA graph per resident batch instance: host-to-device copies of the inputs, the
 *     transform launch, device-to-host copies of the results (only the copy addresses change between
 *     replays); requests whose host buffers are not page-locked go through plain stream-ordered
 *     copies instead;
 *   - polls completion events (no blocking synchronisation on the hot path) and stamps the
 *     latencies.
 * A request's result does not depend on what else is in flight: the kernels a request goes through
 * depend only on its key and N, and each transform of a batch is computed independently.
 *
 * Ownership: the caller owns the host buffers of a request; they must stay valid until its
 * completion is returned by fftu_server_poll (or the server is destroyed).  Requests of one server
 * may be submitted from any thread.
 */
#ifndef FFTU_SERVE_H
#define FFTU_SERVE_H

#include <stdint.h>

#include "fftu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftu_server_st *fftu_server;

typedef struct {
    int64_t device_bytes; /* budget for request buffers, plans and their workspaces; 0 = half the free memory */
    int max_batch;        /* requests per batched launch, 1..128; 0 = 64 */
    int streams;          /* CUDA streams, 1..16; 0 = 8 (half for batched requests, half for solo ones) */
    int64_t large_elems;  /* requests with N >= large_elems run alone through their own plan; 0 = 2^22 */
    int use_graphs;       /* nonzero: replay captured CUDA graphs for page-locked requests */
    int max_inflight;     /* launches in flight at once, 1..256; 0 = 2 x streams.  Requests that
                             arrive while the limit is reached queue, and join one launch */
    int copy_piece_mib;   /* > 0: host copies in pieces of this many MiB, one after another, so that
                             other requests' copies can run between them; 0 = one copy per array */
    int max_inflight_solo; /* solo (large) launches in flight at once, 1..256; 0 = one per solo stream.
                             More solo requests queue in the server, holding no instance */
    int reserved[4];      /* must be zero */
} fftu_server_config;

typedef struct {
    int d;                        /* 1..FFTU_MAX_DIMS */
    int64_t n[FFTU_MAX_DIMS];     /* powers of two, row-major array, last axis contiguous */
    int dtype;                    /* fftu_dtype */
    int dir;                      /* fftu_dir */
    const void *in;               /* host input, N elements (interleaved re, im) */
    void *out;                    /* host output, N elements; may equal in */
    uint64_t tag;                 /* returned unchanged in the completion */
} fftu_request;

typedef struct {
    uint64_t tag;
    int status;        /* fftu_status of this request */
    int batch_size;    /* requests in the launch that computed it (0 if it never ran) */
    double submit_s;   /* server clock (seconds since creation) at fftu_server_submit */
    double start_s;    /* when its batch was issued to the GPU */
    double done_s;     /* when the server saw its batch's completion event */
} fftu_completion;

typedef struct {
    int64_t submitted, completed, rejected;
    int64_t batches, graph_replays, graph_builds, direct_launches;
    int64_t kernel_launches;        /* launches of this library's kernels made by the server */
    int64_t instances, plans;       /* resident batch instances and plans */
    int64_t bytes_in_use, peak_bytes, budget_bytes;
    int64_t evictions;
    int64_t bytes_h2d, bytes_d2h;   /* request bytes copied each way */
    int64_t instance_creations;     /* resident batch instances created (device buffers, plan or batch, graph) */
    double creation_s;              /* host time the server thread spent creating them */
    double max_launch_s;            /* longest host time of issuing one launch (copies, graph, kernels) */
    double max_loop_gap_s;          /* longest time between two passes of the server loop */
    int last_cuda_error;            /* last CUDA error the server met (cudaError_t; 0 = none) */
    int last_error_site;            /* where: 1 input copy, 2 transform launch, 3 output copy, 4 event record,
                                       5 completion event, 6 graph build, 7 graph replay */
} fftu_server_stats;

/* Start a server (cfg may be NULL = defaults).  FFTU_ERR_ARG on an invalid config. */
fftu_status fftu_server_create(const fftu_server_config *cfg, fftu_server *out);

/* Queue one request.  Shape or type errors are returned here (nothing is queued). */
fftu_status fftu_server_submit(fftu_server s, const fftu_request *req);

/* Warm-up before a latency-sensitive stream (no counterpart in the paper): create, for the key of
 * `like` (shape, dtype, direction), idle resident instances for every power-of-two batch size up to
 * max_k (one batch instance of each size per batched stream; max_inflight_solo solo instances for a key
 * with N >= large_elems), so that overlapping launches of the key each find one free, each with its
 * device buffers, batch or plan,
 * and, when `like`'s host buffers are page-locked, its CUDA graph.  The graphs are built with those
 * buffers as placeholders (every replay re-points the copies), so later requests of the key replay
 * an existing graph instead of waiting for a build.  Blocks until done, at most timeout_s seconds:
 * FFTU_OK, FFTU_ERR_TIMEOUT, FFTU_ERR_NOMEM (the budget cannot hold the instances) or the error a
 * request of the key would get.  No transform runs and no completion is produced; `like`'s buffers
 * are only read as addresses.  Validation errors as for fftu_server_submit. */
fftu_status fftu_server_warm(fftu_server s, const fftu_request *like, int max_k, double timeout_s);

/* Move up to max completions into out (oldest first); returns how many, or -1 on a bad argument. */
int fftu_server_poll(fftu_server s, fftu_completion *out, int max);

/* Wait until every submitted request has completed (its completion may still be unpolled),
 * at most timeout_s seconds: FFTU_OK, or FFTU_ERR_TIMEOUT. */
fftu_status fftu_server_drain(fftu_server s, double timeout_s);

fftu_status fftu_server_stats_get(fftu_server s, fftu_server_stats *st);

/* Stop the thread after the work in flight finishes and free everything the server holds.
 * Requests still queued complete with FFTU_ERR_ARG and are dropped. */
fftu_status fftu_server_destroy(fftu_server s);

#ifdef __cplusplus
}
#endif

#endif /* FFTU_SERVE_H */
