/*
 * lic_serve.h -- the serving form: many concurrent frame streams of mixed
 * resolutions through one codec configuration on one GPU (liblic.so).
 *
 * The paper pipelines frames through task queues -- one control thread per
 * GPU workload, worker threads for the CPU stages, a FIFO between each pair
 * (Sec. III-A) -- so that the stages of successive frames overlap; its
 * streaming demo sends 720p30 video through the codec (Sec. V).  Here every
 * stage runs on the GPU, so the pipeline becomes:
 *
 *   submit (any host thread) -> per-resolution bucket FIFO -> dispatcher
 *   thread forms a batch (full, or its oldest frame waited max_wait_ms) ->
 *   one of the bucket's lanes (a codec + CUDA stream, its encode+decode
 *   chain replayed as a CUDA graph) -> completion callback -> result queue.
 *
 * Lanes of one bucket and the buckets of different resolutions run on their
 * own streams, so batches overlap on the GPU (frames in flight together).
 * Admission: a request is refused with LIC_E_BUSY when max_pending requests
 * are in flight, and a new resolution is refused with LIC_E_OOM when its
 * lanes would take the device memory the server holds above hbm_budget.
 * That memory is what the lanes' codecs count at each allocation they make
 * (lic_codec_device_bytes) plus the frame slabs, never the device's free
 * memory (which other users of the GPU move); a resolution's cost is
 * estimated from its geometry (lic_codec_workspace_bytes) and checked before
 * its workspaces are allocated, then charged as counted.
 *
 * Each request is one frame encoded and decoded again (the round trip the
 * paper's demo makes); its bitstream and decoded frame stay in device memory
 * (the decoded frame is copied out only when the caller gives a buffer).
 * A frame's bitstream and reconstruction do not depend on which other frames
 * share its batch (every kernel computes each frame on its own).
 * Conventions are those of lic.h.
 */
#ifndef LIC_SERVE_H
#define LIC_SERVE_H

#include <stdint.h>

#include "lic.h"

#ifdef __cplusplus
extern "C" {
#endif

/* too many requests in flight (lic_server_submit) */
#ifndef LIC_E_BUSY
#define LIC_E_BUSY (-7)
#endif

typedef struct lic_server lic_server;

typedef struct {
    int max_batch;        /* frames per batch, 1 .. 64 */
    int lanes;            /* codecs (and streams) per resolution, 1 .. 8 */
    int max_pending;      /* requests admitted and not yet completed, >= 1 */
    int graphs;           /* 1: replay each lane's encode+decode as a CUDA graph */
    double max_wait_ms;   /* a partial batch starts once its oldest frame waited this long, >= 0 */
    int64_t hbm_budget;   /* device bytes the server may hold (workspaces, slabs), > 0 */
    int reserved[4];      /* must be 0 */
} lic_server_options;

/* Create a server whose lanes are codecs lic_codec_create(kind, N, M,
 * weights, codec_opt) would make (weights are copied once per lane).
 * No device memory is taken until a resolution is first prepared. */
int lic_server_create(lic_kind kind, int N, int M, const lic_weights *weights, const lic_options *codec_opt,
                      const lic_server_options *opt, lic_server **out);

/* Stops the dispatcher after the requests in flight complete, then frees
 * everything. */
void lic_server_destroy(lic_server *server);

/* Make the bucket of H x W frames ready (its lanes' codecs, workspaces and
 * graphs for every batch size) so that the first request does not pay for
 * it.  LIC_E_OOM when it would exceed hbm_budget (refused before any
 * workspace is allocated when the estimate already exceeds it; only the
 * first lane's weights are created to make the estimate).  Idempotent. */
int lic_server_prepare(lic_server *server, int H, int W);

/* Queue one frame (float32 3 x H x W in [0, 1], host memory -- pinned for
 * asynchronous copies -- or device memory) of stream `stream_id`.  The
 * buffer must stay valid until the request's result is polled.  If
 * `decoded` is non-null the reconstruction (3 x H x W float32, host or
 * device) is written there before the request completes.  *ticket receives
 * the request's number (consecutive from 0).  Errors: LIC_E_BUSY (too many
 * in flight; nothing queued), LIC_E_OOM (a new resolution over budget),
 * LIC_E_INVALID_ARG. */
int lic_server_submit(lic_server *server, int stream_id, const float *frame, int H, int W, float *decoded,
                      uint64_t *ticket);

typedef struct {
    uint64_t ticket;
    int stream_id;
    int status;          /* LIC_OK or the error of its batch (lic_sync's codes) */
    int H, W;
    int batch;           /* frames in the batch it ran in */
    int64_t bytes;       /* size of its bitstream */
    double t_submit_ms;  /* server clock: ms since lic_server_create */
    double t_start_ms;   /* its batch was issued to the GPU */
    double t_done_ms;    /* the batch's completion callback ran */
} lic_server_result;

/* Move up to `cap` completed results into `out`, oldest first, waiting up
 * to wait_ms for the first one.  Returns the number written (>= 0). */
int lic_server_poll(lic_server *server, lic_server_result *out, int cap, double wait_ms);

/* Block until every admitted request has completed (or timeout_ms passed:
 * LIC_E_TIMEOUT). */
int lic_server_drain(lic_server *server, double timeout_ms);

typedef struct {
    int64_t submitted, completed, refused_busy, refused_budget, batches, graph_replays;
    int64_t device_bytes;   /* held by the prepared buckets */
    int buckets;
} lic_server_stats;

int lic_server_stats_get(lic_server *server, lic_server_stats *out);

/* The server clock (ms since lic_server_create). */
double lic_server_clock_ms(lic_server *server);

#ifdef __cplusplus
}
#endif

#endif /* LIC_SERVE_H */
