/*
 * rmusic_serve.h -- C ABI of the serving loop: continuous batching of camera frame streams onto
 * the FP32-batched demodulation path of rmusic.h (one GPU).
 *
 * The method is single-shot per frame (Sec. 5 of the paper stresses single-frame operation), so
 * a stream needs no temporal state beyond its frames: each open stream owns a ring of device
 * frame slots (input frame, output map, status map) carved from arenas allocated once when the
 * server is created, under its HBM budget. Streams are admitted while their rings fit.
 *
 * A worker thread forms batches from the submitted frames in arrival order and launches one as
 * soon as one of the server's batch slots is free: frames that arrive while other batches run on
 * the GPU join the next batch (continuous batching), and the host-to-device copies, the kernels
 * and the device-to-host copies of different batches overlap on separate CUDA streams. Because
 * every pixel's arithmetic is independent of how frames are batched, a frame's maps are the same
 * alone or in any mix (bit for bit).
 *
 * Buffers passed to rmusic_serve_submit stay owned by the caller and must remain valid, and the
 * output buffers untouched, until the frame's completion is returned by rmusic_serve_poll.
 * Pinned host memory makes the copies asynchronous DMA; pageable memory also works, but a
 * pageable output buffer makes the worker wait for its batch before it can launch the next one.
 * A server may be used from several host threads.
 */
#ifndef RMUSIC_SERVE_H
#define RMUSIC_SERVE_H

#include "rmusic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmusic_server rmusic_server;

/* Server configuration.
 *   max_streams        streams that may be open at once (1 .. 4096).
 *   ring_depth         frame slots per stream: frames of one stream that may be queued or in
 *                      flight at once (1 .. 64); a submit beyond that returns RMUSIC_EAGAIN.
 *   max_batch_frames   frames one device batch may take (1 .. 1024).
 *   max_batch_pixels   pixels one device batch may take; also the largest frame a stream may have.
 *   inflight_batches   batches that may be on the GPU at once, each with its own CUDA stream and
 *                      workspace (1 .. 8).
 *   hbm_budget_bytes   device memory the server may hold: the batch workspaces (8 B per
 *                      max_batch_pixels pixel each) and the stream arenas (9 B per pixel slot).
 */
typedef struct {
    int32_t max_streams;
    int32_t ring_depth;
    int32_t max_batch_frames;
    int32_t inflight_batches;
    uint64_t max_batch_pixels;
    uint64_t hbm_budget_bytes;
} rmusic_serve_config;

/* One finished frame. Times are seconds on the host's monotonic clock: submitted, launched in a
 * batch, and seen finished by the worker (latency = t_done - t_submit). */
typedef struct {
    int32_t stream_id;
    int32_t status;        /* RMUSIC_OK, or the error code of the frame's batch */
    uint64_t tag;          /* the caller's tag from rmusic_serve_submit */
    double t_submit;
    double t_launch;
    double t_done;
    int32_t batch_frames;  /* frames in the batch this frame ran in */
    int32_t pad_;
} rmusic_completion;

typedef struct {
    uint64_t frames_done;
    uint64_t pixels_done;
    uint64_t batches;
    uint64_t submits_rejected;  /* RMUSIC_EAGAIN returned by submit */
    uint64_t opens_rejected;    /* RMUSIC_ENOMEM returned by open_stream */
    uint64_t device_bytes;      /* device memory the server holds */
    uint64_t arena_free_pixels; /* pixel slots still free for new streams */
    int32_t streams_open;
    int32_t frames_queued;
    int32_t batches_inflight;
    int32_t pad_;
} rmusic_serve_stats;

/* Create a server on `device` for the given estimator parameters (precision must be
 * RMUSIC_FP32_BATCHED, geometry RMUSIC_GEOM_ROW). Allocates its arenas and starts its worker
 * thread.
 * Errors: RMUSIC_EINVAL, RMUSIC_EUNSUPPORTED, RMUSIC_ENOMEM, RMUSIC_ECUDA. */
int rmusic_serve_create(const rmusic_params* params, int device, const rmusic_serve_config* cfg,
                        rmusic_server** out);

/* Admit a stream of height x width frames of type dtype (RMUSIC_DTYPE_*). Reserves its ring of
 * ring_depth slots in the arenas; RMUSIC_ENOMEM if the budget cannot hold it (or max_streams are
 * open, or the frame exceeds max_batch_pixels). On success *stream_id receives its id. */
int rmusic_serve_open_stream(rmusic_server* s, int32_t height, int32_t width, int32_t dtype,
                             int32_t* stream_id);

/* Queue one frame of a stream. h_frame: height x width samples (dense rows) in host memory;
 * h_out: height x width float32 for the derivative map; h_status: height x width uint8 or NULL.
 * RMUSIC_EAGAIN if all ring slots of the stream are busy; RMUSIC_EINVAL for a bad stream id. */
int rmusic_serve_submit(rmusic_server* s, int32_t stream_id, const void* h_frame, float* h_out,
                        uint8_t* h_status, uint64_t tag);

/* Copy up to max finished frames into out (oldest first), waiting up to timeout_ms for the first
 * one (0 = do not wait). Returns the number copied (>= 0) or a negative error. */
int rmusic_serve_poll(rmusic_server* s, rmusic_completion* out, int32_t max, int32_t timeout_ms);

/* Close a stream: waits until its queued and in-flight frames have finished (their completions
 * stay available to poll), then returns its ring to the arenas. */
int rmusic_serve_close_stream(rmusic_server* s, int32_t stream_id);

int rmusic_serve_get_stats(rmusic_server* s, rmusic_serve_stats* out);

/* Stop the worker after the frames already submitted have finished, and free everything. NULL is
 * allowed. */
void rmusic_serve_destroy(rmusic_server* s);

#ifdef __cplusplus
}
#endif

#endif /* RMUSIC_SERVE_H */
