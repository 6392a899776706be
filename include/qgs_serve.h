/*
 * qgs_serve.h - serving loop of the quadric Gaussian splatting rasterizer.
 *
 * The paper renders one view at a time during training (Sec. 4.1); serving novel views
 * of resident scenes is this library's own layer around the same forward render
 * (include/qgs.h: render_forward, Sec. 3.1-3.2 and the supplementary). It implements
 * continuous batching:
 *   - scenes are copied once into server-owned device memory (serve_load_scene);
 *   - serve_submit enqueues a view request (forward, or forward + backward with upstream
 *     gradients) and returns at once (bounded FIFO queue);
 *   - worker slots, each with its own rendering context and CUDA stream, take requests
 *     from the head of the queue as soon as a slot is free AND the request's estimated
 *     memory (projected primitives, tile keys and their sort buffers, residue, result
 *     planes) fits in the remaining HBM budget; requests that arrive while others run
 *     are admitted as slots and memory free up, and their kernels overlap on the GPU;
 *   - on a server with a single slot (max_slots = 1), the slot that takes the head also
 *     takes up to max_batch - 1 further queued forward requests of the same scene (queue
 *     order, each only while the budget still holds it) with frames of at most 512x384
 *     pixels, and renders them, at their own resolutions, in shared launches
 *     (render_forward_batch), which saves each view its launches and host round trip; a
 *     batch of one runs render_forward. With several slots those fixed costs are hidden
 *     by the other slots' kernels and concurrent single renders are faster, so no batches
 *     form there;
 *   - serve_wait returns a finished result (host or device destination) with a bounded
 *     wait; serve_stats reports p50/p99 latency (submit to result ready) and frames/s.
 * All functions are thread-safe. Status codes as in qgs.h; nothing aborts.
 */
#ifndef QGS_SERVE_H_
#define QGS_SERVE_H_

#include "qgs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qgs_server qgs_server;

typedef struct {
  int64_t submitted;       /* accepted by serve_submit */
  int64_t completed;       /* finished (ok or failed) */
  int64_t failed;          /* finished with an error status */
  int64_t rejected;        /* refused by serve_submit (queue full: QGS_EBUSY) */
  int64_t max_in_flight;   /* most requests running at once */
  double p50_ms, p99_ms, mean_ms;  /* latency submit -> result ready, completed requests */
  double frames_per_s;     /* completed / (last completion - first submission) */
  int64_t bytes_budget;    /* HBM budget given to serve_create */
  int64_t bytes_reserved_peak; /* most estimated bytes admitted at once */
  int64_t batches;         /* batches started (each of >= 1 request) */
  int64_t max_batch;       /* most requests in one batch */
} qgs_serve_stats;

/* Create a server on CUDA device `device` with `max_slots` worker slots in [1, 64],
 * batches of at most `max_batch` requests in [1, 1024] (max_slots = max_batch = 1 is
 * plain one-request-at-a-time serving), a queue of `queue_capacity` requests and an HBM
 * budget for in-flight requests. device = -1 creates a host-only server whose workers
 * do not touch a GPU and take `fake_us_per_mpix` microseconds per million pixels of a
 * batch (for testing the queue, admission, batching and accounting without a GPU;
 * results are zero). Errors: EINVAL, ECUDA, ENOMEM. */
qgs_status serve_create(qgs_server** out, int32_t device, int64_t hbm_budget_bytes, int32_t max_slots,
                        int32_t max_batch, int32_t queue_capacity, double fake_us_per_mpix);

/* Stop the workers after the running requests finish, drop queued requests, free
 * everything. NULL is ignored. */
void serve_destroy(qgs_server* srv);

/* Copy a scene (device pointers, layouts of qgs_scene) into server-owned device memory;
 * *scene_id receives its id. The copy is ordered after work on the legacy default stream
 * (work on other streams that writes the source must be finished by the caller) and is
 * complete when the call returns. Not counted in the per-request budget. Errors: EINVAL,
 * ENOMEM, ECUDA. */
qgs_status serve_load_scene(qgs_server* srv, const qgs_scene* scene, int32_t* scene_id);

/* Enqueue a render of scene `scene_id` from `cam`; returns with a ticket once queued.
 * want_backward = 0: forward only (on a single-slot server, batched with other queued
 * forward views of the scene).
 * want_backward = 1: forward, then the backward of sum(grad_out . planes) (render_backward;
 * the paper's training step, Sec. 3.3, without the optimiser); grad_out's four base planes
 * (rgb 3HW, alpha HW, depth HW, normal 3HW; host or device; a NULL plane or grad_out = NULL
 * means zero) are copied before the call returns; its extra planes must be NULL. A backward
 * request runs alone and its parameter gradients are returned by serve_wait.
 * Errors: EINVAL (bad camera, size or plane), ENOTFOUND (scene), EBUSY (queue full),
 * ECAPACITY (the request alone exceeds the budget), ENOMEM/ECUDA (upstream copy). */
qgs_status serve_submit(qgs_server* srv, int32_t scene_id, const qgs_camera* cam, int32_t want_backward,
                        const qgs_image* grad_out, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: no limit) for a ticket to finish, then copy its planes
 * into `out` (rgb 3HW, alpha HW, depth HW, normal 3HW floats; any plane may be NULL;
 * host or device pointers; the extra planes of qgs_image are not served and must be
 * NULL) and, for a backward request, its parameter gradients into `grad` (float32 arrays
 * in qgs_scene layouts, sh float32 [n*48]; overwritten, not added; any array may be NULL;
 * grad must be NULL for a forward request: EINVAL), then release the ticket. The copies
 * are ordered after work on the legacy default stream; work on other streams that writes
 * the destinations must be finished by the caller. Returns after the copies have
 * completed. Errors: ENOTFOUND (unknown or already released ticket), ETIMEDOUT (still
 * running; the ticket stays valid), EINVAL, the request's own error status, ECUDA. */
qgs_status serve_wait(qgs_server* srv, uint64_t ticket, int32_t timeout_ms, const qgs_image* out,
                      const qgs_scene_grad* grad);

/* Statistics since creation or the last serve_reset_stats. */
qgs_status serve_stats(qgs_server* srv, qgs_serve_stats* stats);
qgs_status serve_reset_stats(qgs_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* QGS_SERVE_H_ */
