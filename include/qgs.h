/*
 * qgs.h - C ABI of the GB300 (sm_103a) quadric Gaussian splatting rasterizer.
 *
 * The library renders and differentiates the paraboloid Gaussian primitives of
 * "Quadratic Gaussian Splatting" (arXiv 2411.16392):
 *   - primitive parameters: Sec. 3.2 (position c, rotation R, scales, signed curvature);
 *     here mean, quaternion (w, x, y, z), in-surface scales (s_u, s_v) = (|s1|, |s2|),
 *     curvatures (a, b) = (sign(s1) s3 / s1^2, sign(s2) s3 / s2^2) of the local surface
 *     z = a x^2 + b y^2 (the lambda_1, lambda_2 of the curvature paragraph), opacity and
 *     degree-3 SH colour (Sec. 3.1);
 *   - geodesic Gaussian G = exp(-l^2 / (2 sigma(theta)^2)) with the closed-form arc
 *     length l (Sec. 3.2, geodesic Eq.);
 *   - ray-splat intersection and near/far hit selection within 3 sigma (Sec. 3.2.1 and
 *     the supplementary's intersection section);
 *   - front-to-back alpha blending of colour, alpha, depth and normal (Sec. 3.1 blending
 *     Eq., Sec. 3.2 normal/curvature-map Eq.);
 *   - 16x16 tiles ordered by 64-bit (tile << 32 | depth bits) keys (supplementary,
 *     per-tile sorting);
 *   - the reverse-order backward of the supplementary's dX/d(alpha) formula.
 *
 * Conventions for every entry point:
 *   - Every function returns a qgs_status; nothing aborts or exits. On failure the
 *     context keeps a message readable with qgs_last_error().
 *   - Pointers inside qgs_scene, qgs_image and qgs_scene_grad are DEVICE pointers on
 *     the context's device, owned by the caller, and must stay valid until the work
 *     enqueued on `stream` has finished. Inputs are never modified.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     All device work is enqueued on it. render_forward synchronises the stream once
 *     (to size the tile-instance buffers from the instance count); render_backward
 *     does not synchronise.
 *   - The radix sorts wait for each other's chunks with bounded waits. A wait that runs
 *     out (which should not happen on a healthy GPU) makes the frame's later kernels do
 *     nothing, and render_forward has already returned by then: the failure is reported
 *     as QGS_ECUDA by the first later call on the context that waits for the frame:
 *     qgs_check_frame, render_backward, qgs_get_frame_stats, qgs_copy_binning,
 *     qgs_copy_residue, or else the next render_forward / render_forward_batch. The
 *     frame is then discarded (render_backward refuses it).
 *   - A context is not thread-safe; use one per host thread. The serving object
 *     (qgs_server) is thread-safe.
 *   - Images are planar float32: rgb[c*H*W + y*W + x], alpha[y*W + x], ...
 */
#ifndef QGS_H_
#define QGS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QGS_OK = 0,
  QGS_EINVAL = 1,      /* bad argument (null pointer, size, non-finite camera, ...) */
  QGS_ENOMEM = 2,      /* device or host allocation failed */
  QGS_ECAPACITY = 3,   /* a fixed-capacity buffer (serving) is too small for a frame */
  QGS_ECUDA = 4,       /* a CUDA runtime call or kernel launch failed */
  QGS_ETIMEDOUT = 5,   /* a bounded wait ran out */
  QGS_EBUSY = 6,       /* the serving queue is full */
  QGS_ENOTFOUND = 7,   /* unknown scene id or ticket */
  QGS_ESTATE = 8       /* call out of order (backward without a matching forward) */
} qgs_status;

typedef void* qgs_stream; /* cudaStream_t */

/* Pinhole camera. x_cam = R_cw * x_world + t_cw (R_cw row-major). The ray through
 * pixel (px, py) goes through its centre: d_cam = ((px+0.5-cx)/fx, (py+0.5-cy)/fy, 1),
 * so the ray parameter t is the camera-space z depth. Hits with t <= near_plane are
 * ignored and primitives whose centre has z <= near_plane are culled. */
typedef struct {
  int32_t W, H;
  float fx, fy, cx, cy;
  float R_cw[9];
  float t_cw[3];
  float near_plane;
} qgs_camera;

/* Scene: n primitives, device pointers (float32 unless stated). */
typedef struct {
  int64_t n;
  const float* mean;      /* [n*3] world-space centre */
  const float* quat;      /* [n*4] (w, x, y, z), any nonzero norm */
  const float* scale;     /* [n*2] (s_u, s_v) > 0 */
  const float* curv;      /* [n*2] (a, b) */
  const float* opacity;   /* [n]   in (0, 1) */
  const uint16_t* sh;     /* [n*48] bfloat16 bits, index k*3 + c (SH coefficient k, channel c) */
} qgs_scene;

/* Image planes (device pointers). Output of render_forward (fully overwritten) or the
 * upstream gradient given to render_backward (read only). The last three planes are
 * optional extra channels (NULL: not rendered / zero gradient); the first four are
 * required in a forward. Planar layout, row-major, w_i = alpha_i T_i of the i-th blended
 * pair in list order, t_i its hit depth. */
typedef struct {
  float* rgb;      /* [3*H*W] */
  float* alpha;    /* [H*W]   1 - final transmittance */
  float* depth;    /* [H*W]   sum_i w_i t_i (unnormalised expected z depth) */
  float* normal;   /* [3*H*W] sum_i w_i n_i, camera space, each n_i facing the camera */
  float* curvature;    /* [H*W] sum_i w_i K_i, K_i the Gaussian curvature 4ab/(1+4a^2x^2+4b^2y^2)^2
                          at the local hit (x, y) (Sec. 3.2.1, curvature and N/K Eqs.) */
  float* distortion;   /* [H*W] sum_i sum_{j<i} w_i w_j (t_i - t_j)^2 (Sec. 3.3 depth distortion) */
  float* median_depth; /* [H*W] max t_i over blended pairs with T_i > 0.5, 0 if none (Sec. 4.1);
                          forward only: its gradient plane must be NULL */
} qgs_image;

/* Gradients of a scalar loss with respect to the scene parameters (device pointers,
 * float32, same layouts as qgs_scene; sh is float32 [n*48]). render_backward ADDS into
 * them; the caller zeroes them when needed. */
typedef struct {
  float* mean;
  float* quat;
  float* scale;
  float* curv;
  float* opacity;
  float* sh;
} qgs_scene_grad;

/* Blending constants and pipeline options. qgs_config_default() gives the values the
 * oracle and the tests use: alpha_max 0.99, alpha_min 1/255, T_min 1e-4,
 * grazing_eps 1e-5 (roots whose discriminant D satisfies |D| <= grazing_eps * B^2 are
 * re-solved in FP64), sort_mode 0, density 0, order 0. */
typedef struct {
  float alpha_max;
  float alpha_min;
  float T_min;
  float grazing_eps;
  int32_t sort_mode;   /* 0: per-primitive depth sort, then a stable sort of the
                          (tile, primitive) instances by tile: the same order as sorting
                          the 64-bit keys, with fewer passes over the instances.
                          1: one radix sort of the full 64-bit tile|depth keys. */
  int32_t density;     /* 0: geodesic Gaussian (the paper's, Sec. 3.2); 1: Euclidean-distance
                          Gaussian, l = sqrt(rho^2 + z^2) from the vertex with the same
                          sigma(theta) (the "w/ Euclid" variant of Sec. 4.3) */
  int32_t order;       /* 0: tile lists by centre depth; 1: StopThePop ordering
                          (supplementary, per-tile sorting and per-pixel resorting): lists
                          sorted by each primitive's depth on the tile pixel ray closest to
                          its projected vertex, then per-pixel resorting in a buffer of 8
                          entries, with a front-to-back backward. sort_mode is ignored;
                          render_forward_batch refuses it (EINVAL). */
} qgs_config;

/* Counters of the last render_forward / render_backward. Pair counters classify the
 * (pixel, listed primitive) pairs visited before each pixel stopped. Stage times are
 * CUDA-event times on the caller's stream, filled only while profiling is enabled
 * (qgs_set_profiling), else -1. The pair counters read -1 when the frame ran without
 * them (qgs_set_pair_counters). */
typedef struct {
  int64_t n_primitives;
  int64_t n_visible;        /* primitives with a nonempty tile rectangle */
  int64_t n_instances;      /* (tile, primitive) pairs = sort length */
  int64_t n_tiles;
  int64_t pair_evals;       /* forward: pairs visited (the pair that stopped a pixel included) */
  int64_t pair_isect;       /* forward: pairs inside the primitive's screen conic (quadratic solved) */
  int64_t pair_hits;        /* forward: pairs with a root within 3 sigma */
  int64_t pair_blended;     /* forward: pairs blended */
  int64_t grazing_resolves; /* forward: pairs whose roots were re-solved in FP64 */
  int64_t bwd_pairs;        /* backward: pairs recomputed */
  int64_t bwd_contrib;      /* backward: pairs that produced a gradient */
  int64_t launches_fwd;     /* kernels launched by the last render_forward */
  int64_t launches_bwd;     /* kernels launched by the last render_backward */
  float ms_preprocess, ms_depth_sort, ms_emit, ms_tile_sort, ms_raster_fwd;
  float ms_raster_bwd, ms_preprocess_bwd;
} qgs_frame_stats;

typedef struct qgs_ctx qgs_ctx;

/* Default constants (see qgs_config). Never fails. */
void qgs_config_default(qgs_config* cfg);

/* Create a rendering context on CUDA device `device`. The context owns its work
 * buffers (projected primitives, keys, tile ranges, per-pixel residue), grown on
 * demand. cfg may be NULL for the defaults. Errors: EINVAL, ECUDA, ENOMEM. */
qgs_status qgs_create(qgs_ctx** out, const qgs_config* cfg, int32_t device);

/* Free a context and its device buffers (waits for its work). NULL is ignored. */
void qgs_destroy(qgs_ctx* ctx);

/* Message of the last failure on this context ("" if none). Valid until the next call. */
const char* qgs_last_error(const qgs_ctx* ctx);

/* Forward render (Sec. 3.1-3.2, supplementary): preprocessing, tile binning, radix sort,
 * per-tile compositing. Writes the four base planes of `out` (W*H from `cam`) and each
 * non-NULL extra plane. Keeps the per-pixel residue (final transmittance, the count of
 * listed primitives up to the last blended one and, when an extra plane was requested,
 * the distortion's moments) and the sorted lists in the context for render_backward.
 * Errors: EINVAL, ENOMEM, ECUDA. */
qgs_status render_forward(qgs_ctx* ctx, const qgs_scene* scene, const qgs_camera* cam,
                          const qgs_image* out, qgs_stream stream);

/* Forward render of n_views views of ONE scene in shared launches: the serving path's
 * batch (the paper renders one view at a time, Sec. 4.1; the per-view arithmetic is that
 * of render_forward, Sec. 3.1-3.2 and the supplementary). cams[v] and outs[v] (host
 * arrays of n_views structs; the planes are device pointers, W*H of cams[v]) may all
 * differ in resolution. One preprocessing launch covers views x primitives, one depth
 * sort orders all (view, primitive) entries, the tile instances of view v are numbered
 * from the sum of the earlier views' tile counts, one tile sort and one compositing
 * launch cover every view. Each view's planes equal render_forward's for that camera
 * bit for bit. Work buffers scale with n_views * n primitive entries; n_views * n must
 * stay below 2^31 and n_views in [1, 1024]. Extra planes may be requested per view.
 * The instance order is always the factorised one (qgs_config.sort_mode is ignored). No
 * residue is kept:
 * render_backward cannot follow it, and the context's last frame is cleared.
 * Errors: EINVAL, ENOMEM, ECUDA. */
qgs_status render_forward_batch(qgs_ctx* ctx, const qgs_scene* scene, int32_t n_views,
                                const qgs_camera* cams, const qgs_image* outs, qgs_stream stream);

/* Backward of the last render_forward on this context (same scene pointers, same camera):
 * reverse-order traversal per pixel with transmittance recomputed from the residue
 * (supplementary, dX/d(alpha) back-to-front form), then the chain rule to every primitive
 * parameter. grad_out holds dL/d(rgb, alpha, depth, normal, curvature, distortion); a
 * NULL plane means zero; median_depth must be NULL (EINVAL). A distortion gradient needs
 * a forward that rendered at least one extra plane (ESTATE otherwise).
 * Results are ADDED into `grad`. Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
qgs_status render_backward(qgs_ctx* ctx, const qgs_scene* scene, const qgs_camera* cam,
                           const qgs_image* grad_out, const qgs_scene_grad* grad,
                           qgs_stream stream);

/* Counters (and, when profiling, stage times) of the last forward and backward.
 * Synchronises the context's last stream. Errors: EINVAL, ESTATE, ECUDA. */
qgs_status qgs_get_frame_stats(qgs_ctx* ctx, qgs_frame_stats* stats);

/* Enable (1) or disable (0) CUDA-event timing of each pipeline stage on the caller's
 * stream. Off by default; costs a few event records per call. Errors: EINVAL, ECUDA. */
qgs_status qgs_set_profiling(qgs_ctx* ctx, int32_t enable);

/* Collect (1, the default) or skip (0) the per-pair counters of qgs_frame_stats in the
 * compositing kernels of the base ordering (the StopThePop kernels always count). Without
 * them the forward runs a few percent faster and the pair counters read -1; nothing else
 * changes. Takes effect at the next render call. Errors: EINVAL. */
qgs_status qgs_set_pair_counters(qgs_ctx* ctx, int32_t enable);

/* Capacity, in 32-bit words, of the context's tile-mask store: the tile-count pass keeps
 * each primitive's per-tile test results (one bit per tile of its rectangle) so that the
 * instance emission replays them instead of testing again. Primitives that do not fit are
 * tested again (same lists, more time); the store grows by itself after a frame that
 * overflowed it. 0 disables the store until it is set again. Takes effect at the next
 * forward; does not change any result. Errors: EINVAL (ctx null or words < 0). */
qgs_status qgs_set_tile_mask_capacity(qgs_ctx* ctx, int64_t words);

/* Wait until the sorts of the last render_forward / render_forward_batch have run and
 * report them: QGS_OK, or QGS_ECUDA when a look-back wait ran out (the frame's lists and
 * images are invalid and the frame is discarded). Returns QGS_OK at once when the frame
 * has already been checked. Errors: EINVAL, ECUDA. */
qgs_status qgs_check_frame(qgs_ctx* ctx);

/* Test hook for the failure path of the sorts' bounded waits (the paper has no
 * counterpart). With spins > 0, the next forward's first radix sort that runs its passes
 * as single kernels with decoupled look-back (sorts of 2,049 to 2M keys: the depth sort
 * of that many visible primitives) withholds chunk 0 of its first pass, so the chunks
 * after it wait for digit counts that are never published; each wait gives up after
 * `spins` polls (about a microsecond each), the sort's failure word is set, and the
 * frame fails as described in the conventions above. One-shot: the hook is consumed by
 * the next forward. spins <= 0 clears it. Errors: EINVAL. */
qgs_status qgs_debug_withhold_sort_chunk(qgs_ctx* ctx, int32_t spins);

/* Debug bounds checks (the paper has no counterpart). A library built with
 * -DQGS_DEBUG_CHECKS (paper_2411_16392_gb300.build.build(debug_checks=True), which writes
 * libqgs_check.so beside libqgs.so) checks the computed indices of its binning kernels: the
 * slot of every emitted tile instance against the frame's instance count (bit 1), every
 * tile id of the range pass against the tile grid (bit 2), and every scatter position of the
 * radix sort against its chunk and its key count (bit 4). A failed check sets its bit and
 * skips the access (nothing traps). This call waits for the device `device`, then reports
 * whether the checks are compiled in (*compiled_in, 0 or 1) and the bits set since the last
 * call on that device (*word, cleared by the read). In the normal build *compiled_in and
 * *word are 0 and the device is not touched. Errors: EINVAL (NULL pointer, bad device),
 * ECUDA. */
qgs_status qgs_debug_check_word(int32_t device, int32_t* compiled_in, uint32_t* word);

/* Copy the last forward's tile binning to HOST memory, for inspection and tests:
 * keys[i] = (tile << 32) | float bits of the primitive's view depth, vals[i] = primitive
 * index, in sorted order (cap entries at most); ranges[2*t], ranges[2*t+1] = [start, end)
 * of tile t; rects[4*i] = (tx0, tx1, ty0, ty1) of primitive i (-1s when culled).
 * Any pointer may be NULL. *n_instances receives the instance count.
 * Errors: EINVAL, ESTATE, ECAPACITY (cap too small), ECUDA. */
qgs_status qgs_copy_binning(qgs_ctx* ctx, uint64_t* keys, uint32_t* vals, int64_t cap,
                            uint32_t* ranges, int32_t* rects, int64_t* n_instances);

/* Copy the last forward's per-pixel residue to HOST memory: final transmittance and
 * n_contrib (index + 1, within the pixel's tile list, of its last blended primitive). */
qgs_status qgs_copy_residue(qgs_ctx* ctx, float* T_final, uint32_t* n_contrib);

/* Forward render that allocates nothing. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory at render time, e.g. a host
 * process whose memory manager takes the GPU's memory in one pool at start-up and
 * refuses other allocations, or a real-time loop that forbids cudaMalloc/cudaFree after
 * warm-up because they can block and fragment memory. It computes the same planes as
 * render_forward with the default qgs_config, bit for bit: the same kernels and the same
 * tile lists (the tile test against the parallelogram and the conic), with only the
 * intermediate layout changed (64-bit instances, primitive-indexed state, no tile-mask
 * store). Every work buffer comes from one statically sized device array (about 27 MB)
 * that each GPU loading the library holds until the process exits; it calls no
 * cudaMalloc, cudaFree or allocating library routine, and needs no context.
 *   Limits: n <= 32768 primitives, W*H <= 262144 pixels, at most 4096 16x16 tiles, and at
 *   most 1,048,576 (tile, primitive) instances in the frame; beyond them it returns
 *   QGS_ECAPACITY (the instance count is known only after the tile test, so that case is
 *   reported after a synchronisation of `stream`, with `out` unspecified).
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *   with that device current; make that first call before any stream capture.
 *   All calls in the process share the array and leave their contents in it (each call
 *   clears what must start at zero): calls whose GPU work overlaps (concurrent streams,
 *   host threads) race and corrupt each other's results; serialise them.
 *   Scene/camera/output pointers follow the conventions above (base planes only: the
 *   extra planes must be NULL); the call synchronises `stream` twice (for the instance
 *   count, and at the end to read its sorts' failure word, so a look-back wait that ran
 *   out is reported by this call as QGS_ECUDA). Errors: EINVAL, ECAPACITY, ECUDA. No
 *   per-call residue is kept, so render_backward cannot follow it. */
qgs_status render_forward_noalloc(const qgs_scene* scene, const qgs_camera* cam, const qgs_image* out,
                                  qgs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* QGS_H_ */
