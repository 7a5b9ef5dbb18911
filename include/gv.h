/*
 * gv.h -- C ABI of libgv, a GB300-native (sm_103a) differentiable tile-based rasterizer
 * of 3D Gaussians into video frames, forward and backward: the hot path of the
 * per-frame training loop of GaussianVideo (arXiv 2501.04782).
 *
 * What the library computes (paper passages):
 *   Sec. 3.1  each Gaussian has a mean mu, a covariance Sigma = (R S)(R S)^T with R a
 *             rotation (unit quaternion) and S a diagonal scale, a colour c (degree-0
 *             spherical harmonics) and an opacity o; the Gaussians are projected and
 *             rasterized onto the image plane and optimised through a reconstruction
 *             loss.  render(gaussians, camera_t, H, W) -> image, and its adjoint.
 *   Sec. 3.2  Eq. 3: colour and opacity constant over time, the mean time-dependent;
 *             here mu_t = mu_0 + t * vel (linear drift), so frames of one clip can share
 *             one Gaussian set and their gradients are summed.
 *   Sec. 3.4  constant pinhole intrinsics (fx, fy, cx, cy), per-frame extrinsics (R, t).
 *   Sec. 4.1  L2 reconstruction loss; the optimiser step (Adam here).
 *
 * Conventions (the paper defers the rasterizer to prior work; these are fixed readings):
 *   scale = exp(log_scale); quaternion (w,x,y,z), normalised inside; opacity =
 *   sigmoid(logit); colour used raw.  World -> camera x_c = R x_w + t (R row-major);
 *   u = fx x/z + cx, v = fy y/z + cy; pixel (i, j) sampled at (i + 0.5, j + 0.5); near
 *   cull z <= 0.2.  EWA: Sigma2 = J R Sigma R^T J^T + 0.3 I, conic = Sigma2^{-1}.
 *   alpha = min(0.99, o exp(-1/2 d^T conic d)); alpha < 1/255 is skipped; front to back
 *   by camera depth (ties by Gaussian index); a Gaussian is composited and then the pixel
 *   stops if T < 1e-4.  image = sum_i c_i alpha_i T_i + T_final * bg.
 *   Binning: the alpha >= 1/255 region of a Gaussian is the ellipse d^T Sigma2^{-1} d <= tau,
 *   tau = 2 ln(255 o).  Its extent box [u - sqrt(tau Sigma2_xx), u + sqrt(tau Sigma2_xx)] x
 *   [v - sqrt(tau Sigma2_yy), ...] (pixel centres inside it) gives a rectangle of tiles; a
 *   tile of that rectangle is kept when one of its pixel columns has its centre between
 *   the two ends of the ellipse over the band of pixel-centre rows of the tile's row
 *   (near-singular footprints, Sigma2_xx Sigma2_yy > 64 det, keep the whole rectangle).
 *   Every pixel that can reach alpha >= 1/255 is therefore in a kept tile, so the image
 *   does not depend on the tile shape.
 *
 * Memory and ownership.  Every pointer below is a DEVICE pointer unless marked host.
 * The caller owns every buffer; render calls never allocate.  All Gaussian parameter and
 * gradient arrays are structure-of-arrays FP32 planes of length N (plane k of mean at
 * mean + k*N).  Images are planar [3][H][W] FP32 per frame; final_T [H][W] FP32;
 * last_idx [H][W] int32.  Frame f's outputs start at pixel_offset (image: 3*pixel_offset).
 *
 * Streams.  Every call is asynchronous and stream-ordered on `stream` (a cudaStream_t).
 * Calls that share a workspace must not overlap on the GPU.  Device-side failures
 * (key capacity overflow, a bounded wait that gave up) are recorded in the workspace
 * and reported by gv_read_status, which synchronises the stream.
 *
 * Errors.  No exception crosses this ABI.  Every call returns a gv_status; the message
 * of the last failure on a context is available from gv_last_error.
 */
#ifndef GV_H_
#define GV_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GV_API __attribute__((visibility("default")))
#else
#define GV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gv_stream; /* same type as cudaStream_t; NULL = legacy default */

typedef enum {
    GV_OK = 0,
    GV_ERR_INVALID_ARG = 1,   /* bad pointer, size, tile shape, frame table ... */
    GV_ERR_CAPACITY = 2,      /* more (tile, Gaussian) keys than the workspace holds */
    GV_ERR_TIMEOUT = 3,       /* a bounded device-side wait gave up */
    GV_ERR_CUDA = 4,          /* a CUDA runtime call failed (message has the CUDA error) */
    GV_ERR_UNIMPLEMENTED = 5,
} gv_status;

typedef struct gv_ctx gv_ctx;

/* Pinhole camera of one frame (Sec. 3.4). */
typedef struct {
    int32_t W, H;        /* image size in pixels */
    float fx, fy, cx, cy;
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];          /* world -> camera translation */
    float time;          /* t in mu_t = mu_0 + t * vel (ignored when vel is NULL) */
} gv_camera;

/* Gaussian parameter planes (Sec. 3.1), each plane N floats. */
typedef struct {
    int64_t N;
    const float *mean;          /* [3][N] */
    const float *vel;           /* [3][N] or NULL (static Gaussians) */
    const float *log_scale;     /* [3][N] */
    const float *quat;          /* [4][N] (w,x,y,z), need not be normalised */
    const float *opacity_logit; /* [N] */
    const float *rgb;           /* [3][N] */
    /* Time-parameterised form (Sec. 3.2): used when n_ctrl > 0, then mean and vel are
     * ignored (may be NULL) and the camera's time t is read in [0, 1] (clamped).
     * Eq. 2: mu(t) = sum_i N_{i,3}(t) P_i, a clamped cubic B-spline over n_ctrl in [4, 64]
     * control points ctrl [3][n_ctrl][N] (knots: four at 0, four at 1, the others evenly
     * spaced).  Eq. 3: log_scale(t) = log_scale + t a1 + t^2 a2 + t^3 a3 with log_scale_t
     * [3][3][N] = (a1, a2, a3) by axis, quat(t) likewise with quat_t [3][4][N] (each NULL:
     * constant in time).  Colour and opacity stay constant. */
    int32_t n_ctrl;
    const float *ctrl;
    const float *log_scale_t;
    const float *quat_t;
    /* View-dependent colour (Sec. 3.1: colour as spherical harmonics of order d_c), used
     * when sh_degree is 1, 2 or 3 (0: the colour is rgb alone).  sh [3][K][N] with
     * K = (sh_degree + 1)^2 - 1: per channel the coefficients of degrees 1..sh_degree in
     * the order (l, m = -l..l); the degree-0 term is rgb itself, so
     *   colour = rgb + sum_k Y_k(d) sh[ch][k],
     * Y_k the real spherical harmonics (orthonormal on the sphere, Condon-Shortley phase:
     * Y_{1,-1} = -sqrt(3/(4 pi)) y, Y_{1,0} = sqrt(3/(4 pi)) z, Y_{1,1} = -sqrt(3/(4 pi)) x,
     * ...) at the unit direction d from the camera centre -R^T t to the mean, in the
     * world frame.  No offset and no clamp. */
    int32_t sh_degree;
    const float *sh;
    /* Optional OUTPUT of the forward (device, [N] bytes, or NULL): for every Gaussian i with
     * at least one kept (tile, Gaussian) key on some frame of the call -- its alpha can
     * reach 1/255 on a pixel of that frame -- the forward sets visible[i] = 1.  It never
     * clears: zero the array, render any number of frames, and the Gaussians left at 0
     * were drawn on none of them (the candidates of the paper's warping of invisible
     * Gaussians, Sec. 4.1).  The backward ignores it. */
    uint8_t *visible;
} gv_gaussians;

/* Gradient planes, same layout; the backward ACCUMULATES (+=) into them.  vel may be
 * NULL (its gradient is then dropped); with the time-parameterised form, mean and vel
 * get nothing and ctrl, log_scale_t, quat_t receive the gradients of those planes.  camera, if not NULL, is [F][16] FP32 (device):
 * per frame of the call the gradient w.r.t. its camera (Sec. 3.4: the extrinsics and the
 * intrinsics), dR[9] (R row-major, taken as a general matrix: the caller maps it to its
 * rotation parameters), dt[3], dfx, dfy, dcx, dcy; also accumulated (+=). */
#define GV_CAMERA_GRAD 16
typedef struct {
    float *mean, *vel, *log_scale, *quat, *opacity_logit, *rgb;
    float *camera;
    float *ctrl, *log_scale_t, *quat_t; /* time-parameterised form: same layouts, or NULL */
    float *sh;                          /* spherical-harmonic coefficients, [3][K][N], or NULL */
} gv_gaussians_grad;

/* One frame of a batch: its camera, the Gaussian subset [gauss_offset, gauss_offset +
 * gauss_count) it renders, and where its outputs start.  The subsets of a batch must be
 * either all the same (one shared set, gradients summed over frames) or pairwise
 * disjoint (one set per frame). */
typedef struct {
    gv_camera cam;
    int64_t gauss_offset, gauss_count;
    int64_t pixel_offset;
} gv_frame_desc;

/* Launch configuration: tile shape (8x8, 16x8, 16x16, 32x16 or 32x32) and the number of Gaussians
 * staged through shared memory per batch (32, 64, 128 or 256); background colour. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t stage_depth;
    float bg[3];
} gv_options;

#define GV_MAX_FRAMES 1024

/* ---- context ---------------------------------------------------------------------- */

/* Create a context bound to the current CUDA device.  opt may be NULL (16x16 tiles,
 * 256 Gaussians per stage, black background).  *ctx is a host object; it owns one
 * non-blocking CUDA stream and two events on that device, with which a backward call runs
 * its FP64 chain-rule kernel beside the FP32 one (forked from and joined back into the
 * call's stream, so the call stays stream-ordered and capturable).  A context is not
 * thread-safe: one call at a time. */
GV_API gv_status gv_create(gv_ctx **ctx, const gv_options *opt);
GV_API gv_status gv_destroy(gv_ctx *ctx);
GV_API gv_status gv_get_options(const gv_ctx *ctx, gv_options *opt);
GV_API gv_status gv_set_options(gv_ctx *ctx, const gv_options *opt);
/* Last failure message on this context (host string owned by the context). */
GV_API const char *gv_last_error(const gv_ctx *ctx);
GV_API const char *gv_status_string(gv_status s);

/* ---- workspace -------------------------------------------------------------------- */

/* Bytes of device workspace for rendering this batch with up to key_capacity
 * (tile, Gaussian) keys (key_capacity <= 0: 16 keys per (frame, Gaussian) pair plus
 * 65536).  frames is a HOST array of F descriptors.  The forward writes, and the
 * backward reads, the workspace; it must stay untouched in between.  The key capacity of
 * a call is derived from ws_bytes, so fwd and bwd must pass the same ws_bytes. */
GV_API gv_status gv_workspace_size(const gv_ctx *ctx, const gv_frame_desc *frames, int32_t F,
                            int64_t key_capacity, size_t *bytes);

/* ---- rendering (Sec. 3.1 forward / adjoint) --------------------------------------- */

/* Forward of F frames in one launch sequence (batched form).  Writes image, final_T and
 * last_idx (position of the last composited Gaussian in the sorted key list, -1 if none)
 * for every pixel of every frame.  frames: HOST array. */
GV_API gv_status gv_render_batch_fwd(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames,
                              int32_t F, void *workspace, size_t ws_bytes, float *image,
                              float *final_T, int32_t *last_idx, gv_stream stream);

/* Adjoint of gv_render_batch_fwd for the upstream gradient dL_dimage (same layout as
 * image).  Reads the workspace, final_T and last_idx written by the forward (nothing is
 * recomputed) and ACCUMULATES the parameter gradients into grad (+=; zero them first).
 * For a shared Gaussian set the per-frame gradients are summed; vel gets sum_t t dmu_t. */
GV_API gv_status gv_render_batch_bwd(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames,
                              int32_t F, void *workspace, size_t ws_bytes, const float *final_T,
                              const int32_t *last_idx, const float *dL_dimage,
                              gv_gaussians_grad *grad, gv_stream stream);

/* Single frame (the plain per-frame renderer): the whole set under one camera (host). */
GV_API gv_status gv_render_fwd(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam, void *workspace,
                        size_t ws_bytes, float *image, float *final_T, int32_t *last_idx,
                        gv_stream stream);
GV_API gv_status gv_render_bwd(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam, void *workspace,
                        size_t ws_bytes, const float *final_T, const int32_t *last_idx,
                        const float *dL_dimage, gv_gaussians_grad *grad, gv_stream stream);

/* The forward with the L2 reconstruction loss of Sec. 4.1 fused into its compositing
 * pass: besides image, final_T and last_idx it writes dL_dimage = 2 scale (image -
 * target) (if not NULL) and adds scale * sum (image - target)^2 to *loss (if not NULL;
 * one device float, accumulated: zero it first), the same values gv_l2_loss_grad computes
 * from the image (the loss up to the order of the float additions).  target: device
 * array in the image's layout, required.  Saves the loss kernel and its re-read of the
 * image. */
GV_API gv_status gv_render_batch_fwd_l2(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames,
                                 int32_t F, void *workspace, size_t ws_bytes, float *image,
                                 float *final_T, int32_t *last_idx, const float *target, float scale,
                                 float *dL_dimage, float *loss, gv_stream stream);
GV_API gv_status gv_render_fwd_l2(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam, void *workspace,
                           size_t ws_bytes, float *image, float *final_T, int32_t *last_idx,
                           const float *target, float scale, float *dL_dimage, float *loss,
                           gv_stream stream);

/* Synchronise `stream` and report device-side failures recorded in the workspace by the
 * last render call: GV_ERR_CAPACITY (then *keys_needed, if not NULL, is the key capacity
 * the call needs: its kept keys, or more when its cells -- the tiles of the Gaussians'
 * extent boxes, up to 2 per key of capacity -- did not fit), GV_ERR_TIMEOUT, else GV_OK
 * (then *keys_needed is the number of keys).  After a failure the call's tile lists are
 * incomplete: the forward renders every tile empty (background, T = 1, last index -1)
 * and the backward adds nothing. */
GV_API gv_status gv_read_status(gv_ctx *ctx, const void *workspace, size_t ws_bytes, gv_stream stream,
                         int64_t *keys_needed);

/* OR the device-side failure bits the last render call recorded in `workspace` into *acc
 * (a DEVICE int32 the caller zeroes), stream-ordered and without host synchronisation, so
 * a failure in any of many launches (steps of a captured graph, say) stays visible until
 * the caller reads *acc: bit 0 key capacity exceeded (gv_read_status's GV_ERR_CAPACITY),
 * bit 1 a device-side wait gave up (GV_ERR_TIMEOUT).  Not part of the paper's method: a
 * record for callers that launch many steps before they synchronise. */
GV_API gv_status gv_status_accumulate(gv_ctx *ctx, const void *workspace, int32_t *acc, gv_stream stream);

/* Synchronise `stream` and read the work counters of the last forward / backward on this
 * workspace (HOST out[6]): [0] keys emitted, [1] (frame, Gaussian) pairs, [2] (pixel,
 * Gaussian) pairs the forward evaluated, [3] pairs with a non-empty extent box (the pairs
 * the depth sort orders after its first pass drops the others), [4] pairs the backward
 * evaluated, [5] of those the pairs replayed (alpha >= 1/255; exactly the pairs the
 * forward composited; counted only by a backward run in profile mode 2 of
 * gv_profile_enable, else 0: the count costs inner-loop instructions).  "Evaluated" counts,
 * per pixel, the list entries up to the pixel's stop (the algorithmic work of compositing). */
GV_API gv_status gv_read_counters(gv_ctx *ctx, const void *workspace, gv_stream stream, int64_t *out);

/* ---- loss and optimiser (Sec. 4.1) ------------------------------------------------ */

/* L2 loss: loss += scale * sum_i (image_i - target_i)^2 (loss is one device float,
 * accumulated; zero it first), dL_dimage = 2 scale (image - target).  n elements. */
GV_API gv_status gv_l2_loss_grad(gv_ctx *ctx, const float *image, const float *target, int64_t n,
                          float scale, float *dL_dimage, float *loss, gv_stream stream);

/* One fused Adam step with bias correction over n parameters:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr (m / (1-b1^step)) /
 * (sqrt(v / (1-b2^step)) + eps).  If zero_grad, g is set to 0 afterwards. */
GV_API gv_status gv_adam_step(gv_ctx *ctx, float *param, float *grad, float *m, float *v, int64_t n,
                       int64_t step, float lr, float beta1, float beta2, float eps,
                       int32_t zero_grad, gv_stream stream);

/* One fused Adan step (Sec. 4.1: the paper trains with Adan; the update of Algorithm 1 of
 * its authors, betas as the weights of the new term, e.g. 0.02, 0.08, 0.01) over n
 * parameters: with d = grad - g_prev,
 *   m = (1-b1) m + b1 grad,  v = (1-b2) v + b2 d,  nsq = (1-b3) nsq + b3 (grad + (1-b2) d)^2,
 *   param = (param - lr (m + (1-b2) v) / (sqrt(nsq) + eps)) / (1 + weight_decay lr),
 * then g_prev = grad (and grad = 0 if zero_grad).  step is 1-based; step 1 starts the
 * moments from grad (m = grad, v = 0, nsq = grad^2).
 * bias_correction != 0: the debiased form the Adan authors use in practice -- step 1
 * starts the moments from zero with d = 0 (m = b1 grad, v = 0, nsq = b3 grad^2), and the
 * update uses m / (1-(1-b1)^step), v / (1-(1-b2)^step), nsq / (1-(1-b3)^step) in place of
 * m, v, nsq (every beta must then be > 0, else GV_ERR_INVALID_ARG).
 * All arrays device FP32 [n]; the moments and g_prev are state owned by the caller, kept
 * between steps (their contents before step 1 are ignored). */
GV_API gv_status gv_adan_step(gv_ctx *ctx, float *param, float *grad, float *m, float *v, float *nsq, float *g_prev,
                              int64_t n, int64_t step, float lr, float beta1, float beta2, float beta3, float eps,
                              float weight_decay, int32_t bias_correction, int32_t zero_grad, gv_stream stream);

/* ---- autotuner -------------------------------------------------------------------- */

/* Time forward + backward of this batch for every tile shape {8x8, 16x8, 16x16, 32x16,
 * 32x32} and stage depth {64, 128, 256} (reps timed runs each after one warm-up, CUDA
 * events on `stream`) and store the fastest in *best (and in the context).  The buffers
 * are the caller's and are overwritten; grad may be any scratch of the right size.  A
 * configuration whose keys do not fit the workspace is skipped (timing INFINITY).  ms_out
 * (HOST, may be NULL) receives GV_AUTOTUNE_CONFIGS = 15 timings in the order tiles x
 * depths.  Synchronises the stream. */
#define GV_AUTOTUNE_CONFIGS 15
GV_API gv_status gv_autotune(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames, int32_t F,
                      void *workspace, size_t ws_bytes, float *image, float *final_T,
                      int32_t *last_idx, const float *dL_dimage, gv_gaussians_grad *grad,
                      int32_t reps, gv_options *best, float *ms_out, gv_stream stream);

/* ---- CUDA graph of the batched forward + backward ---------------------------------- */

typedef struct gv_graph gv_graph;

/* Capture forward + (if dL_dimage != NULL) backward of the batch into a CUDA graph on
 * `stream` (which must not be the legacy default stream).  Pointers are baked in.  If
 * target != NULL the graph also runs the L2 loss between them: *loss is zeroed, then
 * loss = loss_scale * sum (image - target)^2 and dL_dimage = 2 loss_scale (image -
 * target) (dL_dimage is then an output).  gv_graph_set_frames replaces the frame
 * cameras of an instantiated graph (same sizes, offsets and counts) without recapture.
 * The loss is fused into the forward's compositing pass (gv_render_batch_fwd_l2).
 * Launch with gv_graph_launch. */
GV_API gv_status gv_graph_capture(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames,
                           int32_t F, void *workspace, size_t ws_bytes, float *image,
                           float *final_T, int32_t *last_idx, const float *target, float loss_scale,
                           float *loss, float *dL_dimage, gv_gaussians_grad *grad, gv_stream stream,
                           gv_graph **graph);
GV_API gv_status gv_graph_set_frames(gv_graph *graph, const gv_frame_desc *frames, int32_t F);
GV_API gv_status gv_graph_launch(gv_graph *graph, gv_stream stream);
GV_API gv_status gv_graph_destroy(gv_graph *graph);

/* ---- per-stage timing ------------------------------------------------------------- */

/* Stages of one forward + backward, in launch order. */
typedef enum {
    GV_STAGE_SETUP = 0,         /* frame table upload, per-call state cleared */
    GV_STAGE_PROJECT = 1,       /* projection of every (frame, Gaussian) pair */
    GV_STAGE_DEPTH_SORT = 2,    /* radix sort of the pairs by camera depth */
    GV_STAGE_EMIT = 3,          /* tile-count scan and key emission in depth order */
    GV_STAGE_TILE_SORT = 4,     /* stable radix sort of the keys by tile id */
    GV_STAGE_RANGES = 5,        /* per-tile [start, end) of the sorted list (lists of up to
                                   2^22 keys of capacity: recorded by the kernel that writes
                                   the list, no launch of its own and no events) */
    GV_STAGE_COMPOSITE_FWD = 6, /* front-to-back alpha compositing */
    GV_STAGE_COMPOSITE_BWD = 7, /* back-to-front replay, screen-space gradients */
    GV_STAGE_PROJECT_BWD = 8,   /* chain rule to the raw parameters */
    GV_NUM_STAGES = 9
} gv_stage;

/* Record a CUDA event pair around every stage of later render calls on this context
 * (on the call's stream; not inside graph capture).  on = 0 stops recording; on = 2 also
 * makes the backward count the pairs it replays (gv_read_counters out[5]), which costs it
 * a few per cent. */
GV_API gv_status gv_profile_enable(gv_ctx *ctx, int32_t on);

/* Synchronise the recorded events and write, per stage, the milliseconds of the most
 * recent call that ran it (ms[GV_NUM_STAGES], HOST, -1 when not run) and the number of
 * kernels that call launched (launches[GV_NUM_STAGES], HOST, may be NULL). */
GV_API gv_status gv_profile_read(gv_ctx *ctx, float *ms, int32_t *launches);

/* ---- stage-isolated parity hooks -------------------------------------------------- */

/* Binning + sort only, from caller-given screen-space inputs of n Gaussians of ONE frame
 * (W x H): mean u, v, 2D covariance sxx, sxy, syy (Sigma2), tau (the alpha >= 1/255 level
 * 2 ln(255 o)) and depth (all FP32 device arrays), valid (uint8).  Writes counts [n] (int32,
 * the kept tiles of each Gaussian) and the sorted list: sorted_tile [K], sorted_id [K]
 * (uint32, capacity cap) and *K (host).  Uses the same kernels as the render path. */
GV_API gv_status gv_debug_bin_sort(gv_ctx *ctx, int64_t n, const float *u, const float *v, const float *sxx,
                            const float *sxy, const float *syy, const float *tau, const float *depth,
                            const uint8_t *valid, int32_t W, int32_t H, void *workspace, size_t ws_bytes,
                            int32_t *counts, uint32_t *sorted_tile, uint32_t *sorted_id, int64_t cap,
                            int64_t *K, gv_stream stream);

/* Copy out intermediate state of the last forward on this workspace (device pointers,
 * may be NULL): per (frame, Gaussian) pair: mean2d [2][P], conic [3][P], opacity [P],
 * depth [P], tile count [P]; the sorted list ids [K] (pair index) and tiles [K]; tile
 * ranges [2][tiles].  *P, *K, *tiles (host) get the sizes.  Synchronises the stream. */
GV_API gv_status gv_debug_read(gv_ctx *ctx, const gv_frame_desc *frames, int32_t F, const void *workspace,
                        size_t ws_bytes, float *mean2d, float *conic, float *opacity, float *depth,
                        int32_t *counts, uint32_t *sorted_id, uint32_t *sorted_tile, uint32_t *ranges,
                        int64_t *P, int64_t *K, int64_t *tiles, gv_stream stream);

/* Test hook for the bounded waits: spin_limit is the iteration limit of every device-side
 * wait (<= 0 restores the default); drop_signal != 0 makes the first block of each
 * decoupled look-back never publish, so its successors must give up (GV_ERR_TIMEOUT). */
GV_API gv_status gv_debug_set_wait(gv_ctx *ctx, int64_t spin_limit, int32_t drop_signal);

/* Screen-space gradient of the last backward (per pair: du, dv, dA, dB, dC, do, dr, dg,
 * db as [9][P]); out is a device pointer.  Synchronises the stream. */
GV_API gv_status gv_debug_read_grad2d(gv_ctx *ctx, const gv_frame_desc *frames, int32_t F,
                               const void *workspace, size_t ws_bytes, float *out, gv_stream stream);

/* ---- forward without any allocation ------------------------------------------------ */

/* Largest scratch gv_render_fwd_noalloc can use: 32 MiB. */
#define GV_NOALLOC_SCRATCH_BYTES (32u << 20)

/* gv_render_fwd without a caller workspace, for callers that cannot call cudaMalloc at
 * all: a plug-in whose host application owns every device allocation, or a real-time
 * loop that must never let cudaMalloc / cudaFree synchronise the device.  (The paper has
 * no counterpart; this is a deployment convenience.)
 *
 * The scratch is one file-scope device array of GV_NOALLOC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process exits.  The
 * call allocates nothing (no cudaMalloc, no cudaFree, no allocating library routine);
 * image, final_T and last_idx are the caller's device buffers as for gv_render_fwd, and
 * the results are the same.
 *  - Each call looks up the array's device address in the current context (the current
 *    device's); the first call on a device also loads the library's module there, so that
 *    first call should come before any stream capture.
 *  - Every call on a device shares the one array and leaves the last call's contents in
 *    it; each call clears what must start at zero.  Calls that overlap on the GPU (two
 *    streams, two threads, two contexts of one process) race on the array: serialise them.
 *  - A frame whose Gaussian count does not fit returns GV_ERR_INVALID_ARG, one whose keys
 *    do not fit GV_ERR_CAPACITY (every tile then renders empty: background, T = 1, last
 *    index -1), each with a message naming the limit; an invalid frame (size, counts)
 *    returns GV_ERR_INVALID_ARG with gv_render_fwd's message.  The call synchronises
 *    `stream` before it returns, to report a key-capacity overflow. */
GV_API gv_status gv_render_fwd_noalloc(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam,
                                       float *image, float *final_T, int32_t *last_idx,
                                       gv_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GV_H_ */
