/*
 * exw.h -- C ABI of the ExWarp warping fast path on GB300 (sm_103a).
 *
 * ExWarp (arXiv 2307.12607) inserts three frames P_1, P_2, P_3 at t + 1/4, t + 1/2, t + 3/4 between two rendered
 * frames F_t and F_{t+1}, built from F_t alone (Sec. IV-A, IV-B).  Its fast path warps the last frame with its
 * motion vectors (Sec. I, Sec. II-B, Sec. III-B); the warped frame has invalid pixels ("holes", Sec. III-B,
 * III-C) that are marked and filled.  This library implements that path as three stages:
 *   (a) forward splat of the scaled motion field with z-buffering        -- exw_splat_motion
 *   (b) backward bilinear gather of colour with a hole mask              -- exw_warp
 *   (c) pull-push hole filling                                           -- exw_fill_holes
 * fused into one pass over all fractions (exw_extrapolate, exw_extrapolate_batched), plus the motion bounds that
 * size the splat's search window (exw_motion_bounds) and the adjoint of (b) (exw_warp_backward).
 *
 * The paper does not spell out the warp itself; the library takes these readings (the same ones as the test
 * oracle):
 *   - motion mv(p) is the displacement in pixels of the surface at p over one frame interval, forward in time;
 *     fraction k/denom of it moves p to T(p) = p + floor(1/2 + k mv(p) / denom) per axis (round half up);
 *   - the splat keeps, per target, the nearest depth, ties to the smallest source index:
 *         key[q] = min over {p : T(p) = q} of (bits(depth(p)) << 32) | (y_p * W + x_p),  EMPTY = ~0ull;
 *   - the gather samples colour bilinearly at p + rho, rho = (T(p) - p) - k mv(p)/denom in (-1/2, 1/2], with
 *     taps on rho's side; a tap takes part when in frame and |D(t) - D(p)| <= D(p)/32, and the participating
 *     weights are renormalised;
 *   - mask bit 0 (EMPTY): nothing landed; bit 1 (CRACK): at least 3 in-frame 4-neighbours hold a surface nearer
 *     by more than D_q/32.  Holes (mask != 0) output 0 before the fill;
 *   - the fill is pull-push over a ceil-halving mip pyramid (children averaged in the order (0,0),(0,1),(1,0),
 *     (1,1)); holes take the value of their first valid ancestor; valid pixels are unchanged.
 *
 * Conventions for every entry point:
 *   - All image pointers are DEVICE pointers to dense planar arrays aligned to their element size:
 *       colour [3][H][W] (float32 or float16, exw_dtype), depth [H][W] float32, motion [2][H][W] float32 (plane 0
 *       = x, pixels / frame), keys [H][W] uint64, mask [H][W] uint8.  Pixel (x, y) has index y * W + x.
 *       Workspaces and tile_bounds must be 16-byte aligned.
 *   - Sizes: 1 <= W, H <= 16384.  Fractions: denom is a power of two in [1, 64] and 0 <= k <= denom.
 *   - A source pixel whose depth is not positive and finite, or whose motion is not finite, never lands.
 *   - Work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t; NULL = legacy default stream) and
 *     runs asynchronously.  The caller owns every buffer.  No entry point allocates device memory; scratch comes
 *     from a caller-provided workspace of exw_workspace_bytes() bytes (16-byte aligned), which the call
 *     initialises itself.  Calls that share a workspace must be ordered on one stream.
 *   - Return value: EXW_OK when the work was enqueued; EXW_ERR_INVALID_ARG for a null, misaligned or out-of-range
 *     argument (nothing is enqueued); EXW_ERR_WORKSPACE for a workspace smaller than required; EXW_ERR_CUDA when a
 *     launch failed (including a sticky error left by earlier work); EXW_ERR_UNSUPPORTED for a valid but
 *     unimplemented combination.  Errors found on the device (a bounded wait that ran out) are reported through
 *     exw_device_status().
 */
#ifndef EXW_H
#define EXW_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define EXW_API __attribute__((visibility("default")))
#else
#define EXW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *exw_stream_t; /* identical to cudaStream_t */

typedef enum exw_status {
    EXW_OK = 0,
    EXW_ERR_INVALID_ARG = 1,
    EXW_ERR_UNSUPPORTED = 2,
    EXW_ERR_CUDA = 3,
    EXW_ERR_TIMEOUT = 4,
    EXW_ERR_WORKSPACE = 5
} exw_status;

typedef enum exw_dtype {
    EXW_F32 = 0, /* float32 colour */
    EXW_F16 = 1  /* IEEE binary16 colour; arithmetic in float32, one round-to-nearest on output */
} exw_dtype;

typedef enum exw_op {
    EXW_OP_MOTION_BOUNDS = 0,
    EXW_OP_FILL_HOLES = 1,
    EXW_OP_EXTRAPOLATE = 2,
    EXW_OP_WARP_BACKWARD = 3,
    EXW_OP_STATS = 4,
    EXW_OP_WARP_RECURSIVE = 5,
    EXW_OP_WARP_L2_GRAD = 6
} exw_op;

#define EXW_MASK_EMPTY 1u
#define EXW_MASK_CRACK 2u
#define EXW_KEY_EMPTY 0xFFFFFFFFFFFFFFFFull
#define EXW_BOUNDS_BLOCK 8      /* side of the square tiles of exw_motion_bounds */
#define EXW_FILL_TILE 32        /* side of the fill's shared-memory tiles (pyramid levels 1..5) */
#define EXW_MAX_FRAC 3          /* P_1..P_3 (Sec. IV-B) */

/* Flags of exw_extrapolate / exw_extrapolate_batched. */
#define EXW_FLAG_NO_FILL 1u     /* stop after stage (b): holes stay 0, as exw_warp leaves them */
#define EXW_FLAG_NO_TMA 2u      /* read the source from global memory instead of TMA-staged shared-memory windows
                                   (identical results; the TMA path needs 16-byte aligned bases and W a multiple
                                   of 4 for float32 colour, of 8 for float16 colour, and is used when possible) */

/* One source frame F_t (device pointers, layouts above). */
typedef struct exw_frame {
    const void *color;  /* [3][H][W], cdt */
    const float *depth; /* [H][W] */
    const float *mv;    /* [2][H][W] */
    int W, H;
    exw_dtype cdt;
} exw_frame;

/* One extrapolated frame P_k (device pointers). */
typedef struct exw_frame_out {
    void *color;    /* [3][H][W], same dtype as the source colour */
    uint8_t *mask;  /* [H][W], EXW_MASK_* bits of stage (b) */
} exw_frame_out;

/* Human-readable name of a status code (static storage). */
EXW_API const char *exw_status_string(exw_status s);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
EXW_API int exw_version(void);

/* Bytes of workspace the named operation needs for a W x H frame (nframes frames of nfrac fractions for
 * EXW_OP_EXTRAPOLATE; 1 otherwise).  Returns 0 for invalid arguments. */
EXW_API size_t exw_workspace_bytes(exw_op op, int W, int H, exw_dtype cdt, int nframes, int nfrac);

/* Stage (a0): motion bounds that limit how far any fraction of the motion can carry a source pixel (the halo of
 * the splat's search window; a step of this library that the paper does not have: it reads the per-pixel
 * motion-vector buffer of Sec. III-D that the warp of Sec. III-B uses).  Over the pixels that can land (positive
 * finite depth, finite motion), with each motion component clamped to [-65536, 65536] and -0 read as +0:
 *   tile_bounds  [ceil(H/8)][ceil(W/8)][4] float32 device, or NULL: [min mv_x, max mv_x, min mv_y, max mv_y] per
 *                8 x 8 tile; a tile with no such pixel gets [+inf, -inf, +inf, -inf];
 *   frame_bounds [4] float32 device: the same over the whole frame.
 * The largest offset of fraction k is then max |floor(1/2 + k b / denom)| over the four frame bounds b (the
 * offset is monotone in the motion).  Exact selections: bit-identical to a sequential CPU reduction.
 * Workspace: exw_workspace_bytes(EXW_OP_MOTION_BOUNDS, W, H, ...). */
EXW_API exw_status exw_motion_bounds(const float *depth, const float *mv, int W, int H, float *tile_bounds,
                             float *frame_bounds, void *ws, size_t ws_bytes, exw_stream_t stream);

/* Stage (a): forward z-buffered splat of fraction k/denom of the motion (Sec. II-B: warping maps every location
 * of one image to a location in another; Sec. IV-B: P_k is shown at t + k/4; Sec. V-A2: depth resolves several
 * sources landing on one target).  keys [H][W] uint64 device (output; the callee clears it to EXW_KEY_EMPTY and
 * then takes the 64-bit atomic minimum of (bits(depth) << 32) | source index).  Integer result, bit-exact and
 * independent of scheduling. */
EXW_API exw_status exw_splat_motion(const float *depth, const float *mv, int W, int H, int k, int denom, uint64_t *keys,
                            exw_stream_t stream);

/* Stage (b): backward bilinear gather of colour through splatted keys (Sec. II-B, Sec. III-B: the warped frame
 * and its invalid pixels).  Reads colour (cdt), depth, motion and keys from exw_splat_motion with the same k and
 * denom; writes out_color [3][H][W] (cdt; 0 on holes) and mask [H][W] (EXW_MASK_* bits). */
EXW_API exw_status exw_warp(const void *color, exw_dtype cdt, const float *depth, const float *mv, const uint64_t *keys,
                    int W, int H, int k, int denom, void *out_color, uint8_t *mask, exw_stream_t stream);

/* Stage (c): pull-push fill of the pixels whose mask is non-zero, in place (Sec. III-C: the holes of a warped
 * frame must be filled before it is shown).  color [3][H][W] (cdt) device, read and written; mask [H][W]
 * device, read.  Valid pixels are left bit-identical.  A frame without any valid pixel is filled with 0.
 * Workspace: exw_workspace_bytes(EXW_OP_FILL_HOLES, W, H, cdt, 1, 1). */
EXW_API exw_status exw_fill_holes(void *color, exw_dtype cdt, const uint8_t *mask, int W, int H, void *ws,
                          size_t ws_bytes, exw_stream_t stream);

/* Stage (c) without a workspace: the same pull-push fill as exw_fill_holes (identical results), for callers that
 * cannot allocate device memory when they fill a frame -- renderers that reserve all GPU memory at start-up and
 * forbid allocation inside the frame loop, plugins running inside a host application whose allocator they may not
 * call, code that only receives raw device pointers.  The paper has no counterpart; this is a library facility.
 * Scratch: one built-in device array of 768 KiB, held by every GPU that loads the library until the process exits;
 * frames up to 16384 fill tiles of 32 x 32 pixels (for example 4096 x 4096 or 8192 x 2048) fit, larger ones
 * return EXW_ERR_WORKSPACE.  The call allocates nothing: each call looks up the array's device address on the current
 * device (cudaGetSymbolAddress, so it stays valid after cudaDeviceReset); the first call on a device also loads the
 * library's device code there, so make that first call before any stream capture.  All calls
 * share the one array and each clears the counters it needs at its start: calls that may overlap on the GPU
 * (different streams, or concurrent host threads) race on it and must be serialised by the caller.
 * color [3][H][W] (cdt) device, read and written; mask [H][W] device, read. */
EXW_API exw_status exw_fill_holes_static(void *color, exw_dtype cdt, const uint8_t *mask, int W, int H,
                                         exw_stream_t stream);

/* Stages (a0)+(a)+(b)+(c) fused: P_1..P_nfrac at t + k/4, k = 1..nfrac (Sec. IV-B; nfrac in [1, 3]), for
 * nframes source frames of one size and colour type.  frames [nframes] and out [nframes * nfrac] (frame-major:
 * out[f * nfrac + (k - 1)]) are HOST arrays of descriptors holding device pointers.  Per frame, one pass reads
 * the source once and writes the nfrac outputs; the splat runs in shared memory.  Results are identical to
 * exw_splat_motion + exw_warp (+ exw_fill_holes unless EXW_FLAG_NO_FILL) with k/4: keys and mask bit-exact, the
 * colour bit-identical.  Workspace: exw_workspace_bytes(EXW_OP_EXTRAPOLATE, W, H, cdt, nframes, nfrac). */
EXW_API exw_status exw_extrapolate(const exw_frame *frames, int nframes, int nfrac, unsigned flags, exw_frame_out *out,
                           void *ws, size_t ws_bytes, exw_stream_t stream);

/* exw_extrapolate for frames held in HOST memory (Sec. IV-B, all stages), with the host <-> device copies inside the
 * call and overlapped with the work: the frames go in chunks of `chunk` frames (0: 8); chunk j's inputs are copied in
 * on one internal stream while chunk j - 1 is extrapolated on `stream` and chunk j - 2's outputs are copied back on
 * another. frames_host [nframes] and out_host [nframes * nfrac] are HOST arrays of descriptors holding host pointers
 * (page-locked memory for the copies to overlap; any host memory works), frames_dev and out_dev the same shapes in
 * device memory, owned by the caller and written here (staging: every frame has its own device buffers, nothing is
 * allocated). out_dev NULL: the engine writes the outputs straight into the host buffers, which must then be
 * page-locked and mapped (cudaHostGetDevicePointer; EXW_ERR_INVALID_ARG otherwise).  Workspace:
 * exw_workspace_bytes(EXW_OP_EXTRAPOLATE, W, H, cdt, min(chunk, nframes), nfrac).  The call returns once the work is
 * queued; when `stream` completes, the outputs are in host memory.  The internal streams and events are created at the
 * first call on a device; calls on one device are serialised by the caller.  Errors as exw_extrapolate. */
EXW_API exw_status exw_extrapolate_host(const exw_frame *frames_host, const exw_frame *frames_dev, int nframes,
                                        int nfrac, unsigned flags, const exw_frame_out *out_host,
                                        const exw_frame_out *out_dev, int chunk, void *ws, size_t ws_bytes,
                                        exw_stream_t stream);

/* Depth and motion of a warped frame, so that it can be warped again -- the recursive warps W(P_1), W(P_2) of the
 * decision paths S5 and S6 (Table V; the paper leaves the motion of a predicted frame open, read as the motion of
 * the surface that landed there).  keys [H][W] from exw_splat_motion and mask [H][W] from exw_warp of the same
 * fraction; depth, mv the source frame's.  A target that is not a hole takes its winner's depth and motion (bit
 * copies); a hole gets depth NaN (it never lands again) and motion 0.  depth_out [H][W], mv_out [2][H][W] device
 * float32, written.  Chain: splat, warp (+ fill), carry, then splat and warp the warped colour with the carried
 * depth and motion (k = 1 of 4 per step). */
EXW_API exw_status exw_carry_motion(const uint64_t *keys, const uint8_t *mask, const float *depth, const float *mv,
                                    int W, int H, float *depth_out, float *mv_out, exw_stream_t stream);

/* The recursive warps of decision paths S5 and S6 (Table V): P_1 = W(F_t), P_{i+1} = W(P_i), each a quarter step
 * (k = 1 of 4) of the motion the warped frame carries (exw_carry_motion's reading).  Per step: exw_splat_motion,
 * exw_warp and (unless flags has EXW_FLAG_NO_FILL) exw_fill_holes, then exw_carry_motion for the next step; all
 * on the device, chained in this call.  color [3][H][W] (cdt), depth [H][W], mv [2][H][W]: the source frame
 * (device, read).  out [steps] is a HOST array of descriptors of device buffers: out[i] receives P_{i+1}'s colour
 * (cdt) and hole mask.  steps in [1, 64].  Workspace: exw_workspace_bytes(EXW_OP_WARP_RECURSIVE, W, H, cdt, 1, 1)
 * (the keys, the carried depth and motion, the fill's scratch). */
EXW_API exw_status exw_warp_recursive(const void *color, exw_dtype cdt, const float *depth, const float *mv, int W,
                                      int H, int steps, unsigned flags, exw_frame_out *out, void *ws, size_t ws_bytes,
                                      exw_stream_t stream);

/* Motion-variance features Var_x(F_mv), Var_y(F_mv) of the decision stage's environment vector E_t (Sec. IV-C,
 * Eq. 1; the feature is motivated in Sec. III-D): over every pixel of mv [2][H][W] whose two components are
 * finite, the population variance of the x component and of the y component.  out [3] is a DEVICE float64 array:
 * the number of pixels counted, Var_x, Var_y (0, 0 for an empty set).  FP64 throughout, merged in a fixed order:
 * deterministic.  Workspace: exw_workspace_bytes(EXW_OP_STATS, W, H, cdt, 1, 1). */
EXW_API exw_status exw_mv_variance(const float *mv, int W, int H, double *out, void *ws, size_t ws_bytes,
                                   exw_stream_t stream);

/* Mean squared difference of two colour images a, b [3][H][W] of type cdt over all 3 W H values (FP64, fixed
 * order): the MSE of the reward's PSNR = 10 log10(255^2 / MSE) (Sec. IV-C, Eq. 3) for colours in [0, 1] scaled by
 * 255, i.e. PSNR = -10 log10(out[0]).  out [1] is a DEVICE float64.  Workspace: as exw_mv_variance. */
EXW_API exw_status exw_color_mse(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                                 size_t ws_bytes, exw_stream_t stream);

/* PSNR of the reward (Sec. IV-C, Eq. 3): out [2] DEVICE float64 receives the MSE of exw_color_mse and
 * 10 log10(255^2 / MSE) = -10 log10(MSE) in dB for colours in [0, 1] scaled by 255 (+inf when the images are
 * equal), both computed on the device.  Workspace: as exw_mv_variance. */
EXW_API exw_status exw_psnr(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                            size_t ws_bytes, exw_stream_t stream);

/* Structural similarity of two colour images a, b [3][H][W] of type cdt in [0, 1] (the SSIM of the reward, Sec.
 * IV-C, Eq. 3, read as the standard index: 11 x 11 Gaussian window, sigma 1.5, C1 = 1e-4, C2 = 9e-4, over every
 * window position wholly inside the image, averaged over positions and channels).  Moments in FP32 on values
 * shifted by -1/2, the mean in FP64 in a fixed order.  Needs W, H >= 11.  out [1] is a DEVICE float64.
 * Workspace: as exw_mv_variance. */
EXW_API exw_status exw_ssim(const void *a, const void *b, exw_dtype cdt, int W, int H, double *out, void *ws,
                            size_t ws_bytes, exw_stream_t stream);

/* Adjoint of stage (b) (the gather of Sec. II-B and Sec. III-B; the paper does not differentiate the warp, so this is
 * a library facility for training against it) for fraction k/denom with every integer decision held fixed (target,
 * winner, taps, tap participation, mask). grad_out [3][H][W] float32 = dL/d out_color; accumulates (+=) into grad_color
 * [3][H][W] float32 (dL/d colour: w_t / sum w per participating tap) and grad_mv [2][H][W] float32 (dL/d motion through
 * rho, d rho / d mv = -k/denom). keys: those of the forward pass, or NULL to recompute them into the workspace
 * (activation checkpointing).  Deterministic: each output element is summed by one thread in a fixed order.  Workspace:
 * exw_workspace_bytes(EXW_OP_WARP_BACKWARD, W, H, cdt, 1, 1) (0 bytes suffice when keys is given). */
EXW_API exw_status exw_warp_backward(const float *grad_out, const void *color, exw_dtype cdt, const float *depth,
                             const float *mv, const uint64_t *keys, int W, int H, int k, int denom,
                             float *grad_color, float *grad_mv, void *ws, size_t ws_bytes, exw_stream_t stream);

/* One frame of the training pass exw_warp_l2_grad (device pointers). */
typedef struct exw_train_frame {
    exw_frame src;                     /* F_t: colour (cdt), depth, motion */
    const void *target[EXW_MAX_FRAC];  /* [3][H][W] (cdt): what P_k should be, k = 1..nfrac */
    float *grad_color;                 /* [3][H][W] float32, accumulated (+=): dL/d colour */
    float *grad_mv;                    /* [2][H][W] float32, accumulated (+=): dL/d motion */
} exw_train_frame;

/* The warp of stage (b) (Sec. II-B, Sec. III-B) inside a training loss, for nframes frames of one size and colour
 * type and the fractions k/4, k = 1..nfrac (Sec. IV-B): the forward warp P_k, the loss
 *     L_f = sum over k, over non-hole targets q of P_k and over the 3 channels of (P_k(q) - target_k(q))^2,
 * and its adjoint with every integer decision held fixed, as exw_splat_motion + exw_warp + exw_l2_loss_grad +
 * exw_warp_backward with keys = NULL would give per fraction -- fused: per frame one pass computes the keys of
 * every fraction (activation checkpointing: nothing of the forward is kept between calls), then one pass over
 * 32 x 32 source tiles reads each tile once, recomputes each winner's forward value with stage (b)'s arithmetic
 * and adds the gradients of all fractions (deterministic: each element is summed by one thread, fractions in
 * order, so the gradients equal nfrac exw_warp_backward calls bit for bit).  The paper does not differentiate the
 * warp; this is a library facility.  frames [nframes] is a HOST array of descriptors; loss [nframes] is a DEVICE
 * float64 array, written (summed in FP64 in a fixed order).  Workspace: exw_workspace_bytes(EXW_OP_WARP_L2_GRAD,
 * W, H, cdt, 1, nfrac) (the key planes of one frame; frames run one after another on the stream). */
EXW_API exw_status exw_warp_l2_grad(const exw_train_frame *frames, int nframes, int nfrac, double *loss, void *ws,
                                    size_t ws_bytes, exw_stream_t stream);

/* L2 loss of a warped frame against a target over its non-hole pixels (the loss the differentiation workload
 * trains against): loss += sum over mask == 0 and 3 channels of (out - target)^2 (float32 device scalar,
 * accumulated with atomics, so its last bits depend on scheduling), and grad_out = 2 (out - target) on non-hole
 * pixels, 0 on holes.  out and target [3][H][W] in cdt; grad_out [3][H][W] float32. */
EXW_API exw_status exw_l2_loss_grad(const void *out, const void *target, exw_dtype cdt, const uint8_t *mask, int W, int H,
                            float *grad_out, float *loss, exw_stream_t stream);

/* Device-side status of the last call on a workspace (EXW_OK, or EXW_ERR_TIMEOUT when a bounded wait of the
 * batched path ran out).  Synchronises `stream`, then reads 4 bytes of the workspace. */
EXW_API exw_status exw_device_status(const void *ws, exw_stream_t stream);

/* --- batched path: many independent streams of mixed sizes in one persistent launch ----------------------- */

/* One stream of the batched path: a source frame and its nfrac outputs (device pointers). */
typedef struct exw_stream_desc {
    exw_frame src;
    exw_frame_out out[EXW_MAX_FRAC];
} exw_stream_desc;

typedef struct exw_tuner exw_tuner; /* opaque host-side autotuner state */

EXW_API exw_tuner *exw_tuner_create(void);
EXW_API void exw_tuner_destroy(exw_tuner *t);
/* Make the tuner run one schedule for every batch instead of timing candidates: window shape 0 or 1 (see
 * exw_extrapolate_batched), queue distance lag in [1, 4], pair 0 or 1.  EXW_ERR_INVALID_ARG for other values. */
EXW_API exw_status exw_tuner_fix(exw_tuner *t, int shape, int lag, int pair);
/* Text summary of the tuner's choices (NUL-terminated, truncated to len bytes).  Returns bytes needed. */
EXW_API size_t exw_tuner_report(const exw_tuner *t, char *buf, size_t len);

/* Workspace of exw_extrapolate_batched for n streams (host array of descriptors) with nfrac fractions. */
EXW_API size_t exw_batched_workspace_bytes(const exw_stream_desc *d, int n, int nfrac);

/* Stages (a0)+(a)+(b)+(c) -- P_1..P_nfrac at t + k/4 (Sec. IV-B), as exw_extrapolate -- for n independent streams of
 * possibly different sizes (each with its own colour type) in one persistent kernel launch per 48 streams (the first
 * stream's bounds and plans run as two kernels ahead of it): CTAs pull (stream, stage, tile) work items from a queue in
 * the workspace; a stage waits for the one before it in the same stream with a bounded
 * spin (EXW_ERR_TIMEOUT via exw_device_status if it runs out).  Capturable in a CUDA graph. d [n] is a HOST array. t
 * (nullable) is the autotuner: on the first call for a given set of sizes (outside any stream capture) it times
 * every schedule -- the shape of the shared-memory staging windows (FP32 56 x 48 or 64 x 42, FP16 64 x 56 or
 * 56 x 64 pixels), the queue distance between the stages of a stream (1 or 2) and whether two smooth tiles of a
 * stream share one slot -- and keeps the fastest for later calls; NULL runs the default schedule (the first shape,
 * distance 1, sharing on).  Results are bit-identical to exw_extrapolate on each stream, whatever the schedule. */
EXW_API exw_status exw_extrapolate_batched(const exw_stream_desc *d, int n, int nfrac, unsigned flags, void *ws,
                                   size_t ws_bytes, exw_tuner *t, exw_stream_t stream);

/* --- kernel timing with CUDA events on the launching stream (for benchmarks) ------------------------------- */

/* Enable (1) or disable (0) event pairs around every kernel this library launches; resets the counters. */
EXW_API void exw_timing_enable(int on);
/* After the stream has finished: total milliseconds and launch count of kernel `name` since enabling
 * (synchronises on the recorded events).  Returns 0, or -1 when no such kernel was timed. */
EXW_API int exw_timing_query(const char *name, double *total_ms, int *launches);
/* Comma-separated names of the kernels timed so far (NUL-terminated, truncated to len).  Returns bytes needed. */
EXW_API size_t exw_timing_names(char *buf, size_t len);
/* Number of kernel launches this library has made since load (all entry points). */
EXW_API uint64_t exw_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* EXW_H */
