/*
 * fgs4d.h -- C ABI of the GB300 render path of 4D Gaussian Splatting
 * ("4D Gaussian Splatting: Modeling Dynamic Scenes with Native 4D
 * Primitives", arXiv 2412.20720).
 *
 * The path renders native 4D Gaussians at a timestamp t (Sec. 3.2, Eqs. 5-6):
 * each Gaussian's 4D covariance Sigma = R S S^T R^T with R = L(q_l) R(q_r) is
 * sliced at t into a conditional 3D Gaussian times the marginal p(t)
 * (Sec. 3.2), projected to a 2D conic (Sec. 3.1, Eqs. 3-4), coloured by 4D
 * spherindrical harmonics (Sec. 3.2), binned into screen tiles, sorted by
 * (tile, depth) and composited front to back (Sec. 3.2, Eq. 6), and the whole
 * chain is differentiated (Sec. 3.3, end-to-end optimisation).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All pointers to Gaussian data, images, gradients and the workspace are
 *   DEVICE pointers owned by the caller.  The library never allocates or
 *   frees device memory.  Host structs (views, settings, gaussian pointer
 *   tables) are read during the call only.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every call only enqueues work on it and returns without
 *   synchronising (except fgs4d_get_status), so a sequence of calls can be
 *   captured into a CUDA graph.
 * - One opaque workspace (size from fgs4d_workspace_size for the same n,
 *   views and settings) carries the state from fgs4d_preprocess through
 *   fgs4d_bin_sort and fgs4d_render_fwd to fgs4d_render_bwd.  Calls that
 *   share a workspace must be ordered on one stream.
 * - Return value: FGS4D_OK (0) or a negative FGS4D_ERR_* code.  Argument
 *   errors are detected on the host before anything is enqueued.  Conditions
 *   only the GPU can detect (capacity overflow, a bounded wait that ran out)
 *   are recorded in a status word in the workspace; kernels never trap, and
 *   every write stays inside the caller's buffers.  fgs4d_get_status reads
 *   that word.
 * - Parameter layout (float32, row-major, contiguous): mean [n][4] (x,y,z,t);
 *   log_scale [n][4]; q_l, q_r [n][4] (real part first, any non-zero norm;
 *   normalised inside); opacity_logit [n] (opacity = sigmoid(logit));
 *   sh [n][K][3] with K = (L+1)^2 (n_max+1) and coefficient k =
 *   n (L+1)^2 + l^2 + l + m for temporal order n, degree l, order m.
 */
#ifndef FGS4D_H
#define FGS4D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGS4D_OK 0
#define FGS4D_ERR_ARG (-1)         /* invalid argument (host-side check) */
#define FGS4D_ERR_CUDA (-2)        /* a CUDA runtime call or launch failed */
#define FGS4D_ERR_WORKSPACE (-3)   /* workspace pointer, size or alignment wrong */
#define FGS4D_ERR_CAPACITY (-4)    /* visible or instance capacity exceeded */
#define FGS4D_ERR_TIMEOUT (-5)     /* a bounded inter-block wait ran out */
#define FGS4D_ERR_INTERNAL (-6)    /* an internal consistency check failed */
#define FGS4D_ERR_UNSUPPORTED (-7) /* setting outside the compiled range */

#define FGS4D_MAX_VIEWS 128     /* views per call */
#define FGS4D_MAX_SH_DEGREE 3   /* spatial SH degree L */
#define FGS4D_MAX_T_ORDER 4     /* temporal Fourier order n_max */

/* One (camera, timestamp) to render.  Pinhole camera in the OpenCV
 * convention (x right, y down, z forward); pixel (px, py) is sampled at its
 * centre (px + 0.5, py + 0.5). */
typedef struct fgs4d_view {
  int32_t width, height;   /* image size in pixels, each in [1, 16384] */
  float fx, fy, cx, cy;    /* intrinsics K (Sec. 3.1, Eq. 3) */
  float viewmat[12];       /* extrinsics E: world -> camera, row-major 3x4 [W | T] */
  float campos[3];         /* camera centre in world space (4DSH view direction) */
  float t;                 /* render timestamp */
} fgs4d_view;

/* Render settings.  The paper leaves the rasterizer constants to the tile
 * rasterizer it adapts (Sec. 3.2); the values used by the tests are noted. */
typedef struct fgs4d_settings {
  int32_t sh_degree;     /* spatial SH degree L, 0..FGS4D_MAX_SH_DEGREE */
  int32_t t_order;       /* temporal order n_max, 0..FGS4D_MAX_T_ORDER */
  float period;          /* T of cos(2 pi n dt / T), > 0 (tests: 1) */
  int32_t tile;          /* tile edge in pixels: 16 */
  float near_plane;      /* cull when camera z <= near_plane, > 0 (tests: 0.2) */
  float dilation;        /* added to the 2D covariance diagonal, >= 0 (tests: 0.3) */
  float p_t_min;         /* temporal filter: cull when p(t) < p_t_min (Sec. 8.1.1: 0.05) */
  float bg[3];           /* background colour composited behind the Gaussians */
  int64_t vis_capacity;  /* max visible (view, Gaussian) pairs; 0 = n * nviews */
  int64_t inst_capacity; /* max (tile, Gaussian) instances over all views, > 0 */
  int32_t pixels_per_thread; /* compositor block shape: 0 (default 4), 2, 4 or 8 pixels
                                of one tile column per thread; results are identical */
  int32_t shared_batch;      /* records the compositors stage per shared-memory batch: 0 (= 256), 128 or 256 */
  int32_t stage_blocks_per_sm; /* grids of the latency-bound stages: 0 = full-GPU grids (the lowest
                                  latency for one frame alone); k in 1..8 = at most k resident blocks
                                  per SM for preprocess and the radix passes and 2k for the instance
                                  emission, leaving SMs to other work on the GPU (frames or views
                                  rendered concurrently on other streams); results are identical */
} fgs4d_settings;

/* Gaussian parameters (device pointers, layout in the header comment). */
typedef struct fgs4d_gaussians {
  const float *mean;
  const float *log_scale;
  const float *q_l;
  const float *q_r;
  const float *opacity_logit;
  const float *sh;
  int64_t n; /* number of Gaussians, 0 <= n < 2^31 */
  /* Optional Compact-4DGS significance mask (Sec. 4.3): mask_logit [n] or
   * NULL.  M = sigmoid(m); a Gaussian with M <= mask_threshold is removed
   * (M_hat = 1{M > eps} scales its four scales and its opacity to zero), any
   * other renders unchanged (M_hat = 1).  mask_threshold in [0, 1); the
   * paper's pruning experiments (Sec. 8.3.2) use 0.03. */
  const float *mask_logit;
  float mask_threshold;
} fgs4d_gaussians;

/* Gradient buffers, same shapes as the parameters (device pointers).
 * Gradients are ACCUMULATED (+=); the caller zeroes them when needed. */
typedef struct fgs4d_gaussians_grad {
  float *mean;
  float *log_scale;
  float *q_l;
  float *q_r;
  float *opacity_logit;
  float *sh;
  /* Optional (NULL = off) densification statistics in spacetime (Sec. 3.3,
   * "Densification in spacetime": the magnitude of the spatial position
   * gradient and, as an additional indicator, the gradient of mu_t),
   * float [n][4], 16-byte aligned, ACCUMULATED per (view, visible Gaussian)
   * of each backward call: (|| (dL/du, dL/dv) || in pixels, |dL/dmu_t| of
   * that view, 1 (the view count), 0). */
  float *densify_stats;
  /* dL/dm of the significance mask, [n], used when the parameters carry a
   * mask (NULL = not wanted): the straight-through gradient
   * M (1 - M) (sum_k dL/dlog s_k + dL/dalpha alpha) of each kept Gaussian
   * (Sec. 4.3, M_hat = stop_gradient(1{M > eps} - M) + M). */
  float *mask_logit;
} fgs4d_gaussians_grad;

/* Writable parameter arrays (same layouts as fgs4d_gaussians), n rows. */
typedef struct fgs4d_gaussians_out {
  float *mean;
  float *log_scale;
  float *q_l;
  float *q_r;
  float *opacity_logit;
  float *sh;
  int64_t n;
} fgs4d_gaussians_out;

/* Byte offsets of the workspace regions that hold the documented
 * intermediate results (for inspection and tests; all other bytes are
 * private).  "slot" numbers the visible (view, Gaussian) pairs of a call in
 * (view, Gaussian index) order. */
typedef struct fgs4d_layout {
  size_t bytes;         /* total workspace size */
  size_t counters;      /* uint32: [0] visible pairs, [1] instances, [2] status bits */
  size_t rec_geom;      /* float4 [vis_cap]: (u, v, a1, b1): the exponent in base 2 is power2 = -q,
                           q = (a1 dx)^2 + (b1 dx + b2 dy)^2, (dx, dy) = (u, v) - pixel centre, i.e.
                           (1/2) log2(e) times the conic form of Sigma_2d^-1 as a sum of two squares */
  size_t rec_color;     /* float4 [vis_cap]: (b2, log2 a, r, g) with a = sigmoid(logit) p(t) */
  size_t rec_blue;      /* float  [vis_cap]: b */
  size_t rec_tau;       /* float  [vis_cap]: log2(255 a) + 4e-3; alpha >= 1/255 needs -power2 <= tau */
  size_t rec_meta;      /* int32x4 [vis_cap]: (gaussian, view, x0 | y0 << 16, x1 | y1 << 16) tile rect */
  size_t depth_key;     /* uint32 [vis_cap]: FP32 bits of the camera depth */
  size_t sorted_slots;  /* uint32 [vis_cap]: slots in (depth, slot) order, after fgs4d_bin_sort */
  size_t inst_tile;     /* uint32 [inst_cap]: global tile id of each sorted instance */
  size_t inst_slot;     /* uint32 [inst_cap]: slot of each sorted instance */
  size_t tile_ranges;   /* uint32x2 [total_tiles]: [start, end) into the instance list; a tile
                           without instances holds start >= end */
  size_t pix_T;         /* float  [total_pixels]: final transmittance */
  size_t pix_last;      /* uint32 [total_pixels]: list entries processed up to the last composited one */
  size_t slot_grad;     /* float  [vis_cap][12]: dL/d(u, v, A, B, C, a, r, g, b) per slot */
  int64_t vis_capacity;
  int64_t inst_capacity;
  int64_t total_tiles;  /* sum over views of ceil(W/16) ceil(H/16); view v starts at the sum before it */
  int64_t total_pixels; /* sum over views of W H; view v's image starts at the sum before it */
} fgs4d_layout;

/* Workspace bytes for rendering n Gaussians into `views` with `settings`.
 * Errors: FGS4D_ERR_ARG (bad sizes or pointers), FGS4D_ERR_UNSUPPORTED. */
int fgs4d_workspace_size(const fgs4d_settings *settings, int64_t n, const fgs4d_view *views,
                         int32_t nviews, size_t *bytes_out);

/* Offsets of the documented workspace regions (see fgs4d_layout). */
int fgs4d_workspace_layout(const fgs4d_settings *settings, int64_t n, const fgs4d_view *views,
                           int32_t nviews, fgs4d_layout *layout_out);

/* Per-Gaussian stage for every view (Sec. 3.2 and Sec. 3.1, Eqs. 3-4):
 * activations, R = L(q_l) R(q_r), Sigma = R S S^T R^T, marginal
 * p(t) = exp(-(t - mu_t)^2 / (2 Sigma_44)) and the temporal filter
 * p(t) < p_t_min (Sec. 8.1.1), conditional mean and covariance at t, view
 * transform, near cull, EWA 2D covariance (+ dilation), conic, 3-sigma tile
 * rect, depth, 4DSH colour max(0, sum c cos(2 pi n (t - mu_t)/T) Y_lm(d) +
 * 0.5), effective opacity sigmoid(logit) p(t).  Writes the records of the
 * visible pairs into the workspace (slot order: view, then Gaussian index).
 * Resets the workspace status word.  Device-detected: visible capacity. */
int fgs4d_preprocess(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                     const fgs4d_settings *settings, void *workspace, size_t workspace_bytes, void *stream);

/* Tile binning and sort (the tile rasterizer of Sec. 3.2): every visible
 * slot emits one instance per tile of its rect whose pixel-centre box meets
 * the slot's 1/255 ellipse (tiles it misses would skip the slot at every
 * pixel, so the image is that of the full rect membership); instances are
 * ordered by (global tile, FP32 depth, slot) with a hand-written radix sort,
 * and each tile's [start, end) range is computed.  Reads only what fgs4d_preprocess
 * (or a caller filling rec_meta, depth_key and counters[0]) wrote.
 * Device-detected: instance capacity. */
int fgs4d_bin_sort(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                   void *workspace, size_t workspace_bytes, void *stream);

/* Diagnostic: *count_out = the number of kernels fgs4d_bin_sort launches for
 * these arguments (the count depends on the tile grid's size, which sets the
 * number of tile-sort passes).  Launches nothing; has no counterpart in the
 * paper. */
int fgs4d_bin_sort_kernels(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                           int32_t *count_out);

/* Front-to-back compositing per pixel (Sec. 3.2, Eq. 6) over its tile's
 * sorted list: alpha = min(0.99, a exp(power)), skip when alpha < 1/255,
 * stop before the entry that would take T below 1e-4 (power is a negative
 * semidefinite form; no separate power > 0 test is taken).
 * out_rgb: float [sum_v 3 H W], view v at 3 * (pixels before v), planar
 * [3][H][W].  out_T: optional (may be NULL) float [sum_v H W] final
 * transmittance. */
int fgs4d_render_fwd(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                     void *workspace, size_t workspace_bytes, float *out_rgb, float *out_T, void *stream);

/* fgs4d_render_fwd for a render that no backward pass follows (a viewer, an
 * evaluation sweep): the same image and final transmittance bit for bit, but
 * the compositor does not track each pixel's last contributing entry, which
 * only fgs4d_render_bwd needs; that plane of the workspace is written as 0,
 * so a backward call after this one adds zero gradients.  No counterpart in
 * the paper (a rendering mode of the same Eq. 6). */
int fgs4d_render_image(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                       void *workspace, size_t workspace_bytes, float *out_rgb, float *out_T, void *stream);

/* Auxiliary channels (depth, opacity, optical flow) with the image.
 * Depth and flow are blended with the colour weights of Eq. 6,
 * w_i = alpha_i T_i: depth = sum w_i z_i with z_i the camera-space depth of
 * the sliced mean mu_xyz|t; opacity = 1 - T_final (the O of the sky
 * composition, Sec. 5); flow = sum w_i f_i with f_i the image-plane
 * displacement of mu_xyz|t over flow_dt, pi(pc + W v flow_dt) - pi(pc) with
 * velocity v = Sigma_{1:3,4} / Sigma_44 (Sec. 8.1.3: the trajectory of the
 * conditional mean projected between consecutive frames), 0 when the
 * displaced centre is not in front of the near plane.
 * Call after fgs4d_preprocess and fgs4d_bin_sort on the same workspace,
 * views and settings, with the same gaussians.  out_rgb and out_T as for
 * fgs4d_render_fwd; out_aux: float [sum_v 4 H W], view v at 4 * (pixels
 * before v), planar [4][H][W] = (depth, opacity, flow_u, flow_v), flow in
 * pixels.  Errors: FGS4D_ERR_ARG for a NULL out_rgb or out_aux or a
 * non-finite flow_dt; otherwise as fgs4d_render_fwd.  The image equals
 * fgs4d_render_fwd's bit for bit. */
int fgs4d_render_aux(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                     const fgs4d_settings *settings, void *workspace, size_t workspace_bytes, float flow_dt,
                     float *out_rgb, float *out_T, float *out_aux, void *stream);

/* Diagnostic form of fgs4d_render_fwd: renders identically into out_rgb and
 * ADDS to stats_out (device uint64[3], 8-byte aligned) the number of
 * pixel-entry alpha evaluations, of composited entries, and of the
 * evaluations at list positions up to each pixel's last composited entry
 * (those fgs4d_render_bwd repeats) -- the work counts from which the
 * compositors' algorithmic FLOPs are stated.  Has no counterpart in the
 * paper. */
int fgs4d_render_stats(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                       void *workspace, size_t workspace_bytes, float *out_rgb, uint64_t *stats_out, void *stream);

/* Reverse-mode derivative of the rendered RGB (Sec. 3.3: the chain is
 * optimised end to end): dL_drgb has out_rgb's layout; the gradients of all
 * parameters of the visible Gaussians are ADDED into `grads`.  Reverse
 * traversal recomputes T from the final transmittance; per-Gaussian sums are
 * warp-reduced before atomic accumulation.  Requires the workspace of the
 * matching forward (same n, views, settings, parameters). */
int fgs4d_render_bwd(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                     const fgs4d_settings *settings, void *workspace, size_t workspace_bytes,
                     const float *dL_drgb, const fgs4d_gaussians_grad *grads, void *stream);

/* fgs4d_render_bwd in its two stages, for callers that want the per-slot
 * screen-space gradients alone or time the stages apart; the two calls in
 * this order on one stream do exactly what fgs4d_render_bwd does.
 * fgs4d_render_bwd_composite: the adjoint of the compositing (Eq. 6) over
 * every tile of the matching forward; overwrites the workspace's slot_grad
 * region (fgs4d_layout) with dL/d(u, v, A, B, C, a, r, g, b) per visible
 * slot.  Errors: as fgs4d_render_fwd, FGS4D_ERR_ARG for a NULL dL_drgb.
 * fgs4d_render_bwd_preprocess: the adjoint of the per-Gaussian chain (the
 * 4DSH colour, EWA projection, slice, marginal, rotation and activations of
 * Sec. 3.1-3.2) from the slot gradients; ADDS into `grads` (and the
 * optional densification statistics and mask gradient) as fgs4d_render_bwd
 * does.  Errors: as fgs4d_render_bwd. */
int fgs4d_render_bwd_composite(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                               void *workspace, size_t workspace_bytes, const float *dL_drgb, void *stream);
int fgs4d_render_bwd_preprocess(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                                const fgs4d_settings *settings, void *workspace, size_t workspace_bytes,
                                const fgs4d_gaussians_grad *grads, void *stream);

/* Reverse-mode derivative of a loss on the image and on the depth and
 * opacity channels of fgs4d_render_aux (the inputs of the LiDAR depth loss
 * and the sky composition, Sec. 5).  dL_drgb as for fgs4d_render_bwd;
 * dL_daux has out_aux's layout, planes (depth, opacity, flow_u, flow_v); the
 * flow planes are ignored (flow is rendered for evaluation, not
 * differentiated).  Depth and opacity follow the colour rule with a zero
 * background and x_i = z_i, resp. 1; dL/dz_i flows into the sliced mean.
 * Requires the workspace of the matching fgs4d_render_aux.  Errors: as
 * fgs4d_render_bwd, plus FGS4D_ERR_ARG for a NULL dL_daux. */
int fgs4d_render_aux_bwd(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                         const fgs4d_settings *settings, void *workspace, size_t workspace_bytes,
                         const float *dL_drgb, const float *dL_daux, const fgs4d_gaussians_grad *grads,
                         void *stream);

/* Split sampling in spacetime (Sec. 3.3, "Densification in spacetime";
 * Sec. 8.1.3, "More ablations": new positions are sampled with the complete
 * 4D Gaussian as PDF).  For j in [0, m) and c in [0, k_children), child
 * j * k_children + c of Gaussian idx[j] gets
 *   mean      = mu + R diag(s) eps[j][c]   (a draw from N(mu, Sigma), 4D),
 *   log_scale = log s - log(shrink),
 *   q_l, q_r, opacity_logit and sh copied,
 * with R = L(q_l) R(q_r) of the normalised quaternions and s = exp(log s).
 * eps: device float [m][k_children][4], the standard normal draws (the caller
 * owns the random numbers).  idx: device int32 [m], each in [0, src->n);
 * dst->n >= m * k_children rows; dst must not overlap src.  The SH row
 * length follows settings (sh_degree, t_order).  Errors: FGS4D_ERR_ARG for
 * a bad count, pointer, 16-byte alignment of the float4 rows, or a shrink
 * that is not finite and positive.  An idx entry outside [0, src->n) is not
 * read: its children are written as zeros (the call has no status word, so
 * the caller validates idx).  Needs no workspace. */
int fgs4d_split_gaussians(const fgs4d_gaussians *src, const int32_t *idx, int64_t m, int32_t k_children,
                          const float *eps, float shrink, const fgs4d_settings *settings,
                          const fgs4d_gaussians_out *dst, void *stream);

/* Mask compression loss of Compact-4DGS (Sec. 4.3): L_mask = (1/n) sum_i
 * sigmoid(m_i) is ADDED to *loss_out (device float) and dL_mask/dm_i =
 * sigmoid'(m_i) / n ADDED to grad_out[i] (device float [n]).  n = 0 adds
 * nothing.  Errors: FGS4D_ERR_ARG for a negative n or NULL pointers. */
int fgs4d_mask_loss(const float *mask_logit, int64_t n, float *loss_out, float *grad_out, void *stream);

/* Adam step of the training loop (the optimiser the adapted 3DGS training
 * uses; Sec. 3.3 trains end to end with the rendering loss).  Not part of
 * the paper's method; a streaming kernel so that the optimiser does not
 * dominate the step.  `step` is a device int32 step count t, so a training
 * step can be replayed as a CUDA graph: fgs4d_adam_tick adds 1 to it (call
 * once per step, before the updates), fgs4d_adam_update applies, element by
 * element, m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps).
 * param, grad, exp_avg, exp_avg_sq: device float [count], 16-byte aligned.
 * Errors: FGS4D_ERR_ARG for NULL or misaligned pointers, count < 0,
 * non-finite lr, betas outside [0, 1) or eps <= 0. */
int fgs4d_adam_tick(int32_t *step, void *stream);
int fgs4d_adam_update(float *param, const float *grad, float *exp_avg, float *exp_avg_sq, int64_t count, float lr,
                      float beta1, float beta2, float eps, const int32_t *step, void *stream);

/* The same Adam step over up to FGS4D_ADAM_MAX_TENSORS tensors in one
 * launch (each element gets exactly the update of fgs4d_adam_update, with its
 * tensor's lr).  tensors: HOST array of ntensors descriptors, read during the
 * call only; each tensor's four device arrays hold count floats and are
 * 16-byte aligned; count = 0 is allowed.  With zero_grad != 0 every gradient
 * element is set to 0 after it is read, so the next step can accumulate into
 * the same buffers without clearing them first.  Errors: FGS4D_ERR_ARG for
 * ntensors outside [0, FGS4D_ADAM_MAX_TENSORS], a NULL table or step, NULL or
 * misaligned arrays of a tensor with count > 0, a negative count or
 * non-finite lr, and the scalar conditions of fgs4d_adam_update. */
#define FGS4D_ADAM_MAX_TENSORS 16
typedef struct {
  float *param;
  float *grad; /* written (zeroed) only when zero_grad != 0 */
  float *exp_avg;
  float *exp_avg_sq;
  int64_t count;
  float lr;
} fgs4d_adam_tensor;
int fgs4d_adam_update_set(const fgs4d_adam_tensor *tensors, int32_t ntensors, float beta1, float beta2, float eps,
                          const int32_t *step, int32_t zero_grad, void *stream);

/* Scale-gated feature rendering for 4D segmentation (Sec. 7, "Scale-gated
 * features"): Gaussian i carries features[i][0..D); at a scale s the caller
 * passes the gate vector S(s) (device float [D], values in [0, 1]; NULL =
 * all ones).  f^s = S(s) (.) f is normalised (a zero vector stays zero) and
 * composited with the colour weights of Eq. 6 and a zero background:
 * out_features[c] = sum_i alpha_i T_i fhat_i[c], float [sum_v D H W], view v
 * at D * (pixels before v), planar [D][H][W].  D in {8, 16, 32} (32 is the
 * paper's; others give FGS4D_ERR_UNSUPPORTED); features 16-byte aligned
 * rows.  Call after fgs4d_preprocess and fgs4d_bin_sort on the same
 * workspace, views and settings; the weights equal fgs4d_render_fwd's. */
int fgs4d_render_features(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                          void *workspace, size_t workspace_bytes, const float *features, int32_t D,
                          const float *gate, float *out_features, void *stream);

/* Reverse mode of fgs4d_render_features with the geometry held fixed (the
 * features are trained on a pre-trained 4DGS, Sec. 7 "Training"):
 * dL_dfeatures has out_features' layout; ADDS dL/df into grad_features
 * (device float [n][D]) and, when grad_gate is not NULL, dL/dS(s) into
 * grad_gate (device float [D]).  With g = S (.) f and fhat = g / |g|:
 * dL/dg = (dL/dfhat - fhat (fhat . dL/dfhat)) / |g|, dL/df = S (.) dL/dg,
 * dL/dS = sum_i f_i (.) dL/dg_i. */
int fgs4d_render_features_bwd(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                              void *workspace, size_t workspace_bytes, const float *features, int32_t D,
                              const float *gate, const float *dL_dfeatures, float *grad_features,
                              float *grad_gate, void *stream);

/* Photometric L1 loss (Sec. 3.3, rendering loss only): loss_out[0] +=
 * sum |img - target| / count, dL_dimg = sign(img - target) / count.
 * All device pointers; loss_out must be zeroed by the caller. */
int fgs4d_l1_loss(const float *img, const float *target, int64_t count, float *loss_out, float *dL_dimg,
                  void *stream);

/* One part of an L1 loss averaged over mean_count elements, for a batch whose
 * images are rendered by separate calls: loss_out[0] += sum |img - target| /
 * mean_count over this part's count elements, dL_dimg = sign(img - target) /
 * mean_count.  count <= mean_count; otherwise as fgs4d_l1_loss (the paper's
 * loss is the mean over the batch). */
int fgs4d_l1_loss_part(const float *img, const float *target, int64_t count, int64_t mean_count, float *loss_out,
                       float *dL_dimg, void *stream);

/* Scratch bytes fgs4d_wait_selftest needs. */
#define FGS4D_WAIT_SELFTEST_BYTES 4096

/* Diagnostic of the failure detection; no counterpart in the paper.  Runs the
 * library's two kinds of bounded inter-block wait -- the warp-wide look-back
 * of the compactions (preprocess, pair scan, emission) and the per-digit
 * look-back of the radix passes -- in one block against a predecessor that
 * never posts.  Each wait gives up after its poll limit (about a second),
 * records the timeout in a status word and returns, so the context stays
 * usable; the same bit surfaces as FGS4D_ERR_TIMEOUT from fgs4d_get_status in
 * the render path.  scratch: device memory, at least FGS4D_WAIT_SELFTEST_BYTES,
 * 16-byte aligned, overwritten.  Synchronises the stream.  Returns
 * FGS4D_ERR_TIMEOUT when the timeout was recorded (the expected result),
 * FGS4D_ERR_INTERNAL if it was not, FGS4D_ERR_ARG or FGS4D_ERR_CUDA. */
int fgs4d_wait_selftest(void *scratch, size_t scratch_bytes, void *stream);

/* Largest key count fgs4d_sort_depth_static accepts. */
#define FGS4D_STATIC_SORT_MAX (1 << 20)

/* Depth sort that allocates nothing, for callers that cannot give the
 * library a workspace: plug-ins whose host application owns every device
 * allocation, and per-frame loops that must not call cudaMalloc (it can
 * synchronise the device and fail under a fixed memory budget).  The paper
 * has no counterpart; this is a packaging of the depth-sort step of
 * fgs4d_bin_sort.
 * Input: depth_keys, device uint32 [n] at any 4-byte aligned address (FP32 bit
 * patterns of positive depths; any uint32 keys sort correctly).  Output:
 * sorted_slots, device uint32 [n],
 * the indices 0..n-1 in (key, index) order -- the same permutation
 * fgs4d_bin_sort writes to its sorted_slots region for the same keys.
 * Scratch: one library-owned device array of about 18 MB (FGS4D_STATIC_SORT_MAX
 * keys), present on every GPU that loads the library until the process exits.
 * No device memory is allocated or freed.  The first call on a device looks
 * up that array's address for the current device, so make that first call
 * before capturing a stream into a graph.  Every call reuses the same array
 * (its previous contents are reset as needed), so calls whose work overlaps
 * on the GPU -- on different streams, or from different host threads --
 * race and must be serialised by the caller.
 * Errors: FGS4D_ERR_ARG for n < 0, n > FGS4D_STATIC_SORT_MAX or a null
 * pointer with n > 0; FGS4D_ERR_CUDA if the lookup or a launch fails.  n = 0
 * does nothing. */
int fgs4d_sort_depth_static(const uint32_t *depth_keys, int64_t n, uint32_t *sorted_slots, void *stream);

/* Outcome of the last fgs4d_sort_depth_static call on the current device,
 * as the device saw it.  fgs4d_sort_depth_static only enqueues work, and its
 * radix passes record a bounded wait that ran out, or a position outside the
 * array, in a status word of the library-owned scratch instead of trapping;
 * that word is cleared by the next sort call.  This call synchronises
 * `stream` (the stream of that sort), reads the word and returns FGS4D_OK
 * (the permutation in sorted_slots is valid), FGS4D_ERR_TIMEOUT or
 * FGS4D_ERR_INTERNAL (sorted_slots must not be used); FGS4D_ERR_CUDA if the
 * read fails.  Allocates nothing.  No counterpart in the paper. */
int fgs4d_sort_depth_static_status(void *stream);

/* Synchronises `stream`, then reads the workspace status word.  Returns
 * FGS4D_OK, or the first recorded device condition (FGS4D_ERR_CAPACITY,
 * FGS4D_ERR_TIMEOUT, FGS4D_ERR_INTERNAL).  counts_out (optional, 4 entries):
 * visible pairs, instances, visible pairs needed, instances needed. */
int fgs4d_get_status(const void *workspace, size_t workspace_bytes, void *stream, int64_t *counts_out);

/* Static description of a status code. */
const char *fgs4d_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* FGS4D_H */
