/*
 * fgs4d.h -- C ABI of libfgs4d: the rendering routine of 4D Gaussian
 * Splatting (Yang et al., ICLR 2024, arxiv 2310.10642) and its adjoint, as
 * hand-written CUDA kernels for sm_103a.
 *
 * The path, per (camera, time t) view:
 *   fgs4d_slice_project   4D Gaussian -> conditional 3D Gaussian and marginal
 *                         p(t) (Sec. 3.2, Eq. 7-10), 4DSH colour (Eq. 11),
 *                         EWA projection to a 2D splat (Eq. 3-4)
 *   fgs4d_bin_sort        splat -> screen tiles, ordered by depth (the
 *                         "sorted according to their depth" of Sec. 3.1 and
 *                         the tile-based rasteriser adapted in Sec. 3.2)
 *   fgs4d_render          front-to-back compositing of Eq. 6
 *   fgs4d_render_backward the adjoint of all three (end-to-end training with
 *                         the rendering loss only, Sec. 3.3)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named "device" must point to memory of the current CUDA device;
 *   host arrays (views, options) are read during the call only.  The library
 *   never allocates: the caller owns every buffer, including the per-frame
 *   state whose size fgs4d_state_size() reports.
 * - Every call is asynchronous on `stream` (NULL = legacy default stream),
 *   issues no synchronisation and no allocation, and is safe to capture in a
 *   CUDA graph.  The one exception is fgs4d_read_counters(), which copies
 *   device counters to the host and synchronises the stream.
 * - Argument errors are detected on the host and returned before any work is
 *   enqueued.  Launch errors return FGS4D_ERR_CUDA.  Data-dependent errors
 *   (pair-capacity overflow, non-finite or zero-norm parameters) are recorded
 *   in a device status word inside the state and reported by
 *   fgs4d_read_counters(); no kernel traps, asserts or spins.
 * - Parameters are raw (before activation): log scales, opacity logit and
 *   unnormalised quaternions.  Gradients are returned w.r.t. those raw values.
 * - Images are planar RGB float32: view v occupies
 *   image[3*P_v .. 3*(P_v + W_v*H_v)) as [3][H_v][W_v], where
 *   P_v = sum_{u<v} W_u*H_u ("pixel offset").  final_T and n_last are
 *   [P_v .. P_v + W_v*H_v) as [H_v][W_v].
 * - Pixel (i, j) is sampled at image coordinates (x, y) = (i, j); a camera
 *   maps camera coordinates (X, Y, Z), Z forward, to (fx X/Z + cx, fy Y/Z + cy).
 */
#ifndef FGS4D_H
#define FGS4D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGS4D_ABI_VERSION 5
#define FGS4D_MAX_VIEWS 128   /* views per call */
#define FGS4D_MAX_SH_DEGREE 3 /* L */
#define FGS4D_MAX_FREQ 4      /* K: Fourier orders 0..K */
#define FGS4D_TILE 16         /* default compositing tile: 16 x 16 pixels (32 x 32 selectable) */

typedef struct CUstream_st *fgs4d_stream; /* identical to cudaStream_t */

typedef enum {
    FGS4D_OK = 0,
    FGS4D_ERR_INVALID_ARG = 1, /* bad pointer, size, option or layout */
    FGS4D_ERR_CAPACITY = 2,    /* the state is too small / pair capacity exceeded */
    FGS4D_ERR_CUDA = 3,        /* a CUDA launch or copy failed */
    FGS4D_ERR_TIMEOUT = 4,     /* reserved: no kernel of this library waits */
    FGS4D_ERR_NONFINITE = 5    /* non-finite input or a zero-norm quaternion */
} fgs4d_status;

typedef enum { FGS4D_F32 = 0, FGS4D_BF16 = 1 } fgs4d_dtype;

/* How the 4D rotation R of Sigma = R S S^T R^T is formed.
   FGS4D_ROT_4D: R = L(q_left) R(q_right), Eq. 8 (the method).
   FGS4D_ROT_SPATIAL: the "No-4DRot" variant of the ablation (Sec. 4.3): only
   x, y, z rotate, R = blockdiag(R3(q_left), 1) with R3 the usual rotation
   of a unit quaternion (w, x, y, z); Sigma is block-diagonal, so the slice
   at t leaves the mean and the spatial covariance unchanged (no motion) and
   p(t) depends on s_t alone.  q_right is not read (may be NULL) and its
   gradient is zero.  The kernels take the short path: no Schur complement,
   no velocity term, and neither in the adjoint.
   FGS4D_ROT_STATIC: the special case of a static 3D Gaussian (3D Gaussian
   splatting, the model 4DGS extends in Sec. 3.1): as FGS4D_ROT_SPATIAL with
   no time axis at all.  mu_t and s_t are not read, p(t) = 1 for every view,
   and the 4DSH time basis is evaluated at dt = 0 (every Fourier order counts
   with cos 0 = 1; n_freq = 0 gives plain SH colour).  The gradients of
   q_right, mu_t and log s_t are zero. */
typedef enum { FGS4D_ROT_4D = 0, FGS4D_ROT_SPATIAL = 1, FGS4D_ROT_STATIC = 2 } fgs4d_rotation;

/* Device status bits written into the state (see fgs4d_counters.status). */
#define FGS4D_STATUS_PAIR_OVERFLOW 1u  /* more (splat, tile) pairs than capacity */
#define FGS4D_STATUS_NONFINITE 2u      /* a Gaussian had non-finite values or |q| ~ 0 */

/* 4D Gaussians in structure-of-arrays layout (Sec. 3.2 "Representation of
   4D Gaussian"; Eq. 11 for the coefficients).  All arrays are device memory,
   row-major with the Gaussian index fastest:
     mu            [4][n] float  (mu_x, mu_y, mu_z, mu_t)
     log_scale     [4][n] float  log(s_x, s_y, s_z, s_t); S = diag(exp(.))
     q_left        [4][n] float  q_l = (a, b, c, d), scalar first, any norm > 0
     q_right       [4][n] float  q_r = (p, q, r, s), scalar first, any norm > 0
     opacity_logit [n]    float  alpha = 1 / (1 + exp(-logit))
     shs           [3*(L+1)^2*(K+1)][n]  float32 or bfloat16 (shs_dtype):
                   row (f*(L+1)^2 + j)*3 + ch holds k for Fourier order f,
                   real SH index j = l^2 + l + m and colour channel ch.
   Every array pointer must be 16-byte aligned. */
typedef struct {
    const float *mu;
    const float *log_scale;
    const float *q_left;
    const float *q_right;
    const float *opacity_logit;
    const void *shs;
    int64_t n;       /* 0 <= n < 2^31 / n_views */
    int sh_degree;   /* L, 0..FGS4D_MAX_SH_DEGREE */
    int n_freq;      /* K, 0..FGS4D_MAX_FREQ */
    float period;    /* T of Eq. 11, > 0 */
    int shs_dtype;   /* fgs4d_dtype */
    int rotation;    /* fgs4d_rotation */
} fgs4d_gaussians;

/* One camera at one time t (host memory). */
typedef struct {
    float viewmat[12]; /* row-major 3x4 [W | tau]: x_cam = W x_world + tau; W a rotation */
    float fx, fy, cx, cy;
    int width, height; /* 1..16384 each */
    float t;           /* render time */
    float bg[3];       /* background colour added with the final transmittance */
} fgs4d_view;

/* Rendering options; fgs4d_default_options() fills the values below. */
typedef struct {
    float p_min;      /* 0.05: drop Gaussians with p(t) < p_min (Sec. 4.2) */
    float near_z;     /* 0.2: drop splats with camera depth below near_z */
    float alpha_min;  /* 1/255: skip a splat at a pixel when alpha < alpha_min */
    float alpha_max;  /* 0.99: clamp of alpha */
    float T_min;      /* 1e-4: stop before a splat that would bring T below T_min */
    float dilation;   /* 0.3: added to both diagonal entries of the 2D covariance */
    float clamp_fov;  /* 1.3: clamp x/z to +-clamp_fov*W/(2 fx) inside J; 0 = off */
    int record_fp16;  /* 0: FP32 splat records; 1: FP16 conic (mixed precision) */
    float schur_cond; /* 1e-3: FP64 Schur complement when min_i Sigma3_ii/Sigma_ii is below */
    float conic_cond; /* 1e-4: FP64 2x2 inversion when det/(S00*S11) is below */
    int tile_size;    /* 16 or 32: side of the square compositing tiles (one thread block each);
                         with 32 each thread composites 2x2 pixels */
    int batch_depth;  /* 256: splat records a tile stages in shared memory per batch while
                         compositing (32, 64, 128 or 256); results do not depend on it */
    int aux_channels; /* 0; 1: fgs4d_slice_project also stores, per splat, its camera depth and
                         the displacement of its projected mean from t to t + flow_dt, for
                         fgs4d_render_aux (the state grows by 16 bytes per splat) */
    float flow_dt;    /* 1/300: time step of the optical-flow channels (one frame of 300) */
    int bin_size;     /* 0: tile_size; else 16, 32 or 64 and a multiple of tile_size: side of the
                         binning tiles, the screen cells whose depth-ordered splat lists
                         fgs4d_bin_sort builds; each list serves the (bin_size/tile_size)^2
                         compositing tiles inside its cell.  Larger cells make fewer (splat,
                         tile) pairs to sort when splats span several compositing tiles;
                         results do not depend on it.  "Tile" in the counters, the state
                         layout and fgs4d_bin_sort means a binning tile. */
    int accumulate_grads; /* 0: the backward calls overwrite grads; 1: they add to grads'
                         current contents with atomic adds (nothing is zeroed), so that
                         the adjoints of several view batches of one parameter set, each
                         with its own state, sum into one set of gradients, also when
                         they run concurrently on different streams (the order of the
                         FP32 sums then varies from run to run) */
} fgs4d_options;

/* Gradients w.r.t. the raw parameters, same layouts as fgs4d_gaussians but
   always float32.  Overwritten by fgs4d_render_backward, or added to with the
   option accumulate_grads. */
typedef struct {
    float *mu;
    float *log_scale;
    float *q_left;
    float *q_right;
    float *opacity_logit;
    float *shs;
    float *mean2d_abs; /* optional [n]: sum over views of |dL/d mu_2d| (densification signal); may be NULL */
    float *mu_t_abs;   /* optional [n]: sum over views of |dL/d mu_t| of each view (the temporal
                          densification signal, Sec. 3.4); may be NULL */
} fgs4d_gaussian_grads;

/* Counters read back by fgs4d_read_counters. */
typedef struct {
    uint32_t n_visible;   /* (view, Gaussian) splats that touch at least one tile */
    uint32_t n_pairs;     /* (splat, tile) pairs needed */
    uint32_t status;      /* FGS4D_STATUS_* bits */
    uint32_t pair_capacity;
} fgs4d_counters;

/* Library version (FGS4D_ABI_VERSION). */
int fgs4d_abi_version(void);

/* Number of kernel launches this library has issued in the process so far
   (all threads and devices; for benchmarks that report launch counts). */
uint64_t fgs4d_launch_count(void);

/* Human-readable text of a status code (static storage). */
const char *fgs4d_status_string(fgs4d_status status);

/* Fills *opt with the defaults documented in fgs4d_options. */
void fgs4d_default_options(fgs4d_options *opt);

/* Bytes of per-frame state needed for n Gaussians, these views and room for
   pair_capacity (splat, tile) pairs (4 bytes per pair on the counting-sort
   path of fgs4d_bin_sort, 16 on its radix path).  The same n, views and pair
   capacity must be used by every call that receives this state.  Returns
   INVALID_ARG for bad sizes. */
fgs4d_status fgs4d_state_size(int64_t n, const fgs4d_view *views, int n_views, int64_t pair_capacity,
                              const fgs4d_options *opt, size_t *bytes);

/* Number of pixels over all views (sum W*H): the length of final_T/n_last;
   the image holds three times as many floats. */
int64_t fgs4d_total_pixels(const fgs4d_view *views, int n_views);

/* Slice, colour and project every Gaussian for every view (Eq. 3, 4, 7-11;
   the p(t) filter of Sec. 4.2).  Writes the splat records and per-splat tile
   counts into the state and clears its counters.  state must be 256-byte
   aligned and state_bytes the value fgs4d_state_size() returned. */
fgs4d_status fgs4d_slice_project(const fgs4d_gaussians *g, const fgs4d_view *views, int n_views,
                                 const fgs4d_options *opt, void *state, size_t state_bytes, fgs4d_stream stream);

/* Bin the splats to the binning tiles (bin_size x bin_size pixels) their
   support ellipse reaches and order each tile's list by (depth, Gaussian
   index) on the device (Sec. 3.1/3.2): a radix sort of the visible splats by
   depth, then a stable counting sort of the (tile, splat) pairs when every
   view has at most 4096 binning tiles, else a stable radix sort of the pairs
   by tile id.  Both give the same lists.
   Pairs beyond the capacity are dropped and FGS4D_STATUS_PAIR_OVERFLOW is set. */
fgs4d_status fgs4d_bin_sort(int64_t n, const fgs4d_view *views, int n_views, const fgs4d_options *opt, void *state,
                            size_t state_bytes, fgs4d_stream stream);

/* Front-to-back compositing of Eq. 6 for every pixel of every view.
   image: device float [3 * total_pixels]; final_T: device float
   [total_pixels]; n_last: device int32 [total_pixels] (list entries walked
   up to the last contributing splat).  final_T and n_last are needed by the
   backward pass. */
fgs4d_status fgs4d_render(int64_t n, const fgs4d_view *views, int n_views, const fgs4d_options *opt, void *state,
                          size_t state_bytes, float *image, float *final_T, int32_t *n_last, fgs4d_stream stream);

/* The adjoint in its two steps (fgs4d_render_backward runs both):
   fgs4d_render_backward_2d is the adjoint of Eq. 6 alone.  It writes, into the
   state's grad2d section (zeroed first), the gradient of the loss w.r.t. each
   splat's 2D parameters (u, v, conic a, b, c, alpha_eff, R, G, B), summed over
   the splat's pixels.  fgs4d_project_backward then chains those through the
   projection, the slice and the 4DSH colour (Eq. 3, 4, 7-11) to dL/d(raw
   parameters), summed over views, into grads (overwritten); it consumes the
   grad2d section (reuses it as scratch), so read the 2D gradients before.
   Same arguments and errors as fgs4d_render_backward. */
fgs4d_status fgs4d_render_backward_2d(int64_t n, const fgs4d_view *views, int n_views, const fgs4d_options *opt,
                                      void *state, size_t state_bytes, const float *final_T, const int32_t *n_last,
                                      const float *dL_dimage, fgs4d_stream stream);
fgs4d_status fgs4d_project_backward(const fgs4d_gaussians *g, const fgs4d_view *views, int n_views,
                                    const fgs4d_options *opt, void *state, size_t state_bytes,
                                    fgs4d_gaussian_grads *grads, fgs4d_stream stream);

/* Split sampling in 4D (Sec. 3.4, densification): for j < m, new 4D means
   out_mu[i*m + j] = mu + R diag(s) z_j of Gaussian index[j], i = x, y, z, t,
   so that the samples follow the Gaussian's own 4D density N(mu, Sigma),
   Sigma = R S S^T R^T (Eq. 7-8).  index: device int64 [m]; z: device float
   [4][m], standard normal draws supplied by the caller; out_mu: device float
   [4][m].  An out-of-range index or a Gaussian with non-finite parameters
   yields NaN for that sample. */
fgs4d_status fgs4d_sample_split(const fgs4d_gaussians *g, const int64_t *index, const float *z, int64_t m,
                                float *out_mu, fgs4d_stream stream);

/* Depth and optical-flow maps composited like the colour (Eq. 6 with the
   colour replaced by a per-splat value, background 0), over the lists of the
   last fgs4d_bin_sort: aux_image (device float32, the image's layout, three
   planes per view) receives
     plane 0: sum_i alpha_i T_i z_i, z_i the camera depth of mu_{xyz|t};
              divided by 1 - final_T it is the expected depth;
     planes 1, 2: sum_i alpha_i T_i (u_i(t + flow_dt) - u_i(t)) and likewise
              for v: the flow of the projected conditional means (Eq. 9
              moves mu_{xyz|t} linearly in t), the motion the paper renders
              as optical flow.
   The state must come from fgs4d_slice_project with aux_channels = 1
   (FGS4D_ERR_INVALID_ARG otherwise).  A second walk over the lists: it costs
   about as much as fgs4d_render. */
fgs4d_status fgs4d_render_aux(int64_t n, const fgs4d_view *views, int n_views, const fgs4d_options *opt, void *state,
                              size_t state_bytes, float *aux_image, fgs4d_stream stream);

/* fgs4d_render plus a count of the work its walk did; the paper has no
   counterpart (it measures Eq. 6's cost for throughput accounting).  Writes
   image, final_T and n_last exactly as fgs4d_render does and ADDS to
   stats[0..3] (device, 4 uint64, 8-byte aligned, zeroed by the caller):
     stats[0]  (pixel, splat) pairs with the pixel inside the splat's support
               box (|x - u| <= hx, |y - v| <= hy) before the pixel stopped,
     stats[1]  pairs blended into their pixel (alpha >= alpha_min, not stopped),
     stats[2]  the sum of n_last over all pixels,
     stats[3]  pairs the kernel evaluated: the pixel had not stopped and the
               splat's box reached the group of pixels it is culled with.
   Slower than fgs4d_render (one 64-bit atomic per warp and counter); not
   meant for the training loop. */
fgs4d_status fgs4d_render_stats(int64_t n, const fgs4d_view *views, int n_views, const fgs4d_options *opt,
                                void *state, size_t state_bytes, float *image, float *final_T, int32_t *n_last,
                                uint64_t *stats, fgs4d_stream stream);

/* Adjoint of slice_project + bin_sort + render: given dL/d(image) (same
   layout as image), writes dL/d(raw parameters) summed over all views into
   grads (overwritten).  Transmittance is recomputed from final_T, not stored
   per splat.  g, views, opt and the state must be those of the forward pass. */
fgs4d_status fgs4d_render_backward(const fgs4d_gaussians *g, const fgs4d_view *views, int n_views,
                                   const fgs4d_options *opt, void *state, size_t state_bytes, const float *final_T,
                                   const int32_t *n_last, const float *dL_dimage, fgs4d_gaussian_grads *grads,
                                   fgs4d_stream stream);

/* Byte offsets of the state's sections, for inspection and tests.
   records: one per (view v, Gaussian g) at index v*n + g, record_bytes each
   (FP32 layout: float u, v, conic a, b, c, alpha_eff, R, G, B, depth,
   hx, hy, where outside |x - u| <= hx, |y - v| <= hy the splat's alpha is
   below alpha_min); tiles_touched: uint32 per (v, g), 0 = culled;
   ranges: uint32 pairs [start, end) per global tile (tiles of view v follow
   those of views < v, row-major); pair_vals: uint32 splat index v*n + g per
   list entry, in the buffer that holds the sorted lists; grad2d: 12 floats
   per splat (v*n + g), the first nine dL/d(u, v, a, b, c, alpha_eff, R, G,
   B) after fgs4d_render_backward_2d. */
typedef struct {
    uint64_t counters, records, tiles_touched, ranges, pair_vals;
    uint64_t record_bytes, n_splats, total_tiles, pair_capacity, grad2d;
} fgs4d_state_layout_info;

/* Fills *out for the state of (n, views, opt, state_bytes). Host only. */
fgs4d_status fgs4d_state_layout(int64_t n, const fgs4d_view *views, int n_views, const fgs4d_options *opt,
                                size_t state_bytes, fgs4d_state_layout_info *out);

/* Largest n * n_views accepted by fgs4d_render_backward_noalloc. */
#define FGS4D_NOALLOC_MAX_SPLATS 262144

/* fgs4d_render_backward without caller-provided scratch.  The paper has no
   counterpart: this is an interface for callers that cannot call cudaMalloc
   when they run the backward pass, e.g. real-time loops that reserve all
   device memory once at start-up and may not allocate afterwards, or plugins
   hosted by an engine that owns the device allocator and forbids allocations
   of its own.  Same arguments, results and tolerance as
   fgs4d_render_backward; the forward state is read as input but its
   per-splat gradient section is not used.  That scratch (48 bytes per (view,
   Gaussian) splat, plus the list of visible splats) lives instead in a
   static device array of the library, 13 MiB, which every GPU that loads the
   library holds until the process exits:
   - n * n_views above FGS4D_NOALLOC_MAX_SPLATS returns FGS4D_ERR_CAPACITY
     before anything is enqueued;
   - the first call on a device looks up the array's device address (once per
     device, with that device current); make that first call before any
     stream capture;
   - the looked-up address is kept for the life of the process: calls after
     cudaDeviceReset() (or any other teardown of the device's primary
     context) are not supported;
   - every call clears the part of the array it uses, then reuses it: calls
     that overlap on the GPU (other streams, other threads) race on it and
     must be serialised by the caller;
   - nothing is allocated or freed, on the device or on the host. */
fgs4d_status fgs4d_render_backward_noalloc(const fgs4d_gaussians *g, const fgs4d_view *views, int n_views,
                                           const fgs4d_options *opt, void *state, size_t state_bytes,
                                           const float *final_T, const int32_t *n_last, const float *dL_dimage,
                                           fgs4d_gaussian_grads *grads, fgs4d_stream stream);

/* Copies the state's counters to *out (synchronises `stream`). */
fgs4d_status fgs4d_read_counters(const void *state, fgs4d_counters *out, fgs4d_stream stream);

/* ---------------------------------------------------------------- training step
   The steps around the rendering routine in the paper's end-to-end training
   (Sec. 3.3), with the photometric loss it adopts from 3D Gaussian splatting
   (Sec. 4.1 setup). */

/* Bytes of device scratch fgs4d_loss_l1_dssim needs for these views (0 on bad
   views).  Host only. */
size_t fgs4d_loss_scratch_size(const fgs4d_view *views, int n_views);

/* L = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)) over all pixels
   and channels of the batch, and dL/dx.  x = image, y = target: device, float32,
   the layout of fgs4d_render's image.  SSIM per channel with an 11x11 Gaussian
   window (sigma 1.5, sum 1, zero padding), C1 = 0.01^2, C2 = 0.03^2.  Writes
   *loss (device, one float) and dL_dimage (device, the image's layout; may not
   alias image or target).  scratch: device, 256-byte aligned, at least
   fgs4d_loss_scratch_size() bytes; contents undefined afterwards.
   lambda in [0, 1] (0.2 in the paper's setting).  Argument errors on the host;
   FGS4D_ERR_CAPACITY if scratch is too small. */
fgs4d_status fgs4d_loss_l1_dssim(const fgs4d_view *views, int n_views, const float *image, const float *target,
                                 float lambda, float *loss, float *dL_dimage, void *scratch, size_t scratch_bytes,
                                 fgs4d_stream stream);

/* One parameter group of fgs4d_adam_step: count float32 elements each of the
   parameter, its first and second moment estimates (updated in place) and its
   gradient; all device.  param_bf16 (optional, device): receives the updated
   parameter rounded to bfloat16 (the mixed-precision renderer's copy of the
   4DSH coefficients).  lr_index: which entry of lrs applies. */
typedef struct {
    float *param;
    float *exp_avg;
    float *exp_avg_sq;
    const float *grad;
    void *param_bf16;
    int64_t count;
    int lr_index;
} fgs4d_adam_group;

/* Adam (Kingma and Ba, with bias correction) over up to 8 groups in two
   launches: *step (device int64) is incremented first and t = the new value
   is used, so a captured graph advances it on every replay; lrs (device
   floats) are read at run time for the same reason.  bias_scratch: device,
   two floats.  p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
   The paper has no optimiser of its own (it trains with Adam). */
fgs4d_status fgs4d_adam_step(const fgs4d_adam_group *groups, int n_groups, const float *lrs, float beta1,
                             float beta2, float eps, int64_t *step, float *bias_scratch, fgs4d_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* FGS4D_H */
