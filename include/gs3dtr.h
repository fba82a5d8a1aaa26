/*
 * gs3dtr.h - C ABI of the GB300 hot path of the 3DGS^2-TR optimiser
 * (arXiv 2602.00395, "Scalable Second-Order Trust-Region Method for 3D
 * Gaussian Splatting").
 *
 * One training iteration is six calls, all asynchronous on a caller stream:
 *
 *   gs_project      EWA projection of every Gaussian into every view   (Sec. 3.1)
 *   gs_bin_sort     (tile, depth) keys and their radix sort, tile ranges (Sec. 3.1)
 *   gs_raster_fwd   front-to-back alpha blending (+ forward-mode tangents J z)
 *   gs_raster_bwd   reverse pass: gradient g = (1/m) J^T F           (Sec. 4.1)
 *                   and, fused, the Hutchinson product (1/nu) sum z.(G z)
 *   gs_hvp_diag     the Hutchinson product alone                      (Sec. 4.1)
 *   gs_tr_update    Algorithm 1: EMAs, diagonal Newton step, squared-Hellinger
 *                   radius per parameter, clip, update          (Sec. 4.2, App. B)
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every pointer inside the structs and every array argument is DEVICE memory
 *   owned by the caller, 16-byte aligned, unless marked "host".  The structs
 *   themselves are host memory read during the call only.
 * - No call allocates device memory or synchronises the stream.  Scratch
 *   space comes from the caller through the *_workspace_size queries.
 * - Calls return GS_OK or an error code for invalid arguments or a failed
 *   launch; gs_last_error() then describes the first problem (thread-local).
 *   Conditions found on the device (pair capacity exceeded, non-finite values,
 *   a bounded wait that gave up) are OR-ed into the caller's device status word
 *   (int32, may be NULL) as GS_FLAG_* bits, to be read after the stream completes.
 * - No C++ exception crosses this boundary.
 *
 * Parameter layout (gs_params): one float32 matrix of `rows` rows and row
 * pitch n_pad (n_pad >= n, n_pad % 4 == 0), grouped by type as in Sec. 3.1:
 *     rows 0..2   mean mu                      rows 3..5   log-scale (s = exp)
 *     rows 6..9   quaternion (x, y, z, w), unnormalised
 *     row  10     opacity logit (alpha = sigmoid)
 *     rows 11..   SH coefficient k of channel c at row 11 + 3k + c, K = (deg+1)^2
 *     rows = 11 + 3K (14 for degree 0, 59 for degree 3)
 * Gradient, Hutchinson, EMA and radius buffers use the same struct and layout.
 * Probe entry of row r of Gaussian (column) i: j = i * rows + r (see gs_probe).
 */
#ifndef GS3DTR_H
#define GS3DTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
typedef int32_t gs_status;
enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* a host-checked argument is out of range */
  GS_ERR_CUDA = 2,        /* a kernel launch or async memset failed */
  GS_ERR_UNSUPPORTED = 3  /* valid but not built (e.g. nu > 2, sh_degree > 3) */
};
/* bits of the device status word */
enum {
  GS_FLAG_CAPACITY = 1,  /* gs_bin_sort: more pairs than capacity; *n_pairs holds the need */
  GS_FLAG_NONFINITE = 2, /* gs_tr_update: a non-finite value was written */
  GS_FLAG_TIMEOUT = 4    /* a bounded wait on an asynchronous copy gave up */
};

const char* gs_last_error(void); /* host string, valid until the next call on this thread */
int32_t gs_version(void);        /* major * 10000 + minor * 100 + patch */

/* ------------------------------------------------------------ data */
typedef struct gs_params {
  int32_t n;         /* Gaussians */
  int32_t n_pad;     /* row pitch in elements, multiple of 4, >= n */
  int32_t sh_degree; /* 0..3 */
  int32_t reserved;
  float* data;       /* device, rows x n_pad */
} gs_params;

/* Pinhole camera, world -> camera viewmat (row-major, camera x right, y down,
 * z forward).  Pixel (i, j) is sampled at (i + 0.5, j + 0.5).  Arrays of
 * cameras are DEVICE arrays of this struct. */
typedef struct gs_camera {
  float viewmat[16];
  float fx, fy, cx, cy;
  float near_plane;
  int32_t width, height;
  int32_t reserved;
} gs_camera;

/* Views rendered by one call; every camera of the call has this size.
 * tile_w is 8, 16 or 32, tile_h a power of two >= 8, tile_w * tile_h is 64, 128,
 * 256 or 512 (two pixels per thread; each warp covers an 8 x 8 pixel block).
 * footprint_bins selects the tiles of a splat (see gs_bin_sort): 0 its 3DGS tile
 * square, 1 that square narrowed to its alpha >= 1/255 footprint (its box, then
 * row by row its ellipse).  Both give the same images and derivatives; 1 gives
 * fewer pairs.
 * batch: records a tile's block stages in shared memory per step of its list in
 * the blends (gs_raster_fwd, gs_raster_bwd, gs_hvp_diag): 0 for one per thread,
 * else a multiple of 32 from 32 to 512.  It changes speed, not results. */
typedef struct gs_frame {
  int32_t n_views, width, height, tile_w, tile_h, footprint_bins, batch;
} gs_frame;

/* Rademacher probes z_k (k < nu) of step t: row r of Gaussian i is entry
 * j = i * rows + r (rows = 11 + 3K), and entry j is -1 where bit (j mod 64) of
 * SplitMix64(seed ^ t * 0x9E3779B97F4A7C15 ^ (k << 56) ^ (j / 64)) is set, +1
 * otherwise: 64 entries per hash.
 * t_device (may be NULL): a device int64 read by the kernels in place of t, so
 * that a captured CUDA graph replays successive steps (see gs_step_advance). */
typedef struct gs_probe {
  uint64_t seed;
  int64_t t;
  int32_t nu; /* 0, 1 or 2 */
  int32_t reserved;
  const int64_t* t_device;
} gs_probe;

/* The radius schedule of Sec. 5: eps_t = eps0 (eps1 / eps0)^((t - 1) / (total - 1))
 * (eps0 for total <= 1), evaluated in double precision and rounded to float. */
typedef struct gs_eps_schedule {
  double eps0, eps1;
  int64_t total;
} gs_eps_schedule;

/* Projected splats of V views (device, caller-owned).
 *   rec:     V x n_pad records of 12 floats (48 B):
 *            (mx, my, A, B), (C, opacity, r, g), (b, depth, radius, extents)
 *            where (A, B, C) is the conic, radius is an int32 bit pattern
 *            (0: culled) and extents packs two IEEE half floats (x low, y high):
 *            half-widths of the bounding box of the alpha >= 1/255 footprint
 *            d^T (A B; B C) d <= 2 ln(255 opacity), widened by 0.1% + 0.01 px and
 *            rounded up (-inf: no pixel reaches 1/255; +inf: unbounded).
 *            Binning narrows the splat's tile square to that box, and the
 *            rasteriser skips the splat for an 8 x 8 pixel block outside it.
 *   tangent: NULL or V x n_pad x (1 + nu) records of 12 floats: for each
 *            (view, splat) a copy of its record in rec, then its nu probe
 *            tangent records, the forward-mode derivative of (mx, my, A, B, C,
 *            opacity, r, g, b) along probe k (adjacent, so that the rasteriser
 *            stages all of a splat's records with one copy) */
typedef struct gs_projected {
  float* rec;
  float* tangent;
} gs_projected;

/* Sorted (tile, splat) pairs (device, caller-owned).
 *   keys:     capacity x uint32 (16-byte aligned), key = view * tiles + tile; the
 *             pairs of one key are in (depth, splat index) order
 *   vals:     capacity x uint32, splat index
 *   ranges:   V * tiles x 2 uint32, [start, end) of each tile's pairs
 *   n_pairs:  one uint32, number of pairs the views need (may exceed capacity)
 *   order:    NULL, or V * tiles uint32 that gs_bin_sort fills with the tiles
 *             (view * tiles + tile) from the longest list to the shortest
 *             (lengths grouped in steps of 1/8 of a power of two, any order
 *             within a group); the blends then start the heaviest tiles first.
 *             It changes when a tile runs, never its result.
 *   masks:    NULL, or capacity bytes.  gs_raster_fwd writes, for every pair it
 *             stages, which 8 x 8 pixel blocks of the pair's tile the splat's
 *             footprint reaches (bit w: the block of warp w, see gs_frame);
 *             gs_raster_bwd, gs_hvp_diag and gs_raster_bwd_batch then read those
 *             bits instead of testing the footprint again.  The bits of a pair
 *             are valid once gs_raster_fwd has run on these sorted pairs with the
 *             same frame (the reverse passes read only list positions the
 *             forward staged); pass NULL to a reverse pass otherwise.  Either
 *             way the results are the same. */
typedef struct gs_sorted {
  uint32_t* keys;
  uint32_t* vals;
  uint32_t* ranges;
  uint32_t* n_pairs;
  uint64_t capacity;
  uint32_t* order;
  uint8_t* masks;
} gs_sorted;

enum { GS_LOSS_L1 = 0, GS_LOSS_L2 = 1, GS_LOSS_COTANGENT = 2, GS_LOSS_WEIGHTED = 3 };

/* Per-pixel loss of Sec. 3.2 in least-squares form f = 1/(2m) sum F^2 over the
 * m = 3 H W V residual components r = render - target:
 *   GS_LOSS_L1: F = sqrt(|r|); dL/dC = sign(r)/(2m); GN weight 1/(4 max(|r|, gn_floor)) / m
 *   GS_LOSS_L2: F = r;         dL/dC = r/m;          GN weight 1/m
 *   GS_LOSS_COTANGENT: any objective whose image-space vectors the caller forms:
 *       `target` then holds S cotangent images, S x V x 3 x H x W: first dL/dC
 *       (when the gradient is requested), then for each probe k the vector
 *       u_k whose pull-back J^T u_k is the Gauss-Newton product G z_k (for the
 *       objective of Sec. 3.2, u_k = (1/m) sum_j grad_C F_j (grad_C F_j . J z_k)).
 *       The image is not read, loss_out is left as it is, and the probe count
 *       comes from `probe` alone (image_tangent is not read).
 *   GS_LOSS_WEIGHTED: a least-squares objective whose Gauss-Newton weights the
 *       caller forms per pixel and channel: `target` holds, when the gradient is
 *       requested, the image dL/dC first, then one weight image w (V x 3 x H x W);
 *       the reverse pass forms u_k = w . J z_k itself from image_tangent, so that
 *       G z_k = J^T diag(w) J z_k (Sec. 4.1; for the objective of Sec. 3.2,
 *       w = 1/(4 max(|r|, delta))/m).  The image is not read and loss_out is left
 *       as it is. */
typedef struct gs_loss {
  int32_t kind;
  float gn_floor;
} gs_loss;

/* Algorithm 1 hyper-parameters.  The denominator of the Newton step is
 * max(D_hat, d_floor); the colour radius uses max(DC colour, color_floor);
 * mean_exact = 0 uses Sigma_cc as printed in Sec. 4.2, 1 uses 1/(Sigma^-1)_cc. */
typedef struct gs_tr_config {
  float theta1, theta2, d_floor, color_floor;
  int32_t l, mean_exact;
} gs_tr_config;

/* ------------------------------------------------------------ calls */

/* Sec. 3.1 (projection the paper defers to 3DGS): for every Gaussian and view,
 *   t = W mu + t_w (culled if t_z <= near), Sigma = R diag(s^2) R^T,
 *   Sigma' = J W Sigma W^T J^T + 0.3 I (J the perspective Jacobian with the
 *   image-plane slope clamped at 1.3 x the half field of view), conic = Sigma'^-1,
 *   radius = ceil(3 sqrt(lambda_max)), rgb = max(SH(view dir) + 0.5, 0),
 *   opacity = sigmoid(logit), and the footprint extents described with gs_projected.
 * cams: device array of frame.n_views cameras.  probe may be NULL (no tangents);
 * otherwise out->tangent receives probe->nu tangent records per view. */
gs_status gs_project(const gs_params* x, const gs_camera* cams, gs_frame frame, const gs_probe* probe,
                     gs_projected* out, int32_t* status, void* stream);

/* Sec. 3.1 tile binning and depth order: all (tile, splat) pairs of all views
 * sorted by (view, tile, depth, splat index), and each tile's [start, end).  A splat's tiles
 * are its 3DGS square, decided in FP32 with one rounding per operation:
 *   x0 = clamp(floor((mx - r)/tw), 0, Tx), x1 = clamp(floor((mx + (r + tw - 1))/tw), 0, Tx)
 * (the same for y); with frame.footprint_bins = 1 also
 *   x0 >= clamp(floor((mx - hx)/tw), 0, Tx), x1 <= clamp(floor((mx + hx)/tw) + 1, 0, Tx)
 * with hx, hy the record's footprint extents, and then each tile row ty keeps
 * the tiles from floor(xl/tw) to floor(xr/tw), where [xl, xr] is the footprint
 * ellipse's extent over the row's band [ty th, (ty + 1) th], widened by 1 % of hx
 * + 0.5 px: with rho = -B/sqrt(A C), v = (y - my)/hy, the ends are
 * mx + hx (rho v +- sqrt((1 - rho^2)(1 - v^2))) at v = +-rho clamped into the
 * band (a band outside |v| <= 1 keeps nothing), each step one FP32 rounding.
 * A tile outside the footprint holds no pixel where the splat is blended (its
 * alpha stays below 1/255 there), so this removes pairs but changes no image.  If the pairs
 * exceed out->capacity, GS_FLAG_CAPACITY is raised, *n_pairs holds the need,
 * and the sorted arrays are incomplete (but every access stays in bounds and
 * every range end is at most the capacity). */
size_t gs_bin_sort_workspace_size(int32_t n_pad, gs_frame frame, uint64_t capacity);
gs_status gs_bin_sort(const gs_projected* proj, int32_t n_pad, gs_frame frame, void* workspace,
                      size_t workspace_bytes, gs_sorted* out, int32_t* status, void* stream);

/* gs_bin_sort for callers that cannot allocate device memory (this entry has no
 * counterpart in the paper).  Some callers cannot provide gs_bin_sort's
 * workspace: a server whose allocator is frozen after it reserved its memory, a
 * plugin handed only device pointers by a framework that owns allocation, or a
 * loop that must never pay cudaMalloc's implicit synchronisation.  This call
 * gives the same result as gs_bin_sort with the same arguments, but takes its
 * scratch from a 32 MiB device array inside the library (held on every GPU that
 * loads the library until the process exits) and allocates nothing.
 *   - Limit: gs_bin_sort_workspace_size(n_pad, frame, out->capacity) must be at
 *     most 32 MiB (for example 1 million pairs with 131,072 view x n_pad records);
 *     larger requests return GS_ERR_INVALID_ARG with an explanation.
 *   - The first call on each device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress); make it before any stream
 *     capture.
 *   - Every call shares the one array: calls that may overlap on the GPU race on
 *     it and must be ordered by the caller.  No scratch word needs to start at zero. */
gs_status gs_bin_sort_noalloc(const gs_projected* proj, int32_t n_pad, gs_frame frame, gs_sorted* out,
                              int32_t* status, void* stream);

/* Sec. 3.1 blending: C = sum_i c_i a_i T_i, T_i = prod_{j<i} (1 - a_j),
 * a = min(0.99, o exp(power)), splats with a < 1/255 skipped, stop before T
 * would fall below 1e-4, black background.
 *   image V x 3 x H x W, final_T V x H x W, n_contrib V x H x W (1 + list
 *   position of the last blended splat).  If proj->tangent and probe are given,
 *   image_tangent (probe->nu x V x 3 x H x W) receives J z_k. */
gs_status gs_raster_fwd(const gs_projected* proj, const gs_sorted* sorted, int32_t n_pad, gs_frame frame,
                        const gs_probe* probe, float* image, float* final_T, uint32_t* n_contrib,
                        float* image_tangent, int32_t* status, void* stream);

/* Sec. 4.1: gradient g = (1/m) J^T F of the objective (Eq. objective) over the
 * frame's views, written to grad (overwritten).  If image_tangent and probe are
 * given (S2 = S1), the same reverse pass also writes the Hutchinson diagonal
 * hz = (1/nu) sum_k z_k . ((1/m) J^T diag(w) J z_k) (overwritten).  loss_out
 * (one float, may be NULL) gets the objective added.
 * workspace: device, 16-byte aligned, at least gs_raster_bwd_workspace_size
 *   bytes (a 256-byte header, then the 2-D cotangent rows the reverse blend adds
 *   into).  Any content is accepted on entry.  The call leaves the rows zero
 *   and records that in the header, so a following call on the same workspace
 *   (the same or a smaller frame) skips clearing them; otherwise the call
 *   clears them first.  The same holds for gs_hvp_diag and gs_raster_bwd_batch,
 *   which share this workspace layout. */
size_t gs_raster_bwd_workspace_size(int32_t n_pad, gs_frame frame, int32_t nu);
gs_status gs_raster_bwd(const gs_params* x, const gs_camera* cams, gs_frame frame, const gs_projected* proj,
                        const gs_sorted* sorted, const float* image, const float* target, const float* final_T,
                        const uint32_t* n_contrib, const float* image_tangent, const gs_probe* probe,
                        gs_loss loss, gs_params* grad, gs_params* hz, float* loss_out, void* workspace,
                        size_t workspace_bytes, int32_t* status, void* stream);

/* Sec. 4.1, Hutchinson's estimator alone (for a mini-batch S2 other than S1):
 * hz = (1/nu) sum_k z_k . ((1/m) J^T diag(w) J z_k) (overwritten), from the
 * image tangents J z_k of gs_raster_fwd with the same probe. */
gs_status gs_hvp_diag(const gs_params* x, const gs_camera* cams, gs_frame frame, const gs_projected* proj,
                      const gs_sorted* sorted, const float* image, const float* target, const float* final_T,
                      const uint32_t* n_contrib, const float* image_tangent, const gs_probe* probe,
                      gs_loss loss, gs_params* hz, void* workspace, size_t workspace_bytes, int32_t* status,
                      void* stream);

/* Algorithm 1 for step t >= 1 with radius parameter eps (Sec. 4.2, App. B):
 *   g_ema = theta1 g_ema + (1 - theta1) grad
 *   d_ema = theta2 d_ema + (1 - theta2) hz      when (t - 1) % l == 0 (hz may be NULL otherwise)
 *   step  = clip(-g_ema / max(d_ema, d_floor), -eta, eta),  x += step
 * with eta per parameter from x before the update:
 *   mean       sqrt(-8 Sigma_cc ln(1 - eps/alpha))        (inf if alpha <= eps)
 *   log-scale  sqrt(2 eps / alpha)
 *   quaternion sqrt(-(8/beta_c) ln(1 - eps/alpha))        (inf if beta_c = 0 or alpha <= eps)
 *   logit      sqrt(4 alpha eps) / (alpha (1 - alpha))
 *   SH (k, c)  sqrt(4 C_c eps / alpha) / max|Y_k|         (C_c the floored DC colour)
 * eta_out (may be NULL) receives the radii.  All gs_params share n, n_pad and degree.
 * A non-finite result raises GS_FLAG_NONFINITE. */
gs_status gs_tr_update(gs_params* x, gs_params* g_ema, gs_params* d_ema, const gs_params* grad,
                       const gs_params* hz, const gs_tr_config* cfg, int64_t t, float eps, gs_params* eta_out,
                       int32_t* status, void* stream);

/* gs_tr_update with the step index read on the device from *t_device (>= 1)
 * and eps = eps_t of `schedule`, so that the call can sit in a captured CUDA
 * graph.  Whether this step updates d_ema ((t - 1) % l == 0) is decided on the
 * device; hz must then be given.  A t_device below 1 raises GS_FLAG_NONFINITE
 * and leaves the buffers unchanged. */
gs_status gs_tr_update_dev(gs_params* x, gs_params* g_ema, gs_params* d_ema, const gs_params* grad,
                           const gs_params* hz, const gs_tr_config* cfg, const int64_t* t_device,
                           const gs_eps_schedule* schedule, gs_params* eta_out, int32_t* status, void* stream);

/* Eq. pixel_loss of Sec. 3.2 with the D-SSIM term: per pixel and channel the two
 * residual components F = sqrt((1 - lambda) |r|) and F = sqrt(lambda (1 - S)),
 * S the SSIM of the channel at the pixel (11 x 11 Gaussian window of standard
 * deviation 1.5, zeros outside the image, C1 = 0.01^2, C2 = 0.03^2), and
 * m = 6 H W per view.  Writes the cotangent images that gs_raster_bwd and
 * gs_hvp_diag take with GS_LOSS_COTANGENT (S = want_grad + nu streams,
 * S x V x 3 x H x W):
 *   dL/dC = ((1 - lambda) sign(r) - lambda sum_p dS_p/dC) / (2m)
 *   u_k   = (1 - lambda)/(4 max(|r|, gn_floor))/m . d_k
 *           + A[lambda/(4 max(1 - S, gn_floor))/m . dS[d_k]]
 * with d_k = J z_k from image_tangent (nu x V x 3 x H x W; may be NULL when nu
 * is 0), dS[d] the derivative of the SSIM map along d and A its adjoint.
 * loss_out (one float, may be NULL) gets the objective added.  workspace from
 * gs_dssim_workspace_size. */
size_t gs_dssim_workspace_size(gs_frame frame, int32_t nu);
gs_status gs_dssim_cotangents(gs_frame frame, const float* image, const float* target, const float* image_tangent,
                              int32_t nu, float lambda, float gn_floor, int32_t want_grad, float* cot,
                              float* loss_out, void* workspace, size_t workspace_bytes, int32_t* status,
                              void* stream);

/* Adam hyper-parameters of the ADAM-TR update: beta1, beta2, eps_adam and the
 * learning rate of each row group: lr[0] means, lr[1] log-scales, lr[2]
 * quaternions, lr[3] opacity logit, lr[4] SH DC (rows 11..13), lr[5] the other
 * SH rows. */
typedef struct gs_adam_config {
  float beta1, beta2, eps_adam;
  float lr[6];
} gs_adam_config;

/* ADAM-TR (the ablation of Sec. 5): the trust-region clip of Sec. 4.2 applied
 * to an Adam step, for step t >= 1 with radius parameter eps:
 *   m = beta1 m + (1 - beta1) grad,  v = beta2 v + (1 - beta2) grad^2
 *   step = clip(-lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps_adam), -eta, eta),  x += step
 * with eta from x before the update as in gs_tr_update (cfg supplies
 * color_floor and mean_exact).  m and v are caller-owned state with the layout
 * of x (zero before the first step).  eta_out may be NULL.  A non-finite result
 * raises GS_FLAG_NONFINITE. */
gs_status gs_adam_tr_update(gs_params* x, gs_params* m, gs_params* v, const gs_params* grad,
                            const gs_tr_config* cfg, const gs_adam_config* adam, int64_t t, float eps,
                            gs_params* eta_out, int32_t* status, void* stream);

/* *t_device += 1 on the stream (no paper counterpart: the step counter of a
 * training loop replayed as a CUDA graph). */
gs_status gs_step_advance(int64_t* t_device, void* stream);

/* ------------------------------------------------------------ batches
 * Several independent requests in shared launches (no paper counterpart: the
 * paper trains one scene at a time, Sec. 5).  A batch holds up to GS_BATCH_MAX
 * items of one image size; item b is one view of its own scene, with its own
 * parameters, step index and trust-region state.  The batch's splat records sit
 * in slot b of one set of buffers (records of item b at [b * n_pad_max, ...)),
 * so gs_bin_sort and gs_raster_fwd run on it unchanged as a frame of
 * frame.n_views = n_items views; each item's objective is its own view's
 * (m = 3 H W).  A training step of a batch is
 *   gs_project_batch -> gs_bin_sort -> gs_raster_fwd -> gs_raster_bwd_batch
 *   -> gs_tr_update_batch,
 * a render the first three.  All items share the SH degree, the tile shape
 * and the probe seed and count; n_pad_max >= every item's n, a multiple of 4. */
enum { GS_BATCH_MAX = 16 };

typedef struct gs_batch_item {
  gs_params x;             /* device: the scene's parameters */
  gs_params grad, hz;      /* device: its gradient and Hutchinson diagonal (written; hz.data NULL without probes) */
  gs_params g_ema, d_ema;  /* device: its trust-region state (gs_tr_update_batch updates both in place) */
  const gs_camera* cam;    /* device: the item's camera */
  int64_t t;               /* the scene's step index t >= 1: probes and curvature interval */
  float eps;               /* the radius parameter eps_t of its update */
  int32_t hvp;             /* 1: its update takes d_ema from hz ((t - 1) % l == 0), 0: keeps d_ema */
} gs_batch_item;

/* gs_project for a batch: item b's Gaussians projected into its camera, records
 * (and, with probe, probe->nu tangent records along its probes of step
 * items[b].t) in slot b; columns n..n_pad_max - 1 of a slot are written culled.
 * items: host array of n_items (1..GS_BATCH_MAX); frame.n_views = n_items. */
gs_status gs_project_batch(const gs_batch_item* items, int32_t n_items, int32_t n_pad_max, gs_frame frame,
                           const gs_probe* probe, gs_projected* out, int32_t* status, void* stream);

/* gs_raster_bwd for a batch (Sec. 4.1 per item): item b's gradient
 * (1/m) J^T F of its own view's objective (m = 3 H W) into items[b].grad and,
 * with image_tangent and probe, its Hutchinson diagonal into items[b].hz
 * (overwritten).  loss_out: NULL or n_items floats, item b's objective added
 * to loss_out[b].  workspace from gs_raster_bwd_workspace_size(n_pad_max,
 * frame, nu).  The remaining arguments are those of gs_raster_bwd on the batch's
 * frame. */
gs_status gs_raster_bwd_batch(const gs_batch_item* items, int32_t n_items, int32_t n_pad_max, gs_frame frame,
                              const gs_projected* proj, const gs_sorted* sorted, const float* image,
                              const float* target, const float* final_T, const uint32_t* n_contrib,
                              const float* image_tangent, const gs_probe* probe, gs_loss loss, float* loss_out,
                              void* workspace, size_t workspace_bytes, int32_t* status, void* stream);

/* gs_tr_update for a batch: Algorithm 1 on each item's scene with its own t,
 * eps and hvp (Sec. 4.2, App. B), one launch for all items. */
gs_status gs_tr_update_batch(const gs_batch_item* items, int32_t n_items, const gs_tr_config* cfg, int32_t* status,
                             void* stream);

/* Diagnostics (no paper counterpart): runs, in one warp, the bounded wait that
 * every kernel uses on its asynchronous copies, on an mbarrier that nothing
 * completes, giving up after `limit` tries (1 <= limit <= 2^20).  Raises
 * GS_FLAG_TIMEOUT in *status (device int32) as a kernel does when a staged copy
 * never lands; the kernel then returns and the context stays usable.  Lets
 * the failure path be tested without a fault. */
gs_status gs_wait_check(uint32_t limit, int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GS3DTR_H */
