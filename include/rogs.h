/*
 * rogs.h -- C-ABI of librogs: GB300-native (sm_103a) differentiable splatting
 * of meshgrid Gaussian surfels (RoGs, arXiv 2405.14342).
 *
 * Pointers are plain host or device addresses as stated per argument; sizes
 * are element counts.  No call allocates device memory except rogs_create,
 * rogs_reserve and (when a call needs more scratch than it holds)
 * the first call of a given size; every call is asynchronous on the given
 * stream unless it says it synchronises.  The caller owns every buffer it
 * passes; the library owns only the scratch held in its context.  One
 * context must not be used from two streams at once (its scratch is shared).
 *
 * Errors: every call returns a rogs_status; rogs_last_error() gives a
 * one-line message for the last failing call on that context.  Argument
 * errors are detected on the host (ROGS_ERR_INVALID) before anything is
 * launched.  A data-dependent overflow (more visible surfels or tile pairs
 * than the configured capacities) cannot be seen on the host without a
 * synchronisation: it is recorded in the state header (status word) and
 * returned as ROGS_ERR_CAPACITY by rogs_state_counts(); the frame's outputs
 * are then incomplete and must be recomputed with larger capacities.
 */
#ifndef ROGS_H
#define ROGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rogs_ctx rogs_ctx;
typedef void* rogs_stream; /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
    ROGS_OK = 0,
    ROGS_ERR_INVALID = 1,   /* bad argument, detected on the host */
    ROGS_ERR_CAPACITY = 2,  /* record or pair capacity exceeded (device-detected) */
    ROGS_ERR_OOM = 3,       /* device allocation failed / admission refused */
    ROGS_ERR_CUDA = 4,      /* a CUDA runtime call failed */
    ROGS_ERR_TIMEOUT = 5,   /* a bounded device or host wait gave up */
    ROGS_ERR_BUSY = 6,      /* no free serving slot */
    ROGS_ERR_NOT_READY = 7  /* serving request not finished yet */
} rogs_status;

enum { ROGS_PERSP = 0, ROGS_ORTHO = 1 };

#define ROGS_MAX_VIEWS 128   /* views per render call */
#define ROGS_MAX_CLASSES 54  /* C, semantic logits per surfel */

/* Rendering constants.  Defaults (rogs_default_config): tile 16x16,
   t_min 1e-4, alpha_min 1/255, alpha_max 0.99, eps 0.3 px^2, near 0.2 m,
   box 20 m / 40 m, jac_clamp 1.3, sort_tile 4096.  Tile shape and sort tile
   only change speed, never results. */
typedef struct {
    int32_t tile_w, tile_h;     /* 16x16, 32x8 or 8x8 pixels */
    int32_t num_classes;        /* C in [0, ROGS_MAX_CLASSES] */
    float t_min;                /* stop before T would fall below this (Eq. 6) */
    float alpha_min;            /* a surfel counts at a pixel iff a >= alpha_min */
    float alpha_max;            /* a = min(alpha_max, alpha * g) */
    float eps_dilate;           /* px^2 added to the 2D covariance diagonal */
    float near_plane;           /* perspective: keep iff binary32 depth > near */
    float box_half_x;           /* perspective box cull: |lateral| <= box_half_x (m) */
    float box_depth;            /* and 0 <= forward <= box_depth (m) */
    float jac_clamp;            /* EWA Jacobian evaluated at x/z clamped to +-jac_clamp*W/(2 fx) */
    int32_t sort_tile;          /* pair sort keys per CTA: 1024, 2048, 4096 (default) or 8192 */
    int64_t record_capacity;    /* visible (view, surfel) records per render call */
    int64_t pair_capacity;      /* (tile, record) pairs per render call (<= 2^32-1) */
} rogs_config;

/* One camera.  p_cam = R_wc p_world + t_wc, camera axes x right, y down, z
   forward.  Perspective: u = fx x/z + cx.  Orthographic: u = fx x + cx
   (fx in px per metre).  exposure_idx selects (a, b) of Eq. 7.
   use_box_cull enables the supplementary's perspective box (ignored for
   orthographic cameras). */
typedef struct {
    int32_t kind, width, height, exposure_idx, use_box_cull, reserved;
    float fx, fy, cx, cy;
    float R_wc[9]; /* row-major */
    float t_wc[3];
} rogs_camera;

/* Surfel map (Sec. 3.1, Eq. 3), device pointers, FP32, row-major:
   xyz [n,3], scale [n,2] = (s_x, s_y) (s_z = 0), quat [n,4] = (w,x,y,z)
   (normalised inside), opacity [n] = alpha, rgb [n,3], sem [n,C] logits.
   Optional grid index map of the meshgrid (supplementary "Smooth Loss K
   Nearest Neighbor Acceleration"): grid_index, device int32
   [grid_h][grid_w], the surfel at each grid vertex or -1 where the vertex is
   off the road; NULL (and grid_w = grid_h = 0) when absent.  Only
   rogs_smooth_loss reads it. */
typedef struct {
    const float *xyz, *scale, *quat, *opacity, *rgb, *sem;
    int64_t n;
    const int32_t* grid_index;
    int32_t grid_w, grid_h;
} rogs_surfels;

/* Gradient buffers (device, FP32, same shapes as rogs_surfels plus
   exposure [n_exposure,2]).  rogs_render_bwd ADDS into them.  Any pointer
   may be NULL to skip that gradient. */
typedef struct {
    float *xyz, *scale, *quat, *opacity, *rgb, *sem, *exposure;
} rogs_grads;

/* Counters written by the device into the state header. */
typedef struct {
    uint64_t n_records;      /* visible (view, surfel) records (clamped to capacity) */
    uint64_t n_pairs;        /* (tile, record) pairs (clamped to capacity) */
    uint64_t need_records;   /* records the frame needed */
    uint64_t need_pairs;     /* pairs the frame needed */
    uint64_t composited;     /* (pixel, surfel) pairs composited by the forward */
    uint32_t status;         /* bit 0 record overflow, bit 1 pair overflow */
    uint32_t n_views;
} rogs_counts;

/* Byte offsets of the sections of a render state (device buffer filled by
   rogs_render_fwd and read by rogs_render_bwd).  Pixels of view v start at
   pixel offset pix_base[v] = sum of earlier views' W*H; tiles of view v at
   tile_base[v].  Sections:
     header      rogs_counts
     records     48-byte records: float mean_int[2], mean_frac[2], conic[3]
                 (A,B,C of the inverse 2D covariance), alpha, depth (camera z),
                 key (binary32 sort depth), uint32 surfel, uint32 view;
                 ordered by (view, surfel)
     rects       uint32[2] per record: tx0 | ty0<<16, tx1 | ty1<<16 (inclusive)
     pair_rec    uint32 per pair: record id, ordered by (view, tile, key, surfel)
     tile_range  uint32[2] per tile: [start, end) into pair_rec
     pix_T       float per pixel: final transmittance
     pix_last    uint32 per pixel: entries of its tile list up to and including
                 the last composited one
     tile_order  uint32 per tile: tiles by descending list length (the order in
                 which the compositing kernels are scheduled)
     rec_feat    float[NCP] per record, 16-byte aligned rows: the surfel's rgb,
                 its C logits, the record's depth, then zeros; NCP = 3 + C + 1
                 rounded up to 8, 16, 24, 32 or 64 (what the compositing
                 kernels stage per list entry, one aligned row per record)
     pair_mc     float[8] per pair, in pair_rec order: its record's
                 mean_int, mean_frac, the conic scaled for a base-2
                 exponential (-A/2 log2 e, -B log2 e, -C/2 log2 e) and
                 alpha, so that a list walk reads them without going
                 through the record id
     pair_blk    uint8 per pair: bit w set iff the record's footprint can
                 reach the w-th pixel block of its tile (the 32-pixel block
                 of one compositing warp: 16x2 in 16x16 tiles, 8x4 in 8x8
                 and 32x8 tiles; blocks row-major in the tile; the same
                 conservative test the compositing kernels use) */
typedef struct {
    uint64_t header, records, rects, pair_rec, tile_range, pix_T, pix_last, views, tile_order, rec_feat, pair_mc,
        pair_blk, total_bytes;
    int64_t total_tiles, total_pixels;
} rogs_state_layout;

/* ---------------------------------------------------------- context */

/* Fill *cfg with the defaults above for C classes and the given capacities. */
rogs_status rogs_default_config(int32_t num_classes, int64_t record_capacity, int64_t pair_capacity,
                                rogs_config* cfg);

/* Create a context on the current CUDA device.  Allocates scratch for the
   configured capacities (device memory, owned by the context). */
rogs_status rogs_create(const rogs_config* cfg, rogs_ctx** out);

/* Release the context and its scratch.  Synchronises the device. */
void rogs_destroy(rogs_ctx* ctx);

/* Last error message of this context ("" if none).  Valid until the next call. */
const char* rogs_last_error(const rogs_ctx* ctx);

/* Pre-size scratch so that later calls never allocate, synchronise or free
   (as CUDA-graph capture requires): the visibility scratch for maps of up to
   n_surfels surfels and up to n_views views; and, when `training` is nonzero,
   also the per-record gradient rows of the backward (record_capacity rows,
   cleared here) and, when `cams` (host, n_views entries) is given, the loss
   scratch for calls over those cameras (or any camera set with no more
   pixels and tiles).  After a matching reserve, rogs_render_fwd, rogs_loss,
   rogs_render_bwd and rogs_train_step only enqueue kernels and asynchronous
   copies on their stream.  Without it, the first call that needs more
   scratch grows it: that call synchronises its stream, frees the old buffer
   and allocates (and is refused with ROGS_ERR_CAPACITY during a capture).
   Synchronises the device.  Errors: ROGS_ERR_INVALID for n_surfels < 0 or
   n_views outside [1, ROGS_MAX_VIEWS] or a bad camera; ROGS_ERR_OOM. */
rogs_status rogs_reserve(rogs_ctx* ctx, int64_t n_surfels, const rogs_camera* cams, int32_t n_views,
                         int32_t training);

/* Output and state geometry of a set of cameras (host-side arithmetic).
   out_elems = (3 + C + 1) * total pixels floats: view v occupies
   [(3+C+1) * pix_base[v], ...) laid out as planes [3+C+1][H][W] = rgb after
   exposure (Eq. 7), sem[C], depth (sum of w * camera z). */
rogs_status rogs_state_layout_of(const rogs_ctx* ctx, const rogs_camera* cams, int32_t n_views,
                                 rogs_state_layout* layout, uint64_t* out_elems);

/* Copy the state header to the host (synchronises `stream`).  Returns
   ROGS_ERR_CAPACITY if the frame overflowed a capacity, else ROGS_OK. */
rogs_status rogs_state_counts(rogs_ctx* ctx, const void* state, rogs_counts* counts, rogs_stream stream);

/* ---------------------------------------------------------- the path */

/* Pose-based initialisation (Sec. 3.2, Eq. 4; supplementary Eqs. S1-S2).
   For each grid point (x_i, y_i) find the nearest pose in xy (binary32
   squared distance, ties to the lowest pose index) and set
     z_i = z_v - (n31 (x_i - x_v) + n32 (y_i - y_v)) / n33      (exact_plane = 1)
     z_i = z_v                                                 (exact_plane = 0)
   with n3 the third column of R_v, and R_i = R_v as a unit quaternion
   (w,x,y,z), w >= 0.
   grid_xy: device [n,2]; poses: HOST [n_poses,12] = (x,y,z, R_v row-major);
   out_z: device [n]; out_quat: device [n,4]; out_nearest: device [n] or NULL.
   ROGS_ERR_INVALID if n_poses < 1 or some pose has |n33| < 1e-6 while
   exact_plane = 1.  Synchronises the host copy of the poses. */
rogs_status rogs_init_from_poses(rogs_ctx* ctx, const float* grid_xy, int64_t n, const float* poses,
                                 int64_t n_poses, int32_t exact_plane, float* out_z, float* out_quat,
                                 int32_t* out_nearest, rogs_stream stream);

/* Forward render of n_views cameras in one pass (Sec. 3.3.1, Eqs. 2, 5, 6, 7
   and the supplementary box cull):
     1. cull + EWA projection of every surfel into every view,
     2. tile binning and hand-written radix sorts: pairs ordered by
        (view, tile, binary32 depth, surfel index),
     3. per-tile front-to-back compositing of rgb, C semantic logits and depth
        with the transmittance stop, then the exposure of Eq. 7.
   cams: HOST [n_views]; exposure_ab: device [n_exposure,2] (a, b);
   out: device float[out_elems] (rogs_state_layout_of); state: device buffer
   of layout.total_bytes, 256-byte aligned, written here and read by
   rogs_render_bwd; the layout is that of rogs_state_layout_of for this
   context and these cameras (its sections follow the context's capacities,
   so a state laid out for another context may be too small: the library
   cannot check this).  ROGS_ERR_INVALID for n_views outside [1, ROGS_MAX_VIEWS],
   a camera with non-positive size or focal length, or an exposure index
   outside [0, n_exposure). */
rogs_status rogs_render_fwd(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                            int32_t n_views, const float* exposure_ab, int32_t n_exposure, float* out,
                            void* state, rogs_stream stream);

/* Masked L1 colour + masked cross-entropy semantic loss (Sec. 3.3.2, Eqs. 8,
   9), weighted by lambda_c and lambda_s (Eq. 12), over all views' pixels:
     L = lambda_c/|M| sum_i m_i sum_rgb |c'_i - cbar_i|
       + lambda_s/|M| sum_i m_i CE(softmax(sem_i), label_i)
   |M| = number of mask pixels (L = 0 and zero gradient if |M| = 0).
   out: the forward output; tgt_rgb: device [3][pixels] planes per view (same
   pixel offsets as out); label: device int32 [pixels] in [0, C) (a label
   outside [0, C) drops that pixel's semantic term); mask: device uint8
   [pixels].  Writes loss: device float[1] and grad_out: device
   float[out_elems] = dL/dout (depth plane zero; sign(0) = 0 for L1). */
rogs_status rogs_loss(rogs_ctx* ctx, const rogs_camera* cams, int32_t n_views, const float* out,
                      const float* tgt_rgb, const int32_t* label, const uint8_t* mask, float lambda_c,
                      float lambda_s, float* loss, float* grad_out, rogs_stream stream);

/* The same loss with the targets as 8-bit camera data, the form images and
   segmentation maps are stored in (a third of the bytes of the FP32 / int32
   form): tgt_rgb: device uint8 [3][pixels] planes per view, the colour target
   cbar = value / 255 (rounded to the nearest float, so the loss equals
   rogs_loss given those FP32 values bit for bit); label: device uint8
   [pixels], a class id (a value >= C, 255 say, drops that pixel's semantic
   term); mask as in rogs_loss. */
rogs_status rogs_loss_u8(rogs_ctx* ctx, const rogs_camera* cams, int32_t n_views, const float* out,
                         const uint8_t* tgt_rgb, const uint8_t* label, const uint8_t* mask, float lambda_c,
                         float lambda_s, float* loss, float* grad_out, rogs_stream stream);

/* Backward of rogs_render_fwd (the adjoint of Eqs. 2, 5, 6, 7): reverse
   traversal of each tile's list from each pixel's last composited entry,
   recovering T by division, then the chain through the EWA projection.
   grad_out: device float[out_elems] = dL/dout.  Gradients are ADDED into
   `grads` (device; zero them first for a plain gradient).  state must be the
   one filled by the forward with the same surfels, cameras and exposure. */
rogs_status rogs_render_bwd(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                            int32_t n_views, const float* exposure_ab, int32_t n_exposure, const void* state,
                            const float* grad_out, const rogs_grads* grads, rogs_stream stream);

/* One training step with the loss fused into the backward: rogs_render_fwd,
   then the masked L1 + CE loss of rogs_loss and the backward of
   rogs_render_bwd, except that dL/dout is computed inside the backward kernel
   from `out` and the targets instead of being written to and read back from a
   gradient image (same values as rogs_loss followed by rogs_render_bwd, up to
   FP32 summation order).  With lambda_smooth != 0 the step also takes the
   elevation smoothness loss of rogs_smooth_loss (needs surfels->grid_index),
   so loss[0] = lambda_c L_c + lambda_s L_s + lambda_smooth L_smooth (Eq. 12
   without the LiDAR term); that term runs on a stream owned by the context,
   forked from and joined back into `stream` with events, beside the backward
   compositing.  Arguments as in those calls; gradients are ADDED
   into `grads`; loss: device float[1]. */
rogs_status rogs_train_step(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                            const float* exposure_ab, int32_t n_exposure, float* out, void* state,
                            const float* tgt_rgb, const int32_t* label, const uint8_t* mask, float lambda_c,
                            float lambda_s, float lambda_smooth, float* loss, const rogs_grads* grads,
                            rogs_stream stream);

/* rogs_train_step with 8-bit targets (tgt_rgb, label as in rogs_loss_u8):
   the same results as rogs_train_step given cbar = value / 255 as FP32 and
   the labels as int32, with 5 bytes of supervision per pixel instead of 17. */
rogs_status rogs_train_step_u8(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams, int32_t n_views,
                               const float* exposure_ab, int32_t n_exposure, float* out, void* state,
                               const uint8_t* tgt_rgb, const uint8_t* label, const uint8_t* mask, float lambda_c,
                               float lambda_s, float lambda_smooth, float* loss, const rogs_grads* grads,
                               rogs_stream stream);

/* Elevation smoothness loss (Sec. 3.3.2, smoothness equation, K = 4;
   neighbours as in the supplementary "Smooth Loss K Nearest Neighbor
   Acceleration"):
     L_smooth = (1/4) sum_i sum_{j in N(i)} (z_i - z_j)^2
   where N(i) are the surfels at the grid vertices above, below, left and
   right of surfel i's vertex in surfels->grid_index, and a vertex off the grid
   or holding -1 stands for i itself.  Writes lambda_smooth * L_smooth to
   loss[0] (device float) and ADDS lambda_smooth * dL/dz_i to grad_xyz[3i+2]
   (device [n,3]; NULL skips the gradient).  z_i = surfels->xyz[3i+2]; only
   xyz and the grid fields are read.  Errors: ROGS_ERR_INVALID when the grid
   index or loss pointer is NULL or grid_w, grid_h are not positive.  The sum
   is taken in a fixed order (the result does not depend on timing). */
rogs_status rogs_smooth_loss(rogs_ctx* ctx, const rogs_surfels* surfels, float lambda_smooth, float* loss,
                             float* grad_xyz, rogs_stream stream);

/* Chunked BEV export (supplementary "Orthogonal Rendering Acceleration"):
   a straight-down orthographic render of the map over the ground rectangle
   x in [x0, x0 + width res], y in [y1 - height res, y1] -- image x along +x,
   image y along -y from the top edge y1, res metres per pixel, camera at
   height cam_z -- rendered as a grid of chunk x chunk-pixel orthographic
   cameras (the paper: 2000 x 2000 at 0.05 m/px; edge chunks are smaller),
   `batch` chunks per rogs_render_fwd launch, stitched into `image` (device
   float [3 + C + 1][height][width] planes: rgb after exposure `exposure_idx`,
   the C logits, depth).  Chunks are batched and stitched on `stream`; the
   call synchronises once per batch to check the capacities.  Allocates the
   batch's output and state in the context on first use (not for stream
   capture).  Errors: ROGS_ERR_INVALID for bad sizes, batch outside [1, 16]
   or a bad exposure index; ROGS_ERR_CAPACITY when a batch overflows the
   record or pair capacity (use a smaller batch or larger capacities). */
rogs_status rogs_bev_export(rogs_ctx* ctx, const rogs_surfels* surfels, const float* exposure_ab, int32_t n_exposure,
                            int32_t exposure_idx, double x0, double y1, float res, float cam_z, int32_t width,
                            int32_t height, int32_t chunk, int32_t batch, float* image, rogs_stream stream);

/* LiDAR elevation targets for L_z (Sec. 3.3.2, LiDAR supervision): for each
   surfel, zbar_i = z of the point of `points` (device float [n_points, 3],
   x, y, z) nearest to the surfel centre in the xy-plane, among the points
   within `radius` of it; NaN when there is none; equal distances go to the
   lower point index.  Writes z_target (device float [n]).  Meant to run once
   per point cloud: it may allocate scratch (a spatial hash of the points,
   held by the context), so it is not for stream capture.  Errors:
   ROGS_ERR_INVALID for NULL pointers, radius <= 0 or n_points >= 2^31;
   ROGS_ERR_OOM when the scratch cannot be allocated. */
rogs_status rogs_elev_targets(rogs_ctx* ctx, const rogs_surfels* surfels, const float* points, int64_t n_points,
                              float radius, float* z_target, rogs_stream stream);

/* LiDAR elevation loss (Sec. 3.3.2, L_z = sum_i (z_i - zbar_i)^2 over the
   surfels with a finite target): ADDS lambda_z L_z to loss[0] (device float,
   so it composes with rogs_train_step's loss) and lambda_z dL/dz_i =
   2 lambda_z (z_i - zbar_i) to grad_xyz[3i+2] (NULL skips the gradient).
   The sum is taken in a fixed order. */
rogs_status rogs_elev_loss(rogs_ctx* ctx, const rogs_surfels* surfels, const float* z_target, float lambda_z,
                           float* loss, float* grad_xyz, rogs_stream stream);

/* One parameter tensor of the optimiser step: its k-th element (k < n) is
   param[k * stride] with gradient grad[k * stride] (stride 1 for a whole
   tensor; param = xyz + 2, grad = grad_xyz + 2, stride 3 for the z column
   only); m and v are its Adam moments, dense device float[n], zero before the
   first step.
   Learning rate at step t (Sec. 4.2): lr when decay_steps == 0; otherwise the
   rate falls log-linearly from lr to lr_end over decay_steps steps and stays
   at lr_end, lr_t = lr (lr_end / lr)^min((t - 1) / decay_steps, 1) (the paper
   gives only the two ends of z's rate, 1.6e-4 and 1.6e-6 times the scene
   size; the shape between them is this library's reading).
   zero_lead (0 <= zero_lead < stride): when the step clears gradients, it
   also clears the zero_lead gradient floats just before each element -- for
   the z column of xyz, 2 clears dL/dx and dL/dy, which Sec. 4.2 does not
   learn. */
typedef struct {
    float* param;
    float* grad;
    float* m;
    float* v;
    int64_t n;
    int32_t stride;
    float lr;
    float lr_end;
    int32_t decay_steps;
    int32_t zero_lead;
} rogs_adam_group;

#define ROGS_MAX_ADAM_GROUPS 16

/* One Adam step (Sec. 4.2: Adam with per-tensor learning rates) over up to
   ROGS_MAX_ADAM_GROUPS groups in a single launch, at step number `step` >= 1
   (bias correction and the learning-rate schedule): per element
     m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
     p -= lr_t (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
   With zero_grad != 0 every gradient element (and its zero_lead leading
   floats) is set to 0 after it is read, ready for the next backward (which
   adds).  Groups must not overlap.
   Errors: ROGS_ERR_INVALID for n_groups outside [1, ROGS_MAX_ADAM_GROUPS],
   step < 1, stride < 1, zero_lead outside [0, stride), decay_steps < 0,
   lr or lr_end <= 0 with decay_steps > 0, n < 0 or a NULL pointer in a group
   with n > 0. */
rogs_status rogs_adam_step(rogs_ctx* ctx, const rogs_adam_group* groups, int32_t n_groups, int32_t step, float beta1,
                           float beta2, float eps, int32_t zero_grad, rogs_stream stream);

/* Stable LSD radix sort of (key, value) pairs of uint32 on key bits
   [0, key_bits) -- the sort used inside rogs_render_fwd, exposed for
   testing and reuse.  All pointers device; inputs are not modified; n <=
   the context's pair capacity. */
rogs_status rogs_sort_pairs(rogs_ctx* ctx, const uint32_t* keys_in, const uint32_t* vals_in, int64_t n,
                            int32_t key_bits, uint32_t* keys_out, uint32_t* vals_out, rogs_stream stream);

/* ---------------------------------------------------------- serving */

/* A request loop that keeps one surfel map resident and renders incoming
   BEV-orthographic and perspective requests (the paper's outputs: RGB,
   semantic and elevation maps, Sec. 1 Fig. 1; BEV chunks per the
   supplementary "Orthogonal Rendering Acceleration").  A worker thread takes
   pending requests in arrival order into a batch (up to max_batch_views, as
   long as the batch fits the free device memory), renders the whole batch in
   one forward pass on one of max_inflight streams, packs each request's
   channels and copies them to pinned host memory.  New batches are formed as
   soon as a stream and memory free up, while earlier ones are still running
   (continuous batching).  Each request's result does not depend on what it
   was batched with. */
typedef struct rogs_server rogs_server;

enum { ROGS_CH_RGB = 1, ROGS_CH_SEM = 2, ROGS_CH_ELEV = 4 };

typedef struct {
    int32_t max_batch_views;   /* views per batched forward (1 = plain FIFO path) */
    int32_t max_inflight;      /* batches in flight at once (one stream and context each) */
    int32_t max_queue;         /* pending requests accepted before ROGS_ERR_BUSY */
    int32_t reserved;
    uint64_t memory_budget;    /* device bytes for in-flight batches (outputs + states + packed results) */
    int64_t record_capacity;   /* per batch */
    int64_t pair_capacity;     /* per batch */
    double timeout_s;          /* a batch not finished after this long fails with ROGS_ERR_TIMEOUT */
} rogs_serve_config;

typedef struct {
    uint64_t submitted, completed, failed, batches, views_rendered, pixels_rendered;
    uint32_t pending, inflight;
} rogs_serve_stats;

/* Bytes of a request's packed result: for the requested channels, in this
   order, RGB float32 [3][H][W] (after exposure), ELEV float32 [H][W], SEM
   uint8 [H][W] (argmax of the composited logits).  ELEV is, for an
   orthographic camera looking down, the world height of the composited
   surface: camera z - D / (1 - T) (D = composited depth); for a perspective
   camera the normalised depth D / (1 - T); NaN where 1 - T < 0.5. */
rogs_status rogs_serve_result_bytes(const rogs_camera* cam, int32_t channels, int32_t num_classes, uint64_t* bytes);

/* Start a server on the current device.  `cfg_render` gives the rendering
   constants (tile, classes, thresholds; its capacities are replaced by those
   of `cfg`).  The map (device pointers) and exposure [n_exposure,2] must stay
   valid and unchanged until rogs_serve_close.  Allocates the device pool and
   the contexts. */
rogs_status rogs_serve_open(const rogs_config* cfg_render, const rogs_surfels* map, const float* exposure_ab,
                            int32_t n_exposure, const rogs_serve_config* cfg, rogs_server** out);

/* Queue one request (thread-safe).  ROGS_ERR_INVALID for a bad camera or
   channel set, ROGS_ERR_OOM if the request alone can never fit the memory
   budget, ROGS_ERR_BUSY if max_queue requests are already pending. */
rogs_status rogs_serve_submit(rogs_server* srv, const rogs_camera* cam, int32_t channels, uint64_t* ticket);

/* Non-blocking: if the request is finished, copy its packed result into
   host_out (rogs_serve_result_bytes bytes), set *done = 1, forget the ticket
   and return ROGS_OK; if not, set *done = 0 and return ROGS_ERR_NOT_READY.  A
   failed request returns its error (ROGS_ERR_CAPACITY, ROGS_ERR_TIMEOUT,
   ROGS_ERR_CUDA) once; an unknown ticket gives ROGS_ERR_INVALID. */
rogs_status rogs_serve_poll(rogs_server* srv, uint64_t ticket, void* host_out, int32_t* done);

rogs_status rogs_serve_get_stats(rogs_server* srv, rogs_serve_stats* out);

/* Change the server's timeout_s (thread-safe; > 0).  Batches already in
   flight are checked against the new value from the next check on. */
rogs_status rogs_serve_set_timeout(rogs_server* srv, double timeout_s);

/* Stop the worker, wait (bounded by timeout_s) for batches in flight, free
   everything.  Unpolled results are dropped. */
void rogs_serve_close(rogs_server* srv);

/* ------------------------------------------------------ graph capture */

typedef struct rogs_graph rogs_graph;

/* Capture one training step -- rogs_train_step with exactly these arguments --
   into a CUDA graph (the batched, graph-captured form of the hot path: every
   view of the call is in each stage's single launch, and replaying the graph
   removes the per-kernel launch overhead).  All pointers are fixed in the
   graph; replays read the current contents of the inputs and ADD into
   `grads`.  Scratch is sized before the capture starts (never during it).
   `stream` must not be the legacy default stream (NULL).  Argument errors are
   those of rogs_train_step.  On success *graph receives an executable graph
   owned by the caller (free it with rogs_graph_destroy); ctx must outlive it. */
rogs_status rogs_train_graph_create(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                                    int32_t n_views, const float* exposure_ab, int32_t n_exposure, float* out,
                                    void* state, const float* tgt_rgb, const int32_t* label, const uint8_t* mask,
                                    float lambda_c, float lambda_s, float lambda_smooth, float* loss, const rogs_grads* grads,
                                    rogs_stream stream, rogs_graph** graph);

/* Same, capturing rogs_train_step_u8 (8-bit targets). */
rogs_status rogs_train_graph_create_u8(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                                       int32_t n_views, const float* exposure_ab, int32_t n_exposure, float* out,
                                       void* state, const uint8_t* tgt_rgb, const uint8_t* label, const uint8_t* mask,
                                       float lambda_c, float lambda_s, float lambda_smooth, float* loss,
                                       const rogs_grads* grads, rogs_stream stream, rogs_graph** graph);

/* Same, forward only (rogs_render_fwd). */
rogs_status rogs_render_graph_create(rogs_ctx* ctx, const rogs_surfels* surfels, const rogs_camera* cams,
                                     int32_t n_views, const float* exposure_ab, int32_t n_exposure, float* out,
                                     void* state, rogs_stream stream, rogs_graph** graph);

/* Replay a captured graph on `stream` (asynchronous). */
rogs_status rogs_graph_launch(rogs_graph* graph, rogs_stream stream);

/* Free a captured graph. */
void rogs_graph_destroy(rogs_graph* graph);

/* Largest n accepted by rogs_sort_pairs_noalloc. */
#define ROGS_NOALLOC_MAX_PAIRS 1048576

/* rogs_sort_pairs without a context and without any device allocation (the
   paper has no counterpart; this is a library service).  It exists for
   callers that cannot allocate device memory where they sort -- code that
   enqueues into a stream of a host framework which has reserved all device
   memory itself, loops that forbid allocator calls, plugin hooks that run
   while another component owns the allocator -- and so cannot create a
   rogs_ctx.  Same result as rogs_sort_pairs: stable LSD radix sort of
   (key, value) pairs on key bits [0, key_bits); all pointers device; inputs
   are not modified; keys_out/vals_out must not overlap the inputs.
   Scratch: a fixed array of 2 * ROGS_NOALLOC_MAX_PAIRS + 131328 uint32
   (about 8.9 MB) compiled into the library's device image; every GPU that
   loads the library holds it until the process exits.  Every call looks the
   array's device address up in the current context (cudaGetSymbolAddress);
   the first call on a device also loads the library's device code there, so
   make that first call before any stream capture on that device.
   All calls share the one array, so calls whose executions overlap on the
   GPU (different streams, or concurrent host threads) race and corrupt each
   other's results; serialise them.  Nothing in the array needs clearing
   between calls.  Errors: ROGS_ERR_CAPACITY if n > ROGS_NOALLOC_MAX_PAIRS,
   ROGS_ERR_INVALID for n < 0, key_bits outside [0, 32] or a NULL pointer
   with n > 0, ROGS_ERR_CUDA if the address lookup or a launch fails during
   this call (a CUDA error already pending when the call starts is neither
   reported nor cleared here).  The current device must be the device of
   `stream`. */
rogs_status rogs_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int32_t key_bits,
                                    uint32_t* keys_out, uint32_t* vals_out, rogs_stream stream);

/* ------------------------------------------------------- measurement */

/* Stages timed by the profiler (CUDA events on the call's stream):
   0 cull + projection (records), 1 depth sort, 2 pair scan + emission,
   3 tile sort + tile ranges, 4 forward compositing, 5 loss (the separate
   rogs_loss; rogs_train_step runs its loss pieces on a side stream, untimed),
   6 backward compositing, 7 projection backward. */
#define ROGS_N_STAGES 8
typedef struct {
    double ms[ROGS_N_STAGES];      /* summed device time per stage */
    uint64_t calls[ROGS_N_STAGES]; /* number of timed executions */
} rogs_profile;

/* Enable (1) or disable (0) per-stage event timing on this context and reset
   the totals.  Timing is skipped while a stream is being captured. */
rogs_status rogs_profile_enable(rogs_ctx* ctx, int32_t enable);

/* Wait for the recorded events and return the totals since the last enable. */
rogs_status rogs_profile_read(rogs_ctx* ctx, rogs_profile* out);

/* Measure the current device's FP32 fused multiply-add rate (a measurement
   utility, not part of the method): a kernel of independent FMA chains on
   every SM, timed with CUDA events on `stream`, best of `reps` launches after
   one warm-up; *tflops = 2 x FMAs / time in TFLOP/s, *sm_count (optional) =
   the device's SM count.  Allocates and frees a small buffer and
   synchronises the stream.  Errors: ROGS_ERR_INVALID (reps < 1, NULL
   tflops), ROGS_ERR_OOM, ROGS_ERR_CUDA. */
rogs_status rogs_measure_fp32_peak(int32_t reps, double* tflops, int32_t* sm_count, rogs_stream stream);

/* Number of kernels this library has launched in this process. */
uint64_t rogs_launch_count(void);

/* Test hook for failure handling (the paper has no counterpart): while
   fail_all is nonzero, every device allocation the library makes for its own
   scratch (rogs_create, rogs_reserve, growth inside a call, the serving
   pool) reports out-of-memory, so callers can check that ROGS_ERR_OOM comes
   back cleanly and that nothing leaks.  Process-wide; not for production. */
void rogs_debug_fail_alloc(int32_t fail_all);

/* Bounds-checked builds (the paper has no counterpart): a library compiled
   with -DROGS_CHECKED (paper_2405_14342_gb300.build.build(checked=True),
   librogs_checked.so) tests every index its kernels take from device data
   -- list entries, record ids, surfel ids, scatter positions -- before use,
   skips the access if it is out of range and records a failure code (the
   first one wins; 1xx forward compositing, 2xx backward, 3xx radix sort, 4xx
   binning).  Returns 1 for such a build and stores (then clears) the code, 0
   (code 0) for the normal build, whose kernels carry no tests.  Synchronises
   the device. */
int32_t rogs_bounds_checked(uint32_t* code);

#ifdef __cplusplus
}
#endif

#endif /* ROGS_H */
