/*
 * rgs.h -- C ABI of the GB300 hierarchical 3D Gaussian splatting library
 * (RetinaGS, arXiv 2406.11836).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Tensors are caller-owned, contiguous, device memory unless a name ends in _host.
 *    float = IEEE fp32, int32/int64 as named.  The library never frees caller memory.
 *  - Splat parameters are structure-of-arrays (Sec. 3.1: centre mu, covariance from scale
 *    and rotation, opacity, SH colour):  means [N,3], log_scales [N,3], quats [N,4] stored
 *    (w,x,y,z) and normalised inside, opacity_logits [N], sh [N,(deg+1)^2,3]
 *    (coefficient-major, RGB innermost).
 *  - Cameras: world->camera 4x4 view matrix, row-major, OpenCV axes (x right, y down,
 *    z forward), pinhole intrinsics; pixel (px,py) has its centre at (px+0.5, py+0.5).
 *  - Images are planar: [3,H,W]; partial maps [K,3,H,W] and [K,H,W] are indexed by the
 *    KD leaf (subset) id k, not by the view order.
 *  - Calls taking a `stream` (a cudaStream_t passed as void*) only enqueue work on it and
 *    return without waiting, except where a call says it synchronises.
 *  - Every call returns an int status.  Nothing throws across the ABI.  On failure
 *    rgs_last_error() (thread-local) holds a one-line reason.
 *
 * Readings of the paper that this library implements (the oracle in the test suite
 * implements the same ones):
 *  - depth order along a ray = camera-space depth z_i of the splat centre, ties by
 *    ascending splat index;
 *  - x_i (Sec. 3.2, Eq. 6) = the point of the pixel ray at camera depth z_i;
 *  - a (pixel, splat) pair contributes iff z_i > near_z, d^2 <= trunc_mult^2 (Mahalanobis
 *    distance in the projected 2D Gaussian), |x_i - mu_i| <= D_i and
 *    sigma = min(alpha_max, alpha exp(-d^2/2)) >= alpha_min;
 *  - D_i = trunc_mult * max_j exp(log_scale_j) (Sec. 3.3, "three times the major axis");
 *  - leaf boxes are half-open (left child x[a] < s, right child x[a] >= s);
 *  - the merge order of Eq. 5 is one near-child-first KD traversal per view.
 */
#ifndef RGS_H
#define RGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define RGS_OK 0
#define RGS_EINVAL (-1)     /* invalid argument (see rgs_last_error) */
#define RGS_ENOMEM (-2)     /* a library-internal allocation failed */
#define RGS_ECUDA (-3)      /* a CUDA runtime call failed */
#define RGS_EOVERFLOW (-4)  /* caller workspace too small; rgs_last_required_workspace() */
#define RGS_ETIMEOUT (-5)   /* a bounded wait gave up (serving) */
#define RGS_EAGAIN (-6)     /* not ready yet / no room right now (serving) */

/* ------------------------------------------------------------------ types */
typedef struct {
    const float* means;           /* [N,3] */
    const float* log_scales;      /* [N,3] */
    const float* quats;           /* [N,4] (w,x,y,z) */
    const float* opacity_logits;  /* [N]   */
    const float* sh;              /* [N,(sh_degree+1)^2,3] */
    int64_t n;                    /* N >= 1 */
    int sh_degree;                /* 0..3 */
} rgs_gaussians;

typedef struct {                  /* gradients, same shapes as rgs_gaussians; accumulated (+=) */
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logits;
    float* sh;
} rgs_gaussian_grads;

typedef struct {
    float viewmat[16];            /* world->camera, row-major, OpenCV axes */
    float fx, fy, cx, cy;         /* pixels */
    int width, height;            /* 1..16384 */
    float near_z;                 /* splats with camera depth <= near_z are culled */
} rgs_camera;

typedef struct {
    int tile;                     /* tile edge in pixels; must be 16 */
    float trunc_mult;             /* 3: d^2 <= trunc_mult^2 and D_i = trunc_mult * max scale */
    float eps_T;                  /* 1e-6: a subset stops once its transmittance drops below */
    float alpha_min;              /* 1/255: smaller sigma does not contribute */
    float alpha_max;              /* 0.99: sigma clamp */
    float dilation;               /* 0.3: added to the diagonal of the 2D covariance */
    float bg[3];                  /* background colour behind every ray (merge only) */
    int cull_occluded;            /* 0: every subset is blended on every ray it meets (its
                                     partials are the whole Eq. 3-4).  1: a subset is not
                                     blended on a ray whose transmittance in front of it (the
                                     merge's prod_{m<r} T_{o_m}, Eq. 5) is below eps_T; its
                                     partials there are C = 0, T = 1.  The merged image moves
                                     by less than eps_T times the largest colour. */
    int group_binning;            /* 1 (default): a forward without partial maps bins and
                                     blends the subsets in two groups of view ranks, the first
                                     max(1, K/8) ranks and then the others, the second group
                                     only in tiles where some pixel's transmittance in front is
                                     still at least eps_T; this when K >= 4 and the render's
                                     tile instances average at least 12 per visible splat and
                                     number at least 2^24 (otherwise one group).  The image,
                                     T_final, tile_depth and the lists a backward replays are
                                     those of one group; fewer instances are emitted and
                                     sorted.  Synchronises once more with the stream.  2: as 1
                                     whatever the instance counts (when K >= 4).  0: one
                                     group. */
} rgs_render_opts;

typedef struct rgs_kd rgs_kd;          /* KD partition: splits, leaf boxes, subset lists */
typedef struct rgs_server rgs_server;  /* render server with a device-resident scene */

/* ------------------------------------------------------------------ misc */
const char* rgs_last_error(void);           /* thread-local, never NULL */
size_t rgs_last_required_workspace(void);   /* thread-local; set when a call returns RGS_EOVERFLOW */
int rgs_version(void);                      /* major*10000 + minor*100 + patch */
void rgs_default_opts(rgs_render_opts* opts);

/* ------------------------------------------------------------------ KD partition (Sec. 3.3)
 * rgs_kd_partition: builds a KD tree of depth L (K = 2^L leaves) on the splat centres:
 * level d splits along axis d mod 3 at the median (for an even count the fp32 midpoint
 * of the two middle coordinates, raised to the upper one if it rounds onto the lower;
 * for an odd count the median coordinate itself), so every node's two children differ in
 * size by at most one when coordinates are distinct.  Then forms the overlapping subsets
 * N_k = {i : n.mu_i + d <= D_i for every plane of S_k} (Sec. 3.3) as CSR lists, leaf-major,
 * ascending splat index.  Only means and log_scales are read.  L in [0,8].
 * Synchronises with `stream` before returning (the handle holds host copies of the
 * splits).  Allocates its own device memory; *out is owned by the caller and released
 * with rgs_kd_destroy.  Errors: EINVAL (NULL pointers, N < 1, L out of range,
 * trunc_mult <= 0), ENOMEM, ECUDA. */
int rgs_kd_partition(const rgs_gaussians* g, int depth_L, float trunc_mult, rgs_kd** out, void* stream);

/* A partition with caller-given planes: axis_host [K-1] in {0,1,2} and split_host [K-1]
 * (heap order, as rgs_kd_splits returns them), with the overlapping subsets N_k formed by
 * the same D_i rule as rgs_kd_partition.  Any axis-aligned convex partition of this form
 * is valid for the method (Sec. 3.2 only needs convex subspaces); it restores a saved
 * partition exactly and serves comparison partitions (e.g. a fixed grid).  Errors:
 * EINVAL (axis out of range, non-finite split, L out of [0,8]), ENOMEM, ECUDA. */
int rgs_kd_from_splits(const rgs_gaussians* g, int depth_L, const int32_t* axis_host, const float* split_host,
                       float trunc_mult, rgs_kd** out, void* stream);

/* Depth L, leaf count K and total subset-list length M of a partition. */
int rgs_kd_info(const rgs_kd* kd, int* depth_L, int* K, int64_t* total_members);

/* Splits in heap order (node j has children 2j+1 left, 2j+2 right; leaf k is node K-1+k):
 * axis_host [K-1] int32 in {0,1,2}, split_host [K-1] float.  Either may be NULL. */
int rgs_kd_splits(const rgs_kd* kd, int32_t* axis_host, float* split_host);

/* CSR subset lists: offsets_host [K+1] int64 (host), idx_dev [M] int32 (device, may be
 * NULL to query offsets only).  Synchronous copy. */
int rgs_kd_subsets(const rgs_kd* kd, int64_t* offsets_host, int32_t* idx_dev);

int rgs_kd_destroy(rgs_kd* kd);

/* Merge order o_l of Eq. 5 for every ray of a view: the KD leaves in a near-child-first
 * traversal, where at each node the child containing the camera centre o goes first (o on
 * the plane: the left child).  A ray from o crosses each plane at most once, from o's
 * side, so this order lists the leaves every ray crosses in the order it crosses them.
 * order_host [K] int32 (host).  Pure host computation. */
int rgs_view_order(const rgs_kd* kd, const rgs_camera* cam, int32_t* order_host);

/* ------------------------------------------------------------------ render
 * Workspace bytes for a render of this scene/view whose tile-instance count is at most
 * `instance_capacity` ((subset, tile, splat) triples; unknown until the splats are
 * projected, so rgs_render_fwd/bwd report the exact need via RGS_EOVERFLOW and
 * rgs_last_required_workspace()).  Pure host arithmetic. */
int rgs_render_workspace_size(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                              const rgs_render_opts* opts, int64_t instance_capacity, size_t* bytes);

/* Forward render, Sec. 3.2: projects every splat (EWA, SH colour), bins it into the
 * 16x16 tiles it can touch once per subset N_k that contains it, sorts the instances by
 * (tile, subset position in the view order, depth), and alpha-blends each subset front
 * to back into its partial colour C_k (Eq. 3) and partial transmittance T_k (Eq. 4), with
 * the indicator of Eq. 6 deciding per pixel which subset a straddling splat belongs to.
 * Writes partial_C [K,3,H,W] and partial_T [K,H,W] (a subset a ray never meets gets
 * C = 0, T = 1).  If `image` [3,H,W] is non-NULL the partials are also merged in view
 * order (Eq. 5) with the background behind, and T_final [H,W] (nullable) receives the
 * product of all T_k.  partial_C and partial_T may both be NULL when image is non-NULL:
 * a forward-only render that keeps the partials on chip (no rgs_render_bwd from it); it
 * always culls as opts->cull_occluded = 1 does: a pixel stops at the first subset whose
 * transmittance in front (the merge's prod_{m<r} T_{o_m}) is below eps_T, which changes
 * the image by less than eps_T times the largest colour (T_final is then that
 * transmittance rather than the full product).  With partial maps and cull_occluded = 1
 * the culled (pixel, subset) partials are C = 0, T = 1.  tile_depth (nullable)
 * [ceil(H/16) * ceil(W/16), K] float, indexed by tile then by the subset's position in
 * rgs_view_order, receives per (tile, subset) the camera depth of the last splat blended
 * before every pixel of the tile had dropped below eps_T in that subset (+inf if that did
 * not happen, -inf if culling left no pixel of the tile to blend); rgs_render_bwd uses it
 * to skip splats that cannot matter.  Synchronises once with `stream` to size the
 * instance buffers.
 * Errors: EINVAL (shapes, sh_degree, tile != 16, L > 6 for rendering, non-finite camera,
 * misaligned pointers), EOVERFLOW (workspace too small; required size via
 * rgs_last_required_workspace()), ECUDA. */
int rgs_render_fwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                   float* partial_C, float* partial_T, float* image, float* T_final, float* tile_depth,
                   void* workspace, size_t ws_bytes, void* stream);

/* rgs_render_fwd for callers that cannot allocate device memory (the paper has no
 * counterpart: this is a deployment variant), such as a real-time thread that must not
 * block in the allocator or a host program that hands all device memory out from its own
 * pool.  Same arguments and results as rgs_render_fwd minus the workspace, which comes
 * from a fixed 64 MiB device array inside the library; nothing is allocated.  Like
 * rgs_render_fwd it synchronises `stream` once, after the projection, to size the
 * instance buffers.
 * The first call on a device looks the array up (make it before any stream capture);
 * every GPU that loads the library holds the array until exit.  All calls share it and
 * it keeps the last call's contents (the render clears what must start at zero): calls
 * that overlap on the GPU race and must be serialised by the caller.  A render whose
 * workspace exceeds the array (roughly 150 bytes per splat plus 16 per tile instance)
 * returns RGS_EOVERFLOW; rgs_last_error() gives the render's reason (before binning: the
 * bytes needed for the splats; after binning: the instance count) and
 * rgs_last_required_workspace() the bytes needed (exact after binning; before binning an
 * estimate that assumes 2^20 instances).  Tracing records no events for this call. */
int rgs_render_fwd_noalloc(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                           const rgs_render_opts* opts, float* partial_C, float* partial_T, float* image,
                           float* T_final, float* tile_depth, void* stream);

/* Forward render under the other reading of the intersection point in Sec. 3.2 (a
 * comparison mode, forward only): x_i is the foot of the perpendicular from the centre u_i
 * onto the pixel ray, o + (d^T (u_i - o)) d for the unit ray direction d.  The ball test
 * |x_i - u_i| <= D_i and the indicator of Eq. 6 are taken at the foot, and each ray's
 * contributors are blended in the order of the foot's ray parameter, which differs from
 * pixel to pixel (ties in list order).  The foot lies on the ray, so Eq. 5 still merges
 * the partials exactly.  The instances of each (tile, subset) are sorted by a lower bound
 * of that parameter over the tile, and each pixel holds up to 64 accepted contributors in
 * a buffer ordered by the parameter, blending one once the next instance's bound shows
 * that nothing later can precede it.  The order is exact unless that buffer overflows;
 * *overflow_host (nullable; reading it synchronises with `stream`) receives the number of
 * contributors blended early because it was full.  Arguments, outputs, eps_T stopping and
 * errors as rgs_render_fwd, without tile_depth; the workspace needs 8 more bytes per
 * instance and 16 per splat (EOVERFLOW reports the size).  rgs_render_bwd does not accept
 * its partials (they are not the depth-plane reading's); its backward is
 * rgs_render_bwd_foot. */
int rgs_render_fwd_foot(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                        const rgs_render_opts* opts, float* partial_C, float* partial_T, float* image,
                        float* T_final, void* workspace, size_t ws_bytes, uint64_t* overflow_host, void* stream);

/* Backward of rgs_render_fwd_foot (the comparison reading of Sec. 3.2, flat form of Eq. 2):
 * the reading changes only discrete decisions (which pairs pass the ball test and Eq. 6 at
 * the foot, and each ray's order), whose gradients are zero, so each pair's adjoint is the
 * depth-plane one, dL/dsigma_i = T_i <g, c_i> - <g, C - A_i> / (1 - sigma_i), taken in the
 * foot reading's per-pixel order.  It re-derives the forward's lists and replays its
 * per-pixel order buffer (same pairs, same order, same freeze points and eps_T stopping)
 * from the forward's image ([3,H,W], as written by rgs_render_fwd_foot without partial
 * maps) and dL_dimage [3,H,W]; each blended pair adds its 2D gradients with atomics, then
 * the projection backward accumulates into `grads` (as rgs_render_bwd).  *overflow_host
 * (nullable) as in rgs_render_fwd_foot.  The workspace needs what rgs_render_fwd_foot
 * needs (EOVERFLOW reports the size).  Synchronises once with `stream` (twice when
 * overflow_host is given).  Errors as rgs_render_fwd. */
int rgs_render_bwd_foot(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                        const rgs_render_opts* opts, const float* image, const float* dL_dimage,
                        const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, uint64_t* overflow_host,
                        void* stream);

/* Training on several views of one scene per step (Sec. 4 trains with a batch size per
 * step), through one launch sequence instead of one per view.
 * rgs_render_batch_fwd renders B views (1 <= B <= 16; cams[B] host array, images a host
 * array of B device pointers, images[b] [3,H_b,W_b]; views may differ in size) with the
 * arithmetic of the image-only rgs_render_fwd (merge of the partials per pixel, culling
 * behind a saturated front): one projection of every (view, splat) pair, one depth sort,
 * emission with keys over the batch's tiles, one instance sort and one persistent blend
 * over all views' tiles, every count kept on the device.  A view's image equals its
 * image-only rgs_render_fwd image bit for bit.  The lists stay in `workspace` for
 * rgs_render_batch_bwd.  Synchronises once with `stream` (to read the instance count).
 * Errors: EINVAL (arguments as rgs_render_fwd, B out of range, tile keys of the batch beyond
 * 32 bits), EOVERFLOW (workspace too small: rgs_last_required_workspace() gives the bytes,
 * exact when the instances did not fit, an estimate before binning), ECUDA.
 * rgs_render_batch_bwd: the flat backward (as rgs_render_bwd_flat) of every view of that
 * forward in one persistent launch, then each view's 2D gradients pulled back through its
 * projection; accumulates into `grads` (same shapes as the parameters; the caller zeroes
 * them).  dL_dimages: host array of B device pointers [3,H_b,W_b].  When `workspace` (same
 * pointer and size) no longer holds the lists of the forward with these arguments, the
 * forward is run again first (re-deriving the lists; the images are rewritten with the
 * same values).  Parameters are recognised by their pointers: they must not change between
 * the forward and its backward.  Synchronises with `stream`.  Errors as the forward. */
int rgs_render_batch_fwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cams, int B,
                         const rgs_render_opts* opts, float* const* images, void* workspace, size_t ws_bytes,
                         void* stream);
int rgs_render_batch_bwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cams, int B,
                         const rgs_render_opts* opts, float* const* images, const float* const* dL_dimages,
                         const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, void* stream);

/* Eq. 5 over caller-owned partial maps: image = sum_r C_{o_r} prod_{m<r} T_{o_m} +
 * bg * prod_m T_m.  order_dev [K] int32 (device) lists the subsets front to back.
 * partial_C [K,3,H,W], partial_T [K,H,W], image [3,H,W], T_out [H,W] (nullable). */
int rgs_merge_partials(const float* partial_C, const float* partial_T, const int32_t* order_dev, int K, int H,
                       int W, const float bg[3], float* image, float* T_out, void* stream);

/* Adjoint of rgs_merge_partials: with P_r = prod_{m<r} T_{o_m} and S_r the colour seen
 * behind subset o_r, dL/dC_{o_r} = g P_r and dL/dT_{o_r} = P_r <g, S_r> (+ gT prod_{m!=r}
 * T_{o_m} when dL_dT_out is non-NULL).  Outputs [K,3,H,W] and [K,H,W] are overwritten. */
int rgs_merge_partials_bwd(const float* partial_C, const float* partial_T, const int32_t* order_dev, int K, int H,
                           int W, const float bg[3], const float* dL_dimage, const float* dL_dT_out,
                           float* dL_dpartial_C, float* dL_dpartial_T, void* stream);

/* Stable LSD radix sort of (uint32 key, uint32 value) pairs by the low end_bit bits of the
 * keys (1..32): the primitive that orders the tile instances by (tile, subset), leaving each
 * subset's instances of a tile in the depth order of Eq. 3 (Sec. 3.1-3.2), and the splats
 * by depth.  keys, vals, keys_alt, vals_alt: device arrays of n pairs (0 <= n < 2^32), owned
 * by the caller.  The sorted pairs end up in (keys, vals), or in (keys_alt, vals_alt) when
 * *in_alt is 1 on return; the other two arrays are overwritten as scratch.  Every key must
 * be below 2^end_bit (higher bits may or may not take part in the order); pairs with equal
 * keys keep their input order.  temp:
 * device scratch of at least rgs_sort_temp_bytes(n) bytes.  Asynchronous on `stream`.
 * n = 0 returns at once (*in_alt = 0; the arrays may then be NULL).  RGS_EINVAL on a NULL
 * in_alt, a NULL array when n > 0, n < 0 or end_bit outside 1..32; RGS_EOVERFLOW when temp
 * is too small or n >= 2^32. */
size_t rgs_sort_temp_bytes(int64_t n);
int rgs_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n, int end_bit,
                   void* temp, size_t temp_bytes, void* stream, int* in_alt);

/* Backward of rgs_render_fwd with the merge (the "backward process" of Sec. 3.4): routes
 * dL/dimage [3,H,W] through Eq. 5 to each subset's (C_k, T_k), replays each subset's blend
 * from the stored partials, and pulls the per-splat 2D gradients back through the
 * projection.  Gradients are accumulated into `grads` (same shapes as the parameters; the
 * caller zeroes them).  A splat shared by several subsets accumulates into its single
 * parameter slot.  partial_C/partial_T (and tile_depth when non-NULL) must be the ones
 * rgs_render_fwd wrote for the same inputs.
 * A pixel whose transmittance in front of a subset (the merge's prod_{m<r} T_{o_m}) is
 * below eps_T takes no gradient from that subset or any behind it (they would be scaled by
 * less than eps_T).
 * The per-tile lists: when `workspace` (same pointer and size) still holds the lists of
 * the rgs_render_fwd call that wrote partial_C/partial_T with these kd, g, cam and opts
 * (no render into that workspace since; the forward stamps it), they are replayed as the
 * forward left them, cut back to what it staged, and nothing is re-derived.  Otherwise
 * they are re-derived; with tile_depth they then omit the splats lying behind a (tile,
 * subset) the forward had already saturated.  Neither changes a result.
 * The library recognises "these g" by the parameter POINTERS (and n, sh_degree), not by
 * their contents: the parameters must not change between the forward and its backward
 * (an in-place update with the same pointers would replay lists built for the old values
 * and give wrong gradients).  To back-propagate through changed parameters, render again.
 * Synchronises once with `stream`.  Errors as rgs_render_fwd. */
int rgs_render_bwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                   const float* partial_C, const float* partial_T, const float* dL_dimage, const float* tile_depth,
                   const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, void* stream);

/* Backward of a render through the flat form (an alternative to rgs_render_bwd): Eq. 5
 * equals flat blending (Eq. 2) exactly (the paper's appendix proof), so the gradients of
 * the merged image can be taken over each pixel's concatenated list (the subsets in view
 * order, each in depth order) in ONE front-to-back replay with the global transmittance:
 * dL/dsigma_i = T_i <g, c_i> - <g, C - A_i> / (1 - sigma_i), C the image (background
 * included), A_i the colour blended up to and including pair i.  Needs only the image the
 * forward wrote (rgs_render_fwd with or without partial maps: `image` [3,H,W]) and
 * dL_dimage; no partial maps are read or needed.  It replays the forward's own decisions:
 * each subset from T = 1 with its freeze points, the transmittance in front of it rebuilt
 * from the subset ends, a subset skipped where that is below eps_T.  Lists, tile_depth,
 * accumulation into `grads`, the parameter-pointer rule and errors as rgs_render_bwd (the
 * lists are replayed when `workspace` holds those of the forward that wrote `image`). */
int rgs_render_bwd_flat(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                        const float* image, const float* dL_dimage, const float* tile_depth,
                        const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ Adam (Sec. 4 details)
 * One Adam step over a flat parameter buffer split into `nseg` contiguous segments, each
 * with its own learning rate: seg_offsets_host [nseg+1] (elements), seg_lr_host [nseg].
 * param/grad/m/v [n] float (device, 16-byte aligned).  `step` is 1-based.  If zero_grad
 * is non-zero the gradient is cleared after it is read.  nseg in [1,16]. */
int rgs_adam_step(float* param, float* grad, float* m, float* v, int64_t n, const int64_t* seg_offsets_host,
                  const float* seg_lr_host, int nseg, float beta1, float beta2, float eps, int step, int zero_grad,
                  void* stream);

/* rgs_adam_step with one segment split periodically: inside segment `pseg`, an element
 * whose offset from the segment start is below `head` modulo `period` takes `head_lr`
 * instead of seg_lr_host[pseg].  For the SH block [N, (d+1)^2, 3] of splats (period
 * 3 (d+1)^2, head 3) that gives the degree-0 coefficients of every splat their own rate.
 * 0 <= pseg < nseg, period >= 1, 0 <= head <= period; otherwise as rgs_adam_step. */
int rgs_adam_step_periodic(float* param, float* grad, float* m, float* v, int64_t n, const int64_t* seg_offsets_host,
                           const float* seg_lr_host, int nseg, int pseg, int64_t period, int64_t head, float head_lr,
                           float beta1, float beta2, float eps, int step, int zero_grad, void* stream);

/* Exponential decay of the position learning rate, 1.6e-4 -> 1.6e-6 in the paper
 * (log-linear between lr_init at step 0 and lr_final at max_steps, then constant). */
float rgs_position_lr(int64_t step, int64_t max_steps, float lr_init, float lr_final);

/* ------------------------------------------------------------------ serving
 * A render server keeps one scene resident (the caller's device parameters, which must
 * stay allocated while the server lives; their values may change between requests) with
 * its KD subsets, and renders forward-only requests (Sec. 3.2 and Eq. 5; image only) from
 * a host-side queue.  The paper has no serving component: this is the deployment loop
 * around its renderer.
 *
 * Batched mode (default).  A host thread forms a batch of up to max_slots queued requests
 * whenever a lane is free, admitting requests in arrival order while the batch's tile and
 * instance capacity (set by mem_budget_bytes) has room, and launches the batch as one
 * captured CUDA graph: one projection pass over all (request, splat) pairs, device-counted
 * depth and tile sorts, and a persistent blend kernel whose blocks take (request, tile)
 * work items from a device counter until the batch is done.  With several lanes (each its
 * own graph, stream and buffers) a batch starts while earlier ones still run, so requests
 * that arrive while others are on the GPU overlap with them.  A batch that overflows its
 * instance capacity is re-run with its requests' exact sizes; a request that alone
 * exceeds a lane fails with RGS_EOVERFLOW.  A request's image does not depend on what
 * else shares its batch.
 * Plain mode renders one request at a time, in arrival order, through rgs_render_fwd's
 * path (the comparison baseline). */

typedef struct {
    size_t mem_budget_bytes;    /* device bytes for the server's buffers (all lanes) */
    int max_slots;              /* requests per batch, 1..16 */
    int lanes;                  /* batches in flight, 1..4 */
    int plain;                  /* non-zero: plain mode */
    int max_width, max_height;  /* largest image accepted (1..16384) */
    int max_queue;              /* queued requests beyond which submit returns RGS_EAGAIN */
    float inst_per_pixel;       /* first admission estimate of tile instances per pixel (later:
                                   measured); a low value only costs a re-run of the batch */
    float group_per_splat;      /* batched mode, opts.group_binning set and at least 4 subsets:
                                   a request bins its subsets in two groups of view ranks (as
                                   rgs_render_fwd's image-only forward) once the batches before
                                   measured at its resolution at least this many tile
                                   instances per visible splat ... */
    float group_min_instances;  /* ... and at least this many tile instances; with both 0, or
                                   with group_binning 2, every request is grouped */
    int64_t batch_max_pixels;   /* batched mode: a batch takes more requests only while their
                                   pixels stay within this (the first is always taken), so that
                                   small requests do not wait behind a large one; 0: no limit */
} rgs_serve_config;

typedef struct {
    int64_t submitted, completed, failed, cancelled;
    int64_t batches;            /* launches (batches, or requests in plain mode) */
    int64_t requeued;           /* requests re-run after their batch overflowed */
    int64_t instance_capacity;  /* tile instances per lane */
    double mean_batch;          /* requests per launch */
} rgs_serve_stats;

/* Defaults: 8 GiB, 8 slots, 2 lanes, batched, 4096x4096, 65536 queued, 16 instances
 * per pixel, groups from 12 instances per visible splat and 2^24 instances, batches of at
 * most 2^21 pixels. */
void rgs_serve_default_config(rgs_serve_config* cfg);

/* Device bytes one lane of a batched server with this configuration takes for a capacity
 * of `instance_capacity` tile instances (pure host arithmetic; mem_budget_bytes and
 * lanes are ignored), with the buffers of binning in groups of view ranks when the KD
 * tree has at least 4 subsets (a server whose options set group_binning).  A lane needs
 * at least 65536 instances. */
int rgs_serve_lane_bytes(const rgs_kd* kd, const rgs_gaussians* g, const rgs_serve_config* cfg,
                         int64_t instance_capacity, size_t* bytes);

/* rgs_serve_create_ex with the defaults, mem_budget_bytes and max_slots. */
int rgs_serve_create(const rgs_kd* kd, const rgs_gaussians* g, const rgs_render_opts* opts, size_t mem_budget_bytes,
                     int max_slots, rgs_server** out);

/* Allocates the lanes (within the budget), captures their graphs and starts the
 * scheduler thread on the current device.  kd and g must outlive the server.  Errors:
 * EINVAL (arguments, a budget too small for one request of max_width x max_height),
 * ENOMEM, ECUDA. */
int rgs_serve_create_ex(const rgs_kd* kd, const rgs_gaussians* g, const rgs_render_opts* opts,
                        const rgs_serve_config* cfg, rgs_server** out);

/* Queues a render of `cam` into out_image [3,H,W] (device, caller-owned, untouched by the
 * caller until the request is done).  Never blocks.  *ticket identifies the request.
 * Errors: EINVAL (camera, image larger than the configured maximum, NULL pointers),
 * EAGAIN (queue full or server stopping). */
int rgs_serve_submit(rgs_server* srv, const rgs_camera* cam, float* out_image, uint64_t* ticket);

/* Non-blocking.  *done = 1 once the request has finished, with *latency_ms (nullable) the
 * host time from submit to the scheduler seeing it complete; the ticket is then retired.
 * Returns RGS_OK while pending or after success, the request's error (EOVERFLOW, ECUDA,
 * EAGAIN if cancelled) with *done = 1 if it failed, EINVAL for an unknown ticket. */
int rgs_serve_poll(rgs_server* srv, uint64_t ticket, int* done, double* latency_ms);

int rgs_serve_stats_read(rgs_server* srv, rgs_serve_stats* out);

/* hold != 0: the scheduler starts no new batch (submitted requests wait in the queue;
 * batches already on the GPU finish).  hold == 0 resumes.  For draining and for
 * admitting a known set of requests together. */
int rgs_serve_hold(rgs_server* srv, int hold);

/* Stops the scheduler, cancels queued requests and waits at most 10 s for batches on the
 * GPU.  Returns ETIMEOUT if they did not finish (their buffers are then left allocated
 * rather than freed under a running kernel).  Never hangs. */
int rgs_serve_destroy(rgs_server* srv);

/* ------------------------------------------------------------------ tracing
 * rgs_profile_enable(flags): bit 0 turns on per-pass timing: every pass of the library
 * (projection, compaction, depth sort, offsets, emission, instance sort, ranges, blend
 * forward, blend backward, projection backward, Adam, merge, merge backward, KD build)
 * records a pair of CUDA events on the stream it is launched on (two event records per
 * pass; a batch of views' whole forward is one pass, "batch_fwd").  Bit 1 turns on pair
 * counting: the blend kernels run in a counting variant that
 * tallies the (pixel, splat) pairs they evaluate, the ones that contribute and why the
 * others fail (slower; keep it off where time is measured).  Process-wide.
 * rgs_profile_read synchronises with the recorded events and writes, per stage index
 * 0..rgs_profile_num_stages()-1, the accumulated milliseconds (ms_host) and pass counts
 * (launches_host), and counters_host[16] = {fwd pairs evaluated, fwd pairs contributing,
 * bwd pairs evaluated, bwd pairs contributing, tile instances, visible splats, kernel
 * launches of the library (counted whether or not profiling is on), fwd pairs failing the
 * Mahalanobis test, failing the ball test, failing the Eq. 6 subset test, fwd pairs
 * evaluated for splats held by several subsets, fwd instances staged before their tile's
 * pixels were all done, fwd instances contributing to at least one pixel, fwd warp passes
 * over one record-list entry (pairs evaluated / (32 x passes): the share of a warp's lanes
 * whose pixel is still blending), fwd pairs evaluated where the merged transmittance in
 * front of their subset is below eps_T, bwd warp passes over one record-list entry},
 * summed since the last reset.  Any
 * output pointer may be NULL.  reset != 0 clears the sums. */
int rgs_profile_enable(int flags);
int rgs_profile_num_stages(void);
const char* rgs_profile_stage_name(int stage);
int rgs_profile_read(double* ms_host, int64_t* launches_host, int64_t* counters_host, int reset);

#ifdef __cplusplus
}
#endif
#endif /* RGS_H */
