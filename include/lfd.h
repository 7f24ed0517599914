/*
 * lfd.h - C ABI of the GB300 (sm_103a) subpixel-level 3D Gaussian Splatting
 * renderer for lenticular light-field displays (CoherentRaster,
 * arXiv 2605.04509).
 *
 * The renderer takes a set of 3D Gaussians, the cameras of the display's
 * view cone and the panel's lenticular parameters, and writes the interlaced
 * light-field image I_LF in R^{W x H x 3} (Sec. 4, problem statement;
 * Alg. 1 inputs and output). Every step runs in CUDA kernels of this library.
 *
 * General rules
 *  - Device pointers are CUDA device (or managed) addresses valid on the
 *    current device; host pointers are ordinary CPU memory. The caller owns
 *    every buffer it passes; no call frees or retains caller memory beyond
 *    its own duration. A plan owns its panel tables and its scratch memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Rendering calls enqueue work on it; they block the host once per
 *    frame to read back the pair count P (needed to size the pair buffers),
 *    and again only when stage timing or evaluation counting is enabled.
 *  - A plan may be used by one host thread at a time; frames rendered with
 *    one plan on one stream are ordered. Different plans are independent.
 *  - Return value: LFD_OK (0) or a negative LFD_ERR_* code. No call aborts,
 *    traps or throws. lfd_status_string() gives the text; after
 *    LFD_ERR_CUDA, lfd_last_error() gives the CUDA error message of the
 *    calling thread's last failure.
 *
 * Layouts (row-major, float32 unless stated)
 *  - Gaussians (Sec. 3.3): means [M][3] (FP32); scales [M][3] (activated,
 *    > 0); quats [M][4] in (w, x, y, z) order (normalised inside); opacities
 *    [M] (activated, in [0, 1]); sh [M][(d+1)^2][3] real SH coefficients of
 *    degree d <= 3 in the 3DGS basis; the last four in FP32, FP16 or BF16.
 *  - Camera: world->camera rotation R (row-major 3x3), translation t,
 *    pinhole fx, fy, cx, cy in pixels (x right, y down, z forward). Every
 *    view renders at panel resolution.
 *  - Image: out_rgb [H][W][3]; subpixel (x, y, u) at (y*W + x)*3 + u; values
 *    are not clamped.
 *  - Clusters (Appendix B.1): C = views_per_cluster, K = ceil(N / C); slot l
 *    of cluster k is view min(k*C + l, N-1); the representative is slot
 *    floor(C/2).
 *  - Projected attributes (Eq. 5-6), for k in [0, K), i in [0, M):
 *      means2d       [K][M][C][2]  2D mean of Gaussian i in the view of slot
 *                                  l; NaN where the Gaussian lies at or in
 *                                  front of the near plane z = 0.2 of that
 *                                  view (culled there)
 *      conic_opacity [K][M][4]     (a, b, c, o): inverse of the 2D covariance
 *                                  [[a, b], [b, c]] at the representative
 *                                  view, and the opacity o
 *      color_tau     [K][M][4]     (r, g, b, tau): SH colour at the
 *                                  representative view, and
 *                                  tau = 2 ln(255 o) (the region q <= tau is
 *                                  where alpha >= 1/255); tau < 0 marks a
 *                                  Gaussian culled for the whole cluster
 *      depth         [K][M]        view-space depth at the representative
 */
#ifndef LFD_H
#define LFD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LFD_API __attribute__((visibility("default")))
#else
#define LFD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define LFD_OK 0
#define LFD_ERR_INVALID (-1)  /* bad argument, size or combination           */
#define LFD_ERR_OOM (-2)      /* device allocation failed                    */
#define LFD_ERR_CAPACITY (-3) /* pair count or key width beyond the limits   */
#define LFD_ERR_CUDA (-4)     /* a CUDA call failed; see lfd_last_error()    */
#define LFD_ERR_STATE (-5)    /* the requested data does not exist (yet)     */
#define LFD_ERR_TIMEOUT (-6)  /* a bounded device wait gave up (the sort's
                               * bulk-copy waits); reported at the plan's
                               * next read-back, the frame it hit is wrong  */

/* Key-generation and sort strategy. Both produce the identical sorted list
 * and range table.
 *  LFD_SORT_DEPTH_FIRST: sort the K*M per-cluster depths once, emit the
 *    Gaussian-tile pairs in that order and sort them stably by the
 *    (tile, cluster) bits only.
 *  LFD_SORT_KEY64: emit the 64-bit keys of Eq. 11 in (k, i) order and sort
 *    them stably over their 32 + Bit_K + Bit_T used bits. */
#define LFD_SORT_DEPTH_FIRST 0
#define LFD_SORT_KEY64 1

/* lfd_set_flags() bits */
#define LFD_FLAG_STAGE_TIMING 1 /* fill lfd_stats.ms_* (adds host syncs)  */
#define LFD_FLAG_COUNT_EVALS 2  /* fill lfd_stats.num_visits, num_evals  */
/* Remapped lfd_render frames keep, per subpixel, where its walk stopped and
 * its final transmittance (8 bytes per subpixel, allocated by lfd_set_flags);
 * lfd_render_backward then starts from them instead of re-blending. */
#define LFD_FLAG_KEEP_BLEND_STATE 4

typedef struct lfd_plan lfd_plan;

/* Lenticular panel (Sec. 3.1): resolution W x H, N views (1..255), tan of
 * the grating tilt angle alpha, grating pitch L_x in subpixels (> 0) and the
 * lens-to-panel offset K_offset in subpixels. */
typedef struct {
  int32_t width, height, num_views;
  double tan_slant, pitch, k_offset;
} lfd_panel;

/* Rendering options. tile_w * tile_h <= 1024, both in [4, 64]; C in
 * [1, 32] (C = 1: no attribute reuse); remap 1 = view-coherent remapping
 * (Sec. 4.3), 0 = subpixels in raster order, each thread walking its own list
 * (the ablation "w/o remap"; same image); sort_mode one of LFD_SORT_*; bg is
 * the background colour added as T * bg. subpixels_per_thread (0, 1, 2, 4 or
 * 8) is accepted and has no effect: the blend gives each (tile, cluster) run
 * one warp, which stages 32 list entries per batch and takes the run's live
 * subpixels 32 at a time. */
typedef struct {
  int32_t tile_w, tile_h;
  int32_t views_per_cluster;
  int32_t remap;
  int32_t sort_mode;
  float bg[3];
  int32_t subpixels_per_thread;
} lfd_opts;

/* Storage type of the Gaussians' scales, rotations, opacities and SH
 * coefficients (means are always FP32). Everything after the load - the
 * 2D-covariance inverse, the blend and the transmittance product - is FP32. */
#define LFD_DTYPE_F32 0
#define LFD_DTYPE_F16 1
#define LFD_DTYPE_BF16 2

typedef struct {
  const float *means;                          /* device, FP32 [M][3] */
  const void *scales, *quats, *opacities, *sh; /* device, attr_dtype */
  int64_t count;
  int32_t sh_degree;
  int32_t attr_dtype;                          /* LFD_DTYPE_* (0 = FP32) */
} lfd_gaussians;

typedef struct {
  float R[9], t[3], fx, fy, cx, cy;
} lfd_camera;

typedef struct {
  int32_t num_clusters;   /* K */
  int32_t tiles_x, tiles_y;
  int32_t tile_capacity;  /* 3 * tile_w * tile_h */
  int32_t bit_k, bit_t;   /* ceil(log2 K), ceil(log2 T) */
  int32_t max_segment;    /* largest (tile, cluster) subpixel run */
} lfd_plan_info;

typedef struct {
  int64_t num_pairs;  /* P: Gaussian-(tile, cluster) pairs of the last frame */
  int64_t num_visits; /* list entries walked by all subpixels until they
                         saturate or the list ends (flag)                   */
  int64_t num_evals;  /* E: of those, entries whose region in the
                         subpixel's own view meets the tile, for which the
                         Eq. 10 opacity was evaluated (flag)                 */
  float ms_project, ms_keygen, ms_sort, ms_blend; /* stage times (flag)    */
} lfd_stats;

/* The display's view cone as cameras (Sec. 4 problem statement: the views
 * of the 3D display setup; Alg. 1 inputs). Writes n (1..255) pinhole cameras
 * to the host array out[n]: camera j on a horizontal arc of the given radius
 * around the world origin at angle theta_j = -cone/2 + cone * j / (n - 1)
 * (0 for n = 1), position (radius sin theta, 0, -radius cos theta), looking
 * at the origin (z axis towards it, y axis the world's y, pointing down,
 * x = y cross z: view 0 is the leftmost camera); R holds the x, y, z axes as
 * rows and t = -R * position. fx = fy = (width / 2) / tan(fov_x / 2), principal
 * point (width / 2, height / 2): every view renders at panel size. Angles in
 * degrees; computed in double, stored as float. Host only (no device work).
 * LFD_ERR_INVALID for n outside [1, 255], radius <= 0, fov_x outside (0, 180),
 * cone outside [0, 360), width or height <= 0, or out == NULL. */
LFD_API int lfd_make_arc_cameras(int32_t n, double cone_deg, double radius, double fov_x_deg,
                                 int32_t width, int32_t height, lfd_camera *out);

/* Create a plan for one panel and option set on the current device: builds
 * the view index matrix V (Eq. 1-3, FP64 arithmetic), the per-tile
 * view-sorted subpixel table Psi (Sec. 4.3, Eq. 8; "precomputed once since
 * the lens geometry is fixed") and the per-(tile, cluster) runs inside it.
 * Synchronous. *out receives the plan, or NULL on error. */
LFD_API int lfd_plan_create(const lfd_panel *panel, const lfd_opts *opts, lfd_plan **out);

/* Release a plan and all device memory it owns (synchronises the device). */
LFD_API void lfd_plan_destroy(lfd_plan *plan);

LFD_API int lfd_plan_get_info(const lfd_plan *plan, lfd_plan_info *out);

/* Enable LFD_FLAG_* bits for the following frames. */
LFD_API int lfd_set_flags(lfd_plan *plan, int32_t flags);

/* Copy the panel tables to host memory (each pointer may be NULL):
 *   V      uint8 [H][W][3]  view index per subpixel (Eq. 3)
 *   psi    uint16 [T][3*TW*TH]  per tile, the tile's in-panel subpixels as
 *          local row-major indices (yl*TW + xl)*3 + u, stably sorted by view
 *          (Eq. 8); entries past n_sub[t] are unspecified
 *   n_sub  int32 [T]        in-panel subpixels of each tile
 *   seg    int32 [T][K+1]   first psi position of each cluster's run */
LFD_API int lfd_plan_copy_tables(const lfd_plan *plan, uint8_t *V, uint16_t *psi,
                         int32_t *n_sub, int32_t *seg);

/* Projection with cross-view attribute reuse (Sec. 4.2, Eq. 5-6; Alg. 1
 * stage 1): per-view 2D means for every slot of every cluster, and the
 * covariance, depth and SH colour of each cluster's representative view.
 * cams: host array of num_cams == N cameras. Outputs are caller-owned device
 * buffers in the layouts above. Asynchronous on stream. */
LFD_API int lfd_project(lfd_plan *plan, const lfd_gaussians *g, const lfd_camera *cams,
                int32_t num_cams, float *means2d, float *conic_opacity,
                float *color_tau, float *depth, void *stream);

/* Key generation, sort, range identification and subpixel blending
 * (Sec. 4.2-4.3, Alg. 1 stages 2-4, Alg. 2) from projected attributes in the
 * layouts above, for M Gaussians. Writes out_rgb [H][W][3] (device). A tile
 * of cluster k holds Gaussian i when some view of the cluster's region
 * {q <= tau} contains a pixel centre of the tile. Returns LFD_ERR_CAPACITY
 * (output untouched) when P would exceed 2^32 - 1. stats may be NULL. */
LFD_API int lfd_render_projected(lfd_plan *plan, int64_t M, const float *means2d,
                         const float *conic_opacity, const float *color_tau,
                         const float *depth, float *out_rgb, void *stream,
                         lfd_stats *stats);

/* The whole path (Alg. 1): lfd_project into plan-owned buffers, then
 * lfd_render_projected. */
LFD_API int lfd_render(lfd_plan *plan, const lfd_gaussians *g, const lfd_camera *cams,
               int32_t num_cams, float *out_rgb, void *stream, lfd_stats *stats);

/* Backward of lfd_render (not in the paper): given dL/dI for the image of
 * the plan's last lfd_render frame (grad_rgb, device [H][W][3]) and the same
 * Gaussians and cameras, writes dL/d(means, scales, quats, opacities, sh)
 * into caller-owned FP32 device arrays shaped like the inputs (overwritten).
 * The blend gradient is taken through Eq. 9-10 with the 3DGS rules; each
 * subpixel takes its final transmittance and the position where its walk
 * stopped from the forward frame when that frame kept them
 * (LFD_FLAG_KEEP_BLEND_STATE), else re-blends its list to find them, then
 * walks back to front. The projection gradient follows Eq. 5-6: every view's 2D mean, and
 * the representative view's covariance (with the Jacobian's dependence on the
 * mean and the 1.3 tan(fov/2) clamp), conic inverse and SH colour (including
 * its view direction). Needs FP32 attributes and the remapped blend;
 * LFD_ERR_STATE if the last frame was not an
 * lfd_render of this Gaussian count. Asynchronous on stream. */
LFD_API int lfd_render_backward(lfd_plan *plan, const lfd_gaussians *g, const lfd_camera *cams,
                                int32_t num_cams, const float *grad_rgb, float *grad_means,
                                float *grad_scales, float *grad_quats, float *grad_opacities,
                                float *grad_sh, void *stream);

/* The full-frame baseline the paper compares against (Sec. 1, Sec. 5.1; the
 * "3DGS" rows of T1/T2): every one of the N views rendered as a whole W x H
 * 3DGS image with its own projection (no attribute reuse: one view per
 * cluster) and its own per-tile lists, one alpha per pixel for all three
 * channels, then each subpixel (x, y, u) taken from the image of its view
 * V[x, y, u] (fused into the write). Same arguments and output as
 * lfd_render; the plan's tile shape (its height cut to 512 / tile_w for
 * tiles of more than 512 pixels: one thread per pixel of a tile), sort mode
 * and background apply. The first call builds a one-view-per-cluster companion plan owned by this plan.
 * Renders the same image as lfd_render with views_per_cluster = 1 (up to
 * FP32 rounding) at N x 8/3 the blend work. */
LFD_API int lfd_render_fullframe(lfd_plan *plan, const lfd_gaussians *g, const lfd_camera *cams,
                                 int32_t num_cams, float *out_rgb, void *stream, lfd_stats *stats);

/* End-to-end variant for callers holding HOST buffers: the Gaussians in g
 * and out_rgb are host pointers (pinned memory gives the fastest copies). The
 * call copies the inputs to plan-owned device memory, renders, copies the
 * image back and returns once it is in out_rgb (or, on an error, once every
 * copy it queued has finished). The copies run on plan-owned upload and
 * download streams: the Gaussians go up in four chunks, each projected as it
 * lands, and the image goes back once the blend is done. The image equals
 * lfd_render's bit for bit. It is
 * lfd_render_host_async followed by lfd_render_host_wait. */
LFD_API int lfd_render_host(lfd_plan *plan, const lfd_gaussians *g_host,
                    const lfd_camera *cams, int32_t num_cams, float *out_rgb_host,
                    void *stream, lfd_stats *stats);

/* Pipelined form of lfd_render_host for a stream of frames (same arguments):
 * queues the frame and returns once its pair count has been read back (the
 * frame's one mid-frame synchronisation), while its blend and the copy of
 * its image to out_rgb_host may still be running; the next call's upload then
 * runs under this frame's blend. The plan keeps two sets of device input and
 * image buffers and alternates them frame by frame. The host Gaussian arrays
 * and out_rgb_host of every queued frame must stay valid, the inputs
 * unchanged and out_rgb_host unread, until lfd_render_host_wait returns.
 * Frames of one plan go on one stream. On an error it waits for the copies
 * it queued before returning. */
LFD_API int lfd_render_host_async(lfd_plan *plan, const lfd_gaussians *g_host,
                                  const lfd_camera *cams, int32_t num_cams, float *out_rgb_host,
                                  void *stream, lfd_stats *stats);

/* Wait until every frame queued with lfd_render_host_async on this plan has
 * its image in host memory. LFD_ERR_CUDA if a copy failed. */
LFD_API int lfd_render_host_wait(lfd_plan *plan);

/* Copy the last frame's sorted Gaussian list L (uint32 [P], Gaussian ids),
 * range table (uint32 [T][K][2] = [S, E), (0, 0) when empty) and, with
 * LFD_SORT_KEY64 only, the sorted Eq. 11 keys (uint64 [P]) to host memory.
 * Any pointer may be NULL; capacity is the element count of list/keys.
 * Synchronises the plan's last stream. LFD_ERR_STATE before the first frame
 * or when keys are requested in depth-first mode. */
LFD_API int lfd_plan_copy_lists(const lfd_plan *plan, uint32_t *list, uint32_t *ranges,
                        uint64_t *keys, int64_t capacity);

/* Allocation-free variant of lfd_render_projected, for callers that must
 * not allocate device memory while they render: real-time loops that cannot
 * afford the device-wide synchronisation cudaMalloc and cudaFree imply, and
 * hosts (plug-in and embedding environments) whose own memory manager owns
 * the device heap. The paper has no counterpart. Callers that replay frames
 * from a CUDA graph use capacity mode (lfd_plan_reserve) instead.
 * Same arguments, stages and results (bit for bit) as lfd_render_projected;
 * the plan must have been created beforehand. All scratch memory comes from
 * one fixed array of about 4.9 MB inside the library (every GPU that loads
 * the library holds it until the process exits), which bounds the frame:
 * K * M <= 32768 projected items, T * K <= 16384 (tile, cluster) lists and
 * P <= 131072 Gaussian-tile pairs; larger frames return LFD_ERR_CAPACITY
 * with a message saying which limit, and the output is left untouched when
 * the item or list limit is hit. The call allocates nothing, neither on the
 * device nor on the host; like lfd_render_projected it reads the pair count
 * back (one stream synchronisation). The first call on a device looks up
 * the array's device address once (set-up); make that first call before any
 * stream capture. Every call shares the one array and leaves its contents
 * behind, so calls that overlap on the GPU (other streams, other host
 * threads) race: serialise them. stats may be NULL; only num_pairs is filled.
 * A bounded wait of the sorts that gives up (LFD_ERR_TIMEOUT) is reported by
 * this call when it happens before the pair-count read-back; one in the pair
 * sort after it is reported by this call when stats is non-NULL (the call
 * then synchronises the stream once more before returning), else by the next
 * call. */
LFD_API int lfd_render_projected_noalloc(lfd_plan *plan, int64_t M, const float *means2d,
                                         const float *conic_opacity, const float *color_tau,
                                         const float *depth, float *out_rgb, void *stream,
                                         lfd_stats *stats);

/* ---- Capacity mode: frames without host read-back (CUDA graphs) ----
 * The paper renders with a host-side pair count (Alg. 1 sizes the key
 * buffers from the offsets scan); these calls have no counterpart there.
 *
 * lfd_plan_reserve preallocates every per-frame buffer of the plan for up to
 * max_gaussians Gaussians and max_pairs Gaussian-(tile, cluster) pairs and
 * switches the plan to capacity mode (max_pairs = 0 switches it back).
 * In capacity mode lfd_render / lfd_render_projected never allocate, never
 * synchronise and never read anything back: the pair count P stays on the
 * device, and every kernel after the offsets scan reads it there. A frame
 * with P > max_pairs writes no pairs and leaves out_rgb untouched; it is
 * reported (LFD_ERR_CAPACITY) by the next lfd_plan_status. More Gaussians
 * than reserved fail at once with LFD_ERR_CAPACITY. Stage timing and
 * evaluation counting are off in this mode and stats->num_pairs is -1.
 * Such frames can be captured into a CUDA graph once the plan has rendered
 * one frame outside the capture (which sets kernel attributes); a replay
 * renders the Gaussians and cameras of the captured call (the cameras are
 * baked into the graph; the Gaussians are read from the captured device
 * pointers, so new values in those buffers are rendered).
 * Synchronous; frees and reallocates the plan's buffers when they grow.
 *
 * lfd_plan_status synchronises the device and returns LFD_ERR_CAPACITY if a
 * frame since the previous call overflowed, LFD_ERR_TIMEOUT if a bounded
 * wait gave up, else LFD_OK; *pairs (may be NULL) receives the last frame's
 * pair count, also when it overflowed (reserve that much and render again).
 * The flags are cleared by the call. */
LFD_API int lfd_plan_reserve(lfd_plan *plan, int64_t max_gaussians, int64_t max_pairs);
LFD_API int lfd_plan_status(lfd_plan *plan, int64_t *pairs);

/* ---- Batched rendering of several scenes per frame ----
 * Not in the paper (it renders one panel per frame): the serving form of
 * Alg. 1 for up to 16 scenes, each with its own plan (panel, tiles,
 * clusters; several scenes may share one plan), Gaussians, cameras and
 * image. Projection and per-item binning run per scene; the item sort, the
 * offsets scan, the pair sort and the range search run once for all scenes
 * (pair key = tile << (bits(S) + bits(K_max)) | scene << bits(K_max) |
 * cluster, sorted on the tile bits only: the pairs are emitted scene-major,
 * so every (scene, tile, cluster) run comes out contiguous), and one
 * persistent blend kernel takes the (scene, cluster, tile) runs from a work
 * counter. Each scene's image equals the single-scene lfd_render of that
 * scene bit for bit.
 * Plans must use LFD_SORT_DEPTH_FIRST, remap = 1 and the same
 * subpixels_per_thread; the tile, scene and cluster bits must fit 32.
 * The batch keeps pointers to the plans (their V, Psi and run tables): the
 * plans must outlive it. A batch always runs in capacity mode:
 * lfd_batch_reserve (per-scene Gaussian capacities [num_scenes], total pair
 * capacity) must precede rendering, and lfd_batch_render neither allocates
 * nor synchronises nor reads back, so it can be captured into a CUDA graph
 * (after one uncaptured frame). scenes: num_scenes device Gaussian sets;
 * cams: num_scenes host arrays, array s holding the num_views cameras of
 * scene s's panel; out_rgb: num_scenes device images [H_s][W_s][3].
 * Overflow and wait errors are reported by lfd_batch_status exactly as
 * lfd_plan_status reports them (an overflowing frame leaves every image
 * untouched). */
typedef struct lfd_batch lfd_batch;
LFD_API int lfd_batch_create(lfd_plan *const *plans, int32_t num_scenes, lfd_batch **out);
LFD_API void lfd_batch_destroy(lfd_batch *batch);
LFD_API int lfd_batch_reserve(lfd_batch *batch, const int64_t *max_gaussians, int64_t max_pairs);
LFD_API int lfd_batch_render(lfd_batch *batch, const lfd_gaussians *scenes,
                             const lfd_camera *const *cams, float *const *out_rgb, void *stream);
LFD_API int lfd_batch_status(lfd_batch *batch, int64_t *pairs);

/* Stage times accumulated over frames rendered with LFD_FLAG_STAGE_TIMING,
 * measured with CUDA events on each frame's stream and folded in without
 * extra synchronisation (a frame's events are read at the next frame's
 * pair-count read-back, or here). Synchronises the plan's last stream. */
typedef struct {
  int64_t frames;
  double ms_project, ms_keygen, ms_sort, ms_blend; /* sums over frames */
} lfd_stage_times;

LFD_API int lfd_get_stage_totals(lfd_plan *plan, lfd_stage_times *out, int32_t reset);

/* Self-test of the library's bounded device waits (no counterpart in the
 * paper): a kernel waits on an mbarrier phase that nothing completes, the
 * kind of wait the sort's pipelined scatter makes on its bulk copies.
 * Returns LFD_ERR_TIMEOUT when the wait gave up after its bound and the
 * kernel finished (the expected outcome, after about a quarter of a second),
 * LFD_OK if it did not, or LFD_ERR_CUDA. Synchronises the stream; allocates
 * and frees a 4-byte flag. */
LFD_API int lfd_selftest_wait_timeout(void *stream);

/* Measured ceilings of the blend's arithmetic on the current device (not in
 * the paper; the roofline of Eq. 9-10's per-evaluation work): one kernel of
 * independent FP32 fused multiply-add chains and one of independent
 * ex2.approx chains, each over every SM after an untimed round. Writes FP32
 * lane operations per second (an FMA counts as one) and exp2 evaluations per
 * second to the two host doubles. Synchronises the stream; allocates and
 * frees a small device buffer. LFD_ERR_INVALID for NULL outputs,
 * LFD_ERR_OOM, LFD_ERR_CUDA. */
LFD_API int lfd_measure_alu_peaks(double *fp32_ops_per_s, double *ex2_per_s, void *stream);

/* Number of CUDA kernels this library has launched in the process so far. */
LFD_API uint64_t lfd_kernel_launches(void);

LFD_API const char *lfd_status_string(int status);
LFD_API const char *lfd_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
LFD_API int lfd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LFD_H */
