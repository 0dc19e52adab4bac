/*
 * fdgs.h - C ABI of the GB300 masked 4D Gaussian splatting rasterizer (libfdgs.so).
 *
 * The library renders 4D Gaussian scenes at a timestamp t (4DGS-1K, arXiv 2503.16422):
 * key-frame mask gate (Sec. 4.2.2), slice of each 4D Gaussian into a conditional 3D Gaussian
 * and a temporal weight (Sec. 3, Eq. 1 and Eq. 3), EWA projection, 16x16 tile binning,
 * (tile, depth) ordering and front-to-back alpha compositing (Sec. 3, Eq. 2); its reverse
 * (gradients for fine-tuning, Sec. 4.2.1 "Pruning" and Sec. 5 "Implementation Details"); the
 * spatial-temporal variation score used for pruning (Sec. 4.2.1, Eqs. 4-7); and batched
 * rendering of many (camera, t, resolution) requests in one call.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an fdgs_status. Nothing is thrown across the ABI; on a non-OK status
 *    fdgs_last_error() returns a message for the calling thread.
 *  - Pointers named *_dev are CUDA device pointers on the scene's device; all others are host
 *    pointers. Float arrays are float32, little-endian, densely packed.
 *  - Calls are stream-ordered on the given stream (NULL = legacy default stream). Unless a
 *    call says it synchronises, it may return before the GPU work finishes. Errors detected
 *    on the device (key capacity, spin-wait limit) are recorded in the scene's status word
 *    and returned by fdgs_status_sync() or by the next call that synchronises.
 *  - A scene is not thread-safe: calls on one scene must be serialised by the caller.
 */
#ifndef FDGS_H
#define FDGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared here so that this header needs no CUDA headers. */
typedef struct CUstream_st *fdgs_stream;

typedef enum {
  FDGS_OK = 0,
  FDGS_ERR_INVALID = -1,   /* bad argument (null pointer, size, degree, camera) */
  FDGS_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  FDGS_ERR_OOM = -3,       /* device allocation failed */
  FDGS_ERR_CAPACITY = -4,  /* a fixed-capacity buffer would overflow (batched path) */
  FDGS_ERR_TIMEOUT = -5,   /* a device spin-wait hit its iteration limit */
  FDGS_ERR_STATE = -6      /* call out of order (e.g. backward of a released frame) */
} fdgs_status;

typedef struct fdgs_scene fdgs_scene;   /* opaque, owned by the library */
typedef struct fdgs_frame fdgs_frame;   /* opaque per-render state kept for the backward */

/*
 * Scene description (Sec. 3: mean mu in R^4, scales S_4D, left/right quaternions q_l, q_r,
 * opacity sigma, colour c(d)). Structure of arrays, all device pointers, BORROWED: the
 * scene reads them at every render and never frees them, so in-place parameter updates are
 * seen without re-creating the scene. They must stay valid until fdgs_destroy_scene.
 *   mean4         [n][4]  (x, y, z, t), 16-byte aligned
 *   logscale4     [n][4]  log of the four axis scales; s = exp(logscale), Sigma = R S S^T R^T
 *   q_left        [n][4]  left quaternion (w, x, y, z), normalised by the renderer
 *   q_right       [n][4]  right quaternion (w, x, y, z), normalised by the renderer
 *   opacity_logit [n]     sigma = 1 / (1 + exp(-opacity_logit))
 *   sh            [K][3][n], K = (sh_degree + 1)^2 real spherical-harmonic coefficients per
 *                 channel; colour = max(0, sum_k Y_k(d) sh[k][c] + 0.5), d the unit direction
 *                 from the camera centre to the conditional mean.
 * sh_degree is 0..3. n may be 0. n must be < 2^30.
 */
typedef struct {
  int64_t n;
  int sh_degree;
  const float *mean4;
  const float *logscale4;
  const float *q_left;
  const float *q_right;
  const float *opacity_logit;
  const float *sh;
} fdgs_scene_desc;

/*
 * Pinhole camera. viewmat: world->camera rigid transform, row-major 4x4, OpenCV axes
 * (x right, y down, z forward). Pixel (i, j) is evaluated at image coordinate (i, j), so the
 * image centre is ((width-1)/2, (height-1)/2). Gaussians whose camera-space depth is
 * <= znear are culled. width, height in 1..16384.
 */
typedef struct {
  float viewmat[16];
  float fx, fy, cx, cy;
  int width, height;
  float znear;
} fdgs_camera;

/* use_mask: gate Gaussians by the key-frame masks given to fdgs_set_active_mask (ignored
 * when none are set). bg: background colour added as T_final * bg. */
typedef struct {
  int use_mask;
  float bg[3];
  int tile_sets;  /* fdgs_render: 0 = 3-sigma squares (the reference lists), 1 = the squares
                     cut to the tiles the alpha >= 1/255 ellipse can reach (same image,
                     shorter lists; fdgs_frame_export then returns these). Batches always
                     use 1. */
  int no_temporal_cull;  /* fdgs_render: 1 keeps the Gaussians whose a = sigmoid(o) p(t) is
                            below 1/255 (Sec. 3, Eq. 3) in projection, binning and sorting,
                            as a renderer without that cull would; they reach alpha >= 1/255
                            at no pixel, so the image is the same, only the lists are longer.
                            0 (default) culls them. Batches ignore it (their alpha-tight
                            tile sets are empty for such Gaussians). */
} fdgs_render_opts;

/* Counts of one rendered frame, for reports and tests. */
typedef struct {
  int64_t n_active;    /* Gaussians that passed the mask gate */
  int64_t n_visible;   /* Gaussians that touch at least one tile */
  int64_t n_keys;      /* (tile, Gaussian) pairs, i.e. total length of the tile lists */
  int width, height, tiles_x, tiles_y;
  int key_l, key_r;    /* key-frames used by the mask gate, -1 when unmasked */
  int key_bytes;       /* 4 or 8: width of the packed (tile, depth-rank) sort key */
  int list_builder;    /* how the tile lists were built: 1 emit + radix sort, 2 bitmasks */
} fdgs_frame_stats;

/* Creates a scene on the current CUDA device. Borrows the attribute pointers (see above).
 * Errors: FDGS_ERR_INVALID (null desc/out, n < 0, degree outside 0..3, null attribute pointer
 * with n > 0), FDGS_ERR_CUDA. */
int fdgs_create_scene(const fdgs_scene_desc *desc, fdgs_scene **out);

/* Frees the scene's workspaces and mask copy. Frames of the scene must be released first;
 * any still held are released here. NULL is accepted. Synchronises the device. */
int fdgs_destroy_scene(fdgs_scene *scene);

/* Replaces the scene's attribute pointers (same n and degree rules as creation). */
int fdgs_update_scene(fdgs_scene *scene, const fdgs_scene_desc *desc);

/*
 * Key-frame temporal filter (Sec. 4.2.2). bits_dev: [n_key][ceil(n/8)] bytes, one row per
 * key-frame, Gaussian i active in row k iff bit (i & 7) of byte (i >> 3) is set (LSB-first,
 * the "mask compressed into bits" of Sec. 5). key_times: n_key ascending host floats. The
 * scene COPIES the bits (device to device, on the stream) into its own padded storage.
 * At render time t the active set is the union of rows l and r, where l is the last key-frame
 * with time <= t (0 if t precedes all) and r = min(l + 1, n_key - 1). n_key = 0 clears the
 * masks. Errors: FDGS_ERR_INVALID (null pointers with n_key > 0, times not ascending).
 */
int fdgs_set_active_mask(fdgs_scene *scene, const uint8_t *bits_dev, const float *key_times,
                         int n_key, fdgs_stream stream);

/*
 * Renders the scene from camera cam at time t (Sec. 3, Eqs. 1-3; mask gate Sec. 4.2.2).
 * rgb_out_dev: [3][height][width] float32, written completely. If frame_out is non-NULL
 * a frame holding what the backward needs is returned (release it with
 * fdgs_frame_release); with NULL the scene's own workspace is reused.
 * Synchronises the stream once, after the per-Gaussian stage, to size the key buffers.
 */
int fdgs_render(fdgs_scene *scene, const fdgs_camera *cam, float t,
                const fdgs_render_opts *opts, float *rgb_out_dev, fdgs_frame **frame_out,
                fdgs_stream stream);

/*
 * fdgs_render without any host synchronisation (the same render, Sec. 3, Eqs. 1-3, mask gate
 * Sec. 4.2.2; the paper has no counterpart of the call itself): every stage is enqueued on
 * the stream and the call returns, so renders queue back to back and can be captured in a
 * CUDA graph. Keeps no frame. The tile lists are the coverage-bitmask lists (identical to the
 * other builder's), built into a list capacity fixed before the launch, in buffers of the
 * scene that no other call reallocates. The first call on a scene sizes that capacity with
 * one synchronised render (twice that frame's lists, plus 65536 entries; or set it with
 * fdgs_reserve_render_lists); make it, at the largest image size to be used, before any stream
 * capture (a later call that needs larger per-pixel or per-Gaussian buffers allocates them).
 * A frame whose lists exceed the capacity composites no Gaussian (its image is the background
 * only) and sets FDGS_ERR_CAPACITY in the status word: fdgs_status_sync (or the next call
 * that synchronises) returns it and grows the capacity to fit that frame, after which the
 * render can be repeated (a graph holding it must then be captured again).
 * Errors: as fdgs_render; FDGS_ERR_INVALID when the coverage-bitmask builder is unavailable
 * (fdgs_set_list_builder(1), or (tiles_x + tiles_y) * ceil(n / 256) * 32 B above 512 MiB).
 */
int fdgs_render_async(fdgs_scene *scene, const fdgs_camera *cam, float t,
                      const fdgs_render_opts *opts, float *rgb_out_dev, fdgs_stream stream);

/* List capacity (tile-list entries) of fdgs_render_async; 0 makes its next call size the
 * capacity again. Allocates: call it outside stream capture. FDGS_ERR_INVALID above 2^30 - 1
 * entries. */
int fdgs_reserve_render_lists(fdgs_scene *scene, uint64_t entries);

/*
 * Reverse of fdgs_render for the frame (reverse-order per-tile replay that recovers
 * transmittance by division, then the chain to the 4D parameters). dL_drgb_dev is
 * [3][height][width]. Gradients are ADDED (+=) into the caller's buffers, laid out like the
 * scene attributes: g_mean4 [n][4], g_logscale4 [n][4], g_q_left [n][4], g_q_right [n][4],
 * g_opacity_logit [n], g_sh [K][3][n]. Any gradient pointer may be NULL to skip it.
 * The scene attributes must not have changed since the render.
 * Errors: FDGS_ERR_STATE if the frame does not belong to the scene.
 */
int fdgs_render_backward(fdgs_scene *scene, fdgs_frame *frame, const float *dL_drgb_dev,
                         float *g_mean4, float *g_logscale4, float *g_q_left, float *g_q_right,
                         float *g_opacity_logit, float *g_sh, fdgs_stream stream);

/* Releases a frame (its buffers return to the scene's pool). NULL is accepted. */
int fdgs_frame_release(fdgs_frame *frame);

/* Counts of a frame. Synchronises the frame's stream. */
int fdgs_frame_get_stats(fdgs_frame *frame, fdgs_frame_stats *out);

/*
 * Copies a frame's internals to caller device buffers (for parity tests and tools), on the
 * stream. Any pointer may be NULL.
 *   tile_ranges_dev [tiles_y*tiles_x][2] uint32 [start, end) into the id list
 *   tile_ids_dev    [n_keys] uint32 Gaussian ids, tile-major, each tile's list in blend order
 *   T_final_dev     [height][width] float32 final transmittance
 *   n_contrib_dev   [height][width] uint32 1 + list position of the last blended Gaussian
 *   gauss_flags_dev [n] uint8 per-Gaussian decisions: bit0 passed the mask gate, bit1
 *                   a = sigmoid(o) p(t) >= 1/255, bit2 depth > znear, bit3 2D determinant
 *                   > 0, bit4 visible (non-empty tile rectangle)
 *   records_dev     [n][12] float32 per visible Gaussian (others untouched): u, v, conic
 *                   A, B, C, a, r, g, b, depth, radius, and the tile count as float
 */
int fdgs_frame_export(fdgs_frame *frame, uint32_t *tile_ranges_dev, uint32_t *tile_ids_dev,
                      float *T_final_dev, uint32_t *n_contrib_dev, uint8_t *gauss_flags_dev,
                      float *records_dev, fdgs_stream stream);

/*
 * Renders n_req requests (cams[i], ts[i]; each camera has its own resolution; 1 <= n_req <=
 * 128; n < 2^25) in one device-driven pass: the time- and camera-independent part of the
 * per-Gaussian work once, one launch over all (request, Gaussian) pairs, one global depth
 * sort whose keys carry the request, per-request lists kept per 4x4 block of tiles (each
 * entry with the block's tiles it covers), and ONE persistent blend launch over a queue of
 * all requests' tiles, longest list first, each tile reading its block's list. The first call for a batch geometry (request count, resolutions, mask use, scene
 * attribute pointers) runs eagerly and captures the sequence in a CUDA graph; later calls
 * replay it. rgb_out_dev is a HOST array of n_req device pointers, each [3][h_i][w_i].
 * Results equal n_req calls of fdgs_render. Synchronises the stream once, at the end; if a
 * list capacity was exceeded it grows the buffers and reruns before returning.
 */
int fdgs_render_batch(fdgs_scene *scene, const fdgs_camera *cams, const float *ts, int n_req,
                      const fdgs_render_opts *opts, float *const *rgb_out_dev,
                      fdgs_stream stream);

/* Autotuner of the batched path: renders the batch once per candidate launch shape (each of
 * the blend shapes of fdgs_set_blend_shape x {half, all} of its resident persistent CTAs per
 * SM), keeps the fastest for this batch geometry, and leaves the outputs of a final render in
 * rgb_out_dev. Synchronises. */
int fdgs_batch_autotune(fdgs_scene *scene, const fdgs_camera *cams, const float *ts,
                        int n_req, const fdgs_render_opts *opts, float *const *rgb_out_dev,
                        fdgs_stream stream);

/* Last batch: per-request latency in ms (%globaltimer, from the start of the batch to the
 * completion of the request's last tile) for the first n requests, the launch shape in use,
 * and stage_ms[FDGS_BATCH_STAGES], the durations of its stages from device timestamps
 * (%globaltimer written in stream order between the stages inside the graph; in order:
 * preprocess, depth_sort, gather, tile_scan, lists, queue_sort, blend).
 * Any pointer may be NULL. FDGS_ERR_STATE if no batch was rendered. With a counting profile
 * enabled (fdgs_profile_enable bit1) the next batch runs eagerly with the counting blend and
 * fdgs_profile_read returns its counts. */
#define FDGS_BATCH_STAGES 7
int fdgs_batch_info(fdgs_scene *scene, float *latency_ms, int n, int *footprint,
                    int *ctas_per_sm, float *stage_ms);

/*
 * Key-frame masks (Sec. 4.2.2, "Key-frame based Temporal Filtering"): for each key-frame time
 * key_times[k] (host array), renders the n_cam training views (host array of cameras) without
 * the filter and marks every Gaussian that takes part in some pixel's compositing in one view:
 * blended there (alpha >= 1/255 before the pixel's stop, a positive blend weight) or the
 * entry whose alpha would take T below 1e-4 (it ends that pixel's list, so a filter without it
 * would change the pixel). The union over the views is
 * row k of bits_out_dev, [n_key][ceil(n/8)] bytes on the device, bit i of row k = bit i % 8 of
 * byte i / 8: the layout fdgs_set_active_mask takes. Stream-ordered, asynchronous.
 * FDGS_ERR_INVALID on bad arguments.
 */
int fdgs_build_keyframe_masks(fdgs_scene *scene, const fdgs_camera *cams, int n_cam,
                              const float *key_times, int n_key, uint8_t *bits_out_dev,
                              fdgs_stream stream);

/*
 * Vector-quantised SH (the post-processing of Sec. 5, "Implementation Details", Ours-PP):
 * from now on the renders take the DC coefficients from plane 0 of the description's sh
 * array (only that plane is read, so it may be a [1][3][n] array) and bands k = 1..K-1 from
 * codebook_dev[codes_dev[i]][k - 1][c], codebook_dev [n_code][K - 1][3] float, codes_dev [n]
 * uint16, both device, BORROWED (valid until cleared or the scene is destroyed). A NULL
 * codebook clears it. Needs sh_degree >= 1 and 1 <= n_code <= 65536, else FDGS_ERR_INVALID.
 * fdgs_render_backward on a scene with a codebook returns FDGS_ERR_STATE (the gradients are
 * defined for full coefficients).
 */
int fdgs_set_sh_codebook(fdgs_scene *scene, const float *codebook_dev, int n_code,
                         const uint16_t *codes_dev);

/* Capacity, in block-list entries (one per (Gaussian, 4x4 tile block) pair a request's
 * rectangles meet), that batches of this scene start with; 0 restores the default
 * (8 x requests x Gaussians, at least 2^20). Applies to the current batch plan too. A batch
 * that needs more detects it on the device (its lists are left empty), grows the lists to
 * 1.125 x the need and reruns before fdgs_render_batch returns, so the capacity only trades
 * memory against a first-run retry. */
int fdgs_set_batch_list_capacity(fdgs_scene *scene, uint64_t entries);

/* Last batch: visible Gaussians and (tile, Gaussian) pairs summed over its requests (the
 * entries the tiles composite from their block lists), and the block-list entries the lists
 * hold (one per (Gaussian, 4x4 tile block) pair). The batched lists use, per Gaussian, the
 * 3-sigma tile square intersected with the tiles its alpha >= 1/255 ellipse can reach, so
 * n_keys is at most the per-request renders' total (images are identical). Any pointer may
 * be NULL. FDGS_ERR_STATE if no batch was rendered. */
int fdgs_batch_counts(fdgs_scene *scene, uint64_t *n_visible, uint64_t *n_keys,
                      uint64_t *n_block_entries);

/* Last batch, request req (for tests and tools; synchronises the device): its tile lists in
 * the layout of fdgs_frame_export, copied to HOST buffers.
 *   tile_ranges_host [tiles_y*tiles_x][2] uint32 [start, end) into the request's id list
 *   tile_ids_host    [ids_cap] uint32 Gaussian ids, tile-major, each tile's list in blend
 *                    order (depth, then id)
 * *n_tiles and *n_ids receive the request's tile count and entry count (0 entries if its
 * lists overflowed and were emptied). Any pointer may be NULL. FDGS_ERR_INVALID for a bad
 * request index or ids_cap < count, FDGS_ERR_STATE if no batch was rendered. */
int fdgs_batch_tile_lists(fdgs_scene *scene, int req, uint32_t *tile_ranges_host,
                          uint32_t *tile_ids_host, uint64_t ids_cap, uint64_t *n_tiles,
                          uint64_t *n_ids);

/*
 * Spatial-Temporal Variation Score (Sec. 4.2.1, Eqs. 4-7), reading "per-t product":
 *   S_i = sum over t in ts, camera in cams of  w_i(t, cam) * f_i(t) * gamma_i
 * with w_i = sum over pixels of alpha_i T_i (Eq. 4, the blend weight), f_i(t) =
 * 1 / (0.5 tanh|p''_i(t)| + 0.5) (Eqs. 5-6), gamma_i = clamp(V_i / V_p90, 0, 1)^0.1 with
 * V_i the product of the four scales and V_p90 its nearest-rank 90th percentile over all n
 * (Sec. 4.2.1 "Norm(V)", following LightGaussian). Renders use no mask. score_out_dev [n]
 * float32 is OVERWRITTEN. batch = renders issued between accumulations (>= 1).
 */
int fdgs_variation_score(fdgs_scene *scene, const fdgs_camera *cams, int n_cam,
                         const float *ts, int n_t, int batch, float *score_out_dev,
                         fdgs_stream stream);

/*
 * The scores of the ablation of the Spatial-Temporal Variation Score (Table 4; their formulas
 * are in the supplement's "Variant Settings"), each in the per-t reading of Eq. 7, with w_i,
 * f_i(t) and gamma_i as in fdgs_variation_score:
 *   FDGS_SCORE_FULL             (f, the paper's score)  sum_{t,cam} w_i f_i(t) gamma_i
 *   FDGS_SCORE_SPATIAL          (b, spatial only)       sum_{t,cam} w_i
 *   FDGS_SCORE_TEMPORAL         (c, temporal only)      sum_t f_i(t) gamma_i  (nothing is
 *                                                       rendered; the cameras are ignored)
 *   FDGS_SCORE_FIRST_DERIVATIVE (d)                     sum_{t,cam} w_i f1_i(t) gamma_i, f1 with
 *                               p'_i(t) = -(t - mu_t) / Sigma_t p_i(t) in place of p''_i(t)
 *   FDGS_SCORE_SIGMA_T          (e)                     sum_{t,cam} w_i Sigma_t,i gamma_i
 */
enum {
  FDGS_SCORE_FULL = 0,
  FDGS_SCORE_SPATIAL = 1,
  FDGS_SCORE_TEMPORAL = 2,
  FDGS_SCORE_FIRST_DERIVATIVE = 3,
  FDGS_SCORE_SIGMA_T = 4
};

/* fdgs_variation_score for one of the FDGS_SCORE_* variants (same arguments, same output
 * layout; score_out_dev is OVERWRITTEN). FDGS_ERR_INVALID for an unknown variant. */
int fdgs_variation_score_variant(fdgs_scene *scene, const fdgs_camera *cams, int n_cam,
                                 const float *ts, int n_t, int batch, int variant,
                                 float *score_out_dev, fdgs_stream stream);

/* fdgs_variation_score_variant that ADDS the pass's scores into score_inout_dev [n] instead of
 * overwriting it (the paper has no counterpart of the call). A score pass split into parts over
 * disjoint sets of (t, camera) renders then sums to the scores of the whole pass, up to the
 * order of the float additions, so a long pass can be checkpointed (the partial scores and the
 * parts done) and resumed after an interruption. Same arguments and errors as
 * fdgs_variation_score_variant. */
int fdgs_variation_score_add(fdgs_scene *scene, const fdgs_camera *cams, int n_cam,
                             const float *ts, int n_t, int batch, int variant,
                             float *score_inout_dev, fdgs_stream stream);

/*
 * Pruning keep-set (Sec. 4.2.1 "Pruning"): ranks the n scores by ascending (score, index)
 * and clears the lowest floor(prune_ratio * n). keep_out_dev [n] uint8 gets 1 = keep,
 * 0 = prune. Scores must be finite and >= 0. prune_ratio in [0, 1].
 */
int fdgs_select_keep(fdgs_scene *scene, const float *score_dev, int64_t n, float prune_ratio,
                     uint8_t *keep_out_dev, fdgs_stream stream);

/*
 * Same result as fdgs_select_keep, for callers that cannot allocate device memory. (The paper
 * has no counterpart: this is a deployment variant.) fdgs_select_keep grows buffers with
 * cudaMalloc/cudaFree, which synchronise the whole device and need free HBM; a caller inside a
 * real-time render or training loop, or one whose HBM is fully reserved by another allocator,
 * cannot allow either. This entry point allocates nothing: all of its scratch is one static
 * 18 MiB device array that every GPU loading the library holds until the process exits.
 *   - n must be <= 1048576 (2^20); larger n returns FDGS_ERR_CAPACITY. Other argument errors
 *     return FDGS_ERR_INVALID. No scene is needed.
 *   - The array is reserved when the runtime loads the library's module on a device: by
 *     default (lazy module loading) at the first call on that device, or when the library is
 *     loaded under CUDA_MODULE_LOADING=EAGER. A caller that must allocate nothing after
 *     start-up makes one warm-up call per device at start-up.
 *   - The first call on a device also looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any stream capture on
 *     that device. Calls after cudaDeviceReset of that device are not supported (the cached
 *     address may be stale).
 *   - Every call on a device shares the one array and overwrites it (the parts that must start
 *     at zero are cleared by each call). Calls whose GPU work overlaps (different streams,
 *     or concurrent host threads) race on the array: serialise them.
 *   - The call synchronises the stream before it returns, so that it can report a spin-wait
 *     limit reached inside its sort as FDGS_ERR_TIMEOUT (the keep-set is then unspecified).
 */
int fdgs_select_keep_noalloc(const float *score_dev, int64_t n, float prune_ratio,
                             uint8_t *keep_out_dev, fdgs_stream stream);

/*
 * Stage profiling of the scene's subsequent fdgs_render and fdgs_render_backward calls.
 * flags bit0: record CUDA events on the stream between the stages (FDGS_PROFILE_STAGES of
 * them, in order: preprocess, depth_sort, gather_scan, host_sync (the one mid-frame wait for
 * the key count), tile_scan (tile ranges and the blend's longest-first tile order), emit,
 * tile_sort, blend, written by fdgs_render; then backward_blend (the reverse replay) and
 * backward_gauss (the chain to the 4D parameters), written by fdgs_render_backward);
 * bit1: count the (Gaussian, pixel) evaluations of the blend or of the reverse replay (slower
 * kernel variants; use them in an untimed pass). 0 turns profiling off.
 */
#define FDGS_PROFILE_STAGES 10
int fdgs_profile_enable(fdgs_scene *scene, int flags);

/* Stage times in milliseconds of the last profiled render, and blend_counts[3] of the last
 * counted render or batch: (Gaussian, pixel) evaluations executed, footprint culling tests
 * executed, and evaluations that reached alpha >= 1/255 at a pixel still compositing (the
 * blended ones and the ones that stopped a pixel: the evaluations any blend order must
 * make, whatever its culling). After a counted fdgs_render_backward, blend_counts holds the
 * reverse replay's counts instead: entry evaluations at pixels whose replay reached them
 * (list position below n_contrib), the blended ones among them, and the gradient atomics
 * issued. Either pointer may be NULL. Synchronises the device. */
int fdgs_profile_read(fdgs_scene *scene, float *stage_ms, uint64_t *blend_counts);

/* How single-frame renders (fdgs_render) build the per-tile lists, process-wide. 1: emit one (tile, depth-rank) key
 * per covered tile and radix-sort the keys by tile; 2: AND per-tile-row and per-tile-column
 * coverage bitmasks over the depth ranks (no sort; wins when Gaussians cover many tiles);
 * 0 (default): choose per frame by a traffic estimate. The lists, and so every result, are
 * identical either way. Returns FDGS_ERR_INVALID for other values. */
int fdgs_set_list_builder(int mode);

/* Launch shape of the forward blend, process-wide: the pixel footprint of one warp inside a
 * 16x16 tile and the pixels each lane composites (one CTA of 256 / pixels-per-lane threads per
 * tile): 0: 16x2, 1: 8x4, 2: 4x8 (one pixel per lane), 3: 8x8 (two, the default), 4: 16x8,
 * 5: 8x16 (four), 6: 16x16 (eight: one warp per tile). Each warp culls, by ballot, the
 * Gaussians that cannot reach alpha >= 1/255 anywhere in its footprint; results do not depend
 * on the shape. A render that keeps no frame, on a black background, uses the forward-only
 * blend (no transmittance or n_contrib, the paired FP32 evaluation), whose shape starts at 5
 * and is set by this call too; -1 restores both defaults (3 and 5). The batch autotuner
 * (fdgs_batch_autotune) searches the same shapes for the batched blend. Returns
 * FDGS_ERR_INVALID for other values. */
int fdgs_set_blend_shape(int footprint);

/*
 * Post-pruning fine-tuning (Sec. 4.2.1 "Pruning": the Gaussians the score keeps are optimised
 * further; Sec. 4.2.2: through the key-frame filter when opts->use_mask is set), one iteration
 * in one call. In stream order: render view cam at t with opts (a frame kept for the reverse
 * replay) into a scene-owned image; the L1 loss against target_dev [3][H][W] (device,
 * float32), added to *loss_accum_dev as mean |image - target| (one device float; NULL: not
 * reported); its image gradient sign(image - target) / (3 H W); the reverse replay into
 * scene-owned gradient buffers; and one Adam step (Kingma and Ba, in PyTorch's formulation
 * with bias corrections) that updates the scene's attribute arrays IN PLACE, so they must be
 * writable device memory. lr[7] are the rates of mean4, logscale4, q_left, q_right,
 * opacity_logit, the SH DC plane and the higher SH bands. The scene keeps Adam's moments and
 * step count; fdgs_finetune_reset clears them (and a change of the scene's size does). The
 * call synchronises the stream once (the render sizes its tile lists). FDGS_ERR_INVALID for
 * null arguments, a bad camera or betas outside [0, 1).
 */
typedef struct {
  float lr[7];
  float beta1, beta2, eps;
} fdgs_adam_opts;
int fdgs_finetune_step(fdgs_scene *scene, const fdgs_camera *cam, float t,
                       const fdgs_render_opts *opts, const float *target_dev,
                       const fdgs_adam_opts *adam, float *loss_accum_dev, fdgs_stream stream);
int fdgs_finetune_reset(fdgs_scene *scene);

/* Launch shape of the scene's batched blend (fdgs_render_batch): a blend shape as in
 * fdgs_set_blend_shape and the persistent CTAs per SM (0: the occupancy limit). It applies to
 * the current batch plan (whose next batch runs eagerly and re-captures its graph) and to the
 * plans of new batch geometries, until fdgs_batch_autotune picks a shape for a plan. The
 * default is shape 6 (16x16 warp footprint, eight pixels a lane) at the occupancy limit.
 * Results do not depend on it. FDGS_ERR_INVALID for a shape outside [0, 7) or CTAs outside
 * [0, 64]. */
int fdgs_set_batch_shape(fdgs_scene *scene, int footprint, int ctas_per_sm);

/* How the batched blend (fdgs_render_batch and the batched score and mask passes) stages the
 * blend-ready records of each tile's list entries in shared memory, process-wide; batch graphs
 * are re-captured at their next run after a change. 0 (default): per-thread 16-byte cp.async
 * copies, three per record. 1: TMA, one cp.async.bulk.tensor tile::gather4 copy of four
 * 48-byte records per instruction, completing on a transaction-counting mbarrier (four-pixel
 * blend shapes and the weighted passes; the others, or a driver without the tensor-map
 * encoder, fall back to 0). Results are identical either way; a stage wait that exceeds its
 * spin limit sets FDGS_ERR_TIMEOUT. Returns FDGS_ERR_INVALID for other values. This is the
 * staging of Sec. 3's tile rasterisation (Eq. 2), which the paper leaves to the inherited
 * renderer. */
int fdgs_set_batch_staging(int mode);

/* Reads and clears the scene's device status word (synchronises the device): FDGS_OK, or
 * FDGS_ERR_CAPACITY / FDGS_ERR_TIMEOUT raised by a kernel since the last read. After a
 * capacity overflow of fdgs_render_async it also grows that call's list capacity to fit the
 * longest overflowing frame. */
int fdgs_status_sync(fdgs_scene *scene);

/*
 * Failure injection, process-wide, for tests of the error paths (the paper has no
 * counterpart). Every injected failure is made on the host or by a bounded wait that gives up:
 * none faults or hangs the GPU.
 *   FDGS_INJECT_SPIN_LIMIT (value = polls, 0 = the default 2^20): the spin-wait limit of the
 *     radix sort's decoupled look-back for later sorts. A look-back that reaches it gives up,
 *     sets FDGS_ERR_TIMEOUT in the scene's status word (or, for fdgs_select_keep_noalloc, in
 *     its own error word) and the sort's remaining passes skip their work; every access stays
 *     in bounds, the sorted output is unspecified.
 *   FDGS_INJECT_WITHHOLD_PUBLISH (value = partition index): the next sort pass launched
 *     eagerly (not from a captured graph) has that partition publish nothing in its
 *     look-back, so its successors wait until the spin limit. One-shot.
 *   FDGS_INJECT_FAIL_ALLOCS (value = count): the next `value` device-buffer growths fail with
 *     FDGS_ERR_OOM, as a refused cudaMalloc would.
 *   FDGS_INJECT_TMA_MISSING_ARRIVAL (value ignored): the next batch run with TMA record
 *     staging (fdgs_set_batch_staging(1)) runs eagerly, and in it the first issuing thread of
 *     every CTA neither arrives on its stage barriers nor issues its copy, so no stage
 *     completes; the stage waits give up after 4096 polls, the blend supplies the missing
 *     arrival, waits (bounded) for the copies in flight, sets FDGS_ERR_TIMEOUT and the call
 *     returns it. One-shot.
 *   FDGS_INJECT_NONE: clears all of the above.
 * Returns FDGS_ERR_INVALID for an unknown kind or a value out of range. Not thread-safe.
 */
enum {
  FDGS_INJECT_NONE = 0,
  FDGS_INJECT_SPIN_LIMIT = 1,
  FDGS_INJECT_WITHHOLD_PUBLISH = 2,
  FDGS_INJECT_FAIL_ALLOCS = 3,
  FDGS_INJECT_TMA_MISSING_ARRIVAL = 4
};
int fdgs_debug_inject(int kind, int64_t value);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char *fdgs_last_error(void);

/* FP32 fma throughput of the current device, measured (the paper has no counterpart; this
 * is the denominator of the blend's FP32 roofline). Every thread of a grid of 8 x 256-thread
 * CTAs per SM runs 16 independent fma chains, as scalar fma.rn.f32 (paired = 0) or as
 * fma.rn.f32x2 on pairs (paired = 1), 2^16 steps each; *tflops_out = 2 FLOP per lane fma /
 * the fastest of three launches timed with events on the stream (after one untimed launch).
 * Allocates a small buffer and synchronises. Errors: FDGS_ERR_INVALID (null output, paired
 * not 0 or 1), FDGS_ERR_CUDA. */
int fdgs_measure_fp32_peak(int paired, double *tflops_out, fdgs_stream stream);

/* Library version string. */
const char *fdgs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDGS_H */
