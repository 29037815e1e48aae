/* pcr.h - C ABI of libpcr, a point-cloud rasterizer for NVIDIA GB300 (sm_103a).
 *
 * Method: Schuetz & Wimmer, "Rendering Point Clouds with Compute Shaders" (arXiv 1908.02681).
 *   Section 2.1 (Rasterization via AtomicMin): every point is projected, its depth is computed in double
 *   precision and turned into a 40-bit integer, the integer is shifted left by 24 bits and OR-ed with
 *   the point's 24-bit RGB, and a 64-bit atomicMin writes the key into a per-pixel u64 framebuffer; a
 *   per-pixel pass then turns keys into colours and clears the framebuffer.
 *   Section 2.2 (High-Quality Splatting): a depth pass as above, a second pass that sums R, G, B and a
 *   fragment count over the fragments whose linear depth is at most 1 % larger than the pixel's
 *   closest depth, and a resolve that divides the sums by the count.
 *
 * Conventions used by every entry point
 *   - Points: pcr_point, 16 bytes (float32 x, y, z; RGBA8 word with byte 0 = R), array of structures,
 *     in device memory owned by the caller, 16-byte aligned.
 *   - Framebuffers: opaque, device memory owned by the library, one per pcr_create_framebuffer call,
 *     on the device that was current at creation. Row-major, row 0 = bottom (OpenGL NDC orientation).
 *     Key layout: (depth code << 24) | (rgba & 0xFFFFFF). Empty pixel = 0xFFFFFFFFFFFFFFFF.
 *   - Streams: pcr_stream_t is a cudaStream_t (NULL = legacy default stream). Render, clear and resolve
 *     calls only enqueue work on that stream and return; argument errors are reported synchronously
 *     and enqueue nothing. Calls on one framebuffer from different streams must be ordered by the caller.
 *   - Errors: every call returns a pcr_status; PCR_OK is 0. A failed call leaves a message for the
 *     calling thread in pcr_last_error_message(). No C++ exception crosses this interface and no kernel
 *     traps: conditions found on the device (HQ count overflow) set a status word that
 *     pcr_get_device_status() reports.
 *   - Thread safety: distinct framebuffers may be used from distinct host threads concurrently.
 */
#ifndef PCR_H_
#define PCR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PCR_OK = 0,
  PCR_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment, view or flag; nothing was enqueued */
  PCR_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed; see pcr_last_error_message() */
  PCR_ERR_OOM = 3,         /* device allocation failed */
  PCR_ERR_OVERFLOW = 4,    /* HQ: some pixel received more than 2^24 contributing fragments */
  PCR_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up */
} pcr_status;

typedef void* pcr_stream_t; /* a cudaStream_t */

typedef struct pcr_framebuffer pcr_framebuffer;

/* One point: 16 bytes. rgba byte 0 = R, 1 = G, 2 = B, 3 = A (alpha is not used). */
typedef struct {
  float x, y, z;
  uint32_t rgba;
} pcr_point;

/* Depth-code mappings (Section 2.1: "uniform or customizable" precision).
 *   LINEAR:    q = floor((w - near) * s), s = 2^40 / (far - near), both operations rounded in FP64.
 *   METRIC:    q = floor(w * metric_scale) (the paper's example: metres * 1000 = millimetres).
 *   PIECEWISE: sub-ranges [lo_k, hi_k) at res_k codes per metre, codes of range k following those of
 *              range k-1: q = base_k + floor((w - lo_k) * res_k), base_k = sum_{j<k} ceil((hi_j - lo_j) * res_j);
 *              depths outside every range are culled (Section 2.1's nm / um / mm example).
 * In every mode q = min(q, 2^40 - 2), so that no key equals the empty value. The EXACT transform evaluates all
 * three in single precision with certified bounds (PIECEWISE with one depth table per range that meets
 * [near, far); views whose piecewise codes can reach the cap, like the other views outside its
 * preconditions, run on the FP64 kernels with the same results). */
enum { PCR_DEPTH_LINEAR = 0, PCR_DEPTH_METRIC = 1, PCR_DEPTH_PIECEWISE = 2 };

/* How the per-point transform is evaluated.
 *   EXACT: the result of the FP64 definition, bit for bit (default). The library evaluates most points
 *          in single-precision arithmetic whose error bound proves the FP64 result, and sends the
 *          points that the bound cannot decide through FP64.
 *   FP64:  every point through the FP64 operations directly (same output as EXACT, slower).
 *   DOUBLE_FLOAT: single-precision pair ("double-float") arithmetic without the FP64 arbiter; output may
 *          differ from the FP64 definition in rare depth codes or pixels (precision study only). */
enum { PCR_TRANSFORM_EXACT = 0, PCR_TRANSFORM_FP64 = 1, PCR_TRANSFORM_DOUBLE_FLOAT = 2 };

#define PCR_MAX_DEPTH_RANGES 8

/* A camera. For each point (X, Y, Z) = (double)(x, y, z):
 *   clip_r = fma(M[r][2], Z, fma(M[r][1], Y, fma(M[r][0], X, M[r][3]))) for r = 0 (cx), 1 (cy), 3 (w);
 *   culled unless near <= w < far (NaN culled);
 *   fx = fmaf((float)cx / (float)w, 0.5f, 0.5f) * (float)W, same for fy with cy and H (IEEE single);
 *   culled unless 0 <= fx < W and 0 <= fy < H; pixel = (int)fy * W + (int)fx.
 * Requirements: every matrix entry finite; 0 < near < far < inf; metric_scale > 0 and finite for METRIC;
 * 1 <= n_ranges <= 8 ascending non-overlapping ranges with 0 <= lo < hi, res > 0 for PIECEWISE. */
typedef struct {
  double view_proj[16]; /* row-major 4x4, clip = M * (x, y, z, 1) (OpenGL perspective * lookAt) */
  double near_plane;
  double far_plane;
  int32_t depth_mode;   /* PCR_DEPTH_* */
  int32_t transform;    /* PCR_TRANSFORM_* */
  double metric_scale;  /* METRIC: codes per metre (1000.0 = millimetres) */
  int32_t n_ranges;     /* PIECEWISE: number of used rows of `ranges` */
  int32_t reserved;     /* must be 0 */
  double ranges[PCR_MAX_DEPTH_RANGES][3]; /* PIECEWISE: {lo (m), hi (m), codes per metre} */
} pcr_view;

/* Launch tuning of a framebuffer's point passes (the knobs an autotuner sets). Results never depend on it. */
typedef struct {
  int32_t merge_same_pixel; /* 1: the fragments of one warp that land on the same pixel are merged with warp
                               reductions, then one atomic per pixel; 0 (default): pass 1 issues one atomic
                               per fragment whose key is below the key the pixel holds, and pass 2 merges the
                               additions of two adjacent lanes (consecutive points) that land on one pixel */
  int32_t blocks_per_sm;    /* 256-thread blocks per SM for the point passes, 1..32 (default 8; capped at the
                               blocks that can be resident, 4 for pass 1 and 5 for pass 2) */
  int32_t staging;          /* how each warp brings its tiles of 64 points in: 0 (default) its own 16-byte
                               loads, one tile ahead; 1 bulk copies (cp.async.bulk) into a two-stage
                               shared-memory ring whose waits are bounded (a wait that gives up sets the
                               timeout status, see pcr_get_device_status) */
  int32_t band_filter;      /* 1: pcr_render_atomicmin on an HQ framebuffer (exact transform, LINEAR or METRIC)
                               also records which points may still be in the HQ band of eps <=
                               band_eps_num / band_eps_den, and a following pcr_hq_accumulate of the same
                               points (pointer, count, view; the points unchanged in between) with such an eps
                               skips the others. The records are exact: a stored key only decreases, so a point
                               whose code is already beyond the band of the key its pixel held can never be
                               accepted. pcr_render_hq_splat and pcr_render_frame_host do the same between
                               their two passes. 0 (default): nothing is recorded. It pays off when points come
                               in random order (pass 2 about 17 % faster, the HQ frame about 5 %), not in scan
                               order, where pass 1's extra work outweighs it; the autotuner tries both. The first
                               recording of n points allocates n / 8 bytes of device memory (not during stream
                               capture, where nothing is recorded); a clear drops the record. */
  uint32_t band_eps_num, band_eps_den; /* eps of the records (default 1 / 100); band_eps_den in 1..2^20 */
  int32_t band_bounds;      /* 1: pass 2 with the exact transform first turns each pixel's qmin into its accept
                               bounds {qmin, qmin + floor(eps_num * (qmin + Nq) / eps_den)} (one more kernel,
                               24 B per pixel of traffic) and tests each decided code q by lo <= q <= hi, where
                               the host finds eps_num * (2^40 + Nq) + eps_den * 2^40 <= 2^64 (the same decision
                               as the band test of pcr_render_hq_splat then). The first such pass allocates
                               16 B per pixel (not during stream capture: there the stored-key test is used).
                               0 (default): the band test on the stored key. Faster for points in random order
                               without band records (pass 2 about 1 %), slower in scan order (about 3 %); the
                               autotuner tries both. */
} pcr_tuning;

/* Framebuffer flags. */
#define PCR_FB_HQ 1u /* also allocate the 16 B/pixel HQ accumulation buffer (needed by pcr_render_hq_splat) */

/* Allocates a width x height framebuffer on the current device (keys: 8 B/pixel; with PCR_FB_HQ also
 * sums: 16 B/pixel, and 16 B/pixel of band bounds once a pass 2 runs with pcr_tuning.band_bounds; plus a
 * 96 KB device copy of the depth tables of the view last rendered, re-uploaded on the render call's stream
 * when the view changes) and clears it (synchronously). width, height in 1..16384. */
pcr_status pcr_create_framebuffer(int32_t width, int32_t height, uint32_t flags, pcr_framebuffer** out);

/* Frees the framebuffer (synchronises the device first). NULL is accepted. */
pcr_status pcr_destroy_framebuffer(pcr_framebuffer* fb);

/* Sets the launch tuning used by later render calls on fb (NULL restores the defaults). Not ordered with
 * work already enqueued; calls racing with a render call on another thread are the caller's to avoid. */
pcr_status pcr_set_tuning(pcr_framebuffer* fb, const pcr_tuning* tuning);

/* Current launch tuning of fb. */
pcr_status pcr_get_tuning(const pcr_framebuffer* fb, pcr_tuning* tuning);

/* Autotuner: renders one frame of (d_points, n, view) on fb for every candidate tuning (same-pixel merging
 * on and off, both stagings, 2 / 4 / 6 / 8 blocks per SM, and for HQ framebuffers band records with eps 1/100
 * and pass 2's per-pixel bounds, each on and off), times the point passes with CUDA events on `stream` (pass 1,
 * plus pass 2 with eps 1/100 for HQ framebuffers; best of two runs), and keeps the fastest in fb. Writes it
 * to *best when best is not NULL. Clears fb before every run and at the end; synchronises `stream`.
 * Arguments as for pcr_render_atomicmin; n must be > 0. */
pcr_status pcr_autotune(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                        pcr_stream_t stream, pcr_tuning* best);

/* Size and flags of a framebuffer. Any output pointer may be NULL. */
pcr_status pcr_framebuffer_info(const pcr_framebuffer* fb, int32_t* width, int32_t* height, uint32_t* flags);

/* Section 2.1 (clear value): keys to 0xFFFFFFFFFFFFFFFF and, for HQ framebuffers, sums and counts to 0. */
pcr_status pcr_clear(pcr_framebuffer* fb, pcr_stream_t stream);

/* Section 2.1: rasterizes n points into fb with one 64-bit atomic minimum per visible fragment (keys
 * accumulate with what fb holds; call pcr_clear or resolve with clear_after to start a frame). A fragment
 * whose key is not below the key its pixel already holds skips its atomic: the result is the same.
 * n == 0 is a no-op; n < 2^40. */
pcr_status pcr_render_atomicmin(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                                pcr_stream_t stream);

/* pcr_render_atomicmin that also adds, to d_counts[0..3] (caller-owned device u64, not cleared), how the
 * EXACT transform's single-precision evaluation handled the points: [0] decided by the first tier (float
 * pixel estimate with its error bound, exact depth code), [1] depth code undecided between two
 * neighbours, [2] sent to the FP64 arbiter, [3] deferred to the second tier (double-float clip values; the
 * points of [1] included).
 * For PIECEWISE depth the points the first tier leaves undecided go to the FP64 arbiter directly ([2] and [3]
 * then count the same points). All four stay 0 when the view is evaluated by the FP64 kernels (transform
 * FP64, or a view outside the single-precision preconditions). A diagnostic of the transform; the framebuffer
 * result is the same as pcr_render_atomicmin's. */
pcr_status pcr_render_atomicmin_stats(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n,
                                      const pcr_view* view, uint64_t* d_counts, pcr_stream_t stream);

/* Sections 1 and 2.1, per point and without a framebuffer: the fragment each of the n points gets under the
 * view at width x height. d_pixel[i] = row * width + column (row 0 = bottom) of point i, or 0xFFFFFFFF when
 * the definition culls it; d_key[i] = its key (depth code << 24 | RGB), or 0xFFFFFFFFFFFFFFFF when culled.
 * The view's transform applies: EXACT and FP64 give the FP64 definition bit for bit, DOUBLE_FLOAT its
 * approximation. The framebuffer passes take the same per-point decisions; a framebuffer keeps, per pixel,
 * the smallest key that lands there.
 * d_points: 16-byte aligned device memory, caller-owned; d_pixel (n u32) and d_key (n u64): caller-owned
 * device memory. Asynchronous on stream; argument errors are synchronous and enqueue nothing; n == 0 is a
 * no-op; n < 2^40; width, height in 1..16384. */
pcr_status pcr_project_points(const pcr_point* d_points, uint64_t n, const pcr_view* view, int32_t width,
                              int32_t height, uint32_t* d_pixel, uint64_t* d_key, pcr_stream_t stream);

/* Section 2.2: high-quality splatting of n points into an HQ framebuffer: pass 1 = pcr_render_atomicmin;
 * pass 2 adds (R, G, B, 1) of every fragment with eps_den * (q - qmin) <= eps_num * (qmin + Nq) to its
 * pixel's sums, where qmin = key >> 24 after pass 1 and Nq = floor(near * s) (LINEAR) or 0 (METRIC), i.e.
 * linear depth at most (1 + eps_num / eps_den) times the closest (eps = 1/100 in the paper).
 * Requirements: fb created with PCR_FB_HQ, and cleared; depth_mode LINEAR or METRIC; 1 <= eps_den <= 2^20;
 * eps_num * (2^40 + Nq) < 2^64. Colour sums are u32 per channel: valid while every pixel gets at most 2^24
 * contributing fragments (checked by the HQ resolve, reported as PCR_ERR_OVERFLOW). pcr_tuning.band_bounds
 * selects how pass 2 evaluates the test; the result is the same. */
pcr_status pcr_render_hq_splat(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                               uint32_t eps_num, uint32_t eps_den, pcr_stream_t stream);

/* Section 2.2, second pass only: the band accumulation of pcr_render_hq_splat, for a framebuffer whose
 * keys already hold pass 1 of the same points and view (pcr_render_atomicmin). Same requirements as
 * pcr_render_hq_splat; pcr_render_hq_splat == pcr_render_atomicmin followed by this call. */
pcr_status pcr_hq_accumulate(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                             uint32_t eps_num, uint32_t eps_den, pcr_stream_t stream);

/* Section 2.1 (second shader) / Section 2.2 (third pass): writes one RGBA8 word per pixel into
 * d_rgba_out (caller-owned device memory, width * height u32, row 0 = bottom). For a framebuffer without
 * PCR_FB_HQ: the key's colour with alpha 255, background_rgba where empty. With PCR_FB_HQ: per channel
 * (sum + count / 2) / count with alpha 255, background_rgba where count == 0. clear_after != 0 also
 * clears the framebuffer (as the paper's resolve shader does). */
pcr_status pcr_resolve(pcr_framebuffer* fb, uint32_t* d_rgba_out, uint32_t background_rgba, int32_t clear_after,
                       pcr_stream_t stream);

/* Section 2.1 resolve of the keys of any framebuffer (the basic image of an HQ frame, whose pass 1 holds
 * it). clear_after != 0 clears keys (and HQ sums). */
pcr_status pcr_resolve_basic(pcr_framebuffer* fb, uint32_t* d_rgba_out, uint32_t background_rgba,
                             int32_t clear_after, pcr_stream_t stream);

/* Sections 2.1 and 2.2 resolves of an HQ framebuffer in one pass over its pixels: d_rgba_basic gets the
 * image of pcr_resolve_basic and d_rgba_hq the image of pcr_resolve (the same values, the overflow status
 * as pcr_resolve sets it); both W*H, caller-owned device memory. clear_after != 0 clears the keys and the sums.
 * PCR_ERR_INVALID_ARG without PCR_FB_HQ or with a NULL image. */
pcr_status pcr_resolve_both(pcr_framebuffer* fb, uint32_t* d_rgba_basic, uint32_t* d_rgba_hq, uint32_t background_rgba,
                            int32_t clear_after, pcr_stream_t stream);

/* Read-only device pointers to the key buffer (width * height u64) and, for HQ framebuffers, the sums
 * (width * height pairs of u64: {R | G << 32, B | count << 32}); *d_accum = NULL otherwise. Valid until
 * pcr_destroy_framebuffer. Either output pointer may be NULL. */
pcr_status pcr_framebuffer_keys(const pcr_framebuffer* fb, const uint64_t** d_keys, const uint64_t** d_accum);

/* One complete frame from host memory (Sections 2.1 and 2.2 end to end). It:
 *   - copies the n points from h_points (host memory; pinned for the copies to overlap) into d_points
 *     (caller-owned device buffer of n points, 16-byte aligned) in up to 8 chunks, and runs pass 1 on each
 *     chunk as soon as it has landed;
 *   - then pass 2 (HQ framebuffers), the basic resolve into d_images[0, W*H) and the HQ resolve into
 *     d_images[W*H, 2*W*H), clearing fb;
 *   - copies the images to h_basic and h_hq (host, W*H u32 each; h_hq is unused without PCR_FB_HQ).
 * d_images: caller-owned device scratch of 2*W*H u32. The frame must start from a cleared fb; it leaves fb
 * cleared. Everything is enqueued on `stream`, plus the device's upload queue: one internal copy stream per
 * device, shared by all framebuffers, so that frames from host memory upload back to back in call order and
 * each frame's passes overlap the next frame's upload. It is ordered with `stream` by events (created by the
 * first call on fb); a frame's copies also wait for the work queued on `stream` before the call. Returns at once:
 * synchronise `stream` before reading the host images or reusing h_points or d_points. Requirements as for
 * pcr_render_hq_splat (HQ) or pcr_render_atomicmin. */
pcr_status pcr_render_frame_host(pcr_framebuffer* fb, const pcr_point* h_points, uint64_t n, const pcr_view* view,
                                 uint32_t eps_num, uint32_t eps_den, uint32_t background_rgba, pcr_point* d_points,
                                 uint32_t* d_images, uint32_t* h_basic, uint32_t* h_hq, pcr_stream_t stream);

/* Check of the timeout path (no counterpart in the paper). The point passes wait on shared-memory barriers
 * for their bulk copies, and every such wait gives up after a bounded number of rounds, sets fb's timeout
 * bit and ends the pass, so that a copy that never lands shows up as PCR_ERR_TIMEOUT from
 * pcr_get_device_status instead of a hung kernel. This call runs that wait routine in one warp on a
 * barrier that nothing will complete (no copy is issued), so it gives up after `rounds` rounds (1..2^18;
 * 0 = the passes' own limit of 2^18 rounds, about 1 s on GB300) and sets the bit. Asynchronous on `stream`. */
pcr_status pcr_check_bounded_wait(pcr_framebuffer* fb, uint32_t rounds, pcr_stream_t stream);

/* Synchronises `stream`, then returns and resets the device-side status of fb: PCR_ERR_OVERFLOW if an
 * HQ resolve found a pixel with more than 2^24 fragments, PCR_ERR_TIMEOUT if a bounded wait gave up,
 * else PCR_OK. */
pcr_status pcr_get_device_status(pcr_framebuffer* fb, pcr_stream_t stream);

/* Number of kernels this library has launched in this process (all devices, all streams). Lets a caller
 * check how many GPU launches a region of its own code made. */
uint64_t pcr_kernel_launch_count(void);

/* Static description of a status code. */
const char* pcr_status_string(pcr_status status);

/* Message of the calling thread's last failed call ("" if none). */
const char* pcr_last_error_message(void);


/* ---------------------------------------------------------------------------------------------------
 * Batched rendering of a resident cloud: many views per launch (no counterpart in the paper, which
 * renders one view per frame; the per-point results are those of Sections 2.1 and 2.2).
 * ------------------------------------------------------------------------------------------------- */

typedef struct pcr_cloud pcr_cloud;
typedef struct pcr_batch pcr_batch;

#define PCR_CLOUD_CHUNK 1024   /* points per culling chunk */
#define PCR_MAX_BATCH_VIEWS 256

/* Prepares n caller-owned device points (16-byte aligned, 1 <= n < 2^40) for batched rendering: the
 * bounding box of every chunk of PCR_CLOUD_CHUNK consecutive points is computed on `stream` into
 * library-owned device memory (24 B per chunk). The points are not copied: they must stay valid and
 * unchanged while the cloud is in use. */
pcr_status pcr_cloud_create(const pcr_point* d_points, uint64_t n, pcr_stream_t stream, pcr_cloud** out);

/* Frees the cloud (synchronises the device). Batches made from it must be destroyed first. NULL is accepted. */
pcr_status pcr_cloud_destroy(pcr_cloud* cloud);

/* A frame of `count` views of one cloud (1 <= count <= PCR_MAX_BATCH_VIEWS): view i renders into fbs[i]
 * and resolves into d_outs[i] (caller-owned device memory, width * height u32 of fbs[i]). hq != 0 makes it
 * a high-quality splatting frame (every fbs[i] created with PCR_FB_HQ; eps_num / eps_den as in
 * pcr_render_hq_splat). The framebuffers must be distinct, cleared, on the cloud's device, and used by
 * nothing else while the batch exists. The batch owns its device workspace (per-view constants, chunk
 * visibility masks: 1 bit per chunk per view) and a pinned staging buffer for the views. clear_after != 0: every
 * frame clears the framebuffers after resolving them (ready for the next frame); 0 leaves keys and sums in
 * place (pcr_framebuffer_keys reads them; clear before the next frame). */
pcr_status pcr_batch_create(pcr_cloud* cloud, pcr_framebuffer* const* fbs, uint32_t* const* d_outs, int32_t count,
                            int32_t hq, uint32_t eps_num, uint32_t eps_den, uint32_t background_rgba,
                            int32_t clear_after, pcr_batch** out);

/* Sets the views of the next frames (count of them). Every view must use LINEAR or METRIC depth within
 * the single-precision preconditions (every perspective lookAt camera does), else PCR_ERR_INVALID_ARG.
 * Blocks until the previous frame has copied the earlier views to the device. */
pcr_status pcr_batch_set_views(pcr_batch* batch, const pcr_view* views);

/* Enqueues one frame on `stream`:
 *   - copy the views' constants to the device;
 *   - per view, mark the chunks whose bounding box is certainly outside the view (behind the near plane,
 *     beyond the far plane, or at |ndc| > 1 + 1e-5, with margins covering every rounding);
 *   - pass 1 for all views in one persistent launch that skips those chunks and takes the chunk ranges in
 *     turn for every view (so each range is read from HBM once), then pass 2 (hq) likewise. A frame of at
 *     most 4 views, or of a cloud of at least 10^8 points, instead runs one single-view pass per view,
 *     which is faster there (frames recorded by pcr_batch_capture always use the persistent launch);
 *   - resolve every framebuffer into its output (and clear it, see pcr_batch_create).
 * Framebuffer contents equal those of pcr_render_atomicmin / pcr_render_hq_splat per view, bit for bit. */
pcr_status pcr_batch_render(pcr_batch* batch, pcr_stream_t stream);

/* Records one frame (as pcr_batch_render) into a CUDA graph owned by the batch; pcr_batch_launch
 * replays it. Views set later with pcr_batch_set_views are used by later replays. */
pcr_status pcr_batch_capture(pcr_batch* batch, pcr_stream_t stream);

/* Launches the captured frame graph on `stream`. */
pcr_status pcr_batch_launch(pcr_batch* batch, pcr_stream_t stream);

/* Launch tuning of a batch's frames (the knobs of its autotuner). Results never depend on it. */
typedef struct {
  int32_t route;             /* 0 (default): automatic, single-view passes for frames of at most 4 views or clouds
                                of at least 10^8 points (outside graph capture), else the batch kernel; 1: always
                                the batch kernel; 2: always one single-view pass per view */
  int32_t slice_words;       /* batch kernel work item: 1 (default), 2 or 4 words of a view's chunk mask
                                (32, 64 or 128 chunks of 1024 points) */
  int32_t points_per_thread; /* points a thread classifies per step of the batch kernel: 1 (default) or 2 */
  int32_t blocks_per_sm;     /* 256-thread blocks per SM of the batch kernel, 1..32 (default 4; capped at the
                                blocks that can be resident) */
  int32_t merge_width;       /* 0 (default): one atomic per fragment; 8, 16 or 32: fragments of aligned groups of
                                that many lanes that land on one pixel are merged first (warp match + reduction) */
} pcr_batch_tuning;

/* Sets the tuning used by the batch's later frames (NULL restores the defaults). A captured frame is
 * re-captured by its next pcr_batch_launch (on that call's stream). */
pcr_status pcr_batch_set_tuning(pcr_batch* batch, const pcr_batch_tuning* tuning);

/* Current tuning of the batch. */
pcr_status pcr_batch_get_tuning(const pcr_batch* batch, pcr_batch_tuning* tuning);

/* Autotuner of the batched frame (the paper has no counterpart; its renderer has no tuning): renders the
 * batch's frame (its cloud, views, mode) with candidate tunings on `stream`, times each with CUDA events (the
 * best of two frames after one warm-up), and keeps the fastest in the batch. Candidates are explored one knob
 * at a time from the automatic route's choice (route 1/2, slice_words, points_per_thread, blocks_per_sm,
 * merge_width), keeping a change only when it is at least 2 % faster; two sweeps at most. The result is
 * remembered for the process under the key (GPU name, mode, power-of-two buckets of the frame's pixels, views
 * and points), and appended to the text file named by the environment variable PCR_AUTOTUNE_CACHE when it is
 * set; with force = 0 a remembered result for the key (from the process or that file) is applied without
 * timing anything. The frames rendered while tuning write the batch's framebuffers and images (as a render
 * would). Synchronises `stream`. Writes the chosen tuning to *best when best is not NULL. Needs the views set. */
pcr_status pcr_batch_autotune(pcr_batch* batch, pcr_stream_t stream, int32_t force, pcr_batch_tuning* best);

/* Visible-chunk counts of the last frame per view (host array of count entries; synchronises the
 * device). A diagnostic of the culling. */
pcr_status pcr_batch_visible_chunks(pcr_batch* batch, uint32_t* counts);

/* Frees the batch (synchronises the device). NULL is accepted. */
pcr_status pcr_batch_destroy(pcr_batch* batch);

/* ---------------------------------------------------------------------------------------------------
 * Rendering without device allocation. The paper has no counterpart: its renderer sets up its buffers
 * once and does not consider callers that cannot allocate.
 * ------------------------------------------------------------------------------------------------- */

#define PCR_NOALLOC_MAX_VIEWS 8
#define PCR_NOALLOC_MAX_POINTS 134217728ull /* 2^27 points (131072 chunks of 1024) */

/* One batched frame of count views of n points: the same images as pcr_cloud_create + pcr_batch_create +
 * pcr_batch_set_views + pcr_batch_render (always with the batched persistent launch), but the frame's
 * workspace (chunk bounds, visibility masks, per-view constants, counters) is a fixed device array inside libpcr, so
 * the call allocates nothing: no cudaMalloc, cudaFree or other allocating routine. It is meant for callers
 * that must not allocate while they render: a render loop in which a cudaMalloc or cudaFree would
 * synchronise the device and stall other streams; a process held to a fixed device-memory budget or to
 * its own allocator; code that must still render after an allocation has failed.
 *
 * d_points, n: 1..PCR_NOALLOC_MAX_POINTS points (caller-owned device memory, 16-byte aligned).
 * fbs, d_outs, views, count: 1..PCR_NOALLOC_MAX_VIEWS distinct framebuffers on the current device, their
 * output images (width * height u32 each) and views, as for pcr_batch_create and pcr_batch_set_views.
 * hq, eps_num, eps_den, background_rgba, clear_after: as for pcr_batch_create. A larger n or count returns
 * PCR_ERR_INVALID_ARG, with the limit in pcr_last_error_message(), and enqueues nothing.
 *
 * The array takes about 3.4 MB on every device that loads libpcr, until the process exits. The first call
 * on each device looks up the array's address (cudaGetSymbolAddress) with that device current. All calls
 * on a device share the one array, which keeps what the last call left in it (each call clears what must
 * start at zero). Calls whose work overlaps on the GPU (on different streams, or from different host
 * threads without ordering) race on the array and produce wrong images: put them on one stream or
 * synchronise between them. On the host, calls take a lock. */
pcr_status pcr_render_views_noalloc(const pcr_point* d_points, uint64_t n, pcr_framebuffer* const* fbs,
                                    uint32_t* const* d_outs, const pcr_view* views, int32_t count, int32_t hq,
                                    uint32_t eps_num, uint32_t eps_den, uint32_t background_rgba,
                                    int32_t clear_after, pcr_stream_t stream);

/* ---------------------------------------------------------------------------------------------------
 * Serving: continuous batching of render requests over resident clouds (no counterpart in the paper).
 * A server thread admits requests while framebuffer memory allows, merges requests that arrive while
 * others run into shared frames (same cloud, mode, epsilon and background), and runs frames on several
 * streams so that their work overlaps. Every image equals the single-request result bit for bit.
 * ------------------------------------------------------------------------------------------------- */

typedef struct pcr_server pcr_server;

typedef struct {
  int32_t streams;                   /* concurrent frames on the device, 1..16 */
  int32_t max_batch_views;           /* requests merged into one frame, 1..PCR_MAX_BATCH_VIEWS */
  uint64_t framebuffer_budget_bytes; /* device memory for the framebuffers of admitted requests (pooled) */
  uint64_t max_frame_point_views;    /* work cap of a merged frame: the sum over its requests of their
                                        cloud's point count (0: no cap). A frame always takes its first
                                        request, so one larger request still runs, alone. Bounds how long
                                        a frame holds its stream, hence the wait of requests behind it. */
} pcr_server_config;

typedef struct {
  int32_t cloud;            /* id from pcr_server_add_cloud */
  int32_t width, height;    /* 1..16384 */
  int32_t hq;               /* 0: basic (Section 2.1); 1: high-quality splatting (Section 2.2) */
  uint32_t eps_num, eps_den;
  uint32_t background_rgba;
  int32_t reserved;         /* must be 0 */
  pcr_view view;            /* LINEAR or METRIC, EXACT transform */
  uint32_t* d_out;          /* caller-owned device memory, width * height u32, written before completion */
} pcr_request;

typedef struct {
  uint64_t id;
  int32_t status;           /* pcr_status of the request */
  int32_t batch_views;      /* requests rendered in the same frame */
  double submit_s, start_s, done_s; /* steady-clock seconds since the server was created */
} pcr_completion;

/* Creates a server on the current device and starts its scheduling thread. */
pcr_status pcr_server_create(const pcr_server_config* config, pcr_server** out);

/* Registers a resident cloud (n caller-owned device points, kept unchanged while the server lives) and
 * returns its id. Synchronous (computes the culling bounds). */
pcr_status pcr_server_add_cloud(pcr_server* server, const pcr_point* d_points, uint64_t n, int32_t* cloud_id);

/* Queues a request; returns at once with its id. Arguments are checked here (PCR_ERR_INVALID_ARG). A
 * request larger than the whole framebuffer budget is rejected. The server's streams do not wait on the
 * caller's streams: the cloud's points must be complete and d_out unused until the request completes. */
pcr_status pcr_server_submit(pcr_server* server, const pcr_request* request, uint64_t* request_id);

/* Queues count requests at once (all or none: the first invalid one is reported and nothing is queued);
 * ids[i] receives request i's id. The scheduler sees them together, so requests of one group share frames. */
pcr_status pcr_server_submit_many(pcr_server* server, const pcr_request* requests, int32_t count, uint64_t* ids);

/* Moves up to max completions into out (oldest first); waits up to wait_ms milliseconds for at least one
 * when none is ready. *n_out = number written. */
pcr_status pcr_server_poll(pcr_server* server, pcr_completion* out, int32_t max, int32_t* n_out, int32_t wait_ms);

/* Finishes every submitted request, stops the thread and frees the server (clouds' points stay the
 * caller's). NULL is accepted. */
pcr_status pcr_server_destroy(pcr_server* server);

#ifdef __cplusplus
}
#endif

#endif /* PCR_H_ */
