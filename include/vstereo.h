/*
 * vstereo.h -- C ABI of the B300 (sm_103a) virtual-stereo hot path of
 * "Towards Real-time 3D Reconstruction using Consumer UAVs" (arXiv 1902.09733).
 *
 * One frame pair flows through four steps, each a hand-written CUDA kernel:
 *   vs_rectify_remap     Section 2.1 undistort/rectify remap, fused with the
 *                        Section 2.2 downsample to the stereo resolution
 *   vs_bp_stereo         Eq. 1 hierarchical min-sum belief propagation
 *   vs_guided_upsample   Eq. 2 joint bilateral upsampling to full resolution
 *   vs_reproject         Eq. 3 reprojection to a camera-frame point cloud
 * plus the fused Eq. 2 + Eq. 3 kernel and whole-pair drivers.
 *
 * Conventions shared by every entry point
 *  - Pointers are DEVICE pointers owned by the caller unless a parameter says
 *    "host".  The library never allocates device memory: scratch space is a
 *    caller-provided workspace whose size comes from the matching *_size call.
 *  - Images are row-major.  RGB images are interleaved R,G,B bytes; a pitch is
 *    the distance in bytes between the starts of two rows (>= the row bytes).
 *    Float outputs are contiguous (pitch = width elements).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call only enqueues work and returns; results are ready when the
 *    stream reaches that point.  The host-buffer driver is the one exception:
 *    it synchronises the stream before returning.
 *  - Every call checks its arguments on the host before launching anything
 *    and returns a status: VS_OK (0) or a negative VS_E* code; nothing is
 *    enqueued when a check fails.  VS_ECUDA reports a launch or copy error
 *    (cudaGetLastError after the launch); vs_status_string() names each code.
 *  - Calls on different streams that share a workspace or an output race.
 */
#ifndef VSTEREO_H
#define VSTEREO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VS_OK 0
#define VS_EINVAL (-1)      /* a size, count or parameter is out of range   */
#define VS_EALIGN (-2)      /* a pointer or pitch breaks an alignment rule  */
#define VS_EWORKSPACE (-3)  /* workspace NULL, misaligned or too small      */
#define VS_ECUDA (-4)       /* the CUDA runtime reported an error           */
#define VS_ETIMEOUT (-5)    /* a bounded wait inside a kernel ran out       */

/* Pinhole camera with radial distortion (Section 2.1 and Eq. 3), in pixels of
 * the full-resolution frame: focal lengths fx = f/du, fy = f/dv, principal
 * point (cx, cy) = (u0, v0), radial coefficients k1, k2 (no tangential term). */
typedef struct {
    float fx, fy, cx, cy, k1, k2;
} vs_camera;

/* Eq. 1 parameters.  Data term min(|IL - IR|, data_trunc); smoothness
 * min(smooth_slope * |dp - dq|, smooth_trunc); `labels` disparities
 * 0..labels-1 of the left image (IL(x) is compared with IR(x - d));
 * `levels` pyramid levels with `iters` red-black iterations each.
 * Ranges: w h <= 2^26 pixels, 2 <= labels <= 256, 1 <= levels <= 8,
 * 1 <= iters <= 1000, 0 <= smooth_slope, 0 <= smooth_trunc <= 65535,
 * 0 <= data_trunc with data_trunc * 4^(levels-1) <= 2^28.  Pairs with at
 * most 128 labels, data_trunc and smooth_trunc <= 127 and data_trunc *
 * 4^(levels-1) + 4 * smooth_trunc <= 32767 run the fast path (messages kept
 * in 8 bits, sums of a data term and four messages in 16-bit lanes); all
 * others run the general path (16-bit messages, 32-bit sums, one warp per
 * pixel, about half the speed per label), which computes the same
 * definition.
 * `iters_per_tile` (0..64) chooses how the iterations are launched, never
 * what they compute: 1 runs one kernel per iteration everywhere; k >= 2
 * runs up to k iterations per kernel on every level, each CTA iterating a
 * tile of the level in shared memory with a halo that shrinks by one pixel
 * per iteration (fewer than k where tile and halo would not fit shared
 * memory); 0 (automatic) runs fused tiles on the coarse levels where
 * vs_bp_autotune measured them faster for levels of that size, and on
 * coarse levels of at most 240 000 label-pixels (width x height x padded
 * labels) that it has not measured, one kernel per iteration elsewhere.  The workspace of k != 1 holds one more message
 * buffer (the largest level that may be fused).  The general path runs one
 * kernel per iteration whatever iters_per_tile says. */
typedef struct {
    int32_t labels, levels, iters, data_trunc, smooth_slope, smooth_trunc;
    int32_t iters_per_tile;
} vs_bp_params;

/* Eq. 2 parameters: `scale` s between the full-res and the low-res grid
 * (1..16); window of (2 radius + 1)^2 low-res pixels (0 <= radius <= 3);
 * spatial sigma in low-res pixels, range sigma on 0..255 RGB (both > 0). */
typedef struct {
    int32_t scale, radius;
    float sigma_s, sigma_r;
} vs_jbu_params;

/*
 * Section 2.1 + Section 2.2.  For every destination pixel (u, v) of the
 * W x H frame: the normalised ray ((u-cx)/fx, (v-cy)/fy) is rotated by R^T
 * (R9 = row-major 3x3 rectifying rotation, host pointer, NULL = identity, as
 * when the extrinsics are ignored), distorted by 1 + k1 r^2 + k2 r^4 and
 * mapped back through (fx, fy, cx, cy); the source is sampled bilinearly per
 * channel (taps outside the frame read 0) with the weights quantised to
 * 1/4096, rounded half up and clamped: within 0.06 of the exact bilinear
 * value before rounding, so within 1 of the exactly rounded byte.
 * Rays with a non-positive depth after the rotation give 0.  Arithmetic is
 * FP32.  Optionally the same kernel writes the low-resolution RGB
 * (ceil(W/s) x ceil(H/s), mean of the in-frame pixels of each s x s block,
 * rounded half up) and its grey (77 R + 150 G + 29 B + 128) >> 8.
 *   src, dst      W x H RGB; src_pitch, dst_pitch >= 3 W.  src and dst must
 *                 not overlap.
 *   scale         1..16; ignored when low_rgb and low_gray are both NULL.
 *   low_rgb       nullable, ceil(W/s) x ceil(H/s) RGB with low_rgb_pitch.
 *   low_gray      nullable, ceil(W/s) x ceil(H/s) bytes with low_gray_pitch.
 * Errors: VS_EINVAL (sizes <= 0, pitch too small, NULL src/dst/cam, bad
 * scale, non-finite camera), VS_ECUDA.
 */
int vs_rectify_remap(const uint8_t *src, int W, int H, int src_pitch,
                     const vs_camera *cam, const float *R9,
                     uint8_t *dst, int dst_pitch, int scale,
                     uint8_t *low_rgb, int low_rgb_pitch,
                     uint8_t *low_gray, int low_gray_pitch, void *stream);

/* Bytes of device workspace vs_bp_stereo needs for a w x h pair, or 0 when
 * the parameters are invalid.  The workspace holds the cost pyramid and the
 * message arrays of every level; it may be reused by consecutive calls on one
 * stream and needs no initialisation. */
size_t vs_bp_workspace_size(int w, int h, const vs_bp_params *p);

/*
 * Eq. 1 on a rectified, downsampled grey pair of w x h bytes (row pitch
 * `pitch` for both images).  Level 0 is w x h and every coarser level halves
 * rounding up; the coarse data term of a label is the sum over the in-frame
 * 2 x 2 children.  The coarsest level starts from zero messages and every
 * finer level from its parent pixel's messages (x>>1, y>>1).  At iteration t
 * of a level each pixel with (x + y + t) even sends to its in-frame
 * 4-neighbours the min-sum message of Eq. 1 (its data term plus the messages
 * from its other neighbours, minimised against the truncated-linear
 * smoothness, then shifted to minimum 0); missing neighbours contribute 0.
 * After the last level-0 iteration each pixel gets the smallest d minimising
 * its data term plus its four incoming messages.  Integer arithmetic: the
 * labels are exact, not approximations of a float computation.
 *   labels        w x h bytes out, row pitch labels_pitch >= w.
 *   workspace     >= vs_bp_workspace_size() bytes, 256-byte aligned.
 * Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA.
 */
int vs_bp_stereo(const uint8_t *left, const uint8_t *right, int w, int h, int pitch,
                 const vs_bp_params *p, uint8_t *labels, int labels_pitch,
                 void *workspace, size_t ws_bytes, void *stream);

/* vs_bp_stereo for callers that cannot allocate device memory -- code running
 * where cudaMalloc is off limits (inside a host allocator or memory-pool
 * callback, a plugin whose host owns every allocation, a tight real-time loop
 * that must not allocate).  The paper has no counterpart; this is a
 * deployment convenience.  It runs exactly vs_bp_stereo (same arguments, same
 * results) on a scratch array built into the library: VS_BP_NOALLOC_SCRATCH_BYTES
 * (8 MiB) of device memory that every GPU loading the library keeps until
 * the process exits.  That fits, for example, 320 x 180 with 16 labels and 3
 * levels (the paper's own setting) or 160 x 120 with up to 48 labels; a pair
 * whose vs_bp_workspace_size() exceeds it is rejected with VS_EWORKSPACE
 * before anything is enqueued.  The call allocates nothing.  Each call made
 * outside stream capture looks up the scratch address for the current device
 * (so a module the runtime loads again, e.g. after cudaDeviceReset, is
 * followed); a call during capture reuses the device's last address, so make
 * a device's first call before any stream capture.  All calls share the one
 * scratch and it keeps the last call's contents (nothing needs clearing
 * between calls); calls whose work overlaps on the GPU -- other streams,
 * other host threads -- race on it. */
#define VS_BP_NOALLOC_SCRATCH_BYTES (8u << 20)
int vs_bp_stereo_noalloc(const uint8_t *left, const uint8_t *right, int w, int h, int pitch,
                         const vs_bp_params *p, uint8_t *labels, int labels_pitch, void *stream);

/* vs_bp_status for vs_bp_stereo_noalloc, whose caller never sees the scratch:
 * synchronises `stream` and reports VS_ETIMEOUT if a kernel of the last
 * vs_bp_stereo_noalloc call (with the same w, h and parameters) gave up a
 * bounded wait (its labels are then invalid), else VS_OK.  No counterpart in
 * the paper.  Errors: VS_EINVAL, VS_EWORKSPACE (pair too large for the
 * scratch), VS_ECUDA. */
int vs_bp_noalloc_status(int w, int h, const vs_bp_params *p, void *stream);

/* One pair of a batch for vs_bp_stereo_batch (device pointers as in
 * vs_bp_stereo). */
typedef struct {
    const uint8_t *left, *right;
    int32_t w, h, pitch;
    vs_bp_params params;
    uint8_t *labels;
    int32_t labels_pitch;
} vs_bp_job;

/* Workspace bytes for a batch (the sum of the pairs' BP workspaces), or 0 if
 * a job is invalid or the jobs differ in levels or iters. */
size_t vs_bp_batch_workspace_size(const vs_bp_job *jobs, int n);

/*
 * Eq. 1 for n independent pairs of any sizes and label counts (1 <= n <=
 * 4096), exactly as n vs_bp_stereo calls would compute them.  Two schedules
 * (vs_bp_batch_mode): 0 (default) balances the pairs by size over four
 * library streams forked from `stream` and joined back to it with events,
 * so independent pairs fill each other's idle time; 1 advances all pairs in
 * lockstep, each level-iteration a handful of batched launches (one per
 * label count and kernel variant) whose pair descriptors travel in kernel
 * parameters -- a quarter of the launches, but every pair waits for the
 * largest at each sweep.  Either way the call is enqueued on / ordered after
 * `stream` and can be captured into a CUDA graph and replayed.  All jobs
 * must share `levels` and `iters`; `jobs` is a host array read during the
 * call.  The library streams are per device and shared: do not run batches
 * from several host threads at once.
 * Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA.
 */
int vs_bp_stereo_batch(const vs_bp_job *jobs, int n, void *workspace, size_t ws_bytes, void *stream);
/* Schedule of vs_bp_stereo_batch: 0 streams (default), 1 lockstep.
 * Errors: VS_EINVAL. */
int vs_bp_batch_mode(int mode);

/*
 * Autotuner for the message sweeps (no counterpart in the paper).  Runs
 * vs_bp_stereo on the given pair, then times the sweep kernels (plain,
 * register preload, labels split over two lanes, over four lanes when the
 * padded label count is a multiple of 64) on every level and records
 * the fastest per (padded label count, level size); later vs_bp_stereo and
 * vs_bp_stereo_batch calls on levels of those sizes use it.  Results are
 * identical whichever kernel runs.  Ends with a fresh vs_bp_stereo so labels
 * and workspace hold the pair's result.  Synchronises `stream`; do not call
 * it while the stream is being captured.  chosen (nullable, `levels` ints)
 * receives 0 plain, 1 preload, 2 split in two, 3 split in four per level.
 * vs_bp_autotune_reset
 * forgets every recorded choice.
 */
int vs_bp_autotune(const uint8_t *left, const uint8_t *right, int w, int h, int pitch, const vs_bp_params *p,
                   uint8_t *labels, int labels_pitch, void *workspace, size_t ws_bytes, void *stream, int *chosen);
/* The timings behind the last vs_bp_autotune: milliseconds per launch as
 * [level][variant] (4 per level, -1 where a variant does not apply), up to
 * `max` values written; returns the count. */
int vs_bp_autotune_times(float *ms, int max);
/* With p->iters_per_tile == 0 (automatic), vs_bp_autotune also times every
 * coarse level (level 0 stays one kernel per iteration in the automatic
 * mode), replayed from CUDA graphs, as one kernel per iteration against
 * fused launches of K = 2..10 iterations per tile on several tile shapes
 * and lane counts, and records
 * the fastest for levels of that size, labels and iterations; the
 * automatic mode then uses it.  This reports the last choices as
 * [level][4] = {K, tile_w, tile_h, lanes} (K = 0: one kernel per
 * iteration), up to `max` ints; returns the count. */
int vs_bp_autotune_plans(int *out, int max);
/* The level timings behind those choices, graph replays: [level][2] =
 * {ms of one kernel per iteration, ms of the fastest fused plan} (-1 where
 * not timed), up to `max` floats; returns the count. */
int vs_bp_autotune_level_times(float *ms, int max);
/* Test and measurement aid: run sweep variant `variant` (0 plain, 1 preload,
 * 2 split in two, 3 split in four, 4 staged) on every level where it
 * applies, ahead of any autotuned choice; -1 restores the automatic choice.
 * The staged variant (persistent CTAs that stream each tile's messages and
 * costs through shared memory with bulk asynchronous copies) applies to
 * single-pair sweeps after the first iteration of a level with byte costs
 * and byte-lane sums; by default it runs on such levels of at least 2^16
 * pixels, ahead of the autotuned choice.  Results are identical whichever
 * variant runs.  Errors: VS_EINVAL. */
int vs_bp_select_sweep(int variant);

/* Test and measurement aid for the fused sweeps (iters_per_tile != 1): every
 * fused launch from then on uses cores of tile_w x tile_h pixels (where tile
 * and halo fit shared memory) and `lanes` (1, 2 or 4) threads per direction
 * pair, each running the distance transform over labels / lanes labels;
 * 0, 0, 0 restores the library's own choice.  Results are identical for
 * every tile and lane count.  Errors: VS_EINVAL. */
int vs_bp_select_fused(int tile_w, int tile_h, int lanes);

/* Test aid for the bounded waits: with on = 1, staged sweeps launched from
 * then on announce their tile bytes to the mbarrier but issue no copy, so
 * each wait runs out (about a second per wait) and the call's status becomes
 * VS_ETIMEOUT, its labels invalid; on = 0 restores normal operation.  No
 * fault and no unbounded wait results.  Errors: VS_EINVAL. */
int vs_bp_test_withhold_copies(int on);

/* Synchronises `stream` and reports whether a kernel of the last
 * vs_bp_stereo call on this workspace gave up a bounded wait for its
 * shared-memory copies (VS_ETIMEOUT; the labels are then invalid), else
 * VS_OK.  Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA. */
int vs_bp_status(const void *workspace, size_t ws_bytes, int w, int h, const vs_bp_params *p, void *stream);
void vs_bp_autotune_reset(void);

/* Debug read-out after vs_bp_stereo on the same workspace and stream: the
 * final level-0 incoming messages as int32 [4][h][w][labels], directions
 * 0 = from the left neighbour, 1 = right, 2 = up, 3 = down (zero where the
 * neighbour is missing).  out is a device buffer of 16 h w labels bytes;
 * 4 h w labels must stay below 2^31. */
int vs_bp_export_messages(const void *workspace, size_t ws_bytes, int w, int h,
                          const vs_bp_params *p, int32_t *out, void *stream);

/*
 * Eq. 2.  Full-res pixel p = (x, y) of the W x H guide sits at the low-res
 * position p_down = ((x + 0.5)/s - 0.5, (y + 0.5)/s - 0.5); its window is the
 * (2r+1)^2 low-res pixels around round-half-up(p_down), clipped to the w x h
 * grid.  Weight of q: exp(-|p_down - q|^2 / (2 sigma_s^2)
 * - |I_p - I_q|^2 / (2 sigma_r^2)) with I_p the full-res RGB and I_q the
 * low-res RGB; disp = s * sum(w * label_q) / sum(w), in full-res pixels.
 * FP32, exponents taken relative to one of the largest weights of the window.
 *   labels        w x h bytes, pitch labels_pitch.
 *   guide_low     w x h RGB, pitch guide_low_pitch (the downsampled frame).
 *   guide_full    W x H RGB, pitch guide_full_pitch; w must equal ceil(W/s)
 *                 and h ceil(H/s).
 *   disp          W x H float out.
 * Errors: VS_EINVAL, VS_ECUDA.
 */
int vs_guided_upsample(const uint8_t *labels, int w, int h, int labels_pitch,
                       const uint8_t *guide_low, int guide_low_pitch,
                       const uint8_t *guide_full, int W, int H, int guide_full_pitch,
                       const vs_jbu_params *jp, float *disp, void *stream);

/*
 * Eq. 3.  For each pixel (u, v) with disparity d > 0 (full-res pixels):
 * z = fx B / d, x = (u - cx) B / d, y = (v - cy) (fx / fy) B / d; pixels with
 * d <= 0 or NaN give NaN in all three.  FP32.
 *   disp          W x H float.   xyz  W x H x 3 float out (x, y, z per pixel).
 * Errors: VS_EINVAL (sizes, baseline <= 0), VS_ECUDA.
 */
int vs_reproject(const float *disp, int W, int H, const vs_camera *cam, float baseline,
                 float *xyz, void *stream);

/* Eq. 2 followed by Eq. 3 in one kernel: the same arguments as the two calls
 * above; disp may be NULL when only the point cloud is wanted. */
int vs_guided_upsample_reproject(const uint8_t *labels, int w, int h, int labels_pitch,
                                 const uint8_t *guide_low, int guide_low_pitch,
                                 const uint8_t *guide_full, int W, int H, int guide_full_pitch,
                                 const vs_jbu_params *jp, const vs_camera *cam, float baseline,
                                 float *disp, float *xyz, void *stream);

/* Whole-pair configuration for the drivers below. */
typedef struct {
    int32_t W, H;           /* full-resolution frame size                  */
    vs_camera cam;          /* intrinsics + radial distortion              */
    float baseline;         /* metres between the two views                */
    vs_bp_params bp;        /* Eq. 1                                       */
    vs_jbu_params jbu;      /* Eq. 2; jbu.scale is also the downsample s   */
} vs_pair_config;

/* Bytes of device workspace for one pair: both rectified frames, their
 * low-res RGB and grey, the labels and the BP workspace.  0 if invalid. */
size_t vs_pair_workspace_size(const vs_pair_config *cfg);

/*
 * One virtual-stereo pair, device buffers: rectify + downsample both frames
 * (Section 2.1, 2.2), BP on the grey pair (Eq. 1), fused upsample and
 * reprojection of the left view (Eq. 2, Eq. 3).
 *   left_src, right_src   W x H RGB (pitch 3 W), device.
 *   disp                  nullable W x H float out.   xyz  W x H x 3 float out.
 * Errors: as the steps.
 */
int vs_pair_run(const vs_pair_config *cfg, const uint8_t *left_src, const uint8_t *right_src,
                float *disp, float *xyz, void *workspace, size_t ws_bytes, void *stream);

/* One pair of a whole-pair batch (device buffers as in vs_pair_run). */
typedef struct {
    vs_pair_config cfg;
    const uint8_t *left, *right;   /* W x H RGB (pitch 3 W) */
    float *disp;                   /* nullable W x H */
    float *xyz;                    /* W x H x 3 */
} vs_pair_job;

/* Workspace bytes for a whole-pair batch (the pairs' vs_pair_workspace_size
 * back to back, 256-byte aligned), or 0 if a job is invalid or n is not in
 * 1..4096. */
size_t vs_pair_batch_workspace_size(const vs_pair_job *jobs, int n);

/*
 * n independent pairs (remap of both frames, Eq. 1, Eq. 2 + Eq. 3), each
 * exactly as vs_pair_run computes it, with any sizes, downsample factors,
 * label counts and baselines.  The pairs are balanced, largest first, over
 * the device's four library streams forked from `stream` and joined back to
 * it with events, so the call is ordered after earlier work on `stream`,
 * later work waits for it, and it can be captured into a CUDA graph.  `jobs`
 * is a host array read during the call.  The library streams are shared by
 * the device's batch calls: do not run batches from several host threads at
 * once.  Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA, or a step's status.
 */
int vs_pair_run_batch(const vs_pair_job *jobs, int n, void *workspace, size_t ws_bytes, void *stream);

/*
 * The same pair from and to HOST buffers: copies both frames to the device,
 * runs vs_pair_run and copies the point cloud (and disp if non-NULL) back,
 * then synchronises `stream`.  Host buffers should be page-locked for full
 * copy speed.  `dev_in` is a device buffer of 2 * 3 W H bytes for the frames;
 * dev_xyz (W H 3 floats) and dev_disp (W H floats, nullable) are device
 * outputs the copies read back from.
 *   left_host, right_host   W x H RGB host input.
 *   xyz_host                W x H x 3 float host output.  disp_host nullable.
 */
int vs_pair_run_host(const vs_pair_config *cfg, const uint8_t *left_host, const uint8_t *right_host,
                     float *disp_host, float *xyz_host, uint8_t *dev_in, float *dev_disp, float *dev_xyz,
                     void *workspace, size_t ws_bytes, void *stream);

/*
 * Streaming drivers (overlap of host copies and compute across pairs).
 * A pipeline owns three CUDA streams (host->device copies, compute,
 * device->host copies) and `depth` rotating slots of device buffers, all
 * carved from the caller's workspace (vs_pipeline_workspace_size).  Submit
 * calls enqueue and return; a slot is reused only after its previous pair
 * has been copied back, so at most `depth` pairs are in flight and host
 * buffers handed to a submit must stay valid until that pair completes
 * (vs_pipeline_flush waits for all).  Host buffers should be page-locked.
 *  mode 0 (pairs):  vs_pipeline_submit_pair takes both W x H RGB frames of an
 *                   independent pair; results equal vs_pair_run.
 *  mode 1 (flight): vs_pipeline_submit_frame takes one new frame; frame f is
 *                   remapped once (Section 2.1, 2.2) into a ring of k + 1
 *                   rectified frames, and for f >= k the virtual stereo pair
 *                   (left = frame f - k, right = frame f, Section 3.2) runs
 *                   Eq. 1-3; its cloud (left camera) goes to xyz_host, which
 *                   may be NULL and is ignored while f < k.
 * vs_pipeline_latencies returns, oldest first, the milliseconds from the
 * start of each completed pair's input copy to the end of its output copy.
 * Errors: VS_EINVAL (config, mode, depth 1..16, k 1..64), VS_EWORKSPACE,
 * VS_ECUDA; after an error a pipeline refuses further submits.
 */
typedef struct vs_pipeline vs_pipeline;
size_t vs_pipeline_workspace_size(const vs_pair_config *cfg, int mode, int depth, int k);
int vs_pipeline_create(const vs_pair_config *cfg, int mode, int depth, int k, void *workspace, size_t ws_bytes,
                       vs_pipeline **out);
int vs_pipeline_submit_pair(vs_pipeline *p, const uint8_t *left_host, const uint8_t *right_host, float *xyz_host);
int vs_pipeline_submit_frame(vs_pipeline *p, const uint8_t *frame_host, float *xyz_host);
int vs_pipeline_flush(vs_pipeline *p);
int vs_pipeline_latencies(vs_pipeline *p, float *ms, int max);
void vs_pipeline_destroy(vs_pipeline *p);

/*
 * Temperature-smoothed BP and its adjoint (a differentiable relaxation of
 * Eq. 1; the paper itself only runs min-sum).  The minimum in the Eq. 1
 * message becomes the soft minimum at temperature tau:
 *   m_{r->p}(d) = -tau log sum_d' exp(-(h(d') + V(d, d')) / tau) - (its mean
 *                 over d),  h = D_r + the messages r received from its other
 *                 in-frame neighbours,  V(d, d') = min(lambda |d - d'|, trunc),
 * on one level, every message of iteration t computed from those of t - 1
 * (synchronous; all zero before the first), a missing neighbour sending
 * nothing.  Output after `iters` iterations: beliefs b_p(d) = D_p(d) + the
 * sum of p's incoming messages.  FP32 throughout; as tau -> 0 the messages
 * tend to the min-sum ones.
 *   cost          D, h x w x labels floats, label fastest (device, 16-byte
 *                 aligned).  Any finite values.
 *   beliefs       h x w x labels floats out (device, 16-byte aligned).
 *   labels        16, 32, 48 or 64.  iters 1..64.  w, h >= 1, w h <= 2^22.
 *   ckpt_every    k, 1..iters: the forward pass keeps the messages of every
 *                 k-th iteration in the workspace; the adjoint recomputes the
 *                 k - 1 iterations in between from them.
 *   lambda >= 0, trunc >= 0, tau > 0, trunc / tau <= 50 (keeps every
 *   exp(-V/tau) a normal FP32 number).
 * vs_sp_workspace_size gives the workspace bytes (0 for invalid arguments):
 * (floor((iters-1)/k) + min(k, iters) + 1) message states of 16 w h labels
 * bytes (each rounded up to 256), 32 bytes per 32 pixels (rounded up to 256)
 * and 256 bytes.  The workspace is 256-byte aligned device memory owned by
 * the caller.
 * The label contractions run as FP32 multiply-adds (SIMT kernels);
 * vs_sp_select_kernels(0) switches to tensor-core kernels (tcgen05 MMAs in
 * 3xTF32, about twice the rounding error, slower at 48 labels on B300) and
 * (1) back, for comparison (no counterpart in the paper).
 */
typedef struct {
    int32_t labels;
    int32_t iters;
    int32_t ckpt_every;
    float lambda;
    float trunc;
    float tau;
} vs_sp_params;

size_t vs_sp_workspace_size(int w, int h, const vs_sp_params *p);

/* Forward pass: beliefs, and the checkpoints the adjoint needs, in the
 * workspace.  Errors: VS_EINVAL, VS_EALIGN, VS_EWORKSPACE, VS_ECUDA. */
int vs_sp_forward(const float *cost, int w, int h, const vs_sp_params *p, float *beliefs,
                  void *workspace, size_t ws_bytes, void *stream);

/*
 * Adjoint: given grad_beliefs = dLoss/db (h x w x labels floats), writes
 * grad_cost = dLoss/dD (same shape, overwritten) and grad_params = device
 * array of 3 floats {dLoss/dlambda, dLoss/dtrunc, dLoss/dtau}.  The workspace
 * must hold the checkpoints of a vs_sp_forward with the same cost, sizes and
 * parameters, enqueued earlier (stream order); the adjoint overwrites all but
 * those checkpoints, so it may be run several times after one forward.  At a
 * kink lambda |d - d'| == trunc, V is taken as trunc (its derivative in
 * lambda is 0 there).  grad_params is summed in double in a fixed order, so
 * results are bit-identical from run to run.
 * Errors: VS_EINVAL, VS_EALIGN, VS_EWORKSPACE, VS_ECUDA.
 */
int vs_sp_backward(const float *cost, int w, int h, const vs_sp_params *p, const float *grad_beliefs,
                   float *grad_cost, float *grad_params, void *workspace, size_t ws_bytes, void *stream);

/* Kernel family for the two calls above: 1 SIMT (default), 0 tensor cores.
 * Errors: VS_EINVAL. */
int vs_sp_select_kernels(int family);

/* Test aid for the tensor-core kernels' bounded waits: with on = 1, their
 * launches from then on issue no MMA and no completion signal, so each
 * kernel's wait for its MMAs runs out (about a second, with nothing in
 * flight), the calls' outputs are invalid and vs_sp_status reports
 * VS_ETIMEOUT; on = 0 restores normal operation.  Errors: VS_EINVAL. */
int vs_sp_test_withhold_mma(int on);

/* Synchronises `stream` and reports whether a tensor-core kernel of the
 * vs_sp_forward / vs_sp_backward calls since the last vs_sp_forward on this
 * workspace gave up a bounded wait for its MMAs (VS_ETIMEOUT; its outputs are
 * then invalid).  Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA. */
int vs_sp_status(const void *workspace, size_t ws_bytes, int w, int h, const vs_sp_params *p, void *stream);

/* The checked build (no counterpart in the paper): libvstereo_checked.so is
 * built from the same sources with bounds checks on every global access of
 * the min-sum kernels, tested against the address ranges of the call's
 * buffers; the first access outside them is recorded and skipped, never
 * made.  vs_check_report returns 1 and writes {site, address} to
 * site_addr[0..1] (nullable) if an access was refused since the last
 * report, 0 if none, and -1 in the product library, which carries no
 * checks.  vs_check_test_shrink (test aid, checked build only) registers
 * the BP workspace `bytes` shorter than it is from the next call on, so that
 * an access to its end is refused without leaving the real buffer; 0
 * restores; VS_EINVAL in the product library.  The checked build registers
 * ranges with a synchronous copy per call: not for stream capture. */
int vs_check_report(unsigned long long *site_addr);
int vs_check_test_shrink(long long bytes);

/*
 * Pose between two frames (Section 2.3, Eq. 4-7): Harris corners of frame 1,
 * their matches in frame 2 by zero-mean SSD, and EPnP on the corners' 3D
 * points (from frame 1's point cloud) and the matched pixels.  The paper
 * uses it to re-estimate the relative pose of frames whose stereo
 * assumption fails and to chain point clouds along the flight.
 *   grid          cells per side (1..64); each cell keeps its strongest
 *                 corner (the paper divides the image into 30 x 30 cells).
 *   margin        corners lie at least this far inside the frame
 *                 (radius + 1 .. less than half the frame).
 *   threshold25   25 R must exceed this (R = det M - 0.04 tr(M)^2).
 *   radius        ZSSD patch radius r (1..8): (2r+1)^2 pixels.
 *   search        ZSSD displacements in [-search, search]^2 (0..32).
 */
typedef struct {
    int32_t grid, margin;
    int64_t threshold25;
    int32_t radius, search;
} vs_pose_params;

/* Workspace bytes of vs_harris_corners / vs_pose_estimate (0 if invalid):
 * the W H int64 response map and the per-cell corners, matches and points. */
size_t vs_pose_workspace_size(int W, int H, const vs_pose_params *p);

/* Eq. 4 + Eq. 5 at every pixel of a W x H RGB frame (pitch bytes per row):
 * A, B = central differences of the integer luma (77 R + 150 G + 29 B +
 * 128) >> 8 with the frame edge repeated; M = the 5 x 5 binomial window
 * ([1 4 6 4 1]^T [1 4 6 4 1], a discrete Gaussian; taps outside the frame
 * skipped) of [A^2, AB; AB, B^2]; r25 (W H int64 out) = 25 R = 25 det M -
 * tr(M)^2, exact.  Errors: VS_EINVAL, VS_ECUDA. */
int vs_harris_response(const uint8_t *rgb, int W, int H, int pitch, int64_t *r25, void *stream);

/* Section 3.2: corners (grid^2 x 2 int32 out, (x, y) per cell in row-major
 * cell order, -1 where none): in cell (gx, gy) -- x in [gx W / grid, (gx+1) W
 * / grid), y likewise -- the largest 25 R (the smaller raster index on ties)
 * among pixels inside the margin, above the threshold, that beat each of
 * their 8 neighbours in (R, then the smaller raster index).
 * Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA. */
int vs_harris_corners(const uint8_t *rgb, int W, int H, int pitch, const vs_pose_params *p, int32_t *corners,
                      void *workspace, size_t ws_bytes, void *stream);

/* Matches of n corners (n x 2 int32, -1 = none; n <= 4096) of frame 1 in
 * frame 2 (both W x H RGB, same pitch): the displacement d in [-search,
 * search]^2 with the (2r+1)^2 patch inside frame 2 minimising n Z = n sum D^2
 * - (sum D)^2 (D = patch 1 - patch 2 in luma, exact int64; the first in
 * raster order of (dy, dx) on ties), then on each axis the parabola through
 * the costs at d - 1 and d + 1 where both exist: pos (n x 2 double out,
 * NaN where none), cost (n int64 out, -1 where none).
 * Errors: VS_EINVAL, VS_ECUDA. */
int vs_zssd_match(const uint8_t *rgb1, const uint8_t *rgb2, int W, int H, int pitch, const int32_t *corners, int n,
                  const vs_pose_params *p, double *pos, int64_t *cost, void *stream);

/* Eq. 6 + Eq. 7 (EPnP, FP64): [R, T] with camera point = R P + T from world
 * points (n x 3 double) and their pixels (n x 2 double) in a camera of
 * intrinsics cam (fx, fy, cx, cy; no distortion); rows with a NaN are
 * skipped; 6 <= usable points, n <= 4096.  The points as weighted sums of
 * four control points (centroid and principal axes), the four smallest
 * eigenvectors of the 12 x 12 normal matrix of Eq. 6, N = 1, 2, 3 of them
 * refined by Gauss-Newton on the control-point distances, orthogonal
 * Procrustes, the smallest mean reprojection error; then twice again on the
 * points whose error is below max(2 px, 3 x the median) (the paper names no
 * outlier step).  out (14 doubles, device): R row-major, T, the mean
 * reprojection error of the inliers (px), the inlier count (NaN pose if
 * fewer than 6 usable points).  Errors: VS_EINVAL, VS_ECUDA. */
int vs_epnp(const double *points, const double *uv, int n, const vs_camera *cam, double *out, void *stream);

/* The whole pose step: vs_harris_corners on frame 1, their 3D points read
 * from xyz1 (frame 1's W x H x 3 float cloud, NaN where none, e.g. from
 * vs_pair_run), vs_zssd_match in frame 2, vs_epnp: out as vs_epnp, the pose
 * of camera 2 relative to camera 1 (camera-1 coordinates to camera-2
 * coordinates).  Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA. */
int vs_pose_estimate(const uint8_t *rgb1, const uint8_t *rgb2, const float *xyz1, int W, int H, int pitch,
                     const vs_camera *cam, const vs_pose_params *p, double *out, void *workspace, size_t ws_bytes,
                     void *stream);

/* Section 2.3 ("we calculate poses for both left and right images and
 * average them"): `left` and `right` (14 doubles each, device, as
 * vs_pose_estimate writes them) are the poses of a later stereo pair's left
 * and right cameras relative to frame 1's left camera.  The virtual rig puts
 * the right camera `baseline` metres along the left camera's +x with the
 * same orientation (p_right = p_left - (baseline, 0, 0)), so the right
 * estimate gives the left camera's pose as (R_right, T_right + b).  out (14
 * doubles, device): R = the chordal mean of the two rotations (the rotation
 * nearest to their sum, through the 3 x 3 eigen-decomposition of M^T M,
 * M = R_left + R_right), T = the mean translation, the mean of the two
 * reprojection errors, the sum of the inlier counts.  An estimate with a
 * non-finite R or T is left out (out = the other; all NaN and a count of 0
 * without either).  Errors: VS_EINVAL, VS_ECUDA. */
int vs_pose_average(const double *left, const double *right, double baseline, double *out, void *stream);

/* Workspace bytes of vs_pose_estimate_stereo (0 if invalid). */
size_t vs_pose_stereo_workspace_size(int W, int H, const vs_pose_params *p);

/* The averaged pose of a later stereo pair (left2, right2: W x H RGB, same
 * pitch as left1) relative to frame 1's left camera, whose cloud is xyz1:
 * the corners of left1 once, their ZSSD matches in left2 and in right2,
 * EPnP with its inlier rounds for each (as vs_pose_estimate), then
 * vs_pose_average with `baseline`.  out: 14 doubles as vs_pose_average.
 * Errors: VS_EINVAL, VS_EWORKSPACE, VS_ECUDA. */
int vs_pose_estimate_stereo(const uint8_t *left1, const uint8_t *left2, const uint8_t *right2, const float *xyz1,
                            int W, int H, int pitch, const vs_camera *cam, double baseline,
                            const vs_pose_params *p, double *out, void *workspace, size_t ws_bytes,
                            void *stream);

/* Name of a status code. */
const char *vs_status_string(int status);

/* Total number of kernels this library has enqueued since it was loaded. */
uint64_t vs_kernel_launches(void);

/* Measurement aid (no counterpart in the paper).  vs_profile_enable(n)
 * creates n pairs of CUDA events (0 switches timing off and frees them);
 * while on, each launch of the timed kernels is bracketed by an event pair
 * on its stream, also when the stream is being captured into a CUDA graph.
 * vs_profile_collect synchronises the pending pairs and writes up to `max`
 * (tag, milliseconds) records, oldest first, skipping pairs that have no
 * time (recorded during capture of a graph that has not run); it returns the
 * count.  Tags: 0 level-0 message sweep, 1 coarser-level sweep,
 * 2 remap, 3 upsample (+ reprojection), 4 other BP kernels (cost, pyramid,
 * labels), 5 smoothed-BP forward iteration, 6 smoothed-BP adjoint iteration.  Slots are reused round-robin, so collect before n more launches. */
int vs_profile_enable(int capacity);
int vs_profile_collect(int *tags, float *ms, int max);

#ifdef __cplusplus
}
#endif

#endif /* VSTEREO_H */
