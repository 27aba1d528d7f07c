/*
 * libstitch: GB300 (sm_103a) per-frame panoramic stitching path, C ABI.
 *
 * What the library computes.  The paper (Du et al., "GPU based Parallel Optimization for Real
 * Time Panoramic Video Stitching") describes the per-frame work only in words: each camera
 * frame is "cut and transformed" by the GPU according to pre-corrected parameters (Sec. 4.3,
 * Alg. 4 step 1), and the GPU then transforms the video and blends it into the panorama
 * (Alg. 4 step 6) with multi-band fusion to remove seams (Sec. 1, contribution 3).  Once
 * registration has fixed one homography per camera (Alg. 4 step 5, "transformation matrix"),
 * the library runs, for every frame:
 *   S1 inverse-homography warp of each frame into the canvas with bilinear sampling
 *      (coordinates clamped to the image; pixel centres at integer coordinates),
 *   S2 feather weights: distance to the source-image border, normalised over cameras,
 *   S3 Gaussian pyramids (separable 5-tap [1,4,6,4,1]/16, even-index decimation, reflect-101),
 *   S4 Laplacian bands (EXPAND with weights 2w(x-2k), reflect-101),
 *   S5 per-level blend of the bands by the weight pyramids, renormalised per level,
 *   S6 collapse, coverage mask, clamp to [0,1] and round-half-even to uint8 (or float out).
 * and, for alignment refinement, S7: the overlap photometric loss
 *      sum_{pixels} sum_{i<j} valid_i valid_j |I_i - I_j|^2 with I = gain * bilinear / 255
 *   and its gradient with respect to each camera's 8 canvas->camera homography entries and gain.
 *
 * Conventions common to every call:
 *  - Every pointer documented "device" is CUDA device memory of the device the rig was created
 *    on; "host" pointers are ordinary (preferably pinned) host memory.  The caller owns frames,
 *    outputs, parameters, loss and gradient buffers.  The library owns all scratch memory: it is
 *    allocated by stitch_rig_create / stitch_batch_create and released by the destroy calls;
 *    stitch_frames, stitch_backward and stitch_batch_frames never allocate.
 *  - Frames are RGB, 8 bits per channel, interleaved, rows `pitch` bytes apart (pitch >= 3*W).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All compute calls are
 *    asynchronous on that stream; no call synchronises the device except the create/destroy
 *    calls and stitch_frames_host (which returns after its output copy has completed).
 *  - Errors are reported only through the returned status; no call aborts or throws.  After a
 *    non-OK status from a compute call the outputs are undefined, and the rig stays usable
 *    unless the status is STITCH_ECUDA (a sticky CUDA error poisons the whole context).
 *  - A rig is not thread-safe: use one rig from one host thread and one stream at a time.
 *  - A call that takes a rig, batch or context runs on the device it was created on
 *    (stitch_frames_static: on the current device); no call changes the calling thread's current
 *    CUDA device.
 */
#ifndef STITCH_H
#define STITCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STITCH_OK = 0,
    STITCH_EINVAL = 1,      /* bad argument, descriptor or geometry */
    STITCH_ENOMEM = 2,      /* device or host allocation failed (create calls only) */
    STITCH_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    STITCH_ETIMEOUT = 4,    /* a bounded device-side wait gave up (batched schedule) */
    STITCH_EUNSUPPORTED = 5, /* valid request this build does not handle */
    STITCH_ETOOLARGE = 6     /* request needs more than the fixed static scratch (stitch_frames_static) */
} stitch_status;

/* Limits of this build. */
#define STITCH_MAX_CAMERAS 32
#define STITCH_MAX_LEVELS 12

/* Which implementation of the forward path a rig runs. */
#define STITCH_PATH_FUSED 0 /* fused kernels, pyramid levels kept on chip where they fit */
#define STITCH_PATH_PLAIN 1 /* one kernel per step, FP32 intermediates in HBM (comparison path) */

/* Level-0 blend weights (S2). FEATHER: w_i / sum_j w_j with w the distance to the image border.
 * SEAM: binary masks of the multiresolution spline: 1 for the pixel's owner, the lowest-index
 * camera whose feather weight is > 0 and >= (1 - 1e-9) times the largest, 0 for the others; the
 * owner is decided in FP64 when the rig is created (the pyramids then blend across the seams). */
#define STITCH_WEIGHTS_FEATHER 0
#define STITCH_WEIGHTS_SEAM 1

/* Canvas model. PLANAR: stitch_camera.H is the camera->canvas homography M (inverted by create).
 * CYLINDRICAL: canvas column x is the angle t = (x - cx)/f about the vertical axis and row y the
 * height (y - cy)/f on the unit cylinder; stitch_camera.H is then the camera's 3x3 matrix P
 * (= K R, row-major) that takes the canvas ray (sin t, (y - cy)/f, cos t) to homogeneous source
 * coordinates, used as given (w > 0 in front of the camera).  stitch_backward supports the
 * planar canvas only. */
#define STITCH_CANVAS_PLANAR 0
#define STITCH_CANVAS_CYLINDRICAL 1

typedef struct {
    int32_t width, height; /* source frame size in pixels, >= 1 */
    double H[9];           /* camera->canvas homography, row-major, with m31 u + m32 v + m33 > 0 for
                              the camera's pixels (points in front); its inverse is scaled internally
                              by 1/|a33|, so the canvas->camera map has a33 = +1 or -1 */
    float gain;            /* intensity gain applied to the sampled value (1 = unchanged) */
} stitch_camera;

typedef struct {
    int32_t num_cameras;          /* 1 .. STITCH_MAX_CAMERAS */
    const stitch_camera* cameras; /* host array of num_cameras entries (copied by create) */
    int32_t canvas_w, canvas_h;   /* output canvas size, >= 1 */
    int32_t levels;               /* pyramid levels counting level 0, 1 .. STITCH_MAX_LEVELS */
    int32_t band_fp16;            /* 0: FP32 pyramid storage; 1: FP16 storage of pyramid data
                                     between kernels (all filtering and blending still FP32) */
    int32_t out_float;            /* 0: uint8 RGB output; 1: float RGB output in [0,1] */
    int32_t path;                 /* STITCH_PATH_FUSED or STITCH_PATH_PLAIN */
    int32_t weights;              /* STITCH_WEIGHTS_FEATHER or STITCH_WEIGHTS_SEAM */
    int32_t canvas_model;         /* STITCH_CANVAS_PLANAR or STITCH_CANVAS_CYLINDRICAL */
    double cylinder[3];           /* cylindrical canvas: focal length f (> 0, px per radian), cx, cy */
} stitch_rig_desc;

typedef struct stitch_rig stitch_rig; /* opaque, owned by the library */

/*
 * Validate a rig, plan it and preallocate every buffer the per-frame path needs (the paper
 * precomputes grid/block sizes and static/dynamic memory at start-up, Sec. 4.3.2; this is the
 * counterpart).  Checks: each H is finite and invertible with a non-zero a33 after inversion;
 * each camera's footprint is bounded (w > 0 at the four corners of its image rectangle); w > 0
 * over every canvas region the camera's blend depends on.  `device` is the CUDA ordinal the rig
 * lives on; the caller's current device is restored on return.  On success *out receives the rig;
 * on failure *out is NULL.
 * Status: OK, EINVAL, ENOMEM, ECUDA.
 */
stitch_status stitch_rig_create(const stitch_rig_desc* desc, int device, stitch_rig** out);

/* Release a rig and all its device memory.  NULL-safe.  Synchronises the rig's device. */
void stitch_rig_destroy(stitch_rig* rig);

/*
 * Stitch one frame set (S1-S6).
 *   frames   host array of num_cameras DEVICE pointers, one RGB8 frame per camera
 *   pitches  host array of num_cameras row pitches in bytes (>= 3 * width)
 *   out      DEVICE canvas, canvas_h rows of canvas_w RGB pixels: uint8 (3 bytes per pixel) or
 *            float (12 bytes per pixel) as chosen by desc.out_float
 *   out_pitch  row pitch of `out` in bytes
 * Uncovered canvas pixels are written as 0.  Status: OK, EINVAL, ECUDA.
 */
stitch_status stitch_frames(stitch_rig* rig, const uint8_t* const* frames, const int64_t* pitches, void* out,
                            int64_t out_pitch, void* stream);

/*
 * Same as stitch_frames for HOST buffers: copies the frames host->device into rig-owned
 * staging buffers, stitches, copies the canvas device->host, and returns once `out` is written.
 * The staging buffers are allocated on the first call of this function for a rig (so this call,
 * unlike stitch_frames, may return STITCH_ENOMEM).  Pinned host memory gives asynchronous copies.
 */
stitch_status stitch_frames_host(stitch_rig* rig, const uint8_t* const* host_frames, const int64_t* pitches,
                                 void* host_out, int64_t out_pitch, void* stream);

/*
 * Asynchronous HOST-buffer variant with upload, stitching and download of consecutive calls
 * overlapped (the paper's stream strategy, Sec. 4.3.2 / Fig. 3b: the next frame is uploaded while
 * the current one is processed).  The call only enqueues work: `stream` waits for this call's
 * download, so the canvas in `host_out` is complete once `stream` has reached this point (e.g.
 * after cudaStreamSynchronize(stream)).  Host frames and `host_out` must stay valid and untouched
 * until then; pinned memory makes the copies asynchronous.  The upload is NOT ordered after work
 * queued earlier on `stream` (it reads host memory, which the caller has filled before the call).
 * The rig keeps two staging slots and three streams of its own, created by the first call (which
 * may therefore return ENOMEM).  The stitches run on the rig's compute stream and share the rig's
 * scratch with stitch_frames and stitch_backward: before switching between this call and those on
 * the same rig, let the earlier calls' work finish (synchronise their streams).
 * Status: OK, EINVAL, ENOMEM, ECUDA.
 */
stitch_status stitch_frames_host_async(stitch_rig* rig, const uint8_t* const* host_frames, const int64_t* pitches,
                                       void* host_out, int64_t out_pitch, void* stream);

/*
 * S7: overlap photometric loss and its gradient.
 *   params  DEVICE, num_cameras x 9 doubles per camera: a11 a12 a13 a21 a22 a23 a31 a32 gain of
 *           the canvas->camera map A whose a33 is the rig's (+1 or -1, see stitch_rig_get_camera).
 *           Validity masks are taken from these params.
 *   loss    DEVICE, 1 double: sum over canvas pixels and camera pairs i<j valid at the pixel of
 *           the squared RGB difference of the gained, bilinearly sampled [0,1] intensities
 *   grad    DEVICE, num_cameras x 9 doubles: d loss / d params, masks held constant (may be NULL)
 * Sampling coordinates are clamped to the image as in S1; the derivative along a clamped axis is 0.
 * Pixels where w <= 0 for a camera count as invalid for it.  Status: OK, EINVAL, ECUDA.
 */
stitch_status stitch_backward(stitch_rig* rig, const uint8_t* const* frames, const int64_t* pitches,
                              const double* params, double* loss, double* grad, void* stream);

/* Human-readable name of a status code (static string). */
const char* stitch_status_string(stitch_status s);

/*
 * Stitch one frame set with no device allocation at all (the paper has no counterpart; this is
 * a deployment convenience).  Callers that cannot call cudaMalloc (real-time loops that cannot
 * afford the allocator's implicit device synchronisation, hosts that hand the library a fixed
 * memory budget, plugins whose host application owns every device allocation) describe the rig in `desc`
 * and get the same result as a STITCH_PATH_PLAIN rig's stitch_frames: the plain-path kernels run
 * with every scratch buffer carved from one file-scope device array of STITCH_STATIC_SCRATCH_BYTES
 * (64 MiB) that each GPU loading the library holds until the process exits.
 *   desc     as for stitch_rig_create (path is ignored; band_fp16 must be 0); planned per call on
 *            the host stack, so each call also re-validates the geometry
 *   frames, pitches, out, out_pitch, stream   as for stitch_frames, on the CURRENT device
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it; make that first call before any stream capture.  Calls on a device
 * after cudaDeviceReset are not supported (the kept address belonged to the reset context).  Every
 * call shares the array and keeps the last call's contents; calls whose kernels overlap on the GPU
 * (other streams or host threads) race on it.  A rig
 * needing more scratch than the array holds returns STITCH_ETOOLARGE before any GPU work.
 * Status: OK, EINVAL, ETOOLARGE, ECUDA.
 */
#define STITCH_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
stitch_status stitch_frames_static(const stitch_rig_desc* desc, const uint8_t* const* frames, const int64_t* pitches,
                                   void* out, int64_t out_pitch, void* stream);

/* ------------------------------------------------------------------------------------------ */
/* Introspection and profiling                                                                 */

typedef struct {
    int64_t scratch_bytes;   /* device memory owned by the rig */
    int32_t num_kernels;     /* kernel launches per stitch_frames call */
    int32_t path;            /* STITCH_PATH_* actually used */
    int64_t roi_pixels;      /* sum over cameras of level-0 pixels the path evaluates */
    /* fused path: canvas tiles (64 x 32) by class, and camera tiles of the level-1 pass */
    int32_t tiles_zero;      /* no camera: written as 0 */
    int32_t tiles_solo;      /* one exclusive camera: the pyramid telescopes to its warp */
    int32_t tiles_full2;     /* blended, at most 2 cameras */
    int32_t tiles_full4;     /* blended, 3 or 4 cameras */
    int32_t tiles_general;   /* blended, more than 4 cameras */
    int32_t tiles_down1;     /* camera tiles that build Gaussian level 1 */
    int32_t tiles_down1_staged;    /* of which: source footprint staged in shared memory */
    int32_t tiles_down1_interior;  /* of which: one camera, weight 1, no coordinate clamping */
} stitch_rig_info;

stitch_status stitch_rig_get_info(const stitch_rig* rig, stitch_rig_info* info);

/*
 * Debug build only (libstitch_debug.so, compiled with STITCH_DEBUG; the paper has no counterpart):
 * a memory-safety check standing in for a sanitizer.  That build surrounds every rig allocation
 * with 256-byte guard bands of a NaN word and compiles index checks into the fused kernels, which
 * record the first check that fails and skip the access instead of trapping.  This call waits for
 * the rig's device, then reports the guard words that no longer hold the NaN word
 * (*damaged_words) and the first failed check as (code << 48 | value) (*failed_check, 0 when none;
 * reading it resets it).  Codes: 1 a source tap outside the staged footprint, 2 a footprint larger
 * than the staging capacity, 3 a REDUCE output before its camera's region, 4 a coarse output at a
 * negative position.
 * Status: OK, EINVAL, ECUDA; EUNSUPPORTED from the release build.
 */
stitch_status stitch_rig_debug_check(stitch_rig* rig, int64_t* damaged_words, int64_t* failed_check);

/*
 * The rig's canvas->camera map of camera `index` as used by every kernel: a[9] receives
 * A = H^-1 / |(H^-1)_33| (row-major, a[8] = +1 or -1); *visible is 0 when the camera's footprint
 * misses the canvas.  The first 8 entries and the camera gain are the stitch_backward params of
 * the rig's own geometry.
 */
stitch_status stitch_rig_get_camera(const stitch_rig* rig, int32_t index, double* a, int32_t* visible);

/*
 * Per-kernel CUDA-event timing of stitch_frames (events recorded on the call's stream around
 * every launch).  enable=1 starts accumulating; stitch_rig_kernel_times copies up to `cap`
 * entries: names (static strings), accumulated milliseconds and launch counts, returns the number
 * of distinct kernels in *count.  Reading synchronises the events.  enable=0 stops and resets.
 */
stitch_status stitch_rig_set_profiling(stitch_rig* rig, int enable);
stitch_status stitch_rig_kernel_times(stitch_rig* rig, const char** names, double* ms, int64_t* launches,
                                      int32_t cap, int32_t* count);

/* ------------------------------------------------------------------------------------------ */
/* L-ORB feature extraction (Sec. 4.1, Algorithms 1 and 2): the registration step before the    */
/* per-frame path.  Integer definition (bit-exact against the CPU oracle):                      */
/*   gray = (77 R + 150 G + 29 B + 128) >> 8; candidates inside the detection areas (Algorithm   */
/*   2, step 1) and at least 18 px from the image border; FAST-9 on the radius-3 circle with     */
/*   threshold fast_t (Algorithm 1, step 4); Ix, Iy central differences; A, B, C = their         */
/*   products weighted by the binomial [1,4,6,4,1]^2 (sigma = 1, unnormalised, step 3);          */
/*   R' = 25 (AB - C^2) - (A + B)^2 (25 x the Harris response with alpha = 0.04), kept when      */
/*   R' > harris_t (step 5); non-maximum suppression over the 8-neighbourhood, ties to the lower */
/*   index y W + x (step 6); the max_points strongest, R' descending then index ascending (step  */
/*   7); BRIEF (Sec. 4.1.2) bit k = [S(p + a_k) > S(p + b_k)] with S the binomial-smoothed gray   */
/*   and 256 point pairs given by the caller, stored LSB-first in 32 bytes per point.            */
/* ------------------------------------------------------------------------------------------ */

typedef struct stitch_lorb stitch_lorb; /* opaque: preallocated scratch for images up to a size */

typedef struct {
    int32_t fast_t;     /* FAST intensity threshold, >= 0 */
    int64_t harris_t;   /* keep R' > harris_t */
    int32_t max_points; /* N, <= the context's max_points */
} stitch_lorb_params;

/* Scratch for images up to max_width x max_height (each >= 37) and up to max_points (<= 2048)
 * points, on `device`.  Status: OK, EINVAL, ENOMEM, ECUDA. */
stitch_status stitch_lorb_create(int32_t max_width, int32_t max_height, int32_t max_points, int32_t device,
                                 stitch_lorb** out);
void stitch_lorb_destroy(stitch_lorb* ctx); /* NULL-safe; synchronises the device */

/*
 * Features of one RGB8 device frame (pitch bytes >= 3 width), asynchronous on `stream`.
 *   areas    host array of n_areas (<= 64) rectangles x0, y0, x1, y1 (half-open, image px)
 *   pattern  host array of 256 point pairs ax, ay, bx, by (each in [-15, 15])
 *   xy       device, 2 int32 per point (x, y); resp device, int64 R' per point;
 *   desc     device, 32 bytes per point (4-byte aligned); count device, number of points written
 * The context may serve one call at a time.  Status: OK, EINVAL, ECUDA.
 */
stitch_status stitch_lorb_detect(stitch_lorb* ctx, const uint8_t* frame, int32_t width, int32_t height, int64_t pitch,
                                 const int32_t* areas, int32_t n_areas, const stitch_lorb_params* params,
                                 const int8_t* pattern, int32_t* xy, int64_t* resp, uint8_t* desc, int32_t* count,
                                 void* stream);

/* ------------------------------------------------------------------------------------------ */
/* Feature matching and homography estimation (Sec. 4.2, Algorithm 3): Multi-Probe LSH over     */
/* BRIEF descriptors and PROSAC, bit-exact against the CPU oracle (integer decisions, and IEEE   */
/* double arithmetic without contractions in the order stated):                                  */
/*   M1 table l hashes a descriptor to the k bits bits[l*k + j] (bit j of the key = descriptor   */
/*      bit bits[l*k + j], LSB-first bytes); a query probes its own key and the k keys one bit   */
/*      away in each of the L tables; b1 = nearest probed descriptor of image B (Hamming, ties    */
/*      to the lower index), d2 = distance of the nearest other probed index; the query matches  */
/*      b1 when d1 <= max_dist and (no other, or ratio_den d1 < ratio_num d2);                   */
/*   M2 matches in quality order: d1 ascending, query index ascending;                           */
/*   M3 PROSAC (progressive sampling with the Chum-Matas growth schedule, m = 4, T_N = 200000):  */
/*      iteration t (0-based) draws 4 matches of the top n(t) from rnd[4t..4t+3] (the newest of  */
/*      the top n and 3 of the top n-1, or 4 of the top n once the schedule has passed; the      */
/*      j-th remaining index is taken for word w as j = w mod remaining); coordinates normalised */
/*      per image (centre and 2/extent of the matched points' bounding box); 4-point DLT, h33=1, */
/*      8x8 Gaussian elimination with partial pivoting (pivot magnitude >= 1e-12, else skipped); */
/*      inlier: w > 0 and squared transfer error < (inlier_px * scale_B)^2; best hypothesis:     */
/*      most inliers, ties to the earlier iteration; with >= 4 inliers, least squares on them   */
/*      (normal equations summed in quality order), de-normalised, h33 = 1.                     */
/* ------------------------------------------------------------------------------------------ */

typedef struct stitch_matcher stitch_matcher; /* opaque: preallocated scratch */

typedef struct {
    int32_t tables;    /* L, 1..32 */
    int32_t bits;      /* k, 1..20 */
    int32_t max_dist;  /* accept d1 <= max_dist */
    int32_t ratio_num; /* ratio test den * d1 < num * d2, both >= 1 */
    int32_t ratio_den;
    int32_t iters;     /* PROSAC iterations T, 0..the context's max_iters */
    double inlier_px;  /* inlier threshold in image-B pixels, > 0 */
} stitch_match_params;

/* Scratch for up to max_points (<= 2048) points per image and max_iters (<= 65536) PROSAC
 * iterations on `device`.  Status: OK, EINVAL, ENOMEM, ECUDA. */
stitch_status stitch_matcher_create(int32_t max_points, int32_t max_iters, int32_t device, stitch_matcher** out);
void stitch_matcher_destroy(stitch_matcher* ctx); /* NULL-safe; synchronises the device */

/*
 * Match image A's features to image B's and estimate the homography A -> B, asynchronously on
 * `stream`.  Device arrays: xy_a/xy_b 2 int32 per point; desc_a/desc_b 32 bytes per point
 * (4-byte aligned); count_a/count_b one int32 each (points used: min(count, max_points)) -- the
 * outputs of stitch_lorb_detect chain in directly.  Host arrays: bits (tables x bits bytes,
 * each a descriptor bit 0..255), params.  rnd: device, 4 uint32 per iteration.
 * Outputs (device): matches (3 int32 per match: index a, index b, distance; room for
 * max_points), n_matches (1 int32), H (9 doubles, row-major, h33 = 1; identity when no model),
 * n_inliers (1 int32; 0 when no model), inlier (1 byte per match).
 * The context may serve one call at a time.  Status: OK, EINVAL, ECUDA.
 */
stitch_status stitch_match_homography(stitch_matcher* ctx, const int32_t* xy_a, const uint8_t* desc_a,
                                      const int32_t* count_a, const int32_t* xy_b, const uint8_t* desc_b,
                                      const int32_t* count_b, const stitch_match_params* params, const uint8_t* bits,
                                      const uint32_t* rnd, int32_t* matches, int32_t* n_matches, double* H,
                                      int32_t* n_inliers, uint8_t* inlier, void* stream);

/* ------------------------------------------------------------------------------------------ */
/* Batching: several independent rigs stitched together, replacing per-rig launch sequences      */

typedef struct stitch_batch stitch_batch; /* opaque */

/*
 * Group rigs (all created on the same device, all STITCH_PATH_FUSED) into one batch.  The batch
 * builds a device work list over every rig's tiles, ordered so that each tile's inputs come from
 * earlier items, and preallocates its schedule state.  The rigs must outlive the batch.
 * Status: OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED.
 */
stitch_status stitch_batch_create(stitch_rig* const* rigs, int32_t n, stitch_batch** out);

/*
 * Stitch one frame set for every rig of the batch, with the schedule the batch chose on its first
 * call (stitch_batch_get_schedule): one persistent launch or the staged launches, replayed from a
 * CUDA graph, or every rig's own launch sequence on a stream of its own.
 *   frames       host array of n host arrays of DEVICE frame pointers (one per camera)
 *   pitches      host array of n host arrays of row pitches
 *   outs         host array of n DEVICE output canvases; out_pitches their row pitches
 * The first call times the candidate schedules on these frames and synchronises `stream`; later
 * calls are asynchronous on `stream` (no host synchronisation).  Device-side waits of the
 * persistent launch are bounded; a wait that gave up is reported as STITCH_ETIMEOUT by
 * stitch_batch_sync, or by a later stitch_batch_frames call once the failed call's work has
 * completed (that later call then launches nothing); the outputs of the failed call are undefined.
 * Status: OK, EINVAL, ECUDA, ETIMEOUT.
 */
stitch_status stitch_batch_frames(stitch_batch* batch, const uint8_t* const* const* frames,
                                  const int64_t* const* pitches, void* const* outs, const int64_t* out_pitches,
                                  void* stream);

/*
 * Wait until the batch's last stitch_batch_frames call has completed on the device and report its
 * outcome (and that of any earlier call not yet reported).  Status: OK, EINVAL, ECUDA, ETIMEOUT.
 */
stitch_status stitch_batch_sync(stitch_batch* batch);

void stitch_batch_destroy(stitch_batch* batch);

/*
 * The schedule the batch runs, chosen on its first stitch_batch_frames call by timing every
 * candidate on the real frames.  Candidates:
 *   - the cooperative persistent launch (stage ordering x register variant x tasks per dequeue),
 *     replayed from a CUDA graph;
 *   - the staged schedule (one launch per task type and level over all rigs, no device waits),
 *     replayed from a CUDA graph, with four tile-shape combinations for its REDUCE launches
 *     (32 x 16 outputs, or the column sweep of stitch_frames on 64 x 8) and coarse-level launches
 *     (32 x 32 or 64 x 16);
 *   - the per-rig streams (every rig's own launch sequence on a stream of its own, launched directly).
 * Environment: STITCH_TUNE=off skips timing (persistent defaults); =persistent, =staged or =streams
 * forces that mode (its parameters still timed); =full times even when a cached choice exists.
 * STITCH_TUNE_CACHE=<path> names a file of JSON lines keyed by the GPU's name and SM count and a hash
 * of every rig's description: a batch whose key is found takes the stored choice without timing,
 * and a timed choice is appended to it.
 * Encoding: bit 24 of *order is set when the choice came from the cache.  Below it, 0xE marks the
 * per-rig streams; a low nibble of 0xF the staged schedule, with bits 8-11 its tile shapes (bit 8:
 * 64 x 8 reduce tiles, bit 9: 64 x 16 coarse tiles); otherwise the persistent launch, with bits 0-3
 * the stage ordering (0 ranks every rig's stages from the start, 1 aligns them so every rig
 * finishes together), bits 4-7 the register variant (0: 2 resident blocks per SM, 1: 3) and bits
 * 8-23 the tasks a block dequeues at once.  *grid is the number of persistent blocks; *tasks the
 * number of tile tasks per call.
 */
stitch_status stitch_batch_get_schedule(const stitch_batch* batch, int32_t* order, int32_t* grid, int64_t* tasks);

/*
 * Test hook for the bounded device waits: sets the waits' iteration limit (default 2^22, about a
 * second) and, when rig >= 0, raises that rig's first-stage completion target out of reach so the
 * next stitch_batch_frames call gives up waiting and returns STITCH_ETIMEOUT; rig = -1 restores it.
 */
stitch_status stitch_batch_wait_test(stitch_batch* batch, int32_t spin_limit, int32_t rig);

#ifdef __cplusplus
}
#endif

#endif /* STITCH_H */
