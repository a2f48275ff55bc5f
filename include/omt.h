/*
 * omt.h -- C-ABI of the B300 (sm_103a) box-tracking hot path.
 *
 * The path moves each tracked box from frame t to frame t+1 (Section V-A of
 * the paper: preprocessing -> feature calculation -> prediction):
 *
 *   omt_build_pyramid   Gaussian pyramid + Scharr gradients of a u8 frame
 *   omt_corner_response Shi-Tomasi response of a whole frame (exact integers)
 *   omt_select_corners  Shi-Tomasi corners inside each box of frame t
 *   omt_lk_track        pyramidal Lucas-Kanade from frame t to frame t+1
 *   omt_update_boxes    per-box median (or mean) displacement
 *   omt_fb_check        forward-backward consistency of tracked points
 *   omt_level_u8        the working frame: a pyramid level chosen by resolution
 *
 * Conventions shared by every call
 *   - Pixel centres sit at integer coordinates; a level-L coordinate is the
 *     level-0 coordinate times 2^-L; level sizes are W_L = (W_{L-1} + 1) / 2.
 *   - Boxes are float4 (x0, y0, x1, y1), half-open, in level-0 pixels.
 *   - Points are float2 (x, y) in level-0 pixels.
 *   - Every pointer argument marked "device" must point to device memory of
 *     the current CUDA device.  The caller owns every buffer; the library
 *     never allocates or frees device memory.  One exception: the scratch
 *     of omt_select_corners_static is a fixed array inside the library
 *     (OMT_STATIC_SCRATCH_BYTES on every device that loads it).
 *   - Every call is asynchronous on the given stream (a cudaStream_t passed
 *     as void*, NULL = legacy default stream) with no host synchronisation.
 *   - Arguments are validated on the host before anything is launched; an
 *     invalid call returns OMT_EINVAL and launches nothing.  A failed launch
 *     returns OMT_ECUDA.
 *   - The only device-side waits are waits for tensor copies into shared
 *     memory: the LK kernels' window copies (omt_lk_track and the batched LK
 *     phase) and the pyramid kernels' tile copies (omt_build_pyramid and the
 *     batched pyramid phase).  Each gives up after one second and is
 *     counted; omt_lk_wait_timeouts then reports OMT_ETIMEOUT.  The LK points
 *     it concerns come back OMT_PT_LOST_TIMEOUT; a pyramid CTA whose wait ran
 *     out stops after landing its copies in flight, leaving its remaining
 *     tiles unwritten, so that pyramid must not be used.  No kernel can hang.
 *   - Calls on different streams may run concurrently from different host
 *     threads.  Mutable global state, all of it named here: the count of LK
 *     waits that ran out (omt_lk_wait_timeouts), the LK test hook
 *     (omt_debug_fail_lk_wait), a host cache of encoded TMA descriptors
 *     (thread-safe, keyed by buffer address and shape), and the array of
 *     omt_select_corners_static (calls of it must not overlap on the GPU).
 */
#ifndef OMT_H
#define OMT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */

enum omt_status {
    OMT_OK = 0,
    OMT_EINVAL = -1,   /* bad argument (checked on the host, nothing launched) */
    OMT_ENOMEM = -2,   /* a caller buffer is smaller than the call needs     */
    OMT_ECUDA = -3,    /* a CUDA launch or runtime call failed               */
    OMT_ETIMEOUT = -4, /* a bounded device wait ran out (omt_lk_wait_timeouts) */
    OMT_ECHECK = -5    /* a device-side consistency check failed             */
};

/* Storage of pyramid levels >= 1 and of all gradient planes.  Level 0 is
 * always the u8 frame.  Arithmetic is FP32 in both cases. */
enum omt_storage {
    OMT_F32 = 0, /* levels as float, gradients as float2                       */
    OMT_F16 = 1  /* levels as half(I - 128), gradients as half2 (intensity/px) */
};

/* Per-point status bits written by omt_lk_track (and LOST_FB by the
 * forward-backward check).  Exactly one of OK, LOST_EIG, LOST_OOB, LOST_FB,
 * LOST_TIMEOUT is set; NONCONV may accompany OK. */
enum omt_point_status {
    OMT_PT_OK = 1,       /* tracked                                            */
    OMT_PT_LOST_EIG = 2, /* lambda_min(G)/win^2 < min_eig (or <= 0) at a level */
    OMT_PT_LOST_OOB = 4, /* left the frame (see omt_lk_track)                  */
    OMT_PT_NONCONV = 8,  /* some level hit max_iter without converging (info)  */
    OMT_PT_LOST_FB = 16, /* tracked, but the round trip back did not close    */
    OMT_PT_LOST_TIMEOUT = 32 /* not tracked: a window copy the kernel waited  */
                             /* for did not land within one second (never in  */
                             /* normal operation); reported as its input      */
};

#define OMT_MAX_LEVELS 8
#define OMT_MIN_WIN 3
#define OMT_MAX_WIN 31
#define OMT_MAX_CORNERS 4096

/* ----------------------------------------------------------- parameters */

typedef struct omt_params {
    int32_t levels;      /* pyramid levels, 1..OMT_MAX_LEVELS                     */
    int32_t win;         /* LK window side, odd, OMT_MIN_WIN..OMT_MAX_WIN         */
    int32_t max_iter;    /* LK iterations per level, 1..255                       */
    float eps;           /* LK stops when |eta|^2 < eps^2 (level pixels), >= 0    */
    float min_eig;       /* tau: lost when lambda_min(G)/win^2 < tau, >= 0        */
    int32_t quality_num; /* corner quality as the exact rational num/den:          */
    int32_t quality_den; /*   candidate iff den * R > num * R_max(box)           */
    float min_dist;      /* corners keep dx^2 + dy^2 >= fl32(min_dist^2), >= 0    */
    int32_t max_corners; /* corners per box, 0..OMT_MAX_CORNERS                   */
    int32_t storage;     /* enum omt_storage                                      */
    int32_t aggregator;  /* 0 = median (default), 1 = mean (the paper's choice), */
                         /*   2 = median + median-flow scale (omt_update_boxes)  */
    float fb_max;        /* batched steps: forward-backward check threshold in    */
                         /*   level-0 px (omt_fb_check); < 0 = off (default)     */
} omt_params;

/* Defaults: 3 levels, 21x21 window, 30 iterations, eps 0.01, tau 1e-3,
 * quality 1/100, min distance 5, 50 corners, F32 storage, median, no
 * forward-backward check (fb_max -1). */
void omt_default_params(omt_params *p);

/* OMT_OK if every field is in range, else OMT_EINVAL. */
int omt_validate_params(const omt_params *p);

/* ---------------------------------------------------------------- pyramid */

typedef struct omt_level {
    int32_t w, h;        /* level size                                    */
    int64_t img_off;     /* byte offset of the image plane from base      */
    int64_t img_pitch;   /* bytes per image row (multiple of 128)         */
    int64_t grad_off;    /* byte offset of the (Ix, Iy) plane from base   */
    int64_t grad_pitch;  /* bytes per gradient row (multiple of 128)      */
} omt_level;

/* Describes one frame's pyramid inside a caller-owned device buffer.
 * Layout, level by level: image plane (level 0: u8; level >= 1: float or
 * half(I - 128)), then the gradient plane (float2 or half2, Ix then Iy, in
 * intensity per level pixel).  Every plane starts on a 256-byte boundary. */
typedef struct omt_pyramid {
    int32_t w, h, levels, storage;
    void *base;          /* device, caller-owned, 256-byte aligned        */
    size_t bytes;        /* size of the buffer at base                    */
    omt_level lv[OMT_MAX_LEVELS];
} omt_pyramid;

/* Bytes a pyramid of this shape needs (0 if the shape is invalid). */
size_t omt_pyramid_bytes(int32_t w, int32_t h, int32_t levels, int32_t storage);

/* Fill *pyr for a buffer of `bytes` bytes at device address `base`.
 * OMT_EINVAL on a bad shape or a misaligned base, OMT_ENOMEM if bytes is
 * smaller than omt_pyramid_bytes().  Host-only; launches nothing. */
int omt_pyramid_init(omt_pyramid *pyr, int32_t w, int32_t h, int32_t levels, int32_t storage,
                     void *base, size_t bytes);

/* Section V-A (preprocessing): build the pyramid of one u8 frame.
 *   frame  device, h rows of `pitch` bytes (pitch >= w), read only
 *   pyr    host struct from omt_pyramid_init with the same w, h; its levels
 *          and storage must equal prm->levels and prm->storage
 * Level 0 is a copy of the frame.  Level L >= 1 is the 5x5 binomial
 * ([1 4 6 4 1]/16 each way) of level L-1 with reflect-101 borders,
 * decimated to the even pixels.  Gradients per level:
 *   Ix = sum_d s_d (I(x+1, y+d) - I(x-1, y+d)) / 32, s = (3, 10, 3),
 *   Iy likewise, reflect-101.  In F32 storage levels 0..2 and the gradients
 * of levels 0..1 are exact (dyadic values); deeper levels carry FP32
 * rounding. */
int omt_build_pyramid(const uint8_t *frame, int32_t w, int32_t h, size_t pitch,
                      const omt_params *prm, const omt_pyramid *pyr, void *stream);

/* ---------------------------------------------------------------- corners */

/* Shi-Tomasi response of every pixel of a pyramid's level 0, exact:
 *   a, b, c = 3x3 sums (reflect-101) of gx^2, gx gy, gy^2 with the raw
 *   integer Scharr gx = 32 Ix, gy = 32 Iy of the u8 frame;
 *   R = (a + c) - isqrt((a - c)^2 + 4 b^2)   in [2 lambda_min, 2 lambda_min + 1).
 * out   device uint32[h * w] (row-major, no padding): bits 0..29 hold R,
 *       bit 30 is set where 1 <= x <= w-2, 1 <= y <= h-2 and R is >= each
 *       of its 8 neighbours (non-strict 3x3 maximum). */
int omt_corner_response(const omt_pyramid *pyr, uint32_t *out, void *stream);

/* Scratch bytes omt_select_corners needs for this frame size and box set:
 * the frame's response map (4 bytes per pixel; written only where a box has
 * more than 1,024 candidates), 8 bytes per box-corner slot, and per box a
 * list of up to 1,024 candidate keys (8 KiB) and two counters. */
size_t omt_corner_scratch_bytes(int32_t w, int32_t h, int32_t nboxes, int32_t max_corners);

/* Section V-A (feature calculation, sparse form): Shi-Tomasi corners of
 * frame t inside each box.  Per box, independently:
 *   eligible pixels  x0 <= x < x1, y0 <= y < y1, 1 <= x <= W-2, 1 <= y <= H-2;
 *   candidates       R > 0, den*R > num*R_max (R_max over the eligible pixels),
 *                    and a non-strict 3x3 maximum (neighbours may lie outside
 *                    the box);
 *   order            R descending, then raster index y*W + x ascending;
 *   greedy           keep a candidate if dx^2 + dy^2 >= fl32(min_dist^2) to
 *                    every point kept so far, stop at max_corners.
 * Arguments:
 *   pyr       frame t's pyramid (only level 0 is read)
 *   boxes     device float4[nboxes]
 *   scratch   device, >= omt_corner_scratch_bytes(), 256-byte aligned;
 *             contents on entry are ignored
 *   pts       device float2[nboxes * max_corners]: the kept corners of all
 *             boxes back to back in box order (integer-valued coordinates)
 *   offsets   device int32[nboxes + 1]: CSR, box b owns pts[offsets[b] ..
 *             offsets[b+1]); offsets[nboxes] is the total count
 * The result is deterministic and identical bit for bit to the definition. */
int omt_select_corners(const omt_pyramid *pyr, const float *boxes, int32_t nboxes,
                       const omt_params *prm, void *scratch, size_t scratch_bytes,
                       float *pts, int32_t *offsets, void *stream);

/* Bytes of the device array that omt_select_corners_static uses as scratch.
 * Every GPU that loads this library holds this much memory until the
 * process exits. */
#define OMT_STATIC_SCRATCH_BYTES (16u << 20)

/* omt_select_corners for callers that cannot allocate device memory.  The
 * paper has no counterpart; it exists for callers that only own their
 * inputs and outputs: a plugin inside an application that controls the CUDA
 * allocator, or a real-time loop that must not call cudaMalloc (which can
 * synchronise the whole device).  Same arguments and result as
 * omt_select_corners, minus the scratch: the scratch is one fixed array
 * (OMT_STATIC_SCRATCH_BYTES) inside the library.  It selects through the
 * whole response map (no candidate lists), which needs less scratch.
 *   - Returns OMT_ENOMEM when the scratch it needs exceeds
 *     OMT_STATIC_SCRATCH_BYTES (16 MiB): the frame's response map takes 4
 *     bytes per pixel, each box-corner slot (nboxes x max_corners) 8 more
 *     and each box 4 more (each of the three parts rounded up to 256
 *     bytes, plus one word): a 1920x1080 frame leaves room for about 1.05
 *     million slots (for example 1,000 boxes of 1,000 corners), a 3840x2160
 *     frame for none; the caller must then use omt_select_corners with its
 *     own scratch.
 *   - Allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *     routine.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array, and it keeps whatever the last call
 *     left in it; nothing in it needs to start at zero, because a call
 *     writes every scratch value before reading it.  Calls whose work
 *     overlaps on the GPU (different streams, or different host threads)
 *     race on the array and corrupt each other's results: serialise them. */
int omt_select_corners_static(const omt_pyramid *pyr, const float *boxes, int32_t nboxes,
                              const omt_params *prm, float *pts, int32_t *offsets,
                              void *stream);

/* --------------------------------------------------------------------- LK */

/* Pyramidal iterative Lucas-Kanade (Bouguet), standing in for the dense
 * motion field of Section V-A (feature calculation) / Section IV.
 * For each point u: g = 0 at the top level; for L = levels-1 .. 0:
 *   p = u 2^-L, N = win^2, w = (win-1)/2;
 *   G = sum over (i, j) in [-w, w]^2 of [Ix^2 IxIy; IxIy Iy^2], with I, Ix,
 *       Iy of frame t sampled bilinearly at p + (i, j) (taps clamped);
 *   LOST_EIG if lambda_min(G)/N < min_eig or lambda_min <= 0;
 *   nu = 0; for k = 1..max_iter:
 *       LOST_OOB if the centre c = p + g + nu leaves
 *           [-w, W_L-1+w] x [-w, H_L-1+w];
 *       b = sum (I(p + (i,j)) - J(c + (i,j))) (Ix, Iy), J frame t+1, bilinear;
 *       eta = G^-1 b; nu += eta; stop when eta_x^2 + eta_y^2 < eps^2;
 *   g = 2 (g + nu) for L > 0, else d = g + nu.
 * v = u + d, LOST_OOB if v is outside [0, W-1] x [0, H-1]; lost points
 * report v = u.  NONCONV marks a level that used all max_iter iterations.
 * Arguments:
 *   prev, next  pyramids of frames t and t+1 (same w, h, levels, storage,
 *               equal to prm->levels and prm->storage)
 *   pts         device float2[n_max]
 *   n_max       capacity of the point arrays (host value)
 *   n_dev       device int32 or NULL: if given, only min(*n_dev, n_max)
 *               points are tracked (lets the count come from
 *               omt_select_corners without a host round trip)
 *   pts_out     device float2[n_max]
 *   status      device uint8[n_max] (enum omt_point_status bits)
 *   iters       device uint8[n_max * levels] or NULL: iterations used per
 *               level, entry [i * levels + L]
 * Arithmetic is FP32 with a fixed reduction order: results do not depend on
 * the launch shape or on the other points of the batch. */
int omt_lk_track(const omt_pyramid *prev, const omt_pyramid *next, const float *pts,
                 int32_t n_max, const int32_t *n_dev, const omt_params *prm,
                 float *pts_out, uint8_t *status, uint8_t *iters, void *stream);

/* ------------------------------------------------------------- box update */

/* Section V-A (prediction): every box moves by an aggregate of the
 * displacements pts_out - pts of its OK points; its size is kept.
 * prm->aggregator 0: per-axis median (even count: mean of the two middle
 * values); 1: mean; 2: the median of 0 plus a scale, the median-flow
 * estimate (Kalal, Mikolajczyk and Matas, 2010): the median over all pairs
 * of the box's first 64 OK points (CSR order) of |v_i - v_j| / |u_i - u_j|
 * (u = pts, v = pts_out; FP32; pairs with u_i = u_j skipped; no pair: 1),
 * the box scaled by it about its centre, then moved.  A box without OK
 * points keeps its place, nvalid = 0.
 *   boxes      device float4[nboxes]
 *   offsets    device int32[nboxes + 1] CSR into the point arrays
 *   pts, pts_out, status   device, as written by omt_lk_track
 *   boxes_out  device float4[nboxes] (must not alias boxes)
 *   nvalid     device int32[nboxes] or NULL: OK points per box */
int omt_update_boxes(const float *boxes, const int32_t *offsets, const float *pts,
                     const float *pts_out, const uint8_t *status, int32_t nboxes,
                     const omt_params *prm, float *boxes_out, int32_t *nvalid, void *stream);

/* ------------------------------------------------------- working level
 * Section V-A (preprocessing): the frame is downscaled by the Gaussian
 * pyramid and a level chosen by its resolution is processed.  The working
 * frame of level L is the pyramid's level L rounded to u8; the whole path
 * (omt_build_pyramid, omt_select_corners, omt_lk_track, omt_update_boxes)
 * then runs on the working frames, with boxes in level-L pixels. */

/* Working level of a w x h frame: 0 up to 1280 px wide (SD, HD), 1 up to
 * 2560 (2K), 2 above (4K).  Host only. */
int32_t omt_working_level(int32_t w, int32_t h);

/* The working frame: level `level` of pyr rounded to u8,
 * clamp(floor(v + 0.5), 0, 255) (level 0: the frame itself), into out
 * (device, h_L rows of pitch >= w_L bytes).  pyr must use OMT_F32 storage,
 * whose levels 0-2 are exact, so the working frames of levels 0-2 are the
 * definition's bit for bit.  OMT_EINVAL on a bad pyramid or level.
 * Asynchronous on `stream`. */
int omt_level_u8(const omt_pyramid *pyr, int32_t level, uint8_t *out, size_t pitch,
                 void *stream);

/* boxes_out[i] = boxes[i] * scale (every coordinate); device float4[n],
 * 16-byte aligned (in place allowed).  For scale 2^-L and 2^L (exact),
 * boxes go to and from level-L pixels.  Asynchronous on `stream`. */
int omt_scale_boxes(const float *boxes, int32_t n, float scale, float *boxes_out, void *stream);

/* Forward-backward consistency of tracked points (the round-trip test of
 * Kalal, Mikolajczyk and Matas, 2010), a check on the prediction of Section
 * V-A: after omt_lk_track from frame t to t+1 (pts -> pts_out, status) and
 * back from t+1 to t (pts_out -> pts_back, status_back), every point whose
 * status has OK keeps it only if status_back has OK and its round trip
 * closes, sqrt(dx^2 + dy^2) <= fb_max with (dx, dy) = pts_back - pts (FP32,
 * level-0 px); otherwise its status becomes OMT_PT_LOST_FB (NONCONV
 * dropped).  Other statuses are left as they are.  pts, pts_back: device
 * float2[n]; status_back: device uint8[n]; status: device uint8[n], read
 * and written.  n = min(n_max, *n_dev) if n_dev (device int32) is given,
 * else n_max.  OMT_EINVAL on a NaN fb_max, n_max < 0 or a missing array.
 * Asynchronous on `stream`. */
int omt_fb_check(const float *pts, const float *pts_back, const uint8_t *status_back,
                 int32_t n_max, const int32_t *n_dev, float fb_max, uint8_t *status,
                 void *stream);

/* ---------------------------------------------------------------- batched */

/* Section V-B runs the phases of consecutive frames and of several models
 * concurrently; the batched form carries that to many independent video
 * streams: one step moves every stream's boxes from frame t to frame t+1
 * with one launch per kernel for all streams (a1-a8 in 4 + levels launches).
 * Each stream keeps its own pyramids, points and boxes resident on the
 * device; the step is described by a table packed on the host. */
#define OMT_BATCH_MAX_STREAMS 256

typedef struct omt_batch_stream {
    const uint8_t *frame;  /* device, frame t+1: h rows of frame_pitch bytes        */
    size_t frame_pitch;    /* >= w                                                  */
    omt_pyramid prev;      /* frame t's pyramid (built by an earlier step)          */
    omt_pyramid next;      /* receives frame t+1's pyramid (same shape as prev)     */
    const float *boxes;    /* device float4[nboxes], boxes on frame t               */
    int32_t nboxes;        /* >= 0                                                  */
    int32_t max_corners;   /* per-box corner cap of this stream, <= caps max        */
    void *scratch;         /* device, 256-aligned, omt_corner_scratch_bytes(...)    */
    size_t scratch_bytes;
    float *pts;            /* device float2[nboxes * max_corners]                   */
    float *pts_out;        /* device float2[nboxes * max_corners]                   */
    uint8_t *status;       /* device uint8[nboxes * max_corners]                    */
    uint8_t *iters;        /* device uint8[nboxes * max_corners * levels] or NULL   */
    int32_t *offsets;      /* device int32[nboxes + 1] (CSR of pts per box)         */
    float *boxes_out;      /* device float4[nboxes], must not alias boxes           */
    int32_t *nvalid;       /* device int32[nboxes] or NULL                          */
    float *pts_back;       /* device float2[nboxes * max_corners]: the backward    */
    uint8_t *status_back;  /*   run of the forward-backward check (prm->fb_max >= 0;*/
                           /*   else may be NULL)                                   */
} omt_batch_stream;

/* Capacities a packed table must fit; the launch grids depend on these
 * only, so one captured CUDA graph serves any membership within them. */
typedef struct omt_batch_caps {
    int32_t max_streams;  /* 1..OMT_BATCH_MAX_STREAMS                 */
    int32_t max_boxes;    /* boxes summed over the streams, >= 0      */
    int32_t max_w, max_h; /* largest frame                            */
    int32_t max_corners;  /* largest per-box cap, <= OMT_MAX_CORNERS   */
    /* Launch shape of the batched LK kernel, 0 = the library default: warps
     * per CTA (1..8; default 4), CTAs per SM (0..32; 0 = as many as fit),
     * points a warp takes at a time from the launch's work queue (1..16;
     * default 1).  No result depends on them (each point is computed by one
     * warp in a fixed order), so a tuner may pick any; an autotuner in the
     * Python binding times the candidates on the caller's own batch. */
    int32_t lk_warps, lk_ctas_per_sm, lk_chunk;
    /* CTAs per SM (0..32; 0 = as many as fit) of the pyramid kernels, of the
     * corner-list kernel and of the select kernel: fewer CTAs take more
     * tiles, strips or boxes each.  No result depends on them either. */
    int32_t pyr_ctas_per_sm, corner_ctas_per_sm, select_ctas_per_sm;
    int32_t reserved;     /* 0 */
} omt_batch_caps;

/* Bytes of a packed table (host) and of its device copy (0 on bad caps). */
size_t omt_batch_table_bytes(const omt_batch_caps *caps);

/* Host only: validate nstreams stream descriptions against prm and caps and
 * pack them into `table` (host memory, >= omt_batch_table_bytes).  Every
 * check of omt_build_pyramid / omt_select_corners / omt_lk_track /
 * omt_update_boxes applies per stream; the first failure returns OMT_EINVAL
 * (or OMT_ENOMEM for a short scratch) and leaves `table` unusable. */
int omt_batch_pack(const omt_batch_stream *streams, int32_t nstreams, const omt_params *prm,
                   const omt_batch_caps *caps, void *table, size_t table_bytes);

/* One step for every stream of a packed table: copies the table to
 * dev_table (device, 256-aligned, >= omt_batch_table_bytes) with one
 * cudaMemcpyAsync on `stream`, then builds every frame t+1 pyramid, selects
 * every stream's corners on frame t, tracks all points in one persistent
 * LK launch and updates every box.  Results per stream equal the plain
 * calls' bit for bit.  `table` is read when the copy executes: keep it
 * unchanged until then; under stream capture it must be page-locked host
 * memory, and a replay copies its contents at replay time. */
int omt_batch_step(const void *table, const omt_batch_caps *caps, const omt_params *prm,
                   void *dev_table, size_t dev_table_bytes, void *stream);

/* The same step in pieces, for callers that interleave the phases of
 * consecutive steps (e.g. the next frames' pyramids while this step's
 * points are tracked, Section V-B) or time them separately:
 * omt_batch_upload copies `table` to dev_table; omt_batch_phase runs one
 * phase on an uploaded table.  Phases must run in order on the table's data
 * (the corners read frame t's pyramid, LK reads both pyramids and the
 * corners, the box update reads LK's results). */
enum omt_batch_phase_id {
    OMT_PHASE_PYRAMID = 0, /* frame t+1 pyramids of every stream          */
    OMT_PHASE_CORNERS = 1, /* response maps, selection, CSR compaction    */
    OMT_PHASE_LK = 2,      /* one persistent launch over all points       */
    OMT_PHASE_BOXES = 3,   /* per-box median / mean update                */
    OMT_PHASE_FB = 4       /* backward LK from frame t+1 to t and the     */
                           /*   forward-backward check (between LK and    */
                           /*   BOXES; a no-op when prm->fb_max < 0)      */
};
int omt_batch_upload(const void *table, const omt_batch_caps *caps, void *dev_table,
                     size_t dev_table_bytes, void *stream);
int omt_batch_phase(const void *dev_table, const omt_batch_caps *caps, const omt_params *prm,
                    int32_t phase, void *stream);

/* ------------------------------------------------- dense flow engine
 * Section IV: the paper's flow is a dense TV-L1 field (L1 data term, total
 * variation with the Huber norm, a primal-dual projected gradient scheme)
 * on frames preprocessed by a structure-texture decomposition; Section V-A
 * moves each box by the mean of the field inside it.  The paper gives no
 * parameters; omt_default_flow_params holds the readings used here. */
typedef struct omt_flow_params {
    float st_theta;   /* ROF weight of the structure (Chambolle's projection)   */
    float st_alpha;   /* texture = I - st_alpha * structure                      */
    float st_k;       /* u8 texture = clamp(floor(st_k * texture + 128.5))       */
    int32_t st_iters; /* projection steps (step 1/8), >= 0                      */
    float lambda;     /* weight of the L1 data term (intensities scaled to [0,1])*/
    float eps;        /* Huber parameter of the total variation, >= 0           */
    int32_t warps;    /* warps per pyramid level, >= 1                          */
    int32_t iters;    /* primal-dual iterations per warp, >= 1                  */
    int32_t block;    /* projection steps and primal-dual iterations carried  *
                       * out per kernel launch: 1 or 2.  The results are the  *
                       * same bit for bit; 2 reads and writes the state once  *
                       * per two steps (temporal blocking).                   */
} omt_flow_params;

/* Defaults: st_theta 1/8, st_alpha 0.95, st_k 2, 100 steps; lambda 10,
 * eps 0.05, 3 warps, 30 iterations; 2 per launch. */
void omt_default_flow_params(omt_flow_params *p);

/* Device scratch bytes of omt_structure_texture / omt_tvl1_flow. */
size_t omt_structure_texture_scratch_bytes(int32_t w, int32_t h);
size_t omt_tvl1_scratch_bytes(int32_t w, int32_t h);

/* The u8 texture image of a u8 frame (device, h rows of pitch bytes) into
 * texture (device, h rows of tpitch >= w bytes): the ROF structure S by
 * st_iters steps of Chambolle's dual projection (forward differences, zero
 * at the last row and column; the divergence their negative adjoint), then
 * clamp(floor(st_k (I - st_alpha S) + 128.5), 0, 255), all in FP32.
 * scratch: device, >= omt_structure_texture_scratch_bytes.  Asynchronous. */
int omt_structure_texture(const uint8_t *frame, int32_t w, int32_t h, size_t pitch,
                          const omt_flow_params *fp, uint8_t *texture, size_t tpitch,
                          void *scratch, size_t scratch_bytes, void *stream);

/* Dense Huber-TV-L1 flow from prev (frame t) to next (frame t+1), pyramids
 * of the same shape in OMT_F32 storage (built by omt_build_pyramid, e.g. of
 * texture images), into flow (device float2[w * h], level-0 px, row-major).
 * Per level, coarse to fine: the flow of the level above sampled bilinearly
 * at (x/2, y/2) and doubled (zero at the top), the duals restarted at zero;
 * per warp, frame t+1 and its gradient sampled bilinearly at x + u0 (taps
 * clamped); per iteration (sigma = tau = 1/sqrt(8)) the duals of each flow
 * component p <- P((p + sigma grad ubar) / (1 + sigma eps)), P the
 * projection onto the unit disc, then u <- the pointwise prox of
 * tau lambda |rho| at u + tau div p, ubar = 2 u - u_previous.  flow also
 * serves as working storage of the coarser levels; when the call's work
 * completes it holds the level-0 field.
 * scratch: device, >= omt_tvl1_scratch_bytes.  Asynchronous. */
int omt_tvl1_flow(const omt_pyramid *prev, const omt_pyramid *next, const omt_flow_params *fp,
                  float *flow, void *scratch, size_t scratch_bytes, void *stream);

/* Section V-A prediction from the dense field: box b moves by the mean flow
 * over the pixels x0 <= x < x1, y0 <= y < y1 of the frame (a box without
 * such pixels stays).  flow: device float2[w * h]; boxes, boxes_out: device
 * float4[nboxes], 16-byte aligned.  Asynchronous. */
int omt_box_mean_flow(const float *flow, int32_t w, int32_t h, const float *boxes,
                      int32_t nboxes, float *boxes_out, void *stream);

/* ------------------------------------------------- matching and update
 * Section V-A, matching phase: the predicted scene objects S_t are matched
 * against the detections D_t by a globally optimal assignment (the
 * Hungarian method, Kuhn 1955) with the IoU as score; update phase: scene
 * objects that find no match are flagged lost (kept, excluded from further
 * processing), detections that find none become new scene objects.  Boxes
 * are half-open (x0, y0, x1, y1) floats. */

/* IoU of every pair (a[i], b[j]) into iou[i * nb + j] (device, row-major
 * doubles): area = max(x1 - x0, 0) * max(y1 - y0, 0) per box, the
 * intersection's extents clipped at 0, union = (area_a + area_b) - inter,
 * IoU = inter / union (0 for an empty union), every operation a single
 * rounded FP64 operation (no fused multiply-add), so the matrix is the
 * same bit for bit on any IEEE machine that keeps that order.  a, b: device,
 * 16-byte aligned; na, nb >= 0 (0 is a no-op).  Asynchronous on `stream`. */
int omt_iou_matrix(const float *a, int32_t na, const float *b, int32_t nb, double *iou,
                   void *stream);

/* Host only.  Host workspace bytes for omt_assign on an na x nb matrix. */
size_t omt_assign_workspace_bytes(int32_t na, int32_t nb);

/* Host only.  Maximum-total-IoU assignment of the rows of `iou` (host,
 * na x nb doubles) to its columns; rows with active[i] == 0 take no part
 * (active may be NULL: all rows).  The matrix is padded to a square with
 * zero scores; a row and a column count as matched only when their
 * assigned IoU exceeds iou_min.  match_a[i] = column or -1, match_b[j] = row
 * or -1.  Among several optimal assignments the one returned is a fixed
 * function of the matrix.  OMT_ENOMEM if workspace_bytes is short. */
int omt_assign(const double *iou, int32_t na, int32_t nb, const uint8_t *active, double iou_min,
               void *workspace, size_t workspace_bytes, int32_t *match_a, int32_t *match_b);

/* Host only.  Update phase: entry i < ns of the output is scene object i,
 * with its detection's box and active = 1 when it is active and matched,
 * else its own box and active = 0 (lost, or lost before); the detections
 * that match no scene object follow, active.  boxes_out holds ns + nd
 * boxes, active_out ns + nd flags; *n_out receives the new count. */
int omt_update_tracks(const float *boxes_s, const uint8_t *active_s, int32_t ns,
                      const float *boxes_d, int32_t nd, const int32_t *match_s,
                      const int32_t *match_d, float *boxes_out, uint8_t *active_out,
                      int32_t *n_out);

/* ---------------------------------------------------------------- misc */

/* Synchronous (waits for the device).  *count receives the number of LK
 * window-copy waits (omt_lk_track and the batched LK phase, one per warp
 * and wait) that reached their time limit (one second) since the previous
 * call, and the count restarts at 0; returns OMT_ETIMEOUT when it is not 0,
 * else OMT_OK.  A copy lands in microseconds, so a non-zero count means the
 * copy engine stalled.  No point is computed from a window that did not
 * land: the warp whose wait ran out stops copying and reading windows,
 * waits (again at most a second) for its other copies, and reports every
 * point it held OMT_PT_LOST_TIMEOUT at its input position with zero
 * iterations (in the plain call, all its later points too; in the batched
 * step, the rest of its queue chunk, after which it takes no more work; a
 * point whose backward run was lost so becomes OMT_PT_LOST_TIMEOUT in the
 * forward-backward check).  The count also includes the pyramid kernels'
 * tile waits that ran out (their CTA stopped, leaving tiles of that pyramid
 * unwritten).  The count is process-global.  OMT_EINVAL if count is NULL;
 * OMT_ECUDA on a CUDA error. */
int omt_lk_wait_timeouts(uint32_t *count);

/* Test hook of the wait-failure path (synchronous, current device): from
 * now on, the point with index `point` -- in omt_lk_track its index in pts,
 * in the batched LK phase its position in the step's work queue (the
 * streams' points back to back in stream order) -- declares its first
 * search-window copy 16 bytes larger than the copy delivers, so that its
 * wait runs out after one second with every copy landed and the failure
 * path above runs.  point = -1 (the initial state) turns it off.  The paper
 * has no counterpart.  OMT_ECUDA on a CUDA error. */
int omt_debug_fail_lk_wait(int64_t point);


const char *omt_error_string(int32_t code);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t omt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OMT_H */
