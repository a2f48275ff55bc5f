// omt_internal.cuh -- device helpers and launcher declarations shared by the
// kernels of libomt.  Not part of the public C-ABI (see include/omt.h).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "omt.h"

namespace omt {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Reflect-101 index: mirror about the edge pixel without repeating it, folded
// into [0, n) for any offset; a one-pixel axis maps everything to 0.
__host__ __device__ __forceinline__ int reflect101(int i, int n) {
    if (i >= 0 && i < n) return i;
    if (n == 1) return 0;
    const int period = 2 * n - 2;
    i %= period;
    if (i < 0) i += period;
    return i < n ? i : period - i;
}

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// Integer pixel range [xlo, xhi] x [ylo, yhi] of the pixels a box makes
// eligible for corner selection: x0 <= x < x1, y0 <= y < y1 (float box,
// exact integer comparison) intersected with [1, w-2] x [1, h-2].
// Returns false when the range is empty (including NaN coordinates).
__host__ __device__ __forceinline__ bool box_pixel_range(float4 b, int w, int h, int &xlo,
                                                         int &xhi, int &ylo, int &yhi) {
    if (!(b.x <= b.z) || !(b.y <= b.w)) return false;  // also rejects NaN
    const float lim_x = (float)w + 2.0f, lim_y = (float)h + 2.0f;
    float x0 = fminf(fmaxf(b.x, -2.0f), lim_x), x1 = fminf(fmaxf(b.z, -2.0f), lim_x);
    float y0 = fminf(fmaxf(b.y, -2.0f), lim_y), y1 = fminf(fmaxf(b.w, -2.0f), lim_y);
    xlo = (int)ceilf(x0);
    xhi = (int)ceilf(x1) - 1;
    ylo = (int)ceilf(y0);
    yhi = (int)ceilf(y1) - 1;
    xlo = xlo < 1 ? 1 : xlo;
    ylo = ylo < 1 ? 1 : ylo;
    xhi = xhi > w - 2 ? w - 2 : xhi;
    yhi = yhi > h - 2 ? h - 2 : yhi;
    return xlo <= xhi && ylo <= yhi;
}

// One level of a pyramid as the kernels see it.
struct LevelView {
    const uint8_t *img;   // level 0: u8; else float or half(I-128)
    const uint8_t *grad;  // float2 or half2 (Ix, Iy)
    int64_t img_pitch, grad_pitch;
    int w, h;
};

__host__ inline LevelView level_view(const omt_pyramid &p, int L) {
    LevelView v;
    v.img = (const uint8_t *)p.base + p.lv[L].img_off;
    v.grad = (const uint8_t *)p.base + p.lv[L].grad_off;
    v.img_pitch = p.lv[L].img_pitch;
    v.grad_pitch = p.lv[L].grad_pitch;
    v.w = p.lv[L].w;
    v.h = p.lv[L].h;
    return v;
}

// Image value of level L at an in-range pixel, as float intensity.
template <int ST>
__device__ __forceinline__ float load_level(const LevelView &v, int L, int x, int y) {
    const uint8_t *row = v.img + (int64_t)y * v.img_pitch;
    if (L == 0) return (float)__ldg(row + x);
    if (ST == OMT_F32) return __ldg((const float *)row + x);
    return __half2float(__ldg((const __half *)row + x)) + 128.0f;
}

template <int ST>
__device__ __forceinline__ float2 load_grad(const LevelView &v, int x, int y) {
    const uint8_t *row = v.grad + (int64_t)y * v.grad_pitch;
    if (ST == OMT_F32) return __ldg((const float2 *)row + x);
    return __half22float2(__ldg((const __half2 *)row + x));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(FULL_MASK, v, m);
    return v;
}

// ------------------------------------------------------------ batch table
// Device-side description of a batched step (one entry per stream), packed
// on the host by omt_batch_pack and copied to the device by omt_batch_step.
// Layout: BatchHeader | int32 pyr_prefix[OMT_MAX_LEVELS][S+1] |
// int32 resp_prefix[S+1] | int32 box_prefix[S+1] | StreamEntry[S], with S =
// the capacity in streams; prefixes count tiles or boxes per stream.
struct StreamEntry {
    LevelView P[OMT_MAX_LEVELS];       // frame t's pyramid (read)
    LevelView P_next[OMT_MAX_LEVELS];  // frame t+1's pyramid (K1 writes, K3 reads)
    const uint8_t *frame;              // frame t+1 (u8)
    int64_t frame_pitch;
    const float4 *boxes;
    float4 *boxes_out;
    int32_t *nvalid;
    float2 *pts, *pts_out, *pts_back;
    uint8_t *status, *iters, *status_back;
    int32_t *offsets;
    uint32_t *rmap;                    // scratch: response map
    float2 *pad_pts;                   // scratch: per-box corner lists
    int32_t *pad_counts;               // scratch: per-box counts
    uint64_t *cand;                    // scratch: per-box candidate keys
    uint32_t *cstate;                  // scratch: per-box key count and R_max, overflow word
    int32_t w, h, nboxes, maxc;
    uint32_t tm_ok, tm_ok_back;        // bit 3L + m: LK map m of level L (forward, backward) valid
    uint32_t pyr_maps_ok;              // bit L: the tile map of level L of frame t+1's pyramid
};

// Tensor maps of the LK window copies, per level: the template frame's
// image and gradient planes under the template box, the other frame's image
// plane under the search box (forward: templates on frame t; backward, for
// the forward-backward check: templates on frame t+1).
constexpr int LK_MAP_TI = 0, LK_MAP_TG = 1, LK_MAP_S = 2, LK_MAPS = 3;

struct BatchHeader {
    int32_t nstreams, max_streams, total_boxes, levels, storage, win, max_iter;
    int32_t qnum, qden, aggregator, dmax, cell;
    float eps2, tau_n;
    float fb_max;   // forward-backward threshold (level-0 px)
    int32_t fb_on;  // fb_max >= 0
    int64_t md2c;
    int64_t bytes;  // size of the packed table
    // Words the kernels write: work[0], the next point of the batched LK
    // launch's work queue (reset to 0 on the device before each LK launch);
    // work[1], non-zero when some box's candidate list overflowed in this
    // step's corner phase; work[2], the next strip of the corner-list
    // kernel's queue (both reset by the corner phase's first kernel).
    uint32_t work[4];
};

__host__ __device__ inline size_t batch_entries_offset(int max_streams) {
    size_t off = sizeof(BatchHeader) + sizeof(int32_t) * (size_t)(OMT_MAX_LEVELS + 2) * (max_streams + 1);
    return (off + 15) & ~(size_t)15;
}

// The LK tensor maps follow the stream entries: stream s, direction d
// (0 forward, 1 backward), level L, map m at index
// ((2 s + d) * OMT_MAX_LEVELS + L) * LK_MAPS + m.
__host__ __device__ inline size_t batch_maps_offset(int max_streams) {
    const size_t off = batch_entries_offset(max_streams) + sizeof(StreamEntry) * (size_t)max_streams;
    return (off + 127) & ~(size_t)127;
}

// The pyramid tile maps of the frames t+1 (level 0: the frame; level L:
// the plane of level L) follow the LK maps, OMT_MAX_LEVELS per stream.
__host__ __device__ inline size_t batch_pyr_maps_offset(int max_streams) {
    return batch_maps_offset(max_streams) +
           sizeof(CUtensorMap) * (size_t)max_streams * 2 * OMT_MAX_LEVELS * LK_MAPS;
}

__host__ __device__ inline size_t batch_table_bytes(int max_streams) {
    return batch_pyr_maps_offset(max_streams) + sizeof(CUtensorMap) * (size_t)max_streams * OMT_MAX_LEVELS;
}

struct BatchView {
    const uint8_t *base;
    __host__ __device__ explicit BatchView(const uint8_t *b) : base(b) {}
    __host__ __device__ const BatchHeader &hdr() const { return *(const BatchHeader *)base; }
    __host__ __device__ int nstreams() const { return hdr().nstreams; }
    __host__ __device__ int levels() const { return hdr().levels; }
    __host__ __device__ const int32_t *pyr_prefix(int L) const {
        return (const int32_t *)(base + sizeof(BatchHeader)) + (size_t)L * (hdr().max_streams + 1);
    }
    __host__ __device__ const int32_t *resp_prefix() const { return pyr_prefix(OMT_MAX_LEVELS); }
    __host__ __device__ const int32_t *box_prefix() const { return pyr_prefix(OMT_MAX_LEVELS + 1); }
    __host__ __device__ const StreamEntry &stream(int s) const {
        return ((const StreamEntry *)(base + batch_entries_offset(hdr().max_streams)))[s];
    }
    // stream s's tile map of level L of frame t+1's pyramid
    __host__ __device__ const CUtensorMap *pyr_map(int s, int L) const {
        return (const CUtensorMap *)(base + batch_pyr_maps_offset(hdr().max_streams)) +
               (size_t)s * OMT_MAX_LEVELS + L;
    }
    // stream s's LK maps of direction d (0 forward, 1 backward), LK_MAPS per level
    __host__ __device__ const CUtensorMap *maps(int s, int d) const {
        return (const CUtensorMap *)(base + batch_maps_offset(hdr().max_streams)) +
               (size_t)(2 * s + d) * OMT_MAX_LEVELS * LK_MAPS;
    }
};

// Segment s of a prefix array (pre[0] = 0, non-decreasing, n segments) that
// holds item g < pre[n]: the last s with pre[s] <= g (empty segments skipped).
__host__ __device__ __forceinline__ int find_segment(const int32_t *pre, int n, int g) {
    int lo = 0, hi = n;  // pre[lo] <= g < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// Programmatic dependent launch: a kernel launched by launch_pdl may be
// scheduled while its predecessor in the stream drains; it calls
// pdl_begin() before touching memory its predecessor writes (griddepcontrol
// waits for that grid to complete and its writes to be visible), which also
// lets its own successor be scheduled.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- launchers
// Each returns the cudaError_t of cudaGetLastError() after its launches.

cudaError_t launch_pyramid(const uint8_t *frame, int w, int h, size_t pitch,
                           const omt_pyramid &pyr, cudaStream_t s);

cudaError_t launch_corner_response(const omt_pyramid &pyr, uint32_t *out, const float4 *boxes,
                                   int nboxes, cudaStream_t s);

// lists: the candidate-list path (list, overflow, select kernels); false:
// the map path alone (the map of every strip touching a box, then select),
// whose scratch is smaller.
cudaError_t launch_select_corners(const omt_pyramid &pyr, const float4 *boxes, int nboxes,
                                  const omt_params &prm, void *scratch, float2 *pts,
                                  int32_t *offsets, bool lists, cudaStream_t s);

size_t select_scratch_bytes(int w, int h, int nboxes, int max_corners, bool lists = true);

// omt_select_corners with the path chosen: lists as in launch_select_corners
// (the public call uses the lists; omt_select_corners_static the map path).
int select_corners_entry(const omt_pyramid *pyr, const float *boxes, int32_t nboxes,
                         const omt_params *prm, void *scratch, size_t scratch_bytes, float *pts,
                         int32_t *offsets, bool lists, void *stream);

// The parts of a corner-selection scratch buffer (select_scratch_bytes).
struct SelectScratch {
    uint32_t *rmap;      // w x h response map (written only where a list overflowed)
    float2 *pad_pts;     // nboxes x max_corners selected corners
    int32_t *pad_counts; // nboxes counts
    uint64_t *cand;      // nboxes x 1024 candidate keys (null on the map path)
    uint32_t *cstate;    // nboxes x (count, R_max), then one overflow word (null on the map path)
};
void select_scratch_split(void *scratch, int w, int h, int nboxes, int max_corners, bool lists,
                          SelectScratch &out);

// Batched forms: every launch covers all streams of the table in `table`
// (device memory); grids depend only on the capacities.
int pyramid_tiles(int w, int h);
cudaError_t launch_iou_matrix(const float *a, int na, const float *b, int nb, double *out,
                              cudaStream_t s);
size_t assign_workspace(int n);   // host bytes of the assignment's work arrays
void assign_max_iou(const double *iou, int na, int nb, const uint8_t *active, double iou_min,
                    void *ws, int32_t *match_a, int32_t *match_b);   // K1 tiles of a level of this size
int response_tiles(int w, int h);  // K2 response tiles of a frame of this size
// ctas_per_sm (0 = as many as fit): the launch shapes of omt_batch_caps.
cudaError_t launch_pyramid_batch(const uint8_t *table, int levels, int storage, int max_tiles[],
                                 int max_streams, int ctas_per_sm, cudaStream_t s);
cudaError_t launch_corners_batch(const uint8_t *table, int max_streams, int max_resp_tiles,
                                 int max_boxes, int max_corners, int list_ctas_per_sm,
                                 int select_ctas_per_sm, cudaStream_t s);
// LK over every point of a batch: warps per CTA, CTAs per SM and work-queue
// chunk as in omt_batch_caps (0 = default).
// Encodes the LK window maps of every level of P (frame t) and J (frame
// t+1) for window side win into out[L * LK_MAPS + m]; returns the mask of
// valid maps (bit 3L + m).  Host only; a map that cannot be encoded (or no
// driver) leaves its bit clear and the kernels copy that level row by row.
uint32_t encode_lk_maps(const omt_pyramid &P, const omt_pyramid &J, int win, CUtensorMap *out);

// A 2D tensor map of a plane of esz-byte texels (w x h, pitch bytes apart)
// read in boxes of box_w x box_h texels, zero-filled outside; false when the
// plane's base or pitch is not a multiple of 16 bytes (the map cannot
// describe it).
bool encode_plane_map(const void *base, int esz, int w, int h, int64_t pitch, int box_w, int box_h,
                      CUtensorMap *out);

// The tensor maps of the pyramid tiles' copies (pyramid.cu) for a frame and
// the pyramid built from it: out[0] for the frame, out[L] for level L >= 1
// (up to levels - 1); returns the mask of valid maps (bit L).
uint32_t encode_pyramid_maps(const uint8_t *frame, int64_t frame_pitch, const omt_pyramid &pyr,
                             CUtensorMap *out);

// Box of the level-0 pyramid tiles' tensor copies (pyramid.cu): 16 columns
// either side of a 128-column tile (the copy's x must be a multiple of 16
// bytes) and 2 rows above and below a 32-row tile.
constexpr int L0_BOX_W = 160, L0_BOX_H = 36;

// Reads and clears the count of LK staging waits that hit their limit.
cudaError_t lk_wait_timeouts_take(unsigned *count);
cudaError_t pyr_wait_timeouts_take(unsigned *count);
cudaError_t lk_fail_point_set(long long point);

// backward = 0: the LK phase (frame t -> t+1); 1: the backward run of the
// forward-backward check (frame t+1 -> t from the forward results), each
// point's check applied as it finishes.
cudaError_t launch_lk_batch(const uint8_t *table, int storage, int win, int warps,
                            int ctas_per_sm, int chunk, int backward, cudaStream_t s);

cudaError_t launch_level_u8(const omt_pyramid &p, int level, uint8_t *out, size_t pitch,
                            cudaStream_t s);
cudaError_t launch_scale_boxes(const float4 *in, int n, float scale, float4 *out, cudaStream_t s);

size_t st_scratch_bytes(int w, int h);
size_t tvl1_scratch_bytes(int w, int h);
cudaError_t launch_structure_texture(const uint8_t *frame, int w, int h, size_t pitch,
                                     const omt_flow_params &fp, uint8_t *tex, size_t tpitch,
                                     void *scratch, cudaStream_t s);
cudaError_t launch_tvl1(const omt_pyramid &P0, const omt_pyramid &P1, const omt_flow_params &fp,
                        float2 *flow, void *scratch, cudaStream_t s);
cudaError_t launch_box_mean_flow(const float2 *flow, int w, int h, const float4 *boxes,
                                 int nboxes, float4 *out, cudaStream_t s);

cudaError_t launch_fb_check(const float2 *pts, const float2 *pts_back, const uint8_t *status_back,
                            int n_max, const int32_t *n_dev, float fb_max, uint8_t *status,
                            cudaStream_t s);
cudaError_t launch_update_boxes_batch(const uint8_t *table, int max_boxes, int aggregator,
                                      cudaStream_t s);

cudaError_t launch_lk(const omt_pyramid &prev, const omt_pyramid &next, const float2 *pts,
                      int n_max, const int32_t *n_dev, const omt_params &prm, float2 *out,
                      uint8_t *status, uint8_t *iters, cudaStream_t s);

cudaError_t launch_update_boxes(const float4 *boxes, const int32_t *offsets, const float2 *pts,
                                const float2 *pts_out, const uint8_t *status, int nboxes,
                                int aggregator, float4 *boxes_out, int32_t *nvalid,
                                cudaStream_t s);

}  // namespace omt
