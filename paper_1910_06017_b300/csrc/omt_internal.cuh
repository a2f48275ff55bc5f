// omt_internal.cuh -- device helpers and launcher declarations shared by the
// kernels of libomt.  Not part of the public C-ABI (see include/omt.h).
#pragma once

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

// ---------------------------------------------------------------- launchers
// Each returns the cudaError_t of cudaGetLastError() after its launches.

cudaError_t launch_pyramid(const uint8_t *frame, int w, int h, size_t pitch,
                           const omt_pyramid &pyr, cudaStream_t s);

cudaError_t launch_corner_response(const omt_pyramid &pyr, uint32_t *out, const float4 *boxes,
                                   int nboxes, cudaStream_t s);

cudaError_t launch_select_corners(const omt_pyramid &pyr, const float4 *boxes, int nboxes,
                                  const omt_params &prm, void *scratch, float2 *pts,
                                  int32_t *offsets, cudaStream_t s);

size_t select_scratch_bytes(int w, int h, int nboxes, int max_corners);

cudaError_t launch_lk(const omt_pyramid &prev, const omt_pyramid &next, const float2 *pts,
                      int n_max, const int32_t *n_dev, const omt_params &prm, float2 *out,
                      uint8_t *status, uint8_t *iters, cudaStream_t s);

cudaError_t launch_update_boxes(const float4 *boxes, const int32_t *offsets, const float2 *pts,
                                const float2 *pts_out, const uint8_t *status, int nboxes,
                                int aggregator, float4 *boxes_out, int32_t *nvalid,
                                cudaStream_t s);

}  // namespace omt
