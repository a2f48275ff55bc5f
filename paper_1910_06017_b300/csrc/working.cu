// working.cu -- the working level of a frame (Section V-A, preprocessing:
// the frame is downscaled by the Gaussian pyramid and a level chosen by its
// resolution is processed).
//
// The working frame is pyramid level L (F32 storage) rounded to u8; levels
// 0-2 of an F32 pyramid hold the exact dyadic values of the definition, so
// the rounding decides exactly as the definition's does.  The rest of the
// hot path then runs unchanged on the working frames, with boxes scaled by
// 2^-L into level-L pixels and back (exact: a power of two).
#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int WX = 32, WY = 8;

__global__ void level_u8_kernel(const uint8_t *img, int64_t img_pitch, bool u8, int w, int h,
                                uint8_t *out, int64_t pitch) {
    const int x = blockIdx.x * WX + threadIdx.x, y = blockIdx.y * WY + threadIdx.y;
    if (x >= w || y >= h) return;
    const uint8_t *row = img + (int64_t)y * img_pitch;
    float v;
    if (u8) {
        out[(int64_t)y * pitch + x] = row[x];
        return;
    }
    v = floorf(((const float *)row)[x] + 0.5f);
    out[(int64_t)y * pitch + x] = (uint8_t)(v < 0.f ? 0.f : (v > 255.f ? 255.f : v));
}

__global__ void scale_boxes_kernel(const float4 *in, int n, float s, float4 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 b = in[i];
    out[i] = make_float4(b.x * s, b.y * s, b.z * s, b.w * s);
}

}  // namespace

cudaError_t launch_level_u8(const omt_pyramid &p, int level, uint8_t *out, size_t pitch,
                            cudaStream_t s) {
    const LevelView v = level_view(p, level);
    const dim3 g((v.w + WX - 1) / WX, (v.h + WY - 1) / WY), b(WX, WY);
    level_u8_kernel<<<g, b, 0, s>>>(v.img, v.img_pitch, level == 0, v.w, v.h, out, (int64_t)pitch);
    return cudaGetLastError();
}

cudaError_t launch_scale_boxes(const float4 *in, int n, float scale, float4 *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    scale_boxes_kernel<<<(n + 255) / 256, 256, 0, s>>>(in, n, scale, out);
    return cudaGetLastError();
}

}  // namespace omt
