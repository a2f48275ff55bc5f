// boxes.cu -- K4: per-box displacement update (Section V-A, prediction).
//
// One CTA per box.  The median of dx (and of dy) over the box's OK points is
// found by an exact MSD radix select on order-preserving 32-bit keys of the
// FP32 displacements (four 8-bit digits, shared-memory histograms), so it
// needs no sort, no scratch and works for any number of points per box; an
// even count averages the two middle order statistics.  The mean flag sums
// with a fixed per-thread stride and a fixed tree, so it is deterministic.
#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int BNT = 256;

__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fval(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

struct BoxArgs {
    const float4 *boxes;
    const int32_t *offsets;
    const float2 *pts, *pts_out;
    const uint8_t *status;
    int aggregator;
    float4 *boxes_out;
    int32_t *nvalid;
};

__device__ __forceinline__ float disp(const BoxArgs &a, int i, int axis) {
    return axis == 0 ? a.pts_out[i].x - a.pts[i].x : a.pts_out[i].y - a.pts[i].y;
}

// Value of rank k (0-based, ascending) among the OK displacements of [lo, hi).
__device__ float select_rank(const BoxArgs &a, int lo, int hi, int axis, int k, unsigned *hist,
                             int *s_sel, int *s_k) {
    uint32_t prefix = 0, pmask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += BNT) hist[b] = 0;
        __syncthreads();
        for (int i = lo + threadIdx.x; i < hi; i += BNT) {
            if (!(a.status[i] & OMT_PT_OK)) continue;
            const uint32_t key = fkey(disp(a, i, axis));
            if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned cum = 0;
            int sel = 255;
            for (int b = 0; b < 256; ++b) {
                if (cum + hist[b] > (unsigned)k) {
                    sel = b;
                    break;
                }
                cum += hist[b];
            }
            *s_sel = sel;
            *s_k = k - (int)cum;
        }
        __syncthreads();
        prefix |= (uint32_t)*s_sel << shift;
        pmask |= 0xFFu << shift;
        k = *s_k;
        __syncthreads();
    }
    return fval(prefix);
}

__global__ void __launch_bounds__(BNT) box_update_kernel(BoxArgs a) {
    __shared__ unsigned hist[256];
    __shared__ float red[2][BNT / 32];
    __shared__ int cnt[BNT / 32];
    __shared__ int s_sel, s_k;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int lo = a.offsets[b], hi = a.offsets[b + 1];

    int m = 0;
    float sx = 0.f, sy = 0.f;
    for (int i = lo + tid; i < hi; i += BNT) {
        if (!(a.status[i] & OMT_PT_OK)) continue;
        ++m;
        if (a.aggregator == 1) {
            sx += disp(a, i, 0);
            sy += disp(a, i, 1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_xor_sync(FULL_MASK, m, o);
        sx += __shfl_xor_sync(FULL_MASK, sx, o);
        sy += __shfl_xor_sync(FULL_MASK, sy, o);
    }
    if (lane == 0) {
        cnt[wid] = m;
        red[0][wid] = sx;
        red[1][wid] = sy;
    }
    __syncthreads();
    int total = 0;
    float tx = 0.f, ty = 0.f;
    for (int w = 0; w < BNT / 32; ++w) {
        total += cnt[w];
        tx += red[0][w];
        ty += red[1][w];
    }
    float mx = 0.f, my = 0.f;
    if (total > 0) {
        if (a.aggregator == 1) {
            mx = tx / (float)total;
            my = ty / (float)total;
        } else {
            const int k1 = (total - 1) / 2, k2 = total / 2;
            const float x1 = select_rank(a, lo, hi, 0, k1, hist, &s_sel, &s_k);
            const float y1 = select_rank(a, lo, hi, 1, k1, hist, &s_sel, &s_k);
            if (k2 != k1) {
                const float x2 = select_rank(a, lo, hi, 0, k2, hist, &s_sel, &s_k);
                const float y2 = select_rank(a, lo, hi, 1, k2, hist, &s_sel, &s_k);
                mx = 0.5f * (x1 + x2);
                my = 0.5f * (y1 + y2);
            } else {
                mx = x1;
                my = y1;
            }
        }
    }
    if (tid == 0) {
        const float4 bx = a.boxes[b];
        a.boxes_out[b] = make_float4(bx.x + mx, bx.y + my, bx.z + mx, bx.w + my);
        if (a.nvalid) a.nvalid[b] = total;
    }
}

}  // namespace

cudaError_t launch_update_boxes(const float4 *boxes, const int32_t *offsets, const float2 *pts,
                                const float2 *pts_out, const uint8_t *status, int nboxes,
                                int aggregator, float4 *boxes_out, int32_t *nvalid,
                                cudaStream_t s) {
    if (nboxes <= 0) return cudaSuccess;
    BoxArgs a{boxes, offsets, pts, pts_out, status, aggregator, boxes_out, nvalid};
    box_update_kernel<<<nboxes, BNT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace omt
