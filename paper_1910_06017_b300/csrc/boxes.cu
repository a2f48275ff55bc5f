// boxes.cu -- K4: per-box displacement update (Section V-A, prediction).
//
// One CTA per box.  The median of dx (and of dy) over the box's OK points is
// an exact order statistic: for up to 2048 OK points the displacements are
// gathered in shared memory and the element of rank k is found by counting;
// larger boxes use an MSD radix select on order-preserving 32-bit keys of the
// FP32 displacements (four 8-bit digits, shared-memory histograms).  Neither
// needs a sort or scratch; an even count averages the two middle values.  The mean flag sums
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

// Value of rank k (0-based, ascending) among the OK displacements of [lo, hi),
// for boxes too large for the shared-memory path: MSD radix select, with
// the digit's bin found by a warp scan over the 256-bin histogram.
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
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            unsigned c[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j] = hist[lane * 8 + j];
                sum += c[j];
            }
            unsigned inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(FULL_MASK, inc, o);
                if (lane >= o) inc += t;
            }
            const unsigned exc = inc - sum;
            if (exc <= (unsigned)k && (unsigned)k < inc) {
                unsigned cum = exc;
                for (int j = 0; j < 8; ++j) {
                    if (cum + c[j] > (unsigned)k) {
                        *s_sel = lane * 8 + j;
                        *s_k = k - (int)cum;
                        break;
                    }
                    cum += c[j];
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)*s_sel << shift;
        pmask |= 0xFFu << shift;
        k = *s_k;
        __syncthreads();
    }
    return fval(prefix);
}

// Shared-memory path for boxes with at most SMALL OK points: gather the
// displacements, then the element of rank k is the one with exactly k
// elements before it in the order (value, gather position).
constexpr int SMALL = 2048;

__device__ float rank_pick(const float *v, int m, int k, float *s_out) {
    for (int i = threadIdx.x; i < m; i += BNT) {
        const float x = v[i];
        int r = 0;
        for (int j = 0; j < m; ++j) {
            const float y = v[j];
            r += (y < x) || (y == x && j < i);
        }
        if (r == k) *s_out = x;
    }
    __syncthreads();
    const float out = *s_out;
    __syncthreads();
    return out;
}

// Box b of one stream, whole CTA.
__device__ void box_update_one(const BoxArgs &a, int b) {
    __shared__ unsigned hist[256];
    __shared__ float red[2][BNT / 32];
    __shared__ int cnt[BNT / 32];
    __shared__ int s_sel, s_k, s_n;
    __shared__ float s_val;
    __shared__ float vx[SMALL], vy[SMALL];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int lo = a.offsets[b], hi = a.offsets[b + 1];
    __syncthreads();

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
        } else if (total <= SMALL) {
            if (tid == 0) s_n = 0;
            __syncthreads();
            for (int i = lo + tid; i < hi; i += BNT) {
                if (!(a.status[i] & OMT_PT_OK)) continue;
                const int p = atomicAdd(&s_n, 1);
                vx[p] = disp(a, i, 0);
                vy[p] = disp(a, i, 1);
            }
            __syncthreads();
            const int k1 = (total - 1) / 2, k2 = total / 2;
            const float x1 = rank_pick(vx, total, k1, &s_val);
            const float y1 = rank_pick(vy, total, k1, &s_val);
            if (k2 != k1) {
                const float x2 = rank_pick(vx, total, k2, &s_val);
                const float y2 = rank_pick(vy, total, k2, &s_val);
                mx = 0.5f * (x1 + x2);
                my = 0.5f * (y1 + y2);
            } else {
                mx = x1;
                my = y1;
            }
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

__global__ void __launch_bounds__(BNT) box_update_kernel(BoxArgs a) { box_update_one(a, blockIdx.x); }

__global__ void __launch_bounds__(BNT) box_update_batch_kernel(const uint8_t *table) {
    const BatchView t(table);
    const int32_t *pre = t.box_prefix();
    const int total = pre[t.nstreams()];
    for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
        const int si = find_segment(pre, t.nstreams(), gb);
        const StreamEntry &e = t.stream(si);
        BoxArgs a{e.boxes, e.offsets, e.pts, e.pts_out, e.status, t.hdr().aggregator,
                  e.boxes_out, e.nvalid};
        box_update_one(a, gb - pre[si]);
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

cudaError_t launch_update_boxes_batch(const uint8_t *table, int max_boxes, cudaStream_t s) {
    if (max_boxes <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = max_boxes < sms * 8 ? max_boxes : sms * 8;
    box_update_batch_kernel<<<grid, BNT, 0, s>>>(table);
    return cudaGetLastError();
}

}  // namespace omt
