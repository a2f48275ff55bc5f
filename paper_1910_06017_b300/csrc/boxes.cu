// boxes.cu -- K4: per-box displacement update (Section V-A, prediction).
//
// One CTA per box.  The median of dx (and of dy) over the box's OK points is
// an exact order statistic: for up to 2048 OK points the displacements are
// gathered in shared memory and the elements of the two middle ranks of dx
// and of dy are found by counting, all four in one pass;
// larger boxes use an MSD radix select on order-preserving 32-bit keys of the
// FP32 displacements (four 8-bit digits, shared-memory histograms).  Neither
// needs a sort or scratch; an even count averages the two middle values.  The mean flag sums
// with a fixed per-thread stride and a fixed tree, so it is deterministic.
// The median-flow scale (aggregator 2) takes the box's first 64 OK points in
// CSR order (a block-wide ordered compaction), forms the ratios of their
// pairwise distances after and before into shared memory, and picks their
// median by the same radix select on the ratios' keys.
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

// Warp 0: the bin of a 256-bin histogram holding the element of rank k
// (ascending), and k's rank inside it, by a warp scan.
__device__ __forceinline__ void pick_bin(const unsigned *hist, int k, int *s_sel, int *s_k) {
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
        if (threadIdx.x < 32) pick_bin(hist, k, s_sel, s_k);
        __syncthreads();
        prefix |= (uint32_t)*s_sel << shift;
        pmask |= 0xFFu << shift;
        k = *s_k;
        __syncthreads();
    }
    return fval(prefix);
}

// Key of rank k (ascending) among n 32-bit keys in shared memory: MSD radix
// select, four 8-bit digits.
__device__ uint32_t smem_rank(const uint32_t *keys, int n, int k, unsigned *hist, int *s_sel,
                              int *s_k) {
    uint32_t prefix = 0, pmask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += BNT) hist[b] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += BNT) {
            const uint32_t key = keys[i];
            if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) pick_bin(hist, k, s_sel, s_k);
        __syncthreads();
        prefix |= (uint32_t)*s_sel << shift;
        pmask |= 0xFFu << shift;
        k = *s_k;
        __syncthreads();
    }
    return prefix;
}

// Points of the scale estimate: the box's first SCALE_POINTS OK points in CSR
// order (the strongest corners come first).
constexpr int SCALE_POINTS = 64;

// Shared-memory path for boxes with at most SMALL OK points: gather the
// displacements, then the element of rank k is the one with exactly k
// elements before it in the order (value, gather position).
constexpr int SMALL = 2048;

// The elements of ranks k1 <= k2 of vx and of vy (m each) in one pass: each
// thread ranks its elements of both arrays; out = (x1, x2, y1, y2).
__device__ float4 rank_pick2(const float *vx, const float *vy, int m, int k1, int k2,
                             float *s_out) {
    for (int i = threadIdx.x; i < m; i += BNT) {
        const float x = vx[i], y = vy[i];
        int rx = 0, ry = 0;
        for (int j = 0; j < m; ++j) {
            const float u = vx[j], w = vy[j];
            rx += (u < x) || (u == x && j < i);
            ry += (w < y) || (w == y && j < i);
        }
        if (rx == k1) s_out[0] = x;
        if (rx == k2) s_out[1] = x;
        if (ry == k1) s_out[2] = y;
        if (ry == k2) s_out[3] = y;
    }
    __syncthreads();
    const float4 out = make_float4(s_out[0], s_out[1], s_out[2], s_out[3]);
    __syncthreads();
    return out;
}

// Box b of one stream, whole CTA.  SCALE: the median-flow scale of
// aggregator 2 (compiled only into the kernels that launch for it).
template <bool SCALE>
__device__ void box_update_one(const BoxArgs &a, int b) {
    __shared__ unsigned hist[256];
    __shared__ float red[2][BNT / 32];
    __shared__ int cnt[BNT / 32];
    __shared__ int s_sel, s_k, s_n;
    __shared__ float s_pick[4];
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
            const float4 r = rank_pick2(vx, vy, total, k1, k2, s_pick);
            if (k2 != k1) {
                mx = 0.5f * (r.x + r.y);
                my = 0.5f * (r.z + r.w);
            } else {
                mx = r.x;
                my = r.z;
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
    if (SCALE && a.aggregator == 2) {
        // median-flow scale: the median over all pairs of the first
        // SCALE_POINTS OK points (in CSR order) of |v_i - v_j| / |u_i - u_j|
        __shared__ int s_idx[SCALE_POINTS], wsum[BNT / 32], s_found;
        __shared__ float2 su[SCALE_POINTS], sv[SCALE_POINTS];
        if (tid == 0) s_found = 0;
        __syncthreads();
        for (int base = lo; base < hi; base += BNT) {
            const int i = base + tid;
            const bool ok = i < hi && (a.status[i] & OMT_PT_OK);
            const unsigned bal = __ballot_sync(FULL_MASK, ok);
            if (lane == 0) wsum[wid] = __popc(bal);
            __syncthreads();
            int before = s_found;
            for (int w = 0; w < wid; ++w) before += wsum[w];
            const int p = before + __popc(bal & ((1u << lane) - 1u));
            if (ok && p < SCALE_POINTS) s_idx[p] = i;
            __syncthreads();
            if (tid == 0) {
                int t = s_found;
                for (int w = 0; w < BNT / 32; ++w) t += wsum[w];
                s_found = t;
            }
            __syncthreads();
            if (s_found >= SCALE_POINTS) break;
        }
        const int k = min(s_found, SCALE_POINTS);
        for (int q = tid; q < k; q += BNT) {
            su[q] = a.pts[s_idx[q]];
            sv[q] = a.pts_out[s_idx[q]];
        }
        if (tid == 0) s_n = 0;
        __syncthreads();
        uint32_t *keys = (uint32_t *)vx;  // SCALE_POINTS^2 / 2 < SMALL ratios
        for (int q = tid; q < SCALE_POINTS * SCALE_POINTS; q += BNT) {
            const int i = q / SCALE_POINTS, j = q % SCALE_POINTS;
            if (i >= j || j >= k) continue;
            const float ux = su[i].x - su[j].x, uy = su[i].y - su[j].y;
            const float vx2 = sv[i].x - sv[j].x, vy2 = sv[i].y - sv[j].y;
            const float du = sqrtf(fmaf(ux, ux, uy * uy));
            if (du > 0.f) keys[atomicAdd(&s_n, 1)] = fkey(sqrtf(fmaf(vx2, vx2, vy2 * vy2)) / du);
        }
        __syncthreads();
        const int nr = s_n;
        float scale = 1.f;
        if (nr > 0) {
            const int k1 = (nr - 1) / 2, k2 = nr / 2;
            const float r1 = fval(smem_rank(keys, nr, k1, hist, &s_sel, &s_k));
            scale = k2 != k1 ? 0.5f * (r1 + fval(smem_rank(keys, nr, k2, hist, &s_sel, &s_k))) : r1;
        }
        if (tid == 0) {
            const float4 bx = a.boxes[b];
            const float cx = 0.5f * (bx.x + bx.z) + mx, cy = 0.5f * (bx.y + bx.w) + my;
            const float hw = 0.5f * (bx.z - bx.x) * scale, hh = 0.5f * (bx.w - bx.y) * scale;
            a.boxes_out[b] = make_float4(cx - hw, cy - hh, cx + hw, cy + hh);
            if (a.nvalid) a.nvalid[b] = total;
        }
        return;
    }
    if (tid == 0) {
        const float4 bx = a.boxes[b];
        a.boxes_out[b] = make_float4(bx.x + mx, bx.y + my, bx.z + mx, bx.w + my);
        if (a.nvalid) a.nvalid[b] = total;
    }
}

template <bool SCALE>
__global__ void __launch_bounds__(BNT) box_update_kernel(BoxArgs a) {
    box_update_one<SCALE>(a, blockIdx.x);
}

template <bool SCALE>
__global__ void __launch_bounds__(BNT) box_update_batch_kernel(const uint8_t *table) {
    const BatchView t(table);
    const int32_t *pre = t.box_prefix();
    const int total = pre[t.nstreams()];
    for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
        const int si = find_segment(pre, t.nstreams(), gb);
        const StreamEntry &e = t.stream(si);
        BoxArgs a{e.boxes, e.offsets, e.pts, e.pts_out, e.status, t.hdr().aggregator,
                  e.boxes_out, e.nvalid};
        box_update_one<SCALE>(a, gb - pre[si]);
    }
}

}  // namespace

cudaError_t launch_update_boxes(const float4 *boxes, const int32_t *offsets, const float2 *pts,
                                const float2 *pts_out, const uint8_t *status, int nboxes,
                                int aggregator, float4 *boxes_out, int32_t *nvalid,
                                cudaStream_t s) {
    if (nboxes <= 0) return cudaSuccess;
    BoxArgs a{boxes, offsets, pts, pts_out, status, aggregator, boxes_out, nvalid};
    if (aggregator == 2) box_update_kernel<true><<<nboxes, BNT, 0, s>>>(a);
    else box_update_kernel<false><<<nboxes, BNT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_update_boxes_batch(const uint8_t *table, int max_boxes, int aggregator,
                                      cudaStream_t s) {
    if (max_boxes <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = max_boxes < sms * 8 ? max_boxes : sms * 8;
    if (aggregator == 2) box_update_batch_kernel<true><<<grid, BNT, 0, s>>>(table);
    else box_update_batch_kernel<false><<<grid, BNT, 0, s>>>(table);
    return cudaGetLastError();
}

}  // namespace omt
