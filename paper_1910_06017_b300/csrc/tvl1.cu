// tvl1.cu -- the paper's dense flow engine (Section IV) and the mean-in-box
// prediction (Section V-A).
//
// Structure-texture: the ROF structure S of the u8 frame by Chambolle's dual
// projection (one launch per step, q = div p - I / theta formed in shared
// memory for a tile and its halo, the dual field ping-ponged in global
// memory), then the u8 texture clamp(floor(k (I - alpha S) + 128.5)).
// Huber-TV-L1: per pyramid level (FP32 storage, coarse to fine) the flow of
// the level above is sampled bilinearly at (x/2, y/2) and doubled; per warp
// one launch samples frame t+1 and its gradient at x + u0 (taps clamped) and
// stores grad I1w and rho0, then every primal-dual iteration is one launch
// (pd_kernel): the duals from the extrapolated flow (forward differences, a
// Huber shrink and the projection onto the unit disc, per flow component)
// in shared memory for a tile and its halo, then the flow (backward-
// difference divergence, the pointwise prox of the L1 data term, the
// extrapolation).  Every expression keeps the order of the definition, in
// FP32.  Each iteration reads and writes every field once: the kernel is
// bound by HBM (or L2 for small levels).
#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int TBX = 32, TBY = 8;

// div of an interleaved dual field (px, py), component c of cc, at (x, y).
__device__ __forceinline__ float div_bwd(const float *p, int cc, int c, int w, int h, int x, int y) {
    const int64_t i = (int64_t)y * w + x;
    float d = 0.f;
    if (x + 1 < w) d += p[i * cc + c];
    if (x > 0) d -= p[(i - 1) * cc + c];
    if (y + 1 < h) d += p[i * cc + c + 1];
    if (y > 0) d -= p[(i - w) * cc + c + 1];
    return d;
}

// ------------------------------------------------------ structure-texture
struct StArgs {
    const uint8_t *img;
    int64_t pitch;
    int w, h;
    float theta, step;
    const float *p;  // (px, py) interleaved, w x h
    float *p_out;
};

// One projection step for a TBX x TBY tile: q = div p - I / theta on the
// tile plus its right column and bottom row in shared memory (from p on the
// tile plus one pixel on every side), then the tile's new duals from the
// forward differences of q.  Equal to forming q everywhere and then p.
__global__ void __launch_bounds__(TBX * TBY) st_step_kernel(StArgs a) {
    constexpr int QW = TBX + 1, QH = TBY + 1, RW = TBX + 2, RH = TBY + 2;
    __shared__ float2 spp[RH][RW];
    __shared__ float sq[QH][QW];
    const int tid = threadIdx.y * TBX + threadIdx.x;
    const int bx = blockIdx.x * TBX, by = blockIdx.y * TBY;
    for (int k = tid; k < RW * RH; k += TBX * TBY) {
        const int ry = k / RW, rx = k - ry * RW;
        const int x = bx - 1 + rx, y = by - 1 + ry;
        spp[ry][rx] = (x >= 0 && x < a.w && y >= 0 && y < a.h)
                          ? make_float2(a.p[2 * ((int64_t)y * a.w + x)], a.p[2 * ((int64_t)y * a.w + x) + 1])
                          : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int k = tid; k < QW * QH; k += TBX * TBY) {
        const int ry = k / QW, rx = k - ry * QW;
        const int x = bx + rx, y = by + ry;
        float q = 0.f;
        if (x < a.w && y < a.h) {
            // div p at (x, y): spp holds (x, y) at [ry + 1][rx + 1]
            float d = 0.f;
            if (x + 1 < a.w) d += spp[ry + 1][rx + 1].x;
            if (x > 0) d -= spp[ry + 1][rx].x;
            if (y + 1 < a.h) d += spp[ry + 1][rx + 1].y;
            if (y > 0) d -= spp[ry][rx + 1].y;
            q = d - (float)a.img[(int64_t)y * a.pitch + x] / a.theta;
        }
        sq[ry][rx] = q;
    }
    __syncthreads();
    const int x = bx + threadIdx.x, y = by + threadIdx.y;
    if (x >= a.w || y >= a.h) return;
    const float qc = sq[threadIdx.y][threadIdx.x];
    const float gx = x + 1 < a.w ? sq[threadIdx.y][threadIdx.x + 1] - qc : 0.f;
    const float gy = y + 1 < a.h ? sq[threadIdx.y + 1][threadIdx.x] - qc : 0.f;
    const float m = 1.f + a.step * sqrtf(gx * gx + gy * gy);
    const int64_t i = (int64_t)y * a.w + x;
    const float2 pc = spp[threadIdx.y + 1][threadIdx.x + 1];
    a.p_out[2 * i] = (pc.x + a.step * gx) / m;
    a.p_out[2 * i + 1] = (pc.y + a.step * gy) / m;
}

// Two projection steps for a TBX x TBY tile in one launch: the duals of the
// intermediate step are formed in shared memory on the tile grown by the
// pixels the second step reads (temporal blocking), so a launch reads p and
// I once and writes p once for two steps.  Positions outside the frame are
// formed as zero and never read by a position inside it.  Equal to two
// st_step_kernel launches bit for bit.
__global__ void __launch_bounds__(TBX * TBY) st_step2_kernel(StArgs a) {
    // regions (origin offset, width, height) relative to the tile origin:
    // P0 p^n [-2, TBX+1], Q0 q^n [-1, TBX+1], P1 p^n+1 [-1, TBX], Q1 q^n+1 [0, TBX]
    constexpr int P0W = TBX + 4, P0H = TBY + 4, Q0W = TBX + 3, Q0H = TBY + 3;
    constexpr int P1W = TBX + 2, P1H = TBY + 2, Q1W = TBX + 1, Q1H = TBY + 1;
    __shared__ float2 p0[P0H][P0W];
    __shared__ float q0[Q0H][Q0W];
    __shared__ float i0[Q0H][Q0W];
    __shared__ float2 p1[P1H][P1W];
    __shared__ float q1[Q1H][Q1W];
    const int tid = threadIdx.y * TBX + threadIdx.x;
    const int bx = blockIdx.x * TBX, by = blockIdx.y * TBY;
    auto inside = [&](int x, int y) { return x >= 0 && x < a.w && y >= 0 && y < a.h; };
    for (int k = tid; k < P0W * P0H; k += TBX * TBY) {
        const int ry = k / P0W, rx = k - ry * P0W, x = bx - 2 + rx, y = by - 2 + ry;
        p0[ry][rx] = inside(x, y) ? make_float2(a.p[2 * ((int64_t)y * a.w + x)],
                                                a.p[2 * ((int64_t)y * a.w + x) + 1])
                                  : make_float2(0.f, 0.f);
    }
    for (int k = tid; k < Q0W * Q0H; k += TBX * TBY) {
        const int ry = k / Q0W, rx = k - ry * Q0W, x = bx - 1 + rx, y = by - 1 + ry;
        i0[ry][rx] = inside(x, y) ? (float)a.img[(int64_t)y * a.pitch + x] : 0.f;
    }
    __syncthreads();
    // q^n on Q0: div p^n - I / theta; Q0 (rx, ry) is P0 (rx + 1, ry + 1)
    for (int k = tid; k < Q0W * Q0H; k += TBX * TBY) {
        const int ry = k / Q0W, rx = k - ry * Q0W, x = bx - 1 + rx, y = by - 1 + ry;
        float q = 0.f;
        if (inside(x, y)) {
            float d = 0.f;
            if (x + 1 < a.w) d += p0[ry + 1][rx + 1].x;
            if (x > 0) d -= p0[ry + 1][rx].x;
            if (y + 1 < a.h) d += p0[ry + 1][rx + 1].y;
            if (y > 0) d -= p0[ry][rx + 1].y;
            q = d - i0[ry][rx] / a.theta;
        }
        q0[ry][rx] = q;
    }
    __syncthreads();
    // p^n+1 on P1; P1 (rx, ry) is Q0 (rx, ry) and P0 (rx + 1, ry + 1)
    for (int k = tid; k < P1W * P1H; k += TBX * TBY) {
        const int ry = k / P1W, rx = k - ry * P1W, x = bx - 1 + rx, y = by - 1 + ry;
        float2 pn = make_float2(0.f, 0.f);
        if (inside(x, y)) {
            const float qc = q0[ry][rx];
            const float gx = x + 1 < a.w ? q0[ry][rx + 1] - qc : 0.f;
            const float gy = y + 1 < a.h ? q0[ry + 1][rx] - qc : 0.f;
            const float m = 1.f + a.step * sqrtf(gx * gx + gy * gy);
            const float2 pc = p0[ry + 1][rx + 1];
            pn = make_float2((pc.x + a.step * gx) / m, (pc.y + a.step * gy) / m);
        }
        p1[ry][rx] = pn;
    }
    __syncthreads();
    // q^n+1 on Q1; Q1 (rx, ry) is P1 (rx + 1, ry + 1) and Q0 (rx + 1, ry + 1)
    for (int k = tid; k < Q1W * Q1H; k += TBX * TBY) {
        const int ry = k / Q1W, rx = k - ry * Q1W, x = bx + rx, y = by + ry;
        float q = 0.f;
        if (inside(x, y)) {
            float d = 0.f;
            if (x + 1 < a.w) d += p1[ry + 1][rx + 1].x;
            if (x > 0) d -= p1[ry + 1][rx].x;
            if (y + 1 < a.h) d += p1[ry + 1][rx + 1].y;
            if (y > 0) d -= p1[ry][rx + 1].y;
            q = d - i0[ry + 1][rx + 1] / a.theta;
        }
        q1[ry][rx] = q;
    }
    __syncthreads();
    const int x = bx + threadIdx.x, y = by + threadIdx.y;
    if (x >= a.w || y >= a.h) return;
    const float qc = q1[threadIdx.y][threadIdx.x];
    const float gx = x + 1 < a.w ? q1[threadIdx.y][threadIdx.x + 1] - qc : 0.f;
    const float gy = y + 1 < a.h ? q1[threadIdx.y + 1][threadIdx.x] - qc : 0.f;
    const float m = 1.f + a.step * sqrtf(gx * gx + gy * gy);
    const float2 pc = p1[threadIdx.y + 1][threadIdx.x + 1];
    const int64_t i = (int64_t)y * a.w + x;
    a.p_out[2 * i] = (pc.x + a.step * gx) / m;
    a.p_out[2 * i + 1] = (pc.y + a.step * gy) / m;
}

__global__ void st_texture_kernel(StArgs a, float alpha, float k, uint8_t *tex, int64_t tpitch) {
    const int x = blockIdx.x * TBX + threadIdx.x, y = blockIdx.y * TBY + threadIdx.y;
    if (x >= a.w || y >= a.h) return;
    const float I = (float)a.img[(int64_t)y * a.pitch + x];
    const float S = I - a.theta * div_bwd(a.p, 2, 0, a.w, a.h, x, y);
    const float T = floorf(k * (I - alpha * S) + 128.0f + 0.5f);
    tex[(int64_t)y * tpitch + x] = (uint8_t)(T < 0.f ? 0.f : (T > 255.f ? 255.f : T));
}

// --------------------------------------------------------------- TV-L1
// Bilinear sample of channel c of a cc-channel float plane at (ix + a, iy + b),
// taps clamped to the plane.
__device__ __forceinline__ float bilin(const float *P, int64_t stride, int cc, int c, int w, int h,
                                       int ix, int iy, float a, float b) {
    const int x0 = clampi(ix, 0, w - 1), x1 = clampi(ix + 1, 0, w - 1);
    const int y0 = clampi(iy, 0, h - 1), y1 = clampi(iy + 1, 0, h - 1);
    return (1.f - a) * (1.f - b) * P[y0 * stride + x0 * cc + c] +
           a * (1.f - b) * P[y0 * stride + x1 * cc + c] +
           (1.f - a) * b * P[y1 * stride + x0 * cc + c] + a * b * P[y1 * stride + x1 * cc + c];
}

// Level image texel as float (level 0: u8; F32 storage above).
struct LevelF {
    const uint8_t *img;
    const float *grad;   // (Ix, Iy) interleaved
    int64_t img_pitch, grad_pitch;  // bytes
    int w, h;
    bool u8;
};

__device__ __forceinline__ float level_texel(const LevelF &L, int x, int y) {
    const uint8_t *row = L.img + (int64_t)y * L.img_pitch;
    return L.u8 ? (float)row[x] : ((const float *)row)[x];
}

__device__ __forceinline__ float level_bilin(const LevelF &L, int ix, int iy, float a, float b) {
    const int x0 = clampi(ix, 0, L.w - 1), x1 = clampi(ix + 1, 0, L.w - 1);
    const int y0 = clampi(iy, 0, L.h - 1), y1 = clampi(iy + 1, 0, L.h - 1);
    return (1.f - a) * (1.f - b) * level_texel(L, x0, y0) + a * (1.f - b) * level_texel(L, x1, y0) +
           (1.f - a) * b * level_texel(L, x0, y1) + a * b * level_texel(L, x1, y1);
}

struct FlowLevel {
    int w, h;
    float2 *u;               // flow
    float2 *ub, *ub_out;     // extrapolated flow: read, written (ping-pong)
    float4 *p, *p_out;       // duals (p1x, p1y, p2x, p2y): read, written (ping-pong)
    float2 *gw;              // grad I1 at x + u0, scaled to [0, 1] intensities
    float *r0;
};

__global__ void upsample_kernel(const float2 *coarse, int cw, int ch, float2 *u, int w, int h) {
    const int x = blockIdx.x * TBX + threadIdx.x, y = blockIdx.y * TBY + threadIdx.y;
    if (x >= w || y >= h) return;
    float2 v = make_float2(0.f, 0.f);
    if (coarse) {
        const float cx = 0.5f * x, cy = 0.5f * y;
        const int ix = (int)floorf(cx), iy = (int)floorf(cy);
        const float a = cx - ix, b = cy - iy;
        const float *c = (const float *)coarse;
        v.x = 2.0f * bilin(c, 2 * (int64_t)cw, 2, 0, cw, ch, ix, iy, a, b);
        v.y = 2.0f * bilin(c, 2 * (int64_t)cw, 2, 1, cw, ch, ix, iy, a, b);
    }
    u[(int64_t)y * w + x] = v;
}

__global__ void warp_kernel(FlowLevel f, LevelF I0, LevelF I1) {
    const int x = blockIdx.x * TBX + threadIdx.x, y = blockIdx.y * TBY + threadIdx.y;
    if (x >= f.w || y >= f.h) return;
    const int64_t i = (int64_t)y * f.w + x;
    const float s255 = 1.0f / 255.0f;
    const float2 u0 = f.u[i];
    const float sx = x + u0.x, sy = y + u0.y;
    const int ix = (int)floorf(sx), iy = (int)floorf(sy);
    const float a = sx - ix, b = sy - iy;
    // both scaled intensities rounded on their own (no fused multiply-add
    // across them), so equal frames give rho0 = 0 exactly
    const float I1w = __fmul_rn(level_bilin(I1, ix, iy, a, b), s255);
    const float I0s = __fmul_rn(level_texel(I0, x, y), s255);
    const int64_t gs = I1.grad_pitch / 4;
    const float gx = bilin(I1.grad, gs, 2, 0, I1.w, I1.h, ix, iy, a, b) * s255;
    const float gy = bilin(I1.grad, gs, 2, 1, I1.w, I1.h, ix, iy, a, b) * s255;
    f.gw[i] = make_float2(gx, gy);
    f.r0[i] = I1w - gx * u0.x - gy * u0.y - I0s;
    f.ub[i] = u0;
}

// One primal-dual iteration for a TBX x TBY tile, one pixel per thread.  The
// duals of the tile and of its left column and top row (which the
// divergence needs) are formed in shared memory from the extrapolated flow
// of the tile plus one pixel on every side; the flow then follows.  The
// halo duals are recomputed, not exchanged: a neighbouring tile forms the
// same values from the same inputs, so the result equals a dual launch
// followed by a primal launch.  Reads p and ub, writes p_out and ub_out
// (ping-pong: neighbours read the old fields while this tile writes).
constexpr int PW = TBX + 1, PH = TBY + 1;   // dual region
constexpr int UW = TBX + 2, UH = TBY + 2;   // extrapolated-flow region

__device__ __forceinline__ float4 dual_step(float4 p, float2 c, float2 r, float2 d, float sigma,
                                            float den) {
    const float g1x = r.x - c.x, g1y = d.x - c.x, g2x = r.y - c.y, g2y = d.y - c.y;
    float qx = (p.x + sigma * g1x) / den, qy = (p.y + sigma * g1y) / den;
    float m = sqrtf(qx * qx + qy * qy);
    if (m > 1.0f) {
        qx /= m;
        qy /= m;
    }
    float4 o;
    o.x = qx;
    o.y = qy;
    qx = (p.z + sigma * g2x) / den;
    qy = (p.w + sigma * g2y) / den;
    m = sqrtf(qx * qx + qy * qy);
    if (m > 1.0f) {
        qx /= m;
        qy /= m;
    }
    o.z = qx;
    o.w = qy;
    return o;
}

__global__ void __launch_bounds__(TBX * TBY) pd_kernel(FlowLevel f, float sigma, float eps, float tau,
                                                       float lambda) {
    __shared__ float2 sub[UH][UW];
    __shared__ float4 sp[PH][PW];
    const int tid = threadIdx.y * TBX + threadIdx.x;
    const int x0 = blockIdx.x * TBX - 1, y0 = blockIdx.y * TBY - 1;  // region origins
    for (int k = tid; k < UW * UH; k += TBX * TBY) {
        const int ry = k / UW, rx = k - ry * UW;
        const int x = x0 + rx, y = y0 + ry;
        sub[ry][rx] = (x >= 0 && x < f.w && y >= 0 && y < f.h) ? f.ub[(int64_t)y * f.w + x]
                                                                  : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float den = 1.0f + sigma * eps;
    for (int k = tid; k < PW * PH; k += TBX * TBY) {
        const int ry = k / PW, rx = k - ry * PW;
        const int x = x0 + rx, y = y0 + ry;
        float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x >= 0 && x < f.w && y >= 0 && y < f.h) {
            const float2 c = sub[ry][rx];
            const float2 r = x + 1 < f.w ? sub[ry][rx + 1] : c;
            const float2 d = y + 1 < f.h ? sub[ry + 1][rx] : c;
            pn = dual_step(f.p[(int64_t)y * f.w + x], c, r, d, sigma, den);
        }
        sp[ry][rx] = pn;
    }
    __syncthreads();
    const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;   // this pixel in the regions
    const int x = x0 + tx, y = y0 + ty;
    if (x >= f.w || y >= f.h) return;
    const int64_t i = (int64_t)y * f.w + x;
    const float4 pc = sp[ty][tx];
    f.p_out[i] = pc;
    // div of p1 = (p.x, p.y) and of p2 = (p.z, p.w), as the definition orders it
    float d1 = 0.f, d2 = 0.f;
    if (x + 1 < f.w) {
        d1 += pc.x;
        d2 += pc.z;
    }
    if (x > 0) {
        d1 -= sp[ty][tx - 1].x;
        d2 -= sp[ty][tx - 1].z;
    }
    if (y + 1 < f.h) {
        d1 += pc.y;
        d2 += pc.w;
    }
    if (y > 0) {
        d1 -= sp[ty - 1][tx].y;
        d2 -= sp[ty - 1][tx].w;
    }
    const float2 u = f.u[i];
    const float t1 = u.x + tau * d1, t2 = u.y + tau * d2;
    const float2 g = f.gw[i];
    const float g2 = g.x * g.x + g.y * g.y;
    const float rho = f.r0[i] + g.x * t1 + g.y * t2;
    const float th = tau * lambda * g2;
    float v1 = t1, v2 = t2;
    if (rho < -th) {
        v1 = t1 + tau * lambda * g.x;
        v2 = t2 + tau * lambda * g.y;
    } else if (rho > th) {
        v1 = t1 - tau * lambda * g.x;
        v2 = t2 - tau * lambda * g.y;
    } else if (g2 > 0.f) {
        v1 = t1 - rho * g.x / g2;
        v2 = t2 - rho * g.y / g2;
    }
    f.u[i] = make_float2(v1, v2);
    f.ub_out[i] = make_float2(2.0f * v1 - u.x, 2.0f * v2 - u.y);
}

// -------------------------------------------------------- mean in a box
constexpr int MNT = 256;

__global__ void box_mean_kernel(const float2 *flow, int w, int h, const float4 *boxes,
                                float4 *out) {
    const float4 b = boxes[blockIdx.x];
    // pixels with x0 <= x < x1, y0 <= y < y1 inside the frame
    int xlo = 0, xhi = -1, ylo = 0, yhi = -1;
    if (b.x <= b.z && b.y <= b.w) {  // also rejects NaN
        const float x0 = fminf(fmaxf(b.x, -1.0f), (float)w + 1.0f);
        const float x1 = fminf(fmaxf(b.z, -1.0f), (float)w + 1.0f);
        const float y0 = fminf(fmaxf(b.y, -1.0f), (float)h + 1.0f);
        const float y1 = fminf(fmaxf(b.w, -1.0f), (float)h + 1.0f);
        xlo = max((int)ceilf(x0), 0);
        xhi = min((int)ceilf(x1) - 1, w - 1);
        ylo = max((int)ceilf(y0), 0);
        yhi = min((int)ceilf(y1) - 1, h - 1);
    }
    const bool any = xlo <= xhi && ylo <= yhi;
    float sx = 0.f, sy = 0.f;
    int n = 0;
    if (any) {
        const int nx = xhi - xlo + 1;
        n = nx * (yhi - ylo + 1);
        for (int k = threadIdx.x; k < n; k += MNT) {
            const float2 v = flow[(int64_t)(ylo + k / nx) * w + xlo + k % nx];
            sx += v.x;
            sy += v.y;
        }
    }
    __shared__ float rx[MNT / 32], ry[MNT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(FULL_MASK, sx, o);
        sy += __shfl_xor_sync(FULL_MASK, sy, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rx[threadIdx.x >> 5] = sx;
        ry[threadIdx.x >> 5] = sy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tx = 0.f, ty = 0.f;
        for (int k = 0; k < MNT / 32; ++k) {
            tx += rx[k];
            ty += ry[k];
        }
        const float mx = n ? tx / (float)n : 0.f, my = n ? ty / (float)n : 0.f;
        out[blockIdx.x] = make_float4(b.x + mx, b.y + my, b.z + mx, b.w + my);
    }
}

dim3 grid2(int w, int h) { return dim3((w + TBX - 1) / TBX, (h + TBY - 1) / TBY); }

LevelF level_f(const omt_pyramid &p, int L) {
    const LevelView v = level_view(p, L);
    LevelF f;
    f.img = v.img;
    f.grad = (const float *)v.grad;
    f.img_pitch = v.img_pitch;
    f.grad_pitch = v.grad_pitch;
    f.w = v.w;
    f.h = v.h;
    f.u8 = L == 0;
    return f;
}

}  // namespace

size_t st_scratch_bytes(int w, int h) { return (size_t)w * h * 4 * 5 + 512; }

cudaError_t launch_structure_texture(const uint8_t *frame, int w, int h, size_t pitch,
                                     const omt_flow_params &fp, uint8_t *tex, size_t tpitch,
                                     void *scratch, cudaStream_t s) {
    const size_t n = (size_t)w * h;
    float *base = (float *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
    float *p0 = base, *p1 = base + 2 * n;
    cudaError_t e = cudaMemsetAsync(p0, 0, sizeof(float) * 2 * n, s);
    if (e != cudaSuccess) return e;
    StArgs a{frame, (int64_t)pitch, w, h, fp.st_theta, 0.125f, p0, p1};
    const dim3 g = grid2(w, h), b(TBX, TBY);
    for (int it = 0; it < fp.st_iters; it += 2) {
        if (it + 1 < fp.st_iters) st_step2_kernel<<<g, b, 0, s>>>(a);
        else st_step_kernel<<<g, b, 0, s>>>(a);
        const float *t = a.p;
        a.p = a.p_out;
        a.p_out = const_cast<float *>(t);
    }
    st_texture_kernel<<<g, b, 0, s>>>(a, fp.st_alpha, fp.st_k, tex, (int64_t)tpitch);
    return cudaGetLastError();
}

size_t tvl1_scratch_bytes(int w, int h) {
    // per level-0 pixel: two flow buffers for the levels above (float2 each),
    // the extrapolated flow and the duals twice (ping-pong: float2, float4),
    // the warped gradient (float2) and rho0 (float) -- 76 bytes, plus alignment
    return (size_t)w * h * 76 + 8 * 256;
}

cudaError_t launch_tvl1(const omt_pyramid &P0, const omt_pyramid &P1, const omt_flow_params &fp,
                        float2 *flow, void *scratch, cudaStream_t s) {
    const size_t n0 = (size_t)P0.w * P0.h;
    uint8_t *sp = (uint8_t *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
    auto take = [&](size_t bytes) {
        uint8_t *r = sp;
        sp += (bytes + 255) & ~(size_t)255;
        return r;
    };
    float2 *ua = (float2 *)take(8 * n0), *ucoarse = (float2 *)take(8 * n0);
    float2 *ubuf[2] = {(float2 *)take(8 * n0), (float2 *)take(8 * n0)};
    float4 *pbuf[2] = {(float4 *)take(16 * n0), (float4 *)take(16 * n0)};
    FlowLevel f;
    f.gw = (float2 *)take(8 * n0);
    f.r0 = (float *)take(4 * n0);
    const float sigma = 1.0f / sqrtf(8.0f), tau = 1.0f / sqrtf(8.0f);
    const float2 *coarse = nullptr;
    int cw = 0, ch = 0;
    cudaError_t e = cudaSuccess;
    for (int L = P0.levels - 1; L >= 0; --L) {
        const LevelF I0 = level_f(P0, L), I1 = level_f(P1, L);
        f.w = I0.w;
        f.h = I0.h;
        f.u = L == 0 ? flow : (coarse == ua ? ucoarse : ua);
        const dim3 g = grid2(f.w, f.h), b(TBX, TBY);
        upsample_kernel<<<g, b, 0, s>>>(coarse, cw, ch, f.u, f.w, f.h);
        int cur = 0;  // the p / ub buffers holding the current fields
        e = cudaMemsetAsync(pbuf[cur], 0, sizeof(float4) * (size_t)f.w * f.h, s);
        if (e != cudaSuccess) return e;
        for (int wp = 0; wp < fp.warps; ++wp) {
            f.ub = ubuf[cur];
            warp_kernel<<<g, b, 0, s>>>(f, I0, I1);
            for (int it = 0; it < fp.iters; ++it) {
                f.p = pbuf[cur];
                f.ub = ubuf[cur];
                f.p_out = pbuf[1 - cur];
                f.ub_out = ubuf[1 - cur];
                pd_kernel<<<g, b, 0, s>>>(f, sigma, fp.eps, tau, fp.lambda);
                cur = 1 - cur;
            }
        }
        coarse = f.u;
        cw = f.w;
        ch = f.h;
    }
    return cudaGetLastError();
}

cudaError_t launch_box_mean_flow(const float2 *flow, int w, int h, const float4 *boxes,
                                 int nboxes, float4 *out, cudaStream_t s) {
    if (nboxes <= 0) return cudaSuccess;
    box_mean_kernel<<<nboxes, MNT, 0, s>>>(flow, w, h, boxes, out);
    return cudaGetLastError();
}

}  // namespace omt
