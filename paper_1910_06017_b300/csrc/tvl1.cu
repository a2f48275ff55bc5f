// tvl1.cu -- the paper's dense flow engine (Section IV) and the mean-in-box
// prediction (Section V-A).
//
// Structure-texture: the ROF structure S of the u8 frame by Chambolle's dual
// projection (one or two steps per launch, q = div p - I / theta formed in
// shared memory for a tile and its halo, the dual field ping-ponged in
// global memory), then the u8 texture clamp(floor(k (I - alpha S) + 128.5)).
// Huber-TV-L1: per pyramid level (FP32 storage, coarse to fine) the flow of
// the level above is sampled bilinearly at (x/2, y/2) and doubled; per warp
// one launch samples frame t+1 and its gradient at x + u0 (taps clamped) and
// stores grad I1w and rho0, then the primal-dual iterations run one
// (pd_kernel) or two (pd2_kernel) per launch: the duals from the
// extrapolated flow (forward differences, a Huber shrink and the projection
// onto the unit disc, per flow component) in shared memory for a tile and
// its halo, then the flow (backward-difference divergence, the pointwise
// prox of the L1 data term, the extrapolation).  Every expression keeps the
// order of the definition, in FP32, and both launch forms give the same bits.
// A launch reads and writes every field once: the kernels are bound by HBM
// (or L2 for small levels).
#include <type_traits>

#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int TBX = 32, TBY = 8;   // threads of a CTA
#ifndef OMT_ST_TH
#define OMT_ST_TH 32
#endif
#ifndef OMT_PD_TH
#define OMT_PD_TH 16
#endif
constexpr int ST_TH = OMT_ST_TH, PD_TH = OMT_PD_TH;  // tile rows of the blocked kernels

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

// Asynchronous copy of N (4, 8 or 16) bytes from global into shared memory,
// or N zero bytes when !valid (nothing is read then; gmem must still be a
// valid address).  The copies of a region are issued back to back and
// awaited once, so a thread keeps all of its loads in flight together.
template <int N>
__device__ __forceinline__ void cp_zfill(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int src = valid ? N : 0;
    if constexpr (N == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(N),
                     "r"(src)
                     : "memory");
}

__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Calls fn(rx, ry) for every position of an RW x RH region, RW in
// (TBX, 2 TBX]: the TBX x TBY threads sweep its first TBX columns by rows
// (a warp per row), then the last RW - TBX columns of all rows together,
// numbered row-major across the CTA, so that no warp issues a pass for a
// few lanes per row.
template <int RW, int RH, class F>
__device__ __forceinline__ void sweep(F &&fn) {
    static_assert(RW > TBX && RW <= 2 * TBX, "region width");
    constexpr int XW = RW - TBX;
    for (int ry = threadIdx.y; ry < RH; ry += TBY) fn((int)threadIdx.x, ry);
    for (int e = threadIdx.y * TBX + threadIdx.x; e < XW * RH; e += TBX * TBY) {
        const int ry = e / XW;
        fn(TBX + e - ry * XW, ry);
    }
}

// ------------------------------------------------------ structure-texture
struct StArgs {
    const uint8_t *img;
    int64_t pitch;
    int w, h;
    float theta, rtheta, step;  // rtheta = 1 / theta
    const float *p;  // (px, py) interleaved, w x h
    float *p_out;
};

// Chambolle's projection update of the dual at a position from the forward
// differences (gx, gy) of q = div p - I / theta there.
__device__ __forceinline__ float2 st_dual(float2 pc, float gx, float gy, float step) {
    const float rm = 1.0f / (1.f + step * sqrtf(__fmaf_rn(gx, gx, __fmul_rn(gy, gy))));
    return make_float2((pc.x + step * gx) * rm, (pc.y + step * gy) * rm);
}

// div p - I / theta at an inside position from the duals there (c) and at
// the left (l) and upper (u) neighbours (xr, xl, yd, yu: a right, left,
// lower, upper neighbour inside the frame).
__device__ __forceinline__ float st_q(float2 c, float2 l, float2 u, bool xr, bool xl, bool yd,
                                      bool yu, float img, float rtheta) {
    float d = 0.f;
    if (xr) d += c.x;
    if (xl) d -= l.x;
    if (yd) d += c.y;
    if (yu) d -= u.y;
    return d - img * rtheta;
}

// One projection step for a TBX x TH tile: q on the tile plus its right
// column and bottom row in shared memory (from p on the tile plus one pixel
// on every side), then the tile's new duals from the forward differences
// of q.  Equal to forming q everywhere and then p.
template <int TH>
__global__ void __launch_bounds__(TBX * TBY) st_step_kernel(StArgs a) {
    pdl_begin();
    constexpr int QW = TBX + 1, QH = TH + 1, RW = TBX + 2, RH = TH + 2;
    __shared__ float2 spp[RH][RW];
    __shared__ float sq[QH][QW];
    const int bx = blockIdx.x * TBX, by = blockIdx.y * TH;
    auto inside = [&](int x, int y) { return x >= 0 && x < a.w && y >= 0 && y < a.h; };
    sweep<RW, RH>([&](int rx, int ry) {
        const int x = bx - 1 + rx, y = by - 1 + ry;
        const bool in = inside(x, y);
        cp_zfill<8>(&spp[ry][rx], in ? a.p + 2 * ((int64_t)y * a.w + x) : a.p, in);
    });
    cp_wait_all();
    __syncthreads();
    // q on [0, TBX] x [0, TH]; spp holds (x, y) at [ry + 1][rx + 1]
    sweep<QW, QH>([&](int rx, int ry) {
        const int x = bx + rx, y = by + ry;
        if (inside(x, y))
            sq[ry][rx] = st_q(spp[ry + 1][rx + 1], spp[ry + 1][rx], spp[ry][rx + 1], x + 1 < a.w,
                              x > 0, y + 1 < a.h, y > 0, (float)a.img[(int64_t)y * a.pitch + x],
                              a.rtheta);
    });
    __syncthreads();
    for (int ty = threadIdx.y; ty < TH; ty += TBY) {
        const int tx = threadIdx.x, x = bx + tx, y = by + ty;
        if (x >= a.w || y >= a.h) continue;
        const float qc = sq[ty][tx];
        const float gx = x + 1 < a.w ? sq[ty][tx + 1] - qc : 0.f;
        const float gy = y + 1 < a.h ? sq[ty + 1][tx] - qc : 0.f;
        const float2 pn = st_dual(spp[ty + 1][tx + 1], gx, gy, a.step);
        reinterpret_cast<float2 *>(a.p_out)[(int64_t)y * a.w + x] = pn;
    }
}

// Two projection steps for a TBX x TH tile in one launch: the duals of the
// intermediate step are formed in shared memory on the tile grown by the
// pixels the second step reads (temporal blocking), so a launch reads p and
// I once and writes p once for two steps.  Each stage updates the inside
// positions of its region from the previous stage's values, by the same
// expressions as st_step_kernel, so the result equals two st_step_kernel
// launches bit for bit; positions outside the frame are never read by a
// position inside it.
template <int TH>
__global__ void __launch_bounds__(TBX * TBY) st_step2_kernel(StArgs a) {
    pdl_begin();
    // regions (origin offset, extent) relative to the tile origin:
    // P p^n, then p^n+1 on [-1, TBX]: [-2, TBX + 1]; Q q^n: [-1, TBX + 1], then
    // q^n+1 on [0, TBX]; I the frame on Q's region
    constexpr int PW = TBX + 4, PH = TH + 4, QW = TBX + 3, QH = TH + 3;
    constexpr int P1W = TBX + 2, P1H = TH + 2, Q1W = TBX + 1, Q1H = TH + 1;
    __shared__ float2 sp[PH][PW];
    __shared__ float sq[QH][QW];
    __shared__ float si[QH][QW];
    const int w = a.w, h = a.h;
    const float *p_in = a.p;
    const uint8_t *img = a.img;
    const int64_t pitch = a.pitch;
    const float rtheta = a.rtheta, step = a.step;
    const int bx = blockIdx.x * TBX, by = blockIdx.y * TH;
    // IN: every position of the regions and its right / lower neighbour lie
    // inside the frame, so no position needs an edge test
    auto body = [&](auto in_c) {
        constexpr bool IN = decltype(in_c)::value;
        auto inside = [&](int x, int y) { return IN || (x >= 0 && x < w && y >= 0 && y < h); };
        sweep<PW, PH>([&](int rx, int ry) {
            const int x = bx - 2 + rx, y = by - 2 + ry;
            const bool in = inside(x, y);
            cp_zfill<8>(&sp[ry][rx], in ? p_in + 2 * ((int64_t)y * w + x) : p_in, in);
        });
        sweep<QW, QH>([&](int rx, int ry) {
            const int x = bx - 1 + rx, y = by - 1 + ry;
            if (inside(x, y)) si[ry][rx] = (float)img[(int64_t)y * pitch + x];
        });
        cp_wait_all();
        __syncthreads();
        // q^n on Q; Q (rx, ry) is P (rx + 1, ry + 1)
        sweep<QW, QH>([&](int rx, int ry) {
            const int x = bx - 1 + rx, y = by - 1 + ry;
            if (inside(x, y))
                sq[ry][rx] = st_q(sp[ry + 1][rx + 1], sp[ry + 1][rx], sp[ry][rx + 1],
                                  IN || x + 1 < w, IN || x > 0, IN || y + 1 < h, IN || y > 0,
                                  si[ry][rx], rtheta);
        });
        __syncthreads();
        // p^n+1 on [-1, TBX] x [-1, TH]: Q (rx, ry), P (rx + 1, ry + 1)
        sweep<P1W, P1H>([&](int rx, int ry) {
            const int x = bx - 1 + rx, y = by - 1 + ry;
            if (inside(x, y)) {
                const float qc = sq[ry][rx];
                const float gx = IN || x + 1 < w ? sq[ry][rx + 1] - qc : 0.f;
                const float gy = IN || y + 1 < h ? sq[ry + 1][rx] - qc : 0.f;
                sp[ry + 1][rx + 1] = st_dual(sp[ry + 1][rx + 1], gx, gy, step);
            }
        });
        __syncthreads();
        // q^n+1 on [0, TBX] x [0, TH]: Q (rx + 1, ry + 1), P (rx + 2, ry + 2)
        sweep<Q1W, Q1H>([&](int rx, int ry) {
            const int x = bx + rx, y = by + ry;
            if (inside(x, y))
                sq[ry + 1][rx + 1] = st_q(sp[ry + 2][rx + 2], sp[ry + 2][rx + 1], sp[ry + 1][rx + 2],
                                          IN || x + 1 < w, IN || x > 0, IN || y + 1 < h,
                                          IN || y > 0, si[ry + 1][rx + 1], rtheta);
        });
        __syncthreads();
        for (int ty = threadIdx.y; ty < TH; ty += TBY) {
            const int tx = threadIdx.x, x = bx + tx, y = by + ty;
            if (!IN && (x >= w || y >= h)) continue;
            const float qc = sq[ty + 1][tx + 1];
            const float gx = IN || x + 1 < w ? sq[ty + 1][tx + 2] - qc : 0.f;
            const float gy = IN || y + 1 < h ? sq[ty + 2][tx + 1] - qc : 0.f;
            const float2 pn = st_dual(sp[ty + 2][tx + 2], gx, gy, step);
            reinterpret_cast<float2 *>(a.p_out)[(int64_t)y * w + x] = pn;
        }
    };
    if (blockIdx.x > 0 && blockIdx.y > 0 && bx + TBX + 3 <= w && by + TH + 3 <= h)
        body(std::true_type{});
    else
        body(std::false_type{});
}

__global__ void st_texture_kernel(StArgs a, float alpha, float k, uint8_t *tex, int64_t tpitch) {
    pdl_begin();
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
    float2 *u;               // flow (updated in place by pd_kernel)
    float2 *u_out;           // flow written by pd2_kernel (ping-pong with u)
    float2 *ub, *ub_out;     // extrapolated flow: read, written (ping-pong)
    float4 *p, *p_out;       // duals (p1x, p1y, p2x, p2y): read, written (ping-pong)
    float2 *gw;              // grad I1 at x + u0, scaled to [0, 1] intensities
    float *r0;
};

__global__ void upsample_kernel(const float2 *coarse, int cw, int ch, float2 *u, int w, int h) {
    pdl_begin();
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
    pdl_begin();
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

__device__ __forceinline__ float2 project_unit(float qx, float qy) {
    // sums of two products are rounded in a fixed way (the second product
    // rounded, the first fused), so every kernel forms the same bits
    const float m2 = __fmaf_rn(qx, qx, __fmul_rn(qy, qy));
    const float r = m2 > 1.0f ? rsqrtf(m2) : 1.0f;   // x 1 leaves the value as it is
    return make_float2(qx * r, qy * r);
}

// The dual update of both flow components at a position from the
// extrapolated flow there (c) and at the right (r) and lower (d)
// neighbours: (p + sigma grad ubar) / (1 + sigma eps), then the projection
// onto the unit disc.  rden = 1 / (1 + sigma eps).
__device__ __forceinline__ float4 dual_step(float4 p, float2 c, float2 r, float2 d, float sigma,
                                            float rden) {
    const float g1x = r.x - c.x, g1y = d.x - c.x, g2x = r.y - c.y, g2y = d.y - c.y;
    const float2 q1 = project_unit((p.x + sigma * g1x) * rden, (p.y + sigma * g1y) * rden);
    const float2 q2 = project_unit((p.z + sigma * g2x) * rden, (p.w + sigma * g2y) * rden);
    return make_float4(q1.x, q1.y, q2.x, q2.y);
}

// The primal update at a position from the new duals there (pc) and at the
// left (pl) and upper (pu) neighbours: the backward-difference divergence of
// each dual field in the order the definition writes it (xr, xl, yd, yu: a
// right, left, lower, upper neighbour inside the level), then the pointwise
// prox of tau lambda |rho| at t = u + tau div p, written t - s g with
// s = -tau lambda, tau lambda or rho / |g|^2 (g = 0 leaves t).  tl = tau lambda.
__device__ __forceinline__ float2 primal_step(float4 pc, float4 pl, float4 pu, bool xr, bool xl,
                                              bool yd, bool yu, float2 u, float2 g, float r0,
                                              float tau, float tl) {
    float d1 = 0.f, d2 = 0.f;
    if (xr) {
        d1 += pc.x;
        d2 += pc.z;
    }
    if (xl) {
        d1 -= pl.x;
        d2 -= pl.z;
    }
    if (yd) {
        d1 += pc.y;
        d2 += pc.w;
    }
    if (yu) {
        d1 -= pu.y;
        d2 -= pu.w;
    }
    const float t1 = u.x + tau * d1, t2 = u.y + tau * d2;
    const float g2 = __fmaf_rn(g.x, g.x, __fmul_rn(g.y, g.y));
    const float rho = r0 + g.x * t1 + g.y * t2;
    const float th = tl * g2;
    const float q = rho / g2;
    const float sc = rho < -th ? -tl : (rho > th ? tl : (g2 > 0.f ? q : 0.f));
    return make_float2(t1 - sc * g.x, t2 - sc * g.y);
}

// The extrapolation ubar = 2 u - u_previous.
__device__ __forceinline__ float2 extrapolate(float2 v, float2 u) {
    return make_float2(2.0f * v.x - u.x, 2.0f * v.y - u.y);
}

__global__ void __launch_bounds__(TBX * TBY) pd_kernel(FlowLevel f, float sigma, float rden, float tau,
                                                       float lambda) {
    pdl_begin();
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
    for (int k = tid; k < PW * PH; k += TBX * TBY) {
        const int ry = k / PW, rx = k - ry * PW;
        const int x = x0 + rx, y = y0 + ry;
        float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x >= 0 && x < f.w && y >= 0 && y < f.h) {
            const float2 c = sub[ry][rx];
            const float2 r = x + 1 < f.w ? sub[ry][rx + 1] : c;
            const float2 d = y + 1 < f.h ? sub[ry + 1][rx] : c;
            pn = dual_step(f.p[(int64_t)y * f.w + x], c, r, d, sigma, rden);
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
    const float2 u = f.u[i];
    const float2 v = primal_step(pc, sp[ty][tx - 1], sp[ty - 1][tx], x + 1 < f.w, x > 0, y + 1 < f.h,
                                 y > 0, u, f.gw[i], f.r0[i], tau, tau * lambda);
    f.u[i] = v;
    f.ub_out[i] = extrapolate(v, u);
}

// Two primal-dual iterations for a TBX x TH tile (temporal blocking): the
// first on the tile grown by the reach of the second, in shared memory, so a
// launch reads the state once and writes it once for two iterations.
// Regions relative to the tile origin: B [-2, TBX + 1] holds ub^n (and
// later ub^n+1 on [-1, TBX]); Q [-2, TBX] holds p^n, then p^n+1, then p^n+2
// on [-1, TBX - 1]; V [-1, TBX] holds u^n, then u^n+1, and the warped
// gradient and rho0.  Each stage updates the inside positions of its region
// from the previous stage's values there and at their neighbours, by the
// same expressions as pd_kernel, so the result equals two pd_kernel launches
// bit for bit.  Positions outside the level hold zeros and are never read
// by a position inside it.  u is ping-ponged (u -> u_out), as are p and ub:
// the halos read a neighbouring tile's old state.
template <int TH>
__global__ void __launch_bounds__(TBX * TBY) pd2_kernel(FlowLevel f, float sigma, float rden,
                                                        float tau, float lambda) {
    pdl_begin();
    constexpr int BW = TBX + 4, BH = TH + 4, QW = TBX + 3, QH = TH + 3;
    constexpr int VW = TBX + 2, VH = TH + 2, RW = TBX + 1, RH = TH + 1;
    __shared__ float2 sb[BH][BW];
    __shared__ float4 sq[QH][QW];
    __shared__ float2 su[VH][VW];
    __shared__ float2 sg[VH][VW];
    __shared__ float sr[VH][VW];
    const int w = f.w, h = f.h;
    const float2 *ub = f.ub, *u_in = f.u, *gw = f.gw;
    const float4 *p_in = f.p;
    const float *r0 = f.r0;
    const float tl = tau * lambda;
    const int bx = blockIdx.x * TBX, by = blockIdx.y * TH;
    // IN: the tile and its whole halo (and their right / lower neighbours)
    // lie inside the level, so no position needs an edge test
    auto body = [&](auto in_c) {
        constexpr bool IN = decltype(in_c)::value;
        auto inside = [&](int x, int y) { return IN || (x >= 0 && x < w && y >= 0 && y < h); };
        // the state on the grown regions, zero outside the level
        sweep<QW, QH>([&](int rx, int ry) {
            const int x = bx - 2 + rx, y = by - 2 + ry;
            const bool in = inside(x, y);
            cp_zfill<16>(&sq[ry][rx], in ? p_in + (int64_t)y * w + x : p_in, in);
        });
        sweep<BW, BH>([&](int rx, int ry) {
            const int x = bx - 2 + rx, y = by - 2 + ry;
            const bool in = inside(x, y);
            cp_zfill<8>(&sb[ry][rx], in ? ub + (int64_t)y * w + x : ub, in);
        });
        sweep<VW, VH>([&](int rx, int ry) {
            const int x = bx - 1 + rx, y = by - 1 + ry;
            const bool in = inside(x, y);
            const int64_t i = in ? (int64_t)y * w + x : 0;
            cp_zfill<8>(&su[ry][rx], u_in + i, in);
            cp_zfill<8>(&sg[ry][rx], gw + i, in);
            cp_zfill<4>(&sr[ry][rx], r0 + i, in);
        });
        cp_wait_all();
        __syncthreads();
        // p^n+1 on Q; Q (rx, ry) is B (rx, ry)
        sweep<QW, QH>([&](int rx, int ry) {
            const int x = bx - 2 + rx, y = by - 2 + ry;
            if (inside(x, y)) {
                const float2 c = sb[ry][rx];
                const float2 r = IN || x + 1 < w ? sb[ry][rx + 1] : c;
                const float2 d = IN || y + 1 < h ? sb[ry + 1][rx] : c;
                sq[ry][rx] = dual_step(sq[ry][rx], c, r, d, sigma, rden);
            }
        });
        __syncthreads();
        // u^n+1 and ub^n+1 on V; V (rx, ry) is Q (rx + 1, ry + 1) and B (rx + 1, ry + 1)
        sweep<VW, VH>([&](int rx, int ry) {
            const int x = bx - 1 + rx, y = by - 1 + ry;
            if (inside(x, y)) {
                const float2 u = su[ry][rx];
                const float2 v = primal_step(sq[ry + 1][rx + 1], sq[ry + 1][rx], sq[ry][rx + 1],
                                             IN || x + 1 < w, IN || x > 0, IN || y + 1 < h,
                                             IN || y > 0, u, sg[ry][rx], sr[ry][rx], tau, tl);
                su[ry][rx] = v;
                sb[ry + 1][rx + 1] = extrapolate(v, u);
            }
        });
        __syncthreads();
        // p^n+2 on [-1, TBX - 1] x [-1, TH - 1]; (rx, ry) there is Q and B (rx + 1, ry + 1)
        sweep<RW, RH>([&](int rx, int ry) {
            const int x = bx - 1 + rx, y = by - 1 + ry;
            if (inside(x, y)) {
                const float2 c = sb[ry + 1][rx + 1];
                const float2 r = IN || x + 1 < w ? sb[ry + 1][rx + 2] : c;
                const float2 d = IN || y + 1 < h ? sb[ry + 2][rx + 1] : c;
                sq[ry + 1][rx + 1] = dual_step(sq[ry + 1][rx + 1], c, r, d, sigma, rden);
            }
        });
        __syncthreads();
        // u^n+2 on the tile; a tile pixel is Q (tx + 2, ty + 2) and V (tx + 1, ty + 1)
        for (int ty = threadIdx.y; ty < TH; ty += TBY) {
            const int tx = threadIdx.x, x = bx + tx, y = by + ty;
            if (!IN && (x >= w || y >= h)) continue;
            const int64_t i = (int64_t)y * w + x;
            const float4 pc = sq[ty + 2][tx + 2];
            const float2 u = su[ty + 1][tx + 1];
            const float2 v = primal_step(pc, sq[ty + 2][tx + 1], sq[ty + 1][tx + 2], IN || x + 1 < w,
                                         IN || x > 0, IN || y + 1 < h, IN || y > 0, u,
                                         sg[ty + 1][tx + 1], sr[ty + 1][tx + 1], tau, tl);
            f.p_out[i] = pc;
            f.u_out[i] = v;
            f.ub_out[i] = extrapolate(v, u);
        }
    };
    if (blockIdx.x > 0 && blockIdx.y > 0 && bx + TBX + 2 <= w && by + TH + 2 <= h)
        body(std::true_type{});
    else
        body(std::false_type{});
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
dim3 grid_th(int w, int h, int th) { return dim3((w + TBX - 1) / TBX, (h + th - 1) / th); }

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
    StArgs a{frame, (int64_t)pitch, w, h, fp.st_theta, 1.0f / fp.st_theta, 0.125f, p0, p1};
    const dim3 g = grid2(w, h), gs = grid_th(w, h, ST_TH), b(TBX, TBY);
    for (int it = 0; it < fp.st_iters;) {
        if (fp.block == 2 && it + 1 < fp.st_iters) {
            e = launch_pdl(st_step2_kernel<ST_TH>, gs, b, 0, s, a);
            it += 2;
        } else {
            e = launch_pdl(st_step_kernel<ST_TH>, gs, b, 0, s, a);
            it += 1;
        }
        if (e != cudaSuccess) return e;
        const float *t = a.p;
        a.p = a.p_out;
        a.p_out = const_cast<float *>(t);
    }
    e = launch_pdl(st_texture_kernel, g, b, 0, s, a, fp.st_alpha, fp.st_k, tex, (int64_t)tpitch);
    return e != cudaSuccess ? e : cudaGetLastError();
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
    const float rden = 1.0f / (1.0f + sigma * fp.eps);
    // launches per warp: pairs of iterations (pd2_kernel, u ping-ponged)
    // and single ones (pd_kernel, u in place)
    const int pairs = fp.block == 2 ? fp.iters / 2 : 0, singles = fp.iters - 2 * pairs;
    const bool odd_flips = (fp.warps * pairs) % 2 == 1;
    const float2 *coarse = nullptr;
    int cw = 0, ch = 0;
    cudaError_t e = cudaSuccess;
    for (int L = P0.levels - 1; L >= 0; --L) {
        const LevelF I0 = level_f(P0, L), I1 = level_f(P1, L);
        f.w = I0.w;
        f.h = I0.h;
        // the level's flow ends in dst; its ping-pong partner is a buffer
        // that holds neither the level above nor dst (the output buffer is
        // free until level 0).  The start buffer is chosen so that an odd
        // number of u swaps ends in dst.
        float2 *other_flow = coarse == ua ? ucoarse : ua;
        float2 *dst = L == 0 ? flow : other_flow;
        float2 *partner = L == 0 ? other_flow : flow;
        float2 *ucur = odd_flips ? partner : dst, *unext = odd_flips ? dst : partner;
        const dim3 g = grid2(f.w, f.h), gp = grid_th(f.w, f.h, PD_TH), b(TBX, TBY);
        e = launch_pdl(upsample_kernel, g, b, 0, s, coarse, cw, ch, ucur, f.w, f.h);
        if (e != cudaSuccess) return e;
        int cur = 0;  // the p / ub buffers holding the current fields
        e = cudaMemsetAsync(pbuf[cur], 0, sizeof(float4) * (size_t)f.w * f.h, s);
        if (e != cudaSuccess) return e;
        for (int wp = 0; wp < fp.warps; ++wp) {
            f.u = ucur;
            f.ub = ubuf[cur];
            e = launch_pdl(warp_kernel, g, b, 0, s, f, I0, I1);
            if (e != cudaSuccess) return e;
            for (int it = 0; it < pairs + singles; ++it) {
                f.p = pbuf[cur];
                f.ub = ubuf[cur];
                f.p_out = pbuf[1 - cur];
                f.ub_out = ubuf[1 - cur];
                f.u = ucur;
                if (it < pairs) {
                    f.u_out = unext;
                    e = launch_pdl(pd2_kernel<PD_TH>, gp, b, 0, s, f, sigma, rden, tau, fp.lambda);
                    float2 *t = ucur;
                    ucur = unext;
                    unext = t;
                } else {
                    e = launch_pdl(pd_kernel, g, b, 0, s, f, sigma, rden, tau, fp.lambda);
                }
                if (e != cudaSuccess) return e;
                cur = 1 - cur;
            }
        }
        coarse = ucur;
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
