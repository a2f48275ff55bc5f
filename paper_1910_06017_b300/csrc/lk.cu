// lk.cu -- K3: pyramidal iterative Lucas-Kanade (Bouguet), the sparse
// stand-in for the dense motion field of Section V-A (feature calculation).
//
// One warp per point, lane c owning window column c.  Per level the warp
// walks the (win+1) texel rows of its window: each lane loads the texel of
// its column, takes the right neighbour from lane c+1 with a shuffle, and
// interpolates horizontally, then vertically reusing the previous row.  The
// frame-t window keeps only (Ix, Iy) per tap in registers (its rows are
// loaded in batches of 8); b = sum (I - J) grad I is formed as
// c - sum J grad I with the level constant c = sum I grad I, so an iteration
// reads one frame-(t+1) texel per lane and row.  The sums of b (and of G, c)
// are warp butterfly reductions.
// All lanes end with identical sums, so the control flow stays uniform, and
// the reduction order is fixed: a point's result does not depend on the
// launch shape or on its neighbours in the batch.
//
// Solve: det = Gxx Gyy - Gxy^2 by Kahan's fused form, lambda_min =
// det / lambda_max (no cancellation), eta = G^-1 b by the 2x2 adjugate.
#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int LK_NT = 128;
constexpr int LK_WARPS = LK_NT / 32;

struct LKArgs {
    LevelView P[OMT_MAX_LEVELS];
    LevelView J[OMT_MAX_LEVELS];
    const float2 *pts;
    const int32_t *n_dev;
    float2 *out;
    uint8_t *status;
    uint8_t *iters;
    int levels;
    int n_max;
    int max_iter;
    float eps2;   // eps^2
    float tau_n;  // tau * win^2
};

// a*d - b*b with one rounding error of the result (Kahan).
__device__ __forceinline__ float det2(float a, float d, float b) {
    const float w = b * b;
    const float e = fmaf(-b, b, w);
    const float f = fmaf(a, d, -w);
    return f + e;
}

// Image value at an in-range pixel: u8 for level 0, else float or
// half(I - 128).  One code path for all levels keeps the register budget
// of a single inlined copy; the branch is uniform across the warp.
template <int ST>
__device__ __forceinline__ float texel(const uint8_t *row, int x, bool u8) {
    if (u8) return (float)__ldg(row + x);
    if (ST == OMT_F32) return __ldg((const float *)row + x);
    return __half2float(__ldg((const __half *)row + x)) + 128.0f;
}

// Frame-t window of one level: (Ix, Iy) per tap row in registers, and the
// level constants G (three sums) and c = sum I (Ix, Iy).
template <int ST, int WIN>
__device__ __forceinline__ void template_window(const LevelView &P, int ipx, int ipy, float ax,
                                                float ay, int lane, bool u8, float (&Xw)[WIN],
                                                float (&Yw)[WIN], float &sxx, float &sxy,
                                                float &syy, float &cx, float &cy) {
    constexpr int R = WIN / 2;
    constexpr int CH = 8;  // texel rows loaded per batch (bounds live registers)
    const bool loader = lane <= WIN, tapcol = lane < WIN;
    const int tx = clampi(ipx + lane - R, 0, P.w - 1);
    float pI = 0.f, pX = 0.f, pY = 0.f;
    float cx0 = 0.f, cy0 = 0.f, cx1 = 0.f, cy1 = 0.f;
    sxx = sxy = syy = 0.f;
#pragma unroll
    for (int t0 = 0; t0 <= WIN; t0 += CH) {
        float v[CH];
        float2 g[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int tr = t0 + c;
            v[c] = 0.f;
            g[c] = make_float2(0.f, 0.f);
            if (tr <= WIN && loader) {
                const int ty = clampi(ipy + tr - R, 0, P.h - 1);
                v[c] = texel<ST>(P.img + (int64_t)ty * P.img_pitch, tx, u8);
                g[c] = load_grad<ST>(P, tx, ty);
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int tr = t0 + c;
            if (tr > WIN) break;
            const float v1 = __shfl_down_sync(FULL_MASK, v[c], 1);
            const float g1x = __shfl_down_sync(FULL_MASK, g[c].x, 1);
            const float g1y = __shfl_down_sync(FULL_MASK, g[c].y, 1);
            const float hI = fmaf(ax, v1 - v[c], v[c]);
            const float hX = fmaf(ax, g1x - g[c].x, g[c].x);
            const float hY = fmaf(ax, g1y - g[c].y, g[c].y);
            if (tr > 0) {
                const float I = fmaf(ay, hI - pI, pI);
                const float X = fmaf(ay, hX - pX, pX);
                const float Y = fmaf(ay, hY - pY, pY);
                Xw[tr - 1] = X;
                Yw[tr - 1] = Y;
                sxx = fmaf(X, X, sxx);
                sxy = fmaf(X, Y, sxy);
                syy = fmaf(Y, Y, syy);
                // Same two chains as correlate_window, so that J == I gives
                // c - sum J grad I == 0 exactly (zero flow on equal frames).
                if (tr & 1) {
                    cx0 = fmaf(I, X, cx0);
                    cy0 = fmaf(I, Y, cy0);
                } else {
                    cx1 = fmaf(I, X, cx1);
                    cy1 = fmaf(I, Y, cy1);
                }
            }
            pI = hI;
            pX = hX;
            pY = hY;
        }
    }
    if (!tapcol) sxx = sxy = syy = 0.f;
    cx = tapcol ? cx0 + cx1 : 0.f;
    cy = tapcol ? cy0 + cy1 : 0.f;
}

// ------------------------------------------------------------ J staging
// Each warp stages frame t+1's search region of one level in shared memory:
// SH texel rows around the window with MARGIN texels of slack on every
// side, stored as (J(x), J(x+1)) pairs so that a tap row of an iteration is
// one 8-byte shared load per lane.  Texels are clamped to the level and
// converted to float once, at staging; the region is restaged only when the
// iteration centre moves more than MARGIN texels from where it was staged.
constexpr int MARGIN = 4;

template <int WIN>
struct StageDims {
    static constexpr int R = WIN / 2;
    static constexpr int SH = WIN + 1 + 2 * MARGIN;  // texel rows
    static constexpr int SP = WIN + 2 * MARGIN;      // pairs per row
    static constexpr int PAIRS = SH * SP;            // float2 per warp
};

template <int ST, int WIN>
__device__ __forceinline__ void stage_region(const LevelView &J, bool u8, int jx, int jy, int lane,
                                             float *S) {
    using D = StageDims<WIN>;
    const int sx0 = jx - D::R - MARGIN, sy0 = jy - D::R - MARGIN;
    __syncwarp();
#pragma unroll 2
    for (int r = 0; r < D::SH; ++r) {
        const int y = clampi(sy0 + r, 0, J.h - 1);
        const uint8_t *row = J.img + (int64_t)y * J.img_pitch;
        for (int c = lane; c <= D::SP; c += 32) {
            const float v = texel<ST>(row, clampi(sx0 + c, 0, J.w - 1), u8);
            if (c < D::SP) S[2 * (r * D::SP + c)] = v;
            if (c >= 1) S[2 * (r * D::SP + c - 1) + 1] = v;
        }
    }
    __syncwarp();
}

// Two warp sums at once: lanes 0-15 end with the total of a, lanes 16-31
// with the total of b (one exchange, then butterflies within each half);
// returns both totals in every lane.  Fixed order: every lane gets the same
// bits, and equal inputs give equal outputs whatever they are paired with.
__device__ __forceinline__ void warp_sum2(float &a, float &b, int lane) {
    const bool hi = (lane & 16) != 0;
    float keep = hi ? b : a;
    const float give = hi ? a : b;
    keep += __shfl_xor_sync(FULL_MASK, give, 16);
#pragma unroll
    for (int m = 8; m > 0; m >>= 1) keep += __shfl_xor_sync(FULL_MASK, keep, m);
    a = __shfl_sync(FULL_MASK, keep, 0);
    b = __shfl_sync(FULL_MASK, keep, 16);
}

// sum over the window of J(c + (i, j)) (Ix, Iy) from the staged region; the
// window's top-left tap sits at pair (oy, ox) of the region.
template <int WIN>
__device__ __forceinline__ void correlate_staged(const float2 *S, int ox, int oy, float bx, float by,
                                                 int lane, const float (&Xw)[WIN],
                                                 const float (&Yw)[WIN], float &sx, float &sy) {
    using D = StageDims<WIN>;
    const bool tapcol = lane < WIN;
    const float2 *base = S + oy * D::SP + ox + (tapcol ? lane : 0);
    float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f, ph = 0.f;
#pragma unroll
    for (int tr = 0; tr <= WIN; ++tr) {
        const float2 pv = base[tr * D::SP];
        const float h = fmaf(bx, pv.y - pv.x, pv.x);
        if (tr > 0) {
            const float jv = fmaf(by, h - ph, ph);
            if (tr & 1) {
                ax0 = fmaf(jv, Xw[tr - 1], ax0);
                ay0 = fmaf(jv, Yw[tr - 1], ay0);
            } else {
                ax1 = fmaf(jv, Xw[tr - 1], ax1);
                ay1 = fmaf(jv, Yw[tr - 1], ay1);
            }
        }
        ph = h;
    }
    sx = tapcol ? ax0 + ax1 : 0.f;
    sy = tapcol ? ay0 + ay1 : 0.f;
}

// One level of the pyramidal iteration for one point (the whole warp).
// Returns the status after this level; nu is the level's increment.
template <int ST, int WIN>
__device__ __forceinline__ int track_level(const LevelView &P, const LevelView &J, float px,
                                           float py, float gx, float gy, int max_iter,
                                           float eps2, float tau_n, int lane, bool u8, float *Sw,
                                           float &nux, float &nuy, int &k, bool &conv) {
    constexpr int R = WIN / 2;
    const float fpx = floorf(px), fpy = floorf(py);
    const int ipx = (int)fpx, ipy = (int)fpy;
    const float ax = px - fpx, ay = py - fpy;
    float Xw[WIN], Yw[WIN];
    float sxx, sxy, syy, cx, cy;
    template_window<ST, WIN>(P, ipx, ipy, ax, ay, lane, u8, Xw, Yw, sxx, sxy, syy, cx, cy);
    sxx = warp_sum(sxx);
    sxy = warp_sum(sxy);
    syy = warp_sum(syy);
    warp_sum2(cx, cy, lane);
    const float det = det2(sxx, syy, sxy);
    const float dd = sxx - syy;
    const float lmax = 0.5f * ((sxx + syy) + sqrtf(fmaf(dd, dd, 4.0f * sxy * sxy)));
    const float lmin = det / lmax;
    nux = nuy = 0.f;
    k = 0;
    conv = false;
    if (!(lmin >= tau_n) || !(lmin > 0.f)) return OMT_PT_LOST_EIG;
    const float2 *S = (const float2 *)Sw;
    int sjx = 0, sjy = 0;
    bool staged = false;
    while (k < max_iter) {
        // Centre c = p + g + nu, held as (ipx, ipy) + (ccx, ccy).
        const float ccx = ax + gx + nux, ccy = ay + gy + nuy;
        if (!(fabsf(ccx) < 1.0e8f) || !(fabsf(ccy) < 1.0e8f)) return OMT_PT_LOST_OOB;
        const float fcx = floorf(ccx), fcy = floorf(ccy);
        const int jx = ipx + (int)fcx, jy = ipy + (int)fcy;
        const float bx = ccx - fcx, by = ccy - fcy;
        if (jx < -R || jx > J.w - 1 + R || (jx == J.w - 1 + R && bx > 0.f) || jy < -R ||
            jy > J.h - 1 + R || (jy == J.h - 1 + R && by > 0.f))
            return OMT_PT_LOST_OOB;
        if (!staged || abs(jx - sjx) > MARGIN || abs(jy - sjy) > MARGIN) {
            stage_region<ST, WIN>(J, u8, jx, jy, lane, Sw);
            sjx = jx;
            sjy = jy;
            staged = true;
        }
        float sx, sy;
        correlate_staged<WIN>(S, jx - sjx + MARGIN, jy - sjy + MARGIN, bx, by, lane, Xw, Yw, sx,
                              sy);
        warp_sum2(sx, sy, lane);
        const float bbx = cx - sx, bby = cy - sy;  // b = sum (I - J) grad I
        const float ex = (syy * bbx - sxy * bby) / det;
        const float ey = (sxx * bby - sxy * bbx) / det;
        nux += ex;
        nuy += ey;
        ++k;
        if (ex * ex + ey * ey < eps2) {
            conv = true;
            break;
        }
    }
    return OMT_PT_OK;
}

// The whole pyramidal iteration for one point u (the whole warp); P, J are
// the frame-t and frame-(t+1) level views.  Writes pts_out / status / iters
// entry i.
template <int ST, int WIN>
__device__ __forceinline__ void lk_point(const LevelView *P, const LevelView *J, int levels,
                                         int max_iter, float eps2, float tau_n, float2 u,
                                         int i, float2 *out, uint8_t *status, uint8_t *iters,
                                         float *Sw) {
    const int lane = threadIdx.x & 31;
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f;
    int st = OMT_PT_OK;
    bool nonconv = false;
    unsigned long long itp = 0ull;  // iterations per level, 8 bits each

    for (int L = levels - 1; L >= 0; --L) {
        const float sc = __int_as_float((127 - L) << 23);  // 2^-L, exact
        float nux, nuy;
        int k;
        bool conv;
        st = track_level<ST, WIN>(P[L], J[L], u.x * sc, u.y * sc, gx, gy, max_iter, eps2, tau_n,
                                  lane, L == 0, Sw, nux, nuy, k, conv);
        itp |= (unsigned long long)k << (8 * L);
        if (st != OMT_PT_OK) break;
        if (!conv) nonconv = true;
        if (L > 0) {
            gx = 2.0f * (gx + nux);
            gy = 2.0f * (gy + nuy);
        } else {
            dx = gx + nux;
            dy = gy + nuy;
        }
    }

    float2 v = u;
    if (st == OMT_PT_OK) {
        const float ox = u.x + dx, oy = u.y + dy;
        if (!(ox >= 0.f && ox <= (float)(P[0].w - 1) && oy >= 0.f && oy <= (float)(P[0].h - 1)))
            st = OMT_PT_LOST_OOB;
        else
            v = make_float2(ox, oy);
    }
    if (st == OMT_PT_OK && nonconv) st |= OMT_PT_NONCONV;
    if (lane == 0) {
        out[i] = v;
        status[i] = (uint8_t)st;
    }
    if (iters && lane < levels) iters[(int64_t)i * levels + lane] = (uint8_t)(itp >> (8 * lane));
}

// Staging buffer of this warp in the block's dynamic shared memory.
template <int WIN>
__device__ __forceinline__ float *warp_stage() {
    extern __shared__ __align__(16) float lk_smem[];
    return lk_smem + (size_t)(threadIdx.x >> 5) * StageDims<WIN>::PAIRS * 2;
}

template <int WIN>
constexpr size_t stage_bytes() {
    return (size_t)LK_WARPS * StageDims<WIN>::PAIRS * sizeof(float2);
}

template <int ST, int WIN>
__global__ void __launch_bounds__(LK_NT) lk_kernel(const __grid_constant__ LKArgs a) {
    float *Sw = warp_stage<WIN>();
    int n = a.n_max;
    if (a.n_dev) {
        const int m = *a.n_dev;
        n = m < n ? m : n;
    }
    const int nwarps = gridDim.x * LK_WARPS;
    for (int i = blockIdx.x * LK_WARPS + (threadIdx.x >> 5); i < n; i += nwarps)
        lk_point<ST, WIN>(a.P, a.J, a.levels, a.max_iter, a.eps2, a.tau_n, a.pts[i], i, a.out,
                          a.status, a.iters, Sw);
}

// All points of all streams of a batch: the per-stream counts come from the
// CSR offsets written by the corner step; each CTA forms their prefix in
// shared memory and its warps stride over the concatenated index space.
template <int ST, int WIN>
__global__ void __launch_bounds__(LK_NT) lk_batch_kernel(const uint8_t *table) {
    __shared__ int32_t pre[OMT_BATCH_MAX_STREAMS + 1];
    float *Sw = warp_stage<WIN>();
    const BatchView t(table);
    const BatchHeader &h = t.hdr();
    const int ns = h.nstreams;
    if (threadIdx.x == 0) {
        int acc = 0;
        pre[0] = 0;
        for (int s = 0; s < ns; ++s) {
            const StreamEntry &e = t.stream(s);
            acc += e.offsets[e.nboxes];
            pre[s + 1] = acc;
        }
    }
    __syncthreads();
    const int total = pre[ns];
    const int nwarps = gridDim.x * LK_WARPS;
    for (int g = blockIdx.x * LK_WARPS + (threadIdx.x >> 5); g < total; g += nwarps) {
        const int s = find_segment(pre, ns, g);
        const StreamEntry &e = t.stream(s);
        const int i = g - pre[s];
        lk_point<ST, WIN>(e.P, e.P_next, h.levels, h.max_iter, h.eps2, h.tau_n, e.pts[i], i,
                          e.pts_out, e.status, e.iters, Sw);
    }
}

template <int ST>
cudaError_t launch_st(const LKArgs &a, int win, int grid, cudaStream_t s) {
    switch (win) {
#define OMT_LK_CASE(W)                                                                    \
    case W:                                                                               \
        if (cudaFuncSetAttribute(lk_kernel<ST, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)stage_bytes<W>()) != cudaSuccess)                  \
            return cudaGetLastError();                                                    \
        lk_kernel<ST, W><<<grid, LK_NT, stage_bytes<W>(), s>>>(a);                        \
        break;
        OMT_LK_CASE(3) OMT_LK_CASE(5) OMT_LK_CASE(7) OMT_LK_CASE(9) OMT_LK_CASE(11)
        OMT_LK_CASE(13) OMT_LK_CASE(15) OMT_LK_CASE(17) OMT_LK_CASE(19) OMT_LK_CASE(21)
        OMT_LK_CASE(23) OMT_LK_CASE(25) OMT_LK_CASE(27) OMT_LK_CASE(29) OMT_LK_CASE(31)
#undef OMT_LK_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int ST, int WIN>
cudaError_t launch_batch_win(const uint8_t *table, int sms, cudaStream_t s) {
    const size_t smem = stage_bytes<WIN>();
    cudaError_t e = cudaFuncSetAttribute(lk_batch_kernel<ST, WIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lk_batch_kernel<ST, WIN>, LK_NT, smem);
    if (per_sm < 1) per_sm = 1;
    lk_batch_kernel<ST, WIN><<<sms * per_sm, LK_NT, smem, s>>>(table);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_batch_st(const uint8_t *table, int win, int sms, cudaStream_t s) {
    switch (win) {
#define OMT_LK_CASE(W) \
    case W: return launch_batch_win<ST, W>(table, sms, s);
        OMT_LK_CASE(3) OMT_LK_CASE(5) OMT_LK_CASE(7) OMT_LK_CASE(9) OMT_LK_CASE(11)
        OMT_LK_CASE(13) OMT_LK_CASE(15) OMT_LK_CASE(17) OMT_LK_CASE(19) OMT_LK_CASE(21)
        OMT_LK_CASE(23) OMT_LK_CASE(25) OMT_LK_CASE(27) OMT_LK_CASE(29) OMT_LK_CASE(31)
#undef OMT_LK_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_lk_batch(const uint8_t *table, int storage, int win, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (storage == OMT_F32) return launch_batch_st<OMT_F32>(table, win, sms, s);
    return launch_batch_st<OMT_F16>(table, win, sms, s);
}

cudaError_t launch_lk(const omt_pyramid &prev, const omt_pyramid &next, const float2 *pts,
                      int n_max, const int32_t *n_dev, const omt_params &prm, float2 *out,
                      uint8_t *status, uint8_t *iters, cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    LKArgs a;
    for (int L = 0; L < OMT_MAX_LEVELS; ++L) {
        if (L < prev.levels) {
            a.P[L] = level_view(prev, L);
            a.J[L] = level_view(next, L);
        } else {
            a.P[L] = a.P[0];
            a.J[L] = a.J[0];
        }
    }
    a.pts = pts;
    a.n_dev = n_dev;
    a.out = out;
    a.status = status;
    a.iters = iters;
    a.levels = prev.levels;
    a.n_max = n_max;
    a.max_iter = prm.max_iter;
    a.eps2 = prm.eps * prm.eps;
    a.tau_n = prm.min_eig * (float)(prm.win * prm.win);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = (n_max + LK_WARPS - 1) / LK_WARPS;
    const int cap = sms * 32;
    const int grid = need < cap ? need : cap;
    if (prev.storage == OMT_F32) return launch_st<OMT_F32>(a, prm.win, grid, s);
    return launch_st<OMT_F16>(a, prm.win, grid, s);
}

}  // namespace omt
