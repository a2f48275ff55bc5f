// lk.cu -- K3: pyramidal iterative Lucas-Kanade (Bouguet), the sparse
// stand-in for the dense motion field of Section V-A (feature calculation).
//
// One warp per point, lane c owning window column c.  Per level the warp
// walks the (win+1) texel rows of the window once: each lane loads the texel
// of its column, takes the right neighbour from lane c+1 with a shuffle, and
// interpolates horizontally; the vertical interpolation reuses the previous
// row.  The frame-t window (I, Ix, Iy) stays in registers for all
// iterations, so an iteration reads one frame-(t+1) texel per lane and row,
// and the two sums of b (and the three of G) are warp butterfly reductions.
// All lanes end with identical sums, so the control flow stays uniform, and
// the reduction order is fixed: a point's result does not depend on the
// launch shape or on its neighbours in the batch.
//
// Solve: det = Gxx Gyy - Gxy^2 by Kahan's fused form, lambda_min =
// det / lambda_max (no cancellation), eta = G^-1 b by the 2x2 adjugate.
#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int LK_NT = 256;
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

template <int ST, int WIN>
__global__ void __launch_bounds__(LK_NT) lk_kernel(const __grid_constant__ LKArgs a) {
    constexpr int R = WIN / 2;
    const int lane = threadIdx.x & 31;
    const bool loader = lane <= WIN;  // texel columns 0..WIN
    const bool tapcol = lane < WIN;   // window columns 0..WIN-1
    int n = a.n_max;
    if (a.n_dev) {
        const int m = *a.n_dev;
        n = m < n ? m : n;
    }
    const int nwarps = gridDim.x * LK_WARPS;
    for (int i = blockIdx.x * LK_WARPS + (threadIdx.x >> 5); i < n; i += nwarps) {
        const float2 u = a.pts[i];
        float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f;
        int st = OMT_PT_OK;
        bool nonconv = false;
        unsigned long long itp = 0ull;  // iterations per level, 8 bits each

        for (int L = a.levels - 1; L >= 0; --L) {
            const LevelView &P = a.P[L];
            const LevelView &J = a.J[L];
            const float sc = __int_as_float((127 - L) << 23);  // 2^-L, exact
            const float px = u.x * sc, py = u.y * sc;
            const float fpx = floorf(px), fpy = floorf(py);
            const int ipx = (int)fpx, ipy = (int)fpy;
            const float ax = px - fpx, ay = py - fpy;

            // Frame-t window: I, Ix, Iy at p + (i, j), bilinear.
            float Iw[WIN], Xw[WIN], Yw[WIN];
            {
                const int tx = clampi(ipx + lane - R, 0, P.w - 1);
                float pI = 0.f, pX = 0.f, pY = 0.f;
#pragma unroll
                for (int tr = 0; tr <= WIN; ++tr) {
                    const int ty = clampi(ipy + tr - R, 0, P.h - 1);
                    float v = 0.f;
                    float2 g = make_float2(0.f, 0.f);
                    if (loader) {
                        v = load_level<ST>(P, L, tx, ty);
                        g = load_grad<ST>(P, tx, ty);
                    }
                    const float v1 = __shfl_down_sync(FULL_MASK, v, 1);
                    const float g1x = __shfl_down_sync(FULL_MASK, g.x, 1);
                    const float g1y = __shfl_down_sync(FULL_MASK, g.y, 1);
                    const float hI = fmaf(ax, v1 - v, v);
                    const float hX = fmaf(ax, g1x - g.x, g.x);
                    const float hY = fmaf(ax, g1y - g.y, g.y);
                    if (tr > 0) {
                        Iw[tr - 1] = fmaf(ay, hI - pI, pI);
                        Xw[tr - 1] = fmaf(ay, hX - pX, pX);
                        Yw[tr - 1] = fmaf(ay, hY - pY, pY);
                    }
                    pI = hI;
                    pX = hX;
                    pY = hY;
                }
            }
            float sxx = 0.f, sxy = 0.f, syy = 0.f;
            if (tapcol) {
#pragma unroll
                for (int r = 0; r < WIN; ++r) {
                    sxx = fmaf(Xw[r], Xw[r], sxx);
                    sxy = fmaf(Xw[r], Yw[r], sxy);
                    syy = fmaf(Yw[r], Yw[r], syy);
                }
            }
            sxx = warp_sum(sxx);
            sxy = warp_sum(sxy);
            syy = warp_sum(syy);
            const float det = det2(sxx, syy, sxy);
            const float dd = sxx - syy;
            const float lmax = 0.5f * ((sxx + syy) + sqrtf(fmaf(dd, dd, 4.0f * sxy * sxy)));
            const float lmin = det / lmax;
            if (!(lmin >= a.tau_n) || !(lmin > 0.f)) {
                st = OMT_PT_LOST_EIG;
                break;
            }

            float nux = 0.f, nuy = 0.f;
            int k = 0;
            bool conv = false;
            while (k < a.max_iter) {
                // Centre c = p + g + nu, held as (ipx, ipy) + (cx, cy).
                const float cx = ax + gx + nux, cy = ay + gy + nuy;
                if (!(fabsf(cx) < 1.0e8f) || !(fabsf(cy) < 1.0e8f)) {
                    st = OMT_PT_LOST_OOB;
                    break;
                }
                const float fcx = floorf(cx), fcy = floorf(cy);
                const int jx = ipx + (int)fcx, jy = ipy + (int)fcy;
                const float bx = cx - fcx, by = cy - fcy;
                if (jx < -R || jx > J.w - 1 + R || (jx == J.w - 1 + R && bx > 0.f) ||
                    jy < -R || jy > J.h - 1 + R || (jy == J.h - 1 + R && by > 0.f)) {
                    st = OMT_PT_LOST_OOB;
                    break;
                }
                const int txj = clampi(jx + lane - R, 0, J.w - 1);
                float sbx = 0.f, sby = 0.f, ph = 0.f;
#pragma unroll
                for (int tr = 0; tr <= WIN; ++tr) {
                    const int ty = clampi(jy + tr - R, 0, J.h - 1);
                    const float v = loader ? load_level<ST>(J, L, txj, ty) : 0.f;
                    const float v1 = __shfl_down_sync(FULL_MASK, v, 1);
                    const float hv = fmaf(bx, v1 - v, v);
                    if (tr > 0) {
                        const float jv = fmaf(by, hv - ph, ph);
                        const float dI = Iw[tr - 1] - jv;
                        sbx = fmaf(dI, Xw[tr - 1], sbx);
                        sby = fmaf(dI, Yw[tr - 1], sby);
                    }
                    ph = hv;
                }
                if (!tapcol) {
                    sbx = 0.f;
                    sby = 0.f;
                }
                sbx = warp_sum(sbx);
                sby = warp_sum(sby);
                const float ex = (syy * sbx - sxy * sby) / det;
                const float ey = (sxx * sby - sxy * sbx) / det;
                nux += ex;
                nuy += ey;
                ++k;
                if (ex * ex + ey * ey < a.eps2) {
                    conv = true;
                    break;
                }
            }
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
            if (!(ox >= 0.f && ox <= (float)(a.P[0].w - 1) && oy >= 0.f && oy <= (float)(a.P[0].h - 1)))
                st = OMT_PT_LOST_OOB;
            else
                v = make_float2(ox, oy);
        }
        if (st == OMT_PT_OK && nonconv) st |= OMT_PT_NONCONV;
        if (lane == 0) {
            a.out[i] = v;
            a.status[i] = (uint8_t)st;
        }
        if (a.iters && lane < a.levels)
            a.iters[(int64_t)i * a.levels + lane] = (uint8_t)(itp >> (8 * lane));
    }
}

template <int ST>
cudaError_t launch_st(const LKArgs &a, int win, int grid, cudaStream_t s) {
    switch (win) {
#define OMT_LK_CASE(W) \
    case W: lk_kernel<ST, W><<<grid, LK_NT, 0, s>>>(a); break;
        OMT_LK_CASE(3) OMT_LK_CASE(5) OMT_LK_CASE(7) OMT_LK_CASE(9) OMT_LK_CASE(11)
        OMT_LK_CASE(13) OMT_LK_CASE(15) OMT_LK_CASE(17) OMT_LK_CASE(19) OMT_LK_CASE(21)
        OMT_LK_CASE(23) OMT_LK_CASE(25) OMT_LK_CASE(27) OMT_LK_CASE(29) OMT_LK_CASE(31)
#undef OMT_LK_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

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
    const int cap = sms * 16;
    const int grid = need < cap ? need : cap;
    if (prev.storage == OMT_F32) return launch_st<OMT_F32>(a, prm.win, grid, s);
    return launch_st<OMT_F16>(a, prm.win, grid, s);
}

}  // namespace omt
