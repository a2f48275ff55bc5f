/*
 * omt_oracle.c -- plain, slow FP64 CPU oracle of the box-tracking hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant with the
 * CUDA library; it is written straight from the definitions below, in the
 * order the method states them, with no blocking, fusion or reordering.
 *
 * What the paper fixes and what comes from the published methods:
 *   - Section V-A (preprocessing): the frame is downscaled by a Gaussian
 *     pyramid.  The paper gives no kernel, so the 5-tap binomial
 *     [1 4 6 4 1]/16 in each direction (Burt & Adelson) is used, with a
 *     reflect-101 border, decimation to the even pixels and level sizes
 *     rounded up: W_L = (W_{L-1} + 1) / 2.
 *   - Section V-A (feature calculation) + Section IV: the motion between
 *     I_{t-1} and I_t.  The dense field is replaced by sparse pyramidal
 *     Lucas-Kanade (Bouguet's formulation) on Shi-Tomasi corners.
 *   - Section V-A (prediction): each box moves by an aggregate of the motion
 *     inside it; the paper's aggregate is the mean, the median is the
 *     default here and the mean is a flag.
 * Conventions: pixel centres at integer coordinates; a level-L coordinate
 * is the level-0 coordinate times 2^-L; boxes are (x0, y0, x1, y1) floats,
 * half-open, in level-0 pixels.
 *
 * Pins: every function here is checked by the not-gpu tests against closed
 * forms, invariants, brute force or library routines (see tests/).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 1
#define ORC_LOST_EIG 2
#define ORC_LOST_OOB 4
#define ORC_NONCONV 8
#define ORC_LOST_FB 16

/* ---------------------------------------------------------------- borders */

/* Reflect-101 index (mirror about the edge pixel, edge not repeated);
 * folds any offset back into [0, n).  A single-pixel axis maps to 0. */
static int reflect101(int i, int n)
{
    if (n == 1) return 0;
    int period = 2 * n - 2;
    i %= period;
    if (i < 0) i += period;
    return i < n ? i : period - i;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int orc_reflect101(int i, int n) { return reflect101(i, n); }

/* ---------------------------------------------------------------- pyramid */

/* Size of pyramid level L: each level halves the previous one, rounding up. */
void orc_level_size(int w, int h, int level, int *lw, int *lh)
{
    for (int l = 0; l < level; ++l) { w = (w + 1) >> 1; h = (h + 1) >> 1; }
    *lw = w; *lh = h;
}

/* One Gaussian (binomial 5x5) reduce step, Section V-A preprocessing:
 *   out(X, Y) = sum_{i,j=-2..2} k_i k_j in(r(2X+i), r(2Y+j)) / 256,
 * k = (1, 4, 6, 4, 1), r = reflect-101.  The full 2-D sum is written out,
 * term by term, as the definition states it. */
static void reduce_level(const double *in, int w, int h, double *out, int ow, int oh)
{
    static const double k[5] = {1.0, 4.0, 6.0, 4.0, 1.0};
    for (int Y = 0; Y < oh; ++Y)
        for (int X = 0; X < ow; ++X) {
            double s = 0.0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i) {
                    int x = reflect101(2 * X + i, w), y = reflect101(2 * Y + j, h);
                    s += k[i + 2] * k[j + 2] * in[(size_t)y * w + x];
                }
            out[(size_t)Y * ow + X] = s / 256.0;
        }
}

/* Scharr derivative of one level, in intensity per level pixel:
 *   Ix(x, y) = sum_{d=-1..1} s_d (I(r(x+1), r(y+d)) - I(r(x-1), r(y+d))) / 32
 *   Iy(x, y) = sum_{d=-1..1} s_d (I(r(x+d), r(y+1)) - I(r(x+d), r(y-1))) / 32
 * with s = (3, 10, 3): the central difference [-1 0 1]/2 across, smoothed by
 * [3 10 3]/16 along the other axis.  grad is interleaved (Ix, Iy). */
static void scharr_level(const double *I, int w, int h, double *grad)
{
    static const double s[3] = {3.0, 10.0, 3.0};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double gx = 0.0, gy = 0.0;
            for (int d = -1; d <= 1; ++d) {
                int yy = reflect101(y + d, h), xx = reflect101(x + d, w);
                gx += s[d + 1] * (I[(size_t)yy * w + reflect101(x + 1, w)] -
                                  I[(size_t)yy * w + reflect101(x - 1, w)]);
                gy += s[d + 1] * (I[(size_t)reflect101(y + 1, h) * w + xx] -
                                  I[(size_t)reflect101(y - 1, h) * w + xx]);
            }
            grad[2 * ((size_t)y * w + x) + 0] = gx / 32.0;
            grad[2 * ((size_t)y * w + x) + 1] = gy / 32.0;
        }
}

/* Number of doubles in the packed image planes of all levels. */
size_t orc_pyramid_elems(int w, int h, int levels)
{
    size_t n = 0;
    for (int l = 0; l < levels; ++l) { int lw, lh; orc_level_size(w, h, l, &lw, &lh); n += (size_t)lw * lh; }
    return n;
}

/* Image pyramid and per-level gradients.
 * img:  levels planes packed back to back (level 0 = the frame as doubles);
 * grad: levels planes of interleaved (Ix, Iy), twice img's element count. */
static void pyramid_from_level0(int w, int h, int levels, double *img, double *grad)
{
    size_t off = 0;
    int lw = w, lh = h;
    for (int l = 0; l < levels; ++l) {
        scharr_level(img + off, lw, lh, grad + 2 * off);
        if (l + 1 < levels) {
            int nw = (lw + 1) >> 1, nh = (lh + 1) >> 1;
            reduce_level(img + off, lw, lh, img + off + (size_t)lw * lh, nw, nh);
            off += (size_t)lw * lh;
            lw = nw; lh = nh;
        }
    }
}

void orc_pyramid(const uint8_t *frame, int w, int h, long pitch, int levels,
                 double *img, double *grad)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) img[(size_t)y * w + x] = frame[(size_t)y * pitch + x];
    pyramid_from_level0(w, h, levels, img, grad);
}

/* Same pyramid from an unquantised (real-valued) level 0, for the pins that
 * need renders free of the u8 rounding. */
void orc_pyramid_f64(const double *frame, int w, int h, int levels, double *img, double *grad)
{
    memcpy(img, frame, sizeof(double) * (size_t)w * h);
    pyramid_from_level0(w, h, levels, img, grad);
}

/* ---------------------------------------------------------------- corners */

/* floor(sqrt(D)) by bisection on integers: s*s <= D < (s+1)*(s+1). */
uint64_t orc_isqrt(uint64_t D)
{
    uint64_t lo = 0, hi = 1ull << 32;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (mid * mid <= D) lo = mid; else hi = mid;
    }
    return lo;
}

/* Raw integer Scharr of the u8 frame (32 x the level-0 gradient). */
void orc_scharr_raw(const uint8_t *f, int w, int h, long pitch, int32_t *gx, int32_t *gy)
{
    static const int s[3] = {3, 10, 3};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int ax = 0, ay = 0;
            for (int d = -1; d <= 1; ++d) {
                int yy = reflect101(y + d, h), xx = reflect101(x + d, w);
                ax += s[d + 1] * ((int)f[(size_t)yy * pitch + reflect101(x + 1, w)] -
                                  (int)f[(size_t)yy * pitch + reflect101(x - 1, w)]);
                ay += s[d + 1] * ((int)f[(size_t)reflect101(y + 1, h) * pitch + xx] -
                                  (int)f[(size_t)reflect101(y - 1, h) * pitch + xx]);
            }
            gx[(size_t)y * w + x] = ax;
            gy[(size_t)y * w + x] = ay;
        }
}

/* Shi-Tomasi response in exact integers.  Structure tensor over the 3x3
 * block around each pixel (gradient sampled with reflect-101):
 *   a = sum gx^2, b = sum gx gy, c = sum gy^2,
 * eigenvalues ((a+c) +- sqrt((a-c)^2 + 4 b^2)) / 2, so
 *   R = (a + c) - isqrt((a - c)^2 + 4 b^2)
 * lies in [2 lambda_min, 2 lambda_min + 1). */
void orc_corner_response(const uint8_t *f, int w, int h, long pitch, int64_t *R)
{
    int32_t *gx = (int32_t *)malloc(sizeof(int32_t) * (size_t)w * h);
    int32_t *gy = (int32_t *)malloc(sizeof(int32_t) * (size_t)w * h);
    orc_scharr_raw(f, w, h, pitch, gx, gy);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int64_t a = 0, b = 0, c = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    size_t q = (size_t)reflect101(y + dy, h) * w + reflect101(x + dx, w);
                    a += (int64_t)gx[q] * gx[q];
                    b += (int64_t)gx[q] * gy[q];
                    c += (int64_t)gy[q] * gy[q];
                }
            uint64_t D = (uint64_t)((a - c) * (a - c)) + 4ull * (uint64_t)(b * b);
            R[(size_t)y * w + x] = (a + c) - (int64_t)orc_isqrt(D);
        }
    free(gx);
    free(gy);
}

typedef struct { int64_t R; int64_t idx; int x, y; } cand_t;

static int cand_cmp(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->R != b->R) return a->R > b->R ? -1 : 1;      /* R descending */
    return a->idx < b->idx ? -1 : (a->idx > b->idx);     /* raster index ascending */
}

/* Shi-Tomasi corner selection inside each box, on the u8 frame t.
 *  1. eligible pixels: x0 <= x < x1, y0 <= y < y1, 1 <= x <= W-2, 1 <= y <= H-2;
 *  2. R_max = max R over the eligible pixels;
 *  3. candidates: R > 0, qden * R > qnum * R_max, and R >= R of all 8
 *     neighbours (which may lie outside the box);
 *  4. order by (R descending, y*W + x ascending);
 *  5. greedy: accept a candidate if dx^2 + dy^2 >= fl32(min_dist^2) to every
 *     point accepted so far; stop at max_corners.
 * pts: nboxes * max_corners (x, y) pairs; counts: per box.
 * Returns the number of boxes processed. */
int orc_select_corners(const uint8_t *f, int w, int h, long pitch, const float *boxes, int nboxes,
                       int max_corners, int qnum, int qden, float min_dist,
                       float *pts, int32_t *counts)
{
    int64_t *R = (int64_t *)malloc(sizeof(int64_t) * (size_t)w * h);
    orc_corner_response(f, w, h, pitch, R);
    float md2f = min_dist * min_dist;       /* threshold taken in FP32 */
    double md2 = (double)md2f;
    cand_t *cand = (cand_t *)malloc(sizeof(cand_t) * ((size_t)w * h + 1));
    int *acc = (int *)malloc(sizeof(int) * 2 * (size_t)(max_corners > 0 ? max_corners : 1));
    for (int bi = 0; bi < nboxes; ++bi) {
        double x0 = boxes[4 * bi + 0], y0 = boxes[4 * bi + 1];
        double x1 = boxes[4 * bi + 2], y1 = boxes[4 * bi + 3];
        int64_t rmax = 0;
        for (int y = 1; y <= h - 2; ++y)
            for (int x = 1; x <= w - 2; ++x)
                if (x >= x0 && x < x1 && y >= y0 && y < y1 && R[(size_t)y * w + x] > rmax)
                    rmax = R[(size_t)y * w + x];
        size_t nc = 0;
        for (int y = 1; y <= h - 2; ++y)
            for (int x = 1; x <= w - 2; ++x) {
                if (!(x >= x0 && x < x1 && y >= y0 && y < y1)) continue;
                int64_t r = R[(size_t)y * w + x];
                if (r <= 0 || (int64_t)qden * r <= (int64_t)qnum * rmax) continue;
                int ismax = 1;
                for (int dy = -1; dy <= 1 && ismax; ++dy)
                    for (int dx = -1; dx <= 1; ++dx)
                        if ((dx || dy) && R[(size_t)(y + dy) * w + (x + dx)] > r) { ismax = 0; break; }
                if (!ismax) continue;
                cand[nc].R = r;
                cand[nc].idx = (int64_t)y * w + x;
                cand[nc].x = x;
                cand[nc].y = y;
                ++nc;
            }
        qsort(cand, nc, sizeof(cand_t), cand_cmp);
        int na = 0;
        for (size_t c = 0; c < nc && na < max_corners; ++c) {
            int ok = 1;
            for (int a = 0; a < na; ++a) {
                int64_t dx = cand[c].x - acc[2 * a], dy = cand[c].y - acc[2 * a + 1];
                if ((double)(dx * dx + dy * dy) < md2) { ok = 0; break; }
            }
            if (!ok) continue;
            acc[2 * na] = cand[c].x;
            acc[2 * na + 1] = cand[c].y;
            pts[2 * ((size_t)bi * max_corners + na) + 0] = (float)cand[c].x;
            pts[2 * ((size_t)bi * max_corners + na) + 1] = (float)cand[c].y;
            ++na;
        }
        counts[bi] = na;
    }
    free(acc);
    free(cand);
    free(R);
    return nboxes;
}

/* --------------------------------------------------------------------- LK */

typedef struct { const double *img, *grad; int w, h; } level_t;

/* Bilinear sample of channel k of an ch-channel plane at integer tap
 * (ix, iy) with fractional weights (a, b); each of the four taps is clamped
 * to the plane (replicate border). */
static double bilin(const double *P, int ch, int k, int w, int h, int ix, int iy, double a, double b)
{
    int x0 = clampi(ix, 0, w - 1), x1 = clampi(ix + 1, 0, w - 1);
    int y0 = clampi(iy, 0, h - 1), y1 = clampi(iy + 1, 0, h - 1);
    return (1.0 - a) * (1.0 - b) * P[((size_t)y0 * w + x0) * ch + k] +
           a * (1.0 - b) * P[((size_t)y0 * w + x1) * ch + k] +
           (1.0 - a) * b * P[((size_t)y1 * w + x0) * ch + k] +
           a * b * P[((size_t)y1 * w + x1) * ch + k];
}

/* Pyramidal iterative Lucas-Kanade for one point u (Bouguet's scheme):
 * g = 0 at the top level Lm; for L = Lm..0:
 *   p = u 2^-L, N = win^2, w = (win - 1) / 2;
 *   G = sum over the window (i, j) in [-w, w]^2 of [Ix^2 IxIy; IxIy Iy^2],
 *       I, Ix, Iy sampled bilinearly at p + (i, j) in frame t's level L;
 *   lost (LOST_EIG) if lambda_min(G)/N < tau or lambda_min <= 0;
 *   nu = 0; for k = 1..K:
 *       centre c = p + g + nu; lost (LOST_OOB) if c leaves
 *       [-w, W_L-1+w] x [-w, H_L-1+w];
 *       dI = I(p + (i,j)) - J(c + (i,j)), J frame t+1's level L, bilinear;
 *       b = sum dI (Ix, Iy);  eta = G^{-1} b;  nu += eta;
 *       stop when eta_x^2 + eta_y^2 < eps^2 (else NONCONV after K);
 *   g = 2 (g + nu) if L > 0, else d = g + nu.
 * v = u + d; LOST_OOB if v is outside [0, W-1] x [0, H-1].  A lost point
 * keeps v = u.  iters (per level) and mineig (lambda_min/N per level, NAN
 * where not reached) are optional diagnostics. */
static void lk_point(const level_t *P, const level_t *J, int levels, int win, int max_iter,
                     double eps, double tau, double ux, double uy,
                     double *vx, double *vy, uint8_t *status, uint8_t *iters, double *mineig,
                     double *Ib, double *Ixb, double *Iyb)
{
    const int w = (win - 1) / 2;
    const double N = (double)win * win;
    double gx = 0.0, gy = 0.0, dx = 0.0, dy = 0.0;
    int nonconv = 0;
    uint8_t st = ORC_OK;
    for (int L = 0; L < levels; ++L) {
        if (iters) iters[L] = 0;
        if (mineig) mineig[L] = NAN;
    }
    /* Input domain (a reading: the method assumes points on the frame): a
     * point with a non-finite coordinate or one beyond 2^24 px is lost
     * outside the frame without being tracked. */
    if (!(fabs(ux) <= 16777216.0) || !(fabs(uy) <= 16777216.0)) {
        *vx = ux;
        *vy = uy;
        *status = ORC_LOST_OOB;
        return;
    }
    for (int L = levels - 1; L >= 0; --L) {
        const level_t *pl = &P[L], *jl = &J[L];
        double sc = ldexp(1.0, -L);
        double px = ux * sc, py = uy * sc;
        double fx = floor(px), fy = floor(py);
        int ix = (int)fx, iy = (int)fy;
        double a = px - fx, b = py - fy;
        double Gxx = 0.0, Gxy = 0.0, Gyy = 0.0;
        int t = 0;
        for (int j = -w; j <= w; ++j)
            for (int i = -w; i <= w; ++i, ++t) {
                Ib[t] = bilin(pl->img, 1, 0, pl->w, pl->h, ix + i, iy + j, a, b);
                Ixb[t] = bilin(pl->grad, 2, 0, pl->w, pl->h, ix + i, iy + j, a, b);
                Iyb[t] = bilin(pl->grad, 2, 1, pl->w, pl->h, ix + i, iy + j, a, b);
                Gxx += Ixb[t] * Ixb[t];
                Gxy += Ixb[t] * Iyb[t];
                Gyy += Iyb[t] * Iyb[t];
            }
        double lam = 0.5 * ((Gxx + Gyy) - sqrt((Gxx - Gyy) * (Gxx - Gyy) + 4.0 * Gxy * Gxy));
        if (mineig) mineig[L] = lam / N;
        if (!(lam / N >= tau) || !(lam > 0.0)) { st = ORC_LOST_EIG; break; }
        double det = Gxx * Gyy - Gxy * Gxy;
        double nux = 0.0, nuy = 0.0;
        int k = 0, conv = 0;
        while (k < max_iter) {
            double cx = px + gx + nux, cy = py + gy + nuy;
            if (cx < -w || cx > pl->w - 1 + w || cy < -w || cy > pl->h - 1 + w) { st = ORC_LOST_OOB; break; }
            double fcx = floor(cx), fcy = floor(cy);
            int jx = (int)fcx, jy = (int)fcy;
            double aj = cx - fcx, bj = cy - fcy;
            double bx = 0.0, by = 0.0;
            t = 0;
            for (int j = -w; j <= w; ++j)
                for (int i = -w; i <= w; ++i, ++t) {
                    double dI = Ib[t] - bilin(jl->img, 1, 0, jl->w, jl->h, jx + i, jy + j, aj, bj);
                    bx += dI * Ixb[t];
                    by += dI * Iyb[t];
                }
            double ex = (Gyy * bx - Gxy * by) / det;
            double ey = (Gxx * by - Gxy * bx) / det;
            nux += ex;
            nuy += ey;
            ++k;
            if (ex * ex + ey * ey < eps * eps) { conv = 1; break; }
        }
        if (iters) iters[L] = (uint8_t)k;
        if (st != ORC_OK) break;
        if (!conv) nonconv = 1;
        if (L > 0) { gx = 2.0 * (gx + nux); gy = 2.0 * (gy + nuy); }
        else { dx = gx + nux; dy = gy + nuy; }
    }
    if (st == ORC_OK) {
        double ox = ux + dx, oy = uy + dy;
        if (ox < 0.0 || ox > P[0].w - 1 || oy < 0.0 || oy > P[0].h - 1) st = ORC_LOST_OOB;
        else { *vx = ox; *vy = oy; }
    }
    if (st != ORC_OK) { *vx = ux; *vy = uy; }
    else if (nonconv) st |= ORC_NONCONV;
    *status = st;
}

/* Track n points from frame t (prev) to frame t+1 (next).  Pyramids are
 * given as orc_pyramid() output for each frame.  pts_out is (x, y) doubles;
 * iters is n*levels (level index L), mineig n*levels; both nullable.
 * nthreads <= 0 uses the OpenMP default. */
void orc_lk_track(const double *prev_img, const double *prev_grad,
                  const double *next_img, const double *next_grad,
                  int w, int h, int levels, const float *pts, int n,
                  int win, int max_iter, double eps, double tau,
                  double *pts_out, uint8_t *status, uint8_t *iters, double *mineig, int nthreads)
{
    level_t P[16], J[16];
    size_t off = 0;
    for (int l = 0; l < levels; ++l) {
        int lw, lh;
        orc_level_size(w, h, l, &lw, &lh);
        P[l].img = prev_img + off; P[l].grad = prev_grad + 2 * off; P[l].w = lw; P[l].h = lh;
        J[l].img = next_img + off; J[l].grad = next_grad + 2 * off; J[l].w = lw; J[l].h = lh;
        off += (size_t)lw * lh;
    }
    int nwin = win * win;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double *buf = (double *)malloc(sizeof(double) * 3 * (size_t)nwin);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int i = 0; i < n; ++i)
            lk_point(P, J, levels, win, max_iter, eps, tau, pts[2 * i], pts[2 * i + 1],
                     &pts_out[2 * i], &pts_out[2 * i + 1], &status[i],
                     iters ? iters + (size_t)i * levels : NULL,
                     mineig ? mineig + (size_t)i * levels : NULL,
                     buf, buf + nwin, buf + 2 * nwin);
        free(buf);
    }
}

/* ------------------------------------------------------------- box update */

static int dbl_cmp(const void *pa, const void *pb)
{
    double a = *(const double *)pa, b = *(const double *)pb;
    return a < b ? -1 : (a > b);
}

/* Median of m doubles (sorted in place; even count: mean of the two middle
 * values). */
static double median_of(double *v, int m)
{
    qsort(v, m, sizeof(double), dbl_cmp);
    return (m & 1) ? v[m / 2] : 0.5 * (v[m / 2 - 1] + v[m / 2]);
}

/* Points of the scale estimate: the first ORC_SCALE_POINTS OK points of a box
 * in CSR order (the strongest corners come first). */
#define ORC_SCALE_POINTS 64

/* Section V-A prediction: each box moves by an aggregate of the displacements
 * of its tracked (OK) points.  aggregator 0 = median of dx and of dy
 * separately (even count: mean of the two middle values), 1 = mean (the
 * paper's choice); the size is kept.  aggregator 2 = the median displacement
 * of 0 plus a scale (the median-flow estimate of Kalal, Mikolajczyk and
 * Matas, 2010): the median over all pairs i < j of the box's first 64 OK
 * points of |v_i - v_j| / |u_i - u_j| (pairs with u_i = u_j skipped; no pair:
 * scale 1); the box is scaled by it about its centre, then moved.  offsets is
 * the CSR of points per box (nboxes + 1).  A box with no OK point stays where
 * it is and gets nvalid = 0. */
void orc_update_boxes(const float *boxes, const int32_t *offsets, const float *pts,
                      const float *pts_out, const uint8_t *status, int nboxes, int aggregator,
                      double *boxes_out, int32_t *nvalid)
{
    for (int bi = 0; bi < nboxes; ++bi) {
        int lo = offsets[bi], hi = offsets[bi + 1];
        int cap = hi > lo ? hi - lo : 1;
        double *dx = (double *)malloc(sizeof(double) * cap);
        double *dy = (double *)malloc(sizeof(double) * cap);
        int *ok = (int *)malloc(sizeof(int) * cap);
        int m = 0;
        for (int i = lo; i < hi; ++i)
            if (status[i] & ORC_OK) {
                dx[m] = (double)pts_out[2 * i] - (double)pts[2 * i];
                dy[m] = (double)pts_out[2 * i + 1] - (double)pts[2 * i + 1];
                ok[m] = i;
                ++m;
            }
        double mx = 0.0, my = 0.0, scale = 1.0;
        if (m > 0) {
            if (aggregator == 1) {
                for (int i = 0; i < m; ++i) { mx += dx[i]; my += dy[i]; }
                mx /= m;
                my /= m;
            } else {
                mx = median_of(dx, m);
                my = median_of(dy, m);
            }
        }
        if (aggregator == 2) {
            const int k = m < ORC_SCALE_POINTS ? m : ORC_SCALE_POINTS;
            double *r = (double *)malloc(sizeof(double) * (k * (k - 1) / 2 + 1));
            int nr = 0;
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b) {
                    const int i = ok[a], j = ok[b];
                    const double ux = (double)pts[2 * i] - pts[2 * j];
                    const double uy = (double)pts[2 * i + 1] - pts[2 * j + 1];
                    const double vx = (double)pts_out[2 * i] - pts_out[2 * j];
                    const double vy = (double)pts_out[2 * i + 1] - pts_out[2 * j + 1];
                    const double du = sqrt(ux * ux + uy * uy);
                    if (du > 0.0) r[nr++] = sqrt(vx * vx + vy * vy) / du;
                }
            if (nr > 0) scale = median_of(r, nr);
            free(r);
        }
        const double cx = 0.5 * ((double)boxes[4 * bi + 0] + boxes[4 * bi + 2]);
        const double cy = 0.5 * ((double)boxes[4 * bi + 1] + boxes[4 * bi + 3]);
        if (aggregator == 2) {
            const double hw = 0.5 * ((double)boxes[4 * bi + 2] - boxes[4 * bi + 0]) * scale;
            const double hh = 0.5 * ((double)boxes[4 * bi + 3] - boxes[4 * bi + 1]) * scale;
            boxes_out[4 * bi + 0] = cx + mx - hw;
            boxes_out[4 * bi + 1] = cy + my - hh;
            boxes_out[4 * bi + 2] = cx + mx + hw;
            boxes_out[4 * bi + 3] = cy + my + hh;
        } else {
            boxes_out[4 * bi + 0] = boxes[4 * bi + 0] + mx;
            boxes_out[4 * bi + 1] = boxes[4 * bi + 1] + my;
            boxes_out[4 * bi + 2] = boxes[4 * bi + 2] + mx;
            boxes_out[4 * bi + 3] = boxes[4 * bi + 3] + my;
        }
        nvalid[bi] = m;
        free(dx);
        free(dy);
        free(ok);
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ================================================================ matching
 * Matching and update phases (Section V-A): the predicted scene objects S_t
 * are matched against the detections D_t by a globally optimal assignment
 * (the Hungarian method, Kuhn 1955) of the IoU score; unmatched scene
 * objects are flagged lost, unmatched detections become new scene objects.
 * Boxes are half-open (x0, y0, x1, y1) floats. */

/* IoU of one pair in double, in this order: areas from clipped extents, the
 * intersection's extents clipped at 0, union = (area_a + area_b) - inter,
 * iou = inter / union (0 when the union is empty). */
static double orc_iou1(const float *a, const float *b)
{
    const double aw = fmax((double)a[2] - (double)a[0], 0.0), ah = fmax((double)a[3] - (double)a[1], 0.0);
    const double bw = fmax((double)b[2] - (double)b[0], 0.0), bh = fmax((double)b[3] - (double)b[1], 0.0);
    const double iw = fmax(fmin((double)a[2], (double)b[2]) - fmax((double)a[0], (double)b[0]), 0.0);
    const double ih = fmax(fmin((double)a[3], (double)b[3]) - fmax((double)a[1], (double)b[1]), 0.0);
    const double inter = iw * ih;
    const double uni = (aw * ah + bw * bh) - inter;
    return uni > 0.0 ? inter / uni : 0.0;
}

void orc_iou_matrix(const float *a, int na, const float *b, int nb, double *out)
{
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) out[(size_t)i * nb + j] = orc_iou1(a + 4 * i, b + 4 * j);
}

/* Optimal assignment on an n x n cost matrix (minimum sum), by the
 * Hungarian method with row and column potentials: rows enter one at a
 * time, and each is joined by a shortest augmenting path over reduced costs
 * (Dijkstra over the columns).  p[j] = row of column j (1-based, 0 free). */
static void orc_hungarian(const double *c, int n, int *col_of_row)
{
    double *u = calloc(n + 1, sizeof(double)), *v = calloc(n + 1, sizeof(double));
    double *minv = malloc((n + 1) * sizeof(double));
    int *p = calloc(n + 1, sizeof(int)), *way = calloc(n + 1, sizeof(int));
    char *used = malloc(n + 1);
    for (int i = 1; i <= n; ++i) {
        p[0] = i;
        int j0 = 0;
        for (int j = 0; j <= n; ++j) { minv[j] = INFINITY; used[j] = 0; }
        do {
            used[j0] = 1;
            const int i0 = p[j0];
            double delta = INFINITY;
            int j1 = 0;
            for (int j = 1; j <= n; ++j) {
                if (used[j]) continue;
                const double cur = c[(size_t)(i0 - 1) * n + (j - 1)] - u[i0] - v[j];
                if (cur < minv[j]) { minv[j] = cur; way[j] = j0; }
                if (minv[j] < delta) { delta = minv[j]; j1 = j; }
            }
            for (int j = 0; j <= n; ++j) {
                if (used[j]) { u[p[j]] += delta; v[j] -= delta; }
                else minv[j] -= delta;
            }
            j0 = j1;
        } while (p[j0] != 0);
        do {
            const int j1 = way[j0];
            p[j0] = p[j1];
            j0 = j1;
        } while (j0);
    }
    for (int j = 1; j <= n; ++j)
        if (p[j]) col_of_row[p[j] - 1] = j - 1;
    free(u); free(v); free(minv); free(p); free(way); free(used);
}

/* Maximum-total-IoU assignment of the active rows of an na x nb IoU matrix
 * (the matrix is padded to a square with zero scores); a row and column
 * count as matched only when their assigned IoU exceeds iou_min.
 * match_a[i] = column or -1, match_b[j] = row or -1. */
void orc_assign(const double *iou, int na, int nb, const uint8_t *active, double iou_min,
                int32_t *match_a, int32_t *match_b)
{
    for (int i = 0; i < na; ++i) match_a[i] = -1;
    for (int j = 0; j < nb; ++j) match_b[j] = -1;
    const int n = na > nb ? na : nb;
    if (n == 0) return;
    double *c = calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
            c[(size_t)i * n + j] = (active && !active[i]) ? 0.0 : -iou[(size_t)i * nb + j];
    int *col = malloc(n * sizeof(int));
    orc_hungarian(c, n, col);
    for (int i = 0; i < na; ++i) {
        const int j = col[i];
        if (j < nb && (!active || active[i]) && iou[(size_t)i * nb + j] > iou_min) {
            match_a[i] = j;
            match_b[j] = i;
        }
    }
    free(c);
    free(col);
}

/* Update phase: matched scene objects take their detection's box; active
 * unmatched ones are flagged lost (kept, excluded from further
 * processing); unmatched detections are appended as new scene objects.
 * Outputs hold up to ns + nd entries; *n_out is the new count. */
void orc_update_tracks(const float *boxes_s, const uint8_t *active_s, int ns, const float *boxes_d,
                       int nd, const int32_t *match_s, const int32_t *match_d, float *boxes_out,
                       uint8_t *active_out, int32_t *n_out)
{
    int n = 0;
    for (int i = 0; i < ns; ++i, ++n) {
        const float *src = (active_s[i] && match_s[i] >= 0) ? boxes_d + 4 * match_s[i] : boxes_s + 4 * i;
        for (int k = 0; k < 4; ++k) boxes_out[4 * n + k] = src[k];
        active_out[n] = (uint8_t)(active_s[i] && match_s[i] >= 0);
    }
    for (int j = 0; j < nd; ++j) {
        if (match_d[j] >= 0) continue;
        for (int k = 0; k < 4; ++k) boxes_out[4 * n + k] = boxes_d[4 * j + k];
        active_out[n++] = 1;
    }
    *n_out = n;
}

/* Forward-backward consistency of the tracked points (the round-trip test of
 * Kalal, Mikolajczyk and Matas, 2010), the consistency check that widens the
 * prediction phase of Section V-A: a point tracked from u on frame t to v on
 * frame t+1 is tracked back from v to u' on frame t; it keeps its forward
 * status only if the backward run is OK too and the round trip closes,
 * |u' - u| <= fb_max (Euclidean, level-0 pixels).  Otherwise its status
 * becomes LOST_FB (its NONCONV bit is dropped with the OK bit).  Points whose
 * forward run was lost are left as they are. */
void orc_fb_check(const float *pts, const double *pts_back, const uint8_t *status_back, int n,
                  double fb_max, uint8_t *status)
{
    for (int i = 0; i < n; ++i) {
        if (!(status[i] & ORC_OK)) continue;
        const double dx = pts_back[2 * i] - (double)pts[2 * i];
        const double dy = pts_back[2 * i + 1] - (double)pts[2 * i + 1];
        const int closes = (status_back[i] & ORC_OK) && sqrt(dx * dx + dy * dy) <= fb_max;
        if (!closes) status[i] = ORC_LOST_FB;
    }
}

/* ------------------------------------------------------ dense TV-L1 flow
 * Section IV: the paper's flow engine is a dense TV-L1 motion field (L1 data
 * term, total variation regularised with the Huber norm, solved by a
 * projected (primal-dual) gradient scheme) on frames preprocessed by a
 * structure-texture decomposition; Section V-A moves each box by the mean of
 * the field inside it.  The paper gives no parameters; the readings are:
 *   - structure S = the ROF denoising of I (min_S TV(S) + |S - I|^2 / (2 theta))
 *     by Chambolle's dual projection, texture T = I - alpha S, stored as u8
 *     clamp(floor(k T + 128 + 0.5), 0, 255);
 *   - forward differences with zero at the last row / column for grad, the
 *     negative adjoint (backward differences, zero outside) for div;
 *   - per pyramid level, coarse to fine, the flow of the level above sampled
 *     bilinearly at (x/2, y/2) and doubled (zero at the top), the duals
 *     restarted at zero; per warp, I1 and its gradient sampled bilinearly at
 *     x + u0 (taps clamped, as for LK), rho(u) = rho0 + grad I1w . u with
 *     rho0 = I1w - grad I1w . u0 - I0, intensities scaled to [0, 1];
 *   - per iteration (Chambolle-Pock, sigma = tau = 1/sqrt(8)):
 *       p_d <- P(p_d + sigma grad ubar_d) / (1 + sigma eps), P the projection
 *              onto the unit disc, for each flow component d separately;
 *       u~ = u + tau div p;  u <- the pointwise prox of tau lambda |rho|:
 *              u~ + tau lambda g if rho(u~) < -tau lambda |g|^2,
 *              u~ - tau lambda g if rho(u~) > tau lambda |g|^2,
 *              u~ - rho(u~) g / |g|^2 otherwise (u~ if g = 0), g = grad I1w;
 *       ubar = 2 u - u_previous. */

static void grad_fwd(const double *u, int w, int h, size_t x, size_t y, double *gx, double *gy)
{
    const size_t i = y * w + x;
    *gx = (int)x + 1 < w ? u[i + 1] - u[i] : 0.0;
    *gy = (int)y + 1 < h ? u[i + w] - u[i] : 0.0;
}

/* div of the dual field p (interleaved (px, py)) at (x, y). */
static double div_bwd(const double *p, int w, int h, size_t x, size_t y)
{
    const size_t i = y * w + x;
    double d = 0.0;
    if ((int)x + 1 < w) d += p[2 * i];
    if (x > 0) d -= p[2 * (i - 1)];
    if ((int)y + 1 < h) d += p[2 * i + 1];
    if (y > 0) d -= p[2 * (i - w) + 1];
    return d;
}

/* ROF structure of I by Chambolle's projection (iters steps of 1/8), then
 * the u8 texture.  I: the u8 frame (pitch bytes per row); structure: the
 * w x h structure S (optional). */
void orc_structure_texture(const uint8_t *frame, int w, int h, long pitch, double theta,
                           double alpha, double k, int iters, uint8_t *texture, long tpitch,
                           double *structure)
{
    const size_t n = (size_t)w * h;
    double *I = (double *)malloc(sizeof(double) * n);
    double *p = (double *)calloc(2 * n, sizeof(double));
    double *q = (double *)malloc(sizeof(double) * n);
    double *pn = (double *)malloc(sizeof(double) * 2 * n);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) I[(size_t)y * w + x] = frame[(size_t)y * pitch + x];
    const double step = 0.125;
    for (int it = 0; it < iters; ++it) {
        /* q = div p - I / theta, then p <- (p + step grad q) / (1 + step |grad q|) */
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) q[(size_t)y * w + x] = div_bwd(p, w, h, x, y) - I[(size_t)y * w + x] / theta;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double gx, gy;
                grad_fwd(q, w, h, x, y, &gx, &gy);
                const double m = 1.0 + step * sqrt(gx * gx + gy * gy);
                const size_t i = (size_t)y * w + x;
                pn[2 * i] = (p[2 * i] + step * gx) / m;
                pn[2 * i + 1] = (p[2 * i + 1] + step * gy) / m;
            }
        memcpy(p, pn, sizeof(double) * 2 * n);
    }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            const size_t i = (size_t)y * w + x;
            const double S = I[i] - theta * div_bwd(p, w, h, x, y);
            if (structure) structure[i] = S;
            const double T = floor(k * (I[i] - alpha * S) + 128.0 + 0.5);
            texture[(size_t)y * tpitch + x] = (uint8_t)(T < 0.0 ? 0.0 : (T > 255.0 ? 255.0 : T));
        }
    free(I); free(p); free(q); free(pn);
}

/* grad (forward differences, zero at the last row / column) of a w x h
 * field, interleaved (gx, gy) into g. */
void orc_grad_fwd(const double *u, int w, int h, double *g)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            const size_t i = (size_t)y * w + x;
            grad_fwd(u, w, h, x, y, &g[2 * i], &g[2 * i + 1]);
        }
}

/* div of an interleaved dual field p (the negative adjoint of grad) into d. */
void orc_div_bwd(const double *p, int w, int h, double *d)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) d[(size_t)y * w + x] = div_bwd(p, w, h, x, y);
}

/* The dual step of one pixel and one flow component: the resolvent of the
 * conjugate of the Huber norm, p <- P((p + sigma g) / (1 + sigma eps)), g the
 * forward gradient of ubar there, P the projection onto the unit disc. */
void orc_tvl1_dual(double px, double py, double gx, double gy, double sigma, double eps,
                   double *qx_out, double *qy_out)
{
    double qx = (px + sigma * gx) / (1.0 + sigma * eps);
    double qy = (py + sigma * gy) / (1.0 + sigma * eps);
    const double m = sqrt(qx * qx + qy * qy);
    if (m > 1.0) { qx /= m; qy /= m; }
    *qx_out = qx;
    *qy_out = qy;
}

/* The primal step's data term at one pixel: the prox of tau lambda |rho|,
 * rho(v) = r0 + g . v, evaluated at (t1, t2) = u + tau div p. */
void orc_tvl1_prox(double t1, double t2, double r0, double gx, double gy, double tau,
                   double lambda, double *v1_out, double *v2_out)
{
    const double g2 = gx * gx + gy * gy;
    const double rho = r0 + gx * t1 + gy * t2;
    const double th = tau * lambda * g2;
    double v1 = t1, v2 = t2;
    if (rho < -th) { v1 = t1 + tau * lambda * gx; v2 = t2 + tau * lambda * gy; }
    else if (rho > th) { v1 = t1 - tau * lambda * gx; v2 = t2 - tau * lambda * gy; }
    else if (g2 > 0.0) { v1 = t1 - rho * gx / g2; v2 = t2 - rho * gy / g2; }
    *v1_out = v1;
    *v2_out = v2;
}

/* iters primal-dual iterations (Chambolle-Pock, sigma = tau = 1/sqrt(8)) of
 * one warp of one lw x lh level: the linearised data term rho(u) = r0 +
 * gw . u (gw interleaved), the flow u (interleaved (u1, u2)) and the duals p
 * ((p1x, p1y, p2x, p2y) per pixel) updated in place; the extrapolation ubar
 * starts at u. */
void orc_tvl1_iterations(const double *gw, const double *r0, int lw, int lh, double lambda,
                         double eps, int iters, double *u, double *p)
{
    const double sigma = 1.0 / sqrt(8.0), tau = 1.0 / sqrt(8.0);
    const size_t n = (size_t)lw * lh;
    double *ub = (double *)malloc(sizeof(double) * 2 * n);
    double *uold = (double *)malloc(sizeof(double) * 2 * n);
    double *p1 = (double *)malloc(sizeof(double) * 2 * n), *p2 = (double *)malloc(sizeof(double) * 2 * n);
    double *comp = (double *)malloc(sizeof(double) * n);
    memcpy(ub, u, sizeof(double) * 2 * n);
    for (int it = 0; it < iters; ++it) {
        /* dual step, each flow component on its own */
        for (int d = 0; d < 2; ++d) {
            for (size_t i = 0; i < n; ++i) comp[i] = ub[2 * i + d];
            for (int y = 0; y < lh; ++y)
                for (int x = 0; x < lw; ++x) {
                    const size_t i = (size_t)y * lw + x;
                    double gx, gy;
                    grad_fwd(comp, lw, lh, x, y, &gx, &gy);
                    orc_tvl1_dual(p[4 * i + 2 * d], p[4 * i + 2 * d + 1], gx, gy, sigma, eps,
                                  &p[4 * i + 2 * d], &p[4 * i + 2 * d + 1]);
                }
        }
        /* primal step: u~ = u + tau div p, then the data prox */
        for (size_t i = 0; i < n; ++i) {
            p1[2 * i] = p[4 * i]; p1[2 * i + 1] = p[4 * i + 1];
            p2[2 * i] = p[4 * i + 2]; p2[2 * i + 1] = p[4 * i + 3];
        }
        memcpy(uold, u, sizeof(double) * 2 * n);
        for (int y = 0; y < lh; ++y)
            for (int x = 0; x < lw; ++x) {
                const size_t i = (size_t)y * lw + x;
                const double t1 = u[2 * i] + tau * div_bwd(p1, lw, lh, x, y);
                const double t2 = u[2 * i + 1] + tau * div_bwd(p2, lw, lh, x, y);
                orc_tvl1_prox(t1, t2, r0[i], gw[2 * i], gw[2 * i + 1], tau, lambda, &u[2 * i],
                              &u[2 * i + 1]);
            }
        for (size_t i = 0; i < 2 * n; ++i) ub[i] = 2.0 * u[i] - uold[i];
    }
    free(ub); free(uold); free(p1); free(p2); free(comp);
}

/* The linearisation of a warp: frame t+1 and its gradient sampled
 * bilinearly at x + u0 (taps clamped), intensities scaled to [0, 1]: gw =
 * grad I1w, r0 = I1w - gw . u0 - I0 (I0, I1: lw x lh; G1 interleaved). */
void orc_tvl1_warp(const double *I0, const double *I1, const double *G1, int lw, int lh,
                   const double *u, double *gw, double *r0)
{
    const double s255 = 1.0 / 255.0;
    for (int y = 0; y < lh; ++y)
        for (int x = 0; x < lw; ++x) {
            const size_t i = (size_t)y * lw + x;
            const double sx = x + u[2 * i], sy = y + u[2 * i + 1];
            const int ix = (int)floor(sx), iy = (int)floor(sy);
            const double a = sx - ix, b = sy - iy;
            const double I1w = bilin(I1, 1, 0, lw, lh, ix, iy, a, b) * s255;
            const double gx = bilin(G1, 2, 0, lw, lh, ix, iy, a, b) * s255;
            const double gy = bilin(G1, 2, 1, lw, lh, ix, iy, a, b) * s255;
            gw[2 * i] = gx;
            gw[2 * i + 1] = gy;
            r0[i] = I1w - gx * u[2 * i] - gy * u[2 * i + 1] - I0[i] * s255;
        }
}

/* Dense Huber-TV-L1 flow from frame t (P0) to t+1 (P1), packed pyramids as
 * orc_pyramid writes them, into flow (w x h interleaved (u1, u2), level-0
 * pixels). */
void orc_tvl1(const double *img0, const double *img1, const double *grad1, int w, int h,
              int levels, double lambda, double eps, int warps, int iters, double *flow)
{
    size_t off[64];
    int lw_[64], lh_[64];
    size_t o = 0;
    for (int l = 0; l < levels; ++l) {
        orc_level_size(w, h, l, &lw_[l], &lh_[l]);
        off[l] = o;
        o += (size_t)lw_[l] * lh_[l];
    }
    double *u = NULL;  /* flow of the level above, interleaved */
    for (int L = levels - 1; L >= 0; --L) {
        const int lw = lw_[L], lh = lh_[L];
        const size_t n = (size_t)lw * lh;
        const double *I0 = img0 + off[L], *I1 = img1 + off[L], *G1 = grad1 + 2 * off[L];
        double *uc = (double *)calloc(2 * n, sizeof(double));
        if (u) {
            const int cw = lw_[L + 1], ch = lh_[L + 1];
            for (int y = 0; y < lh; ++y)
                for (int x = 0; x < lw; ++x) {
                    const double cx = 0.5 * x, cy = 0.5 * y;
                    const int ix = (int)floor(cx), iy = (int)floor(cy);
                    const double a = cx - ix, b = cy - iy;
                    const size_t i = (size_t)y * lw + x;
                    uc[2 * i] = 2.0 * bilin(u, 2, 0, cw, ch, ix, iy, a, b);
                    uc[2 * i + 1] = 2.0 * bilin(u, 2, 1, cw, ch, ix, iy, a, b);
                }
            free(u);
        }
        u = uc;
        double *p = (double *)calloc(4 * n, sizeof(double));   /* (p1x, p1y, p2x, p2y) */
        double *gw = (double *)malloc(sizeof(double) * 2 * n);  /* grad I1 at x + u0, scaled */
        double *r0 = (double *)malloc(sizeof(double) * n);
        for (int wp = 0; wp < warps; ++wp) {
            orc_tvl1_warp(I0, I1, G1, lw, lh, u, gw, r0);
            orc_tvl1_iterations(gw, r0, lw, lh, lambda, eps, iters, u, p);
        }
        free(p); free(gw); free(r0);
    }
    memcpy(flow, u, sizeof(double) * 2 * (size_t)w * h);
    free(u);
}

/* Section V-A prediction with the dense field: each box moves by the mean
 * flow over the pixels whose centres lie in it (x0 <= x < x1, y0 <= y < y1,
 * inside the frame); a box without such pixels stays. */
void orc_box_mean_flow(const double *flow, int w, int h, const float *boxes, int nboxes,
                       double *boxes_out)
{
    for (int b = 0; b < nboxes; ++b) {
        const double x0 = boxes[4 * b], y0 = boxes[4 * b + 1], x1 = boxes[4 * b + 2], y1 = boxes[4 * b + 3];
        double sx = 0.0, sy = 0.0;
        long cnt = 0;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x)
                if (x >= x0 && x < x1 && y >= y0 && y < y1) {
                    sx += flow[2 * ((size_t)y * w + x)];
                    sy += flow[2 * ((size_t)y * w + x) + 1];
                    ++cnt;
                }
        const double mx = cnt ? sx / cnt : 0.0, my = cnt ? sy / cnt : 0.0;
        boxes_out[4 * b] = x0 + mx;
        boxes_out[4 * b + 1] = y0 + my;
        boxes_out[4 * b + 2] = x1 + mx;
        boxes_out[4 * b + 3] = y1 + my;
    }
}

/* ----------------------------------------------------------- working level
 * Section V-A (preprocessing): the frame is downscaled by the Gaussian
 * pyramid and a pyramid level chosen by the input resolution is processed.
 * Reading: the working frame is level L of the frame's pyramid (as
 * orc_pyramid builds it) rounded to u8, clamp(floor(v + 0.5), 0, 255); the
 * level is 0 for frames up to 1280 px wide, 1 up to 2560, 2 above (SD, 2K,
 * 4K).  Out: L's w_L x h_L texels, row-major. */
int orc_working_level(int w, int h)
{
    (void)h;
    return w <= 1280 ? 0 : (w <= 2560 ? 1 : 2);
}

void orc_level_u8(const uint8_t *frame, int w, int h, long pitch, int level, uint8_t *out)
{
    const size_t n = orc_pyramid_elems(w, h, level + 1);
    double *img = (double *)malloc(sizeof(double) * n);
    double *grad = (double *)malloc(sizeof(double) * 2 * n);
    orc_pyramid(frame, w, h, pitch, level + 1, img, grad);
    size_t off = 0;
    int lw = w, lh = h;
    for (int l = 0; l < level; ++l) {
        off += (size_t)lw * lh;
        lw = (lw + 1) >> 1;
        lh = (lh + 1) >> 1;
    }
    for (size_t i = 0; i < (size_t)lw * lh; ++i) {
        const double v = floor(img[off + i] + 0.5);
        out[i] = (uint8_t)(v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v));
    }
    free(img);
    free(grad);
}
