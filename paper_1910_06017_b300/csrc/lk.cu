// lk.cu -- K3: pyramidal iterative Lucas-Kanade (Bouguet), the sparse
// stand-in for the dense motion field of Section V-A (feature calculation).
//
// One warp per point.  The warp covers the window in four row bands of
// eight lanes, each lane a few adjacent texel columns of its band (Lanes):
// per level it walks its band's texel rows, loads its columns' texels, takes
// the column right of its last from the next lane with a shuffle, and
// interpolates horizontally, then vertically reusing the previous row.  The
// frame-t window keeps only (Ix, Iy) per tap in registers; b = sum (I - J)
// grad I is formed as c - sum J grad I with the level constant c = sum I
// grad I.  Bilinear sampling of frame t+1 is the weighted sum of four
// integer-shift correlations per lane, kept for the last window position,
// so an iteration at a position already correlated only recombines them.
// The sums of b (and of G, c) are warp reductions.  All lanes end with
// identical sums, so the control flow stays uniform, and the reduction
// order is fixed: a point's result does not depend on the launch shape or
// on its neighbours in the batch.
//
// Solve: det = Gxx Gyy - Gxy^2 by Kahan's fused form; lambda_min =
// det / lambda_max >= tau is tested as det >= tau lambda_max (no
// cancellation, no division); eta = G^-1 b by the 2x2 adjugate.
#include <cudaTypedefs.h>

#include <mutex>
#include <unordered_map>

#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int LK_NT = 128;               // CTA size of the plain launch (and the batched default)
constexpr int LK_WARPS = LK_NT / 32;
constexpr int LK_MAX_NT = 256;           // largest CTA a launch may use

// Registers a thread of the batched kernel may use: 128 (two 256-thread
// CTAs per SM) up to 23x23, where nothing spills; the larger windows hold
// more taps per lane and spilled at 128, so they get 168 (12 resident warps
// per SM instead of 16).  On four 3840x2160 streams at 31x31 (106 k points,
// 5 levels) that took the batched LK from 3.52 to 2.97 ms (F16 storage) and
// from 5.44 to 4.50 ms (F32); at 21x21 the time is the same at 128, 168 or
// 255.
template <int WIN>
constexpr int lk_group();

template <int WIN>
constexpr int lk_batch_regs() { return WIN >= 25 || lk_group<WIN>() == 16 ? 168 : 128; }

// Lanes that track one point together: G = 32 (the whole warp) or 16 (each
// half-warp its own point).  Collectives run on the group's mask, copies
// are issued by the group's lane 0, and every group has its own staging
// buffers and mbarriers.  Every window uses the warp: half-warps measured
// slower at 21x21 (8 streams: 4,952 warp instructions per point instead of
// 5,838, but the two halves' iterations diverge, leaving 24 of 32 lanes
// active per instruction, and at twice the staging per warp only 8 to 10
// warps fit on an SM, which halved the issue rate: 0.717 ms against 0.423).
template <int WIN>
constexpr int lk_group() { return 32; }

template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) return FULL_MASK;
    else return 0xFFFFu << (threadIdx.x & 16);
}

template <int G>
__device__ __forceinline__ int group_lane() { return (int)(threadIdx.x & (G - 1)); }

struct LKArgs {
    CUtensorMap tm[OMT_MAX_LEVELS * LK_MAPS];  // window maps (encode_lk_maps)
    uint32_t tm_ok;                              // valid maps, bit 3L + m
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

// ------------------------------------------------------------ staging
// Per warp and level, the texels the level needs are copied global ->
// shared by the tensor memory accelerator: the (win+1)^2 window of frame t
// under the template (I and (Ix, Iy)) and frame t+1's search region around
// the initial centre, MARGIN texels wider than the window on every side.
// A window whose rows lie inside the level is one 2D tensor copy per plane
// (cp.async.bulk.tensor, issued by lane 0): a box of whole 16-byte chunks
// from the 16-byte aligned column at or before its first column; columns
// past the level's right edge arrive as zeros and are never read, because
// columns are clamped to the level when the raw rows are read back.  A
// window that crosses the top or bottom edge is copied row by row instead
// (cp.async.bulk, one row per lane, each row clamped to the level), and so
// is every window of a level whose map could not be encoded.  Each of the
// warp's three buffers (two templates, one search region) has an mbarrier
// whose phase completes when its fill's bytes have landed.  The region is
// copied again only if the centre moves more than MARGIN texels away.
constexpr int MARGIN = 4;

template <int ST, int WIN>
struct Dims {
    static constexpr int R = WIN / 2;
    static constexpr int T = WIN + 1;                 // template texels per side
    static constexpr int SH = WIN + 1 + 2 * MARGIN;   // search rows
    static constexpr int SP = WIN + 2 * MARGIN;       // search pairs per row
    static constexpr int ESZ = ST == OMT_F32 ? 4 : 2; // bytes of a level >= 1 texel
    static constexpr int GSZ = 2 * ESZ;               // bytes of a gradient texel
    // 4-byte words per raw row: the 16-byte chunks covering the row's bytes
    // from a 16-byte aligned start (at most 15 bytes of lead-in), rounded to
    // whole chunks; a tensor copy's box is one raw row wide.
    static constexpr int chunks(int bytes) { return (bytes + 15 + 15) / 16; }
    static constexpr int RWJ = 4 * chunks((SP + 1) * ESZ);
    static constexpr int RWI = 4 * chunks(T * ESZ);
    static constexpr int RWG = 4 * chunks(T * GSZ);
    // tensor copies land on 128-byte boundaries (32 words)
    static constexpr int a128(int words) { return (words + 31) & ~31; }
    static constexpr int TG = a128(T * RWI);                  // gradient rows in a template buffer
    static constexpr int TRAW = TG + a128(T * RWG);           // one template buffer
    static constexpr int UNION = 2 * TRAW;                    // two template buffers
    static constexpr int BAR = UNION + a128(SH * RWJ);        // the three mbarriers
    static constexpr int WORDS = BAR + 32;                    // per warp, 128-byte multiple
};

constexpr int BUF_SEARCH = 2;
// A fill lands in microseconds; a wait gives up after this long (globaltimer
// nanoseconds) so that a stalled copy cannot hold the warp forever.
constexpr unsigned long long FILL_WAIT_NS = 1000000000ull;

// Waits that ran out FILL_WAIT_NS, one per warp and wait (read and reset by
// omt_lk_wait_timeouts; zero unless the copy engine stalls).
__device__ unsigned lk_wait_timeouts;

// Test hook (omt_debug_fail_lk_wait): the point with this index (the plain
// call's point index, the batched step's position in the work queue) has
// its first search-region fill declared 16 bytes larger than its copies,
// so that the wait for it runs out with every copy landed; -1 = off.
__device__ long long lk_fail_point = -1;
constexpr unsigned FAIL_EXTRA_BYTES = 16;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// Completion state of a warp's three staging buffers.  After a wait runs
// out (failed), a late copy may still land in that buffer: the warp then
// issues no copy and reads no staged texel again, marks the points it
// holds OMT_PT_LOST_TIMEOUT and takes no more work.
struct Fills {
    uint64_t *bar;   // bar[b]: mbarrier of buffer b
    unsigned pend;   // bit b: a fill of buffer b is in flight; FILL_FAILED: a
                     // wait ran out (warp-uniform)
    unsigned phase;  // bit b: parity of buffer b's current phase
};
constexpr unsigned FILL_FAILED = 8u;

template <int G>
__device__ __forceinline__ void fills_init(Fills &f, unsigned *W_bar, int lane) {
    f.bar = (uint64_t *)W_bar;
    f.pend = 0;
    f.phase = 0;
    if (lane == 0) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(f.bar + b)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncwarp(group_mask<G>());
}

// Open a fill of buffer b that will land `bytes` bytes: lane 0 arrives and
// sets the expected count; the copies follow after the warp syncs.
template <int G>
__device__ __forceinline__ void fill_begin(Fills &f, int b, unsigned bytes, int lane) {
    // predicated on lane 0 inside the asm: no divergent branch
    asm volatile(
        "{\n .reg .pred q;\n setp.eq.u32 q, %2, 0;\n"
        " @q mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n}\n" ::"r"(smem_u32(f.bar + b)),
        "r"(bytes), "r"(lane)
        : "memory");
    f.pend |= 1u << b;
    __syncwarp(group_mask<G>());
}

// One row (bytes a multiple of 16, both ends 16-byte aligned).
__device__ __forceinline__ void bulk_row(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// One box of a 2D tensor map at element (x, y), issued by lane 0 only
// (predicated inside the asm); x times the element size is a multiple of
// 16 bytes and dst is 128-byte aligned.
__device__ __forceinline__ void tensor_box(void *dst, const CUtensorMap *map, int x, int y,
                                           uint64_t *bar, int lane) {
    asm volatile(
        "{\n .reg .pred q;\n setp.eq.u32 q, %5, 0;\n"
        " @q cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n}\n" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar)), "r"(lane)
        : "memory");
}

__device__ __forceinline__ unsigned mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait (bounded) until buffer b's fill in flight, if any, has landed.
// Returns false, for the whole group, when the wait ran out its limit: the
// group is then failed (Fills) and the buffer is never waited on again.
template <int G>
__device__ __forceinline__ bool fill_wait(Fills &f, int b) {
    if (!((f.pend >> b) & 1u)) return true;
    const unsigned a = smem_u32(f.bar + b), par = (f.phase >> b) & 1u;
    bool late = false;
    if (!mbar_try_wait(a, par)) {
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(a, par)) {
            if (global_ns() - t0 > FILL_WAIT_NS) {
                late = true;
                break;
            }
        }
    }
    f.pend &= ~(1u << b);
    if (__any_sync(group_mask<G>(), late)) {
        if (group_lane<G>() == 0) atomicAdd(&lk_wait_timeouts, 1u);
        f.pend |= FILL_FAILED;
        return false;
    }
    f.phase ^= 1u << b;
    return true;
}

template <int G>
__device__ __forceinline__ void fill_drain(Fills &f) {
    fill_wait<G>(f, 0);
    fill_wait<G>(f, 1);
    fill_wait<G>(f, BUF_SEARCH);
}

// The bytes of a row to copy for texel columns [x0, x0 + ncols) clamped to
// the level: from the 16-byte aligned byte b0 at or before the first column,
// whole 16-byte chunks through the last.  Rows are 128-byte aligned with
// pitches a multiple of 128, so the chunks never leave the row's pitch.
struct Span {
    int b0;
    unsigned bytes;
};
__device__ __forceinline__ Span row_span(int w, int esz, int x0, int ncols) {
    const int xa = clampi(x0, 0, w - 1), xb = clampi(x0 + ncols - 1, 0, w - 1);
    Span s;
    s.b0 = (xa * esz) & ~15;
    s.bytes = (unsigned)(((xb + 1) * esz - s.b0 + 15) & ~15);
    return s;
}

// log2 of an element size of 1, 2, 4 or 8 bytes.
__device__ __forceinline__ int esz_shift(int esz) { return __ffs(esz) - 1; }

// How a block of `rows` raw rows from level row y0 is filled: one tensor
// copy when it lies inside the level; one tensor copy and then the edge rows
// replicated into the rows outside (fix_rows) when it only overlaps the
// level; row by row (each row clamped) without a map or overlap.
enum FillMode { VIA_TMA, VIA_TMA_EDGE, VIA_ROWS };
__device__ __forceinline__ FillMode fill_mode(const CUtensorMap *tm, int y0, int rows, int h) {
    if (!tm || y0 >= h || y0 + rows <= 0) return VIA_ROWS;
    return y0 >= 0 && y0 + rows <= h ? VIA_TMA : VIA_TMA_EDGE;
}

// After a tensor copy of rows [y0, y0 + rows) that overlaps a level of h
// rows, the rows above the level (zero-filled) take the level's first row
// and those below take its last, as a copy of clamped rows would hold.
template <int RW, int G>
__device__ __forceinline__ void fix_rows(unsigned *blk, int y0, int rows, int h, int lane) {
    const int top = y0 < 0 ? -y0 : 0;                   // rows above the level, < rows
    const int below = h - y0 < rows ? h - y0 : rows;    // first row below the level, > top
    const int n = (top + rows - below) * RW;
    for (int k = lane; k < n; k += G) {
        const int j = k / RW, c = k - j * RW;
        const int r = j < top ? j : below + (j - top);
        const int src = j < top ? top : below - 1;
        blk[r * RW + c] = blk[src * RW + c];
    }
}

// Texel x (level column, clamped) of a raw row whose first byte is level
// column `base`: u8, float or half(I - 128).  Level >= 1 values stay in the
// stored domain (I - 128 for half): only differences and products with the
// template, stored the same way, enter the solve.
template <int ST>
__device__ __forceinline__ float raw_texel(const unsigned *row, int col, bool u8) {
    if (u8) return (float)((const uint8_t *)row)[col];
    if (ST == OMT_F32) return ((const float *)row)[col];
    return __half2float(((const __half *)row)[col]);
}

template <int ST>
__device__ __forceinline__ float2 raw_grad(const unsigned *row, int col) {
    if (ST == OMT_F32) return ((const float2 *)row)[col];
    return __half22float2(((const __half2 *)row)[col]);
}

// Level layout the copies need.
struct LevelCopy {
    int tcol_i, tcol_g;  // level column of the first raw template texel (I, gradients)
    int scol;            // level column of the first raw search texel
    int sx0, sy0;        // search region origin (texels)
};

// The template window to prefetch after this level's template compute.
struct NextTemplate {
    bool has;
    const LevelView *P;     // read only by row copies
    int w, h;               // its level size
    const CUtensorMap *tm;  // the level's maps, or null
    bool u8;
    int ipx, ipy;
};

// A template window copied (or being copied) ahead of its level.
struct Prefetch {
    bool valid;
    int buf;             // template buffer 0 or 1
    int tcol_i, tcol_g;  // as in LevelCopy
};

// Start copying the template window of the level at (ipx, ipy) into buffer
// `buf` (I and gradient rows, one fill); returns its column origins.  tm
// points at the level's maps when they are valid, else null.  The level is
// w x h texels; its view P is read only by the row copies.
template <int ST, int WIN>
__device__ __forceinline__ void issue_template(const LevelView *P, int w, int h,
                                               const CUtensorMap *tm, bool u8, int ipx, int ipy,
                                               int buf, int lane, unsigned *W, Fills &f,
                                               int &tcol_i, int &tcol_g) {
    using D = Dims<ST, WIN>;
    constexpr int G = lk_group<WIN>();
    unsigned *TI = W + buf * D::TRAW, *TGr = TI + D::TG;
    const int esz = u8 ? 1 : D::ESZ;
    const Span si = row_span(w, esz, ipx - D::R, D::T);
    const Span sg = row_span(w, D::GSZ, ipx - D::R, D::T);
    const int y0 = ipy - D::R;
    tcol_i = si.b0 >> esz_shift(esz);
    tcol_g = sg.b0 >> esz_shift(D::GSZ);
    if (fill_mode(tm, y0, D::T, h) != VIA_ROWS) {
        fill_begin<G>(f, buf, D::T * 4 * (D::RWI + D::RWG), lane);
        tensor_box(TI, tm + LK_MAP_TI, tcol_i, y0, f.bar + buf, lane);
        tensor_box(TGr, tm + LK_MAP_TG, tcol_g, y0, f.bar + buf, lane);
    } else {
        fill_begin<G>(f, buf, D::T * (si.bytes + sg.bytes), lane);
        const uint8_t *img = P->img, *grad = P->grad;
        const int64_t ip = P->img_pitch, gp = P->grad_pitch;
        for (int r = lane; r < D::T; r += G) {
            const int64_t y = clampi(y0 + r, 0, h - 1);
            bulk_row(TI + r * D::RWI, img + y * ip + si.b0, si.bytes, f.bar + buf);
            bulk_row(TGr + r * D::RWG, grad + y * gp + sg.b0, sg.bytes, f.bar + buf);
        }
    }
}

// Start copying frame t+1's search region around (jx, jy); tm, w, h and
// the view J as above.
template <int ST, int WIN>
__device__ __forceinline__ void copy_search(const LevelView *J, int w, int h,
                                            const CUtensorMap *tm, bool u8, int jx, int jy,
                                            int lane, unsigned *W, Fills &f, LevelCopy &lc,
                                            unsigned extra = 0) {
    using D = Dims<ST, WIN>;
    constexpr int G = lk_group<WIN>();
    const int esz = u8 ? 1 : D::ESZ;
    lc.sx0 = jx - D::R - MARGIN;
    lc.sy0 = jy - D::R - MARGIN;
    const Span ss = row_span(w, esz, lc.sx0, D::SP + 1);
    lc.scol = ss.b0 >> esz_shift(esz);
    unsigned *S = W + D::UNION;
    if (fill_mode(tm, lc.sy0, D::SH, h) != VIA_ROWS) {
        fill_begin<G>(f, BUF_SEARCH, D::SH * 4 * D::RWJ + extra, lane);
        tensor_box(S, tm, lc.scol, lc.sy0, f.bar + BUF_SEARCH, lane);
    } else {
        fill_begin<G>(f, BUF_SEARCH, D::SH * ss.bytes + extra, lane);
        const uint8_t *img = J->img;
        const int64_t ip = J->img_pitch;
        for (int r = lane; r < D::SH; r += G) {
            const int64_t y = clampi(lc.sy0 + r, 0, h - 1);
            bulk_row(S + r * D::RWJ, img + y * ip + ss.b0, ss.bytes, f.bar + BUF_SEARCH);
        }
    }
}

// Edge rows of a search region that a tensor copy only overlapped.
template <int ST, int WIN>
__device__ __forceinline__ void search_edges(int h, const CUtensorMap *tm, unsigned *W,
                                             const LevelCopy &lc, int lane) {
    using D = Dims<ST, WIN>;
    constexpr int G = lk_group<WIN>();
    if (fill_mode(tm, lc.sy0, D::SH, h) == VIA_TMA_EDGE) {
        __syncwarp(group_mask<G>());
        fix_rows<D::RWJ, G>(W + D::UNION, lc.sy0, D::SH, h, lane);
    }
}

// Two group sums at once: the lower half of the group ends with the total
// of a, the upper half with the total of b (one exchange, then butterflies
// within each half); returns both totals in every lane of the group.  Fixed
// order: every lane gets the same bits, and equal inputs give equal outputs
// whatever they are paired with.
template <int G>
__device__ __forceinline__ void group_sum2(float &a, float &b, int lane) {
    const unsigned m = group_mask<G>();
    const bool hi = (lane & (G / 2)) != 0;
    float keep = hi ? b : a;
    const float give = hi ? a : b;
    keep += __shfl_xor_sync(m, give, G / 2, G);
#pragma unroll
    for (int o = G / 4; o > 0; o >>= 1) keep += __shfl_xor_sync(m, keep, o, G);
    a = __shfl_sync(m, keep, 0, G);
    b = __shfl_sync(m, keep, G / 2, G);
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
    const unsigned m = group_mask<G>();
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o, G);
    return v;
}

// Packed FP32 arithmetic: two lanes of one instruction, each rounded as
// the scalar fmaf / add.
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);  // a - b, one rounding
}

// Four group sums at once: halving exchanges leave each quarter of the
// group with one of the four partial sums, butterflies within the quarter
// finish it, and every lane reads the four totals back.  Fixed order, as
// group_sum2.
template <int G>
__device__ __forceinline__ void group_sum4(float &a, float &b, float &c, float &d, int lane) {
    const unsigned m = group_mask<G>();
    const bool hh = (lane & (G / 2)) != 0, hq = (lane & (G / 4)) != 0;
    float k0 = hh ? c : a, k1 = hh ? d : b;
    const float g0 = hh ? a : c, g1 = hh ? b : d;
    k0 += __shfl_xor_sync(m, g0, G / 2, G);
    k1 += __shfl_xor_sync(m, g1, G / 2, G);
    float keep = hq ? k1 : k0;
    const float give = hq ? k0 : k1;
    keep += __shfl_xor_sync(m, give, G / 4, G);
#pragma unroll
    for (int o = G / 8; o > 0; o >>= 1) keep += __shfl_xor_sync(m, keep, o, G);
    a = __shfl_sync(m, keep, 0, G);
    b = __shfl_sync(m, keep, G / 4, G);
    c = __shfl_sync(m, keep, G / 2, G);
    d = __shfl_sync(m, keep, 3 * G / 4, G);
}

// How a group's lanes cover a window of WIN x WIN taps (texel footprint
// (WIN + 1)^2): NB = G / 8 row bands of eight lanes (four for a warp, two
// for a half-warp).  Lane k of band g holds texel columns CPL k .. CPL k +
// CPL - 1 (taps where the column is below WIN; the column right of its last
// one comes from lane k + 1 by a shuffle) and walks the band's tap rows r0
// .. r0 + nr - 1: the WIN rows split into bands of Q + 1 rows (the first
// REM bands) and Q rows.  A band walks RB rows; a band of Q rows reads its
// last texel row again at step Q, where its taps are zero.  Every lane then
// holds RB x CPL taps, and all lanes take part in every row step (a lane
// per texel column left 10 of 32 lanes idle at WIN = 21).
template <int WIN>
struct Lanes {
    static constexpr int NB = lk_group<WIN>() / 8;       // row bands
    static constexpr int CPL = (WIN + 1 + 7) / 8;       // texel columns per lane
    static constexpr int Q = WIN / NB, REM = WIN % NB;  // band rows: Q + (g < REM)
    static constexpr int RB = Q + (REM > 0 ? 1 : 0);    // row steps of a band
    // a lane holds taps and columns right of the window at once
    static constexpr bool PARTIAL = WIN % CPL != 0;
};

__device__ __forceinline__ int band_r0(int g, int q, int rem) { return g * q + (g < rem ? g : rem); }

// This lane's texel columns of a window whose first column is level column
// x0, clamped to the window's footprint and to the level (w columns), as
// offsets into raw rows that start at level column c0.
template <int WIN>
__device__ __forceinline__ void lane_cols(int x0, int w, int c0, int lane,
                                          int (&col)[Lanes<WIN>::CPL]) {
    using M = Lanes<WIN>;
    const int k = lane & 7;
#pragma unroll
    for (int j = 0; j < M::CPL; ++j) {
        const int c = min(M::CPL * k + j, WIN);
        col[j] = clampi(x0 + c, 0, w - 1) - c0;
    }
}

// Whether this lane holds any tap (lanes whose columns all lie right of the
// window only supply texels to their left neighbour).
template <int WIN>
__device__ __forceinline__ bool lane_owns(int lane) {
    return (lane & 7) * Lanes<WIN>::CPL < WIN;
}

// Frame-t window from the raw template rows: the interpolated (Ix, Iy) of
// this lane's taps stay in registers, with its share of the level constants
// G (three sums).  Taps a lane does not hold (the repeated last row of a
// short band; columns right of the window when a lane straddles its edge)
// are zero; a lane that holds no tap ends with zero sums.
template <int ST, int WIN>
__device__ __forceinline__ void template_window(int w, int tx0, float ax, float ay,
                                                int lane, const unsigned *W, const LevelCopy &lc,
                                                float2 (&XY)[Lanes<WIN>::RB][Lanes<WIN>::CPL],
                                                float &sxx, float &sxy, float &syy) {
    using D = Dims<ST, WIN>;
    using M = Lanes<WIN>;
    constexpr int C = M::CPL;
    const int g = lane >> 3, k = lane & 7;
    const unsigned gm = group_mask<lk_group<WIN>()>();
    const int r0 = band_r0(g, M::Q, M::REM);
    const bool long_band = g < M::REM;
    const unsigned *rawG = W + D::TG;
    int cg[C];
    lane_cols<WIN>(tx0, w, lc.tcol_g, lane, cg);
    const float2 ax2 = f2(ax, ax), ay2 = f2(ay, ay);
    float2 prev[C], sq = f2(0.f, 0.f);  // sq = (sxx, syy)
    sxy = 0.f;
    // horizontal interpolation of texel row r of the footprint
    auto hrow = [&](const unsigned *row, float2 (&h)[C]) {
        float2 t[C];
#pragma unroll
        for (int j = 0; j < C; ++j) t[j] = raw_grad<ST>(row, cg[j]);
        const float2 tn = f2(__shfl_down_sync(gm, t[0].x, 1, 8),
                             __shfl_down_sync(gm, t[0].y, 1, 8));
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float2 t1 = j + 1 < C ? t[j + 1] : tn;
            h[j] = __ffma2_rn(ax2, f2sub(t1, t[j]), t[j]);
        }
    };
    hrow(rawG + r0 * D::RWG, prev);
#pragma unroll
    for (int i = 0; i < M::RB; ++i) {
        const int tr = i < M::Q ? r0 + i + 1 : min(r0 + M::Q + 1, WIN);
        float2 h[C];
        hrow(rawG + tr * D::RWG, h);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            float2 v = __ffma2_rn(ay2, f2sub(h[j], prev[j]), prev[j]);  // vertical
            if (i == M::Q && !long_band) v = f2(0.f, 0.f);
            if (M::PARTIAL && C * k + j >= WIN) v = f2(0.f, 0.f);
            XY[i][j] = v;
            sq = __ffma2_rn(v, v, sq);
            sxy = fmaf(v.x, v.y, sxy);
            prev[j] = h[j];
        }
    }
    sxx = sq.x;
    syy = sq.y;
    if (!lane_owns<WIN>(lane)) sxx = sxy = syy = 0.f;
}

// The four integer-shift correlations of a raw image window with the
// template gradients: S[s] = sum over this lane's taps of V(tap + (b, a))
// (Ix, Iy)(tap), s = 2a + b, for the window whose top tap row sits at raw
// row oy, with this lane's texel columns col (lane_cols).  Bilinear
// sampling at fraction (bx, by) is then the weighted sum (1-bx)(1-by) S0 +
// bx(1-by) S1 + (1-bx)by S2 + bx by S3 (combine4), so a window position is
// correlated once however many iterations revisit it.  The frame-t template
// and the frame-(t+1) search window go through this same code, so equal
// frames give exactly equal sums.  A lane that holds no tap has zero taps
// only when PARTIAL; otherwise its sums are garbage and the caller drops
// them (lane_owns).
template <int ST, bool U8, int WIN>
__device__ __forceinline__ void corr4(const unsigned *raw, int rw, int oy,
                                      const int (&col)[Lanes<WIN>::CPL], int lane,
                                      const float2 (&XY)[Lanes<WIN>::RB][Lanes<WIN>::CPL],
                                      float2 (&S)[4]) {
    using M = Lanes<WIN>;
    constexpr int C = M::CPL;
    const int g = lane >> 3;
    const unsigned gm = group_mask<lk_group<WIN>()>();
    const int r0 = band_r0(g, M::Q, M::REM);
    const unsigned *base = raw + (oy + r0) * rw;
#pragma unroll
    for (int q = 0; q < 4; ++q) S[q] = f2(0.f, 0.f);
    float p[C], pn;
#pragma unroll
    for (int j = 0; j < C; ++j) p[j] = raw_texel<ST>(base, col[j], U8);
    pn = __shfl_down_sync(gm, p[0], 1, 8);
#pragma unroll
    for (int i = 0; i < M::RB; ++i) {
        const unsigned *row = i < M::Q ? base + (i + 1) * rw
                                       : raw + (oy + min(r0 + M::Q + 1, WIN)) * rw;
        float v[C];
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = raw_texel<ST>(row, col[j], U8);
        const float vn = __shfl_down_sync(gm, v[0], 1, 8);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float pr = j + 1 < C ? p[j + 1] : pn;
            const float vr = j + 1 < C ? v[j + 1] : vn;
            const float2 gg = XY[i][j];
            S[0] = __ffma2_rn(f2(p[j], p[j]), gg, S[0]);
            S[1] = __ffma2_rn(f2(pr, pr), gg, S[1]);
            S[2] = __ffma2_rn(f2(v[j], v[j]), gg, S[2]);
            S[3] = __ffma2_rn(f2(vr, vr), gg, S[3]);
        }
#pragma unroll
        for (int j = 0; j < C; ++j) p[j] = v[j];
        pn = vn;
    }
}

// This lane's share of sum over taps of V(tap + (fx, fy)) (Ix, Iy) for the
// window of S, by bilinear weights.
__device__ __forceinline__ void combine4(const float2 (&S)[4], float fx, float fy, float &sx,
                                         float &sy) {
    const float w0 = (1.0f - fx) * (1.0f - fy), w1 = fx * (1.0f - fy);
    const float w2 = (1.0f - fx) * fy, w3 = fx * fy;
    sx = fmaf(w3, S[3].x, fmaf(w2, S[2].x, fmaf(w1, S[1].x, w0 * S[0].x)));
    sy = fmaf(w3, S[3].y, fmaf(w2, S[2].y, fmaf(w1, S[1].y, w0 * S[0].y)));
}

// Level L's maps, or null (row copies).  A pyramid pair's maps are used
// only when every level's encoded.
__device__ __forceinline__ const CUtensorMap *level_maps(const CUtensorMap *tm, int L) {
    return tm ? tm + LK_MAPS * L : nullptr;
}

__device__ __forceinline__ bool all_maps(uint32_t ok, int levels) {
    return ok == (levels >= 32 / LK_MAPS ? ~0u : (1u << (LK_MAPS * levels)) - 1u);
}

__device__ __forceinline__ const CUtensorMap *stream_maps(const BatchView &t, int s, int levels,
                                                          int backward) {
    const StreamEntry &e = t.stream(s);
    return all_maps(backward ? e.tm_ok_back : e.tm_ok, levels) ? t.maps(s, backward) : nullptr;
}

// One level of the pyramidal iteration for one point (the whole warp).
// Returns the status after this level; nu is the level's increment.  Both
// frames' level is w x h texels; the views P and J are read only by row
// copies.  Every branch below depends on warp sums or on values every lane
// holds alike, so the warp never diverges.
template <int ST, int WIN>
__device__ __forceinline__ int track_level(const LevelView *P, const LevelView *J, int w, int h,
                                           float px, float py, float gx, float gy, int max_iter,
                                           float eps2, float tau_n, int lane, bool u8,
                                           const CUtensorMap *tm, unsigned *W, Fills &f,
                                           Prefetch &pf, const NextTemplate &nx, float &nux,
                                           float &nuy, int &k, bool &conv, bool force_fail) {
    using D = Dims<ST, WIN>;
    constexpr int R = D::R;
    constexpr int G = lk_group<WIN>();
    const unsigned gm = group_mask<G>();
    const float fpx = floorf(px), fpy = floorf(py);
    const int ipx = (int)fpx, ipy = (int)fpy;
    const float ax = px - fpx, ay = py - fpy;
    nux = nuy = 0.f;
    k = 0;
    conv = false;
    const CUtensorMap *tms = tm ? tm + LK_MAP_S : nullptr;

    // The template window was prefetched while the previous level (or the
    // previous point) iterated, unless this is the warp's first level; the
    // search region around the initial centre p + g is copied now, and only
    // the template has to land before the template compute starts.
    LevelCopy lc;
    int buf;
    if (pf.valid) {
        buf = pf.buf;
        lc.tcol_i = pf.tcol_i;
        lc.tcol_g = pf.tcol_g;
    } else {
        buf = 0;
        __syncwarp(gm);
        issue_template<ST, WIN>(P, w, h, tm, u8, ipx, ipy, buf, lane, W, f, lc.tcol_i, lc.tcol_g);
    }
    pf.valid = false;
    // The centre c = (ipx, ipy) + (a + g + nu); agx, agy = a + g.
    const float agx = ax + gx, agy = ay + gy;
    const bool c0_ok = fabsf(agx) < 1.0e8f && fabsf(agy) < 1.0e8f;
    int sjx = 0, sjy = 0;
    if (c0_ok) {
        sjx = ipx + (int)floorf(agx);
        sjy = ipy + (int)floorf(agy);
        copy_search<ST, WIN>(J, w, h, tms, u8, sjx, sjy, lane, W, f, lc,
                             force_fail ? FAIL_EXTRA_BYTES : 0u);
    }
    // the template has landed; the search may still run
    if (!fill_wait<G>(f, buf)) return OMT_PT_LOST_TIMEOUT;
    if (fill_mode(tm, ipy - R, D::T, h) == VIA_TMA_EDGE) {
        __syncwarp(gm);
        fix_rows<D::RWI, G>(W + buf * D::TRAW, ipy - R, D::T, h, lane);
        fix_rows<D::RWG, G>(W + buf * D::TRAW + D::TG, ipy - R, D::T, h, lane);
    }
    __syncwarp(gm);

    using M = Lanes<WIN>;
    const bool owns = lane_owns<WIN>(lane);
    float2 XY[M::RB][M::CPL];
    float sxx, sxy, syy, cx, cy;
    template_window<ST, WIN>(w, ipx - R, ax, ay, lane, W + buf * D::TRAW, lc, XY, sxx, sxy, syy);
    float2 S[4];  // integer-shift correlations at the last position visited
    {
        // c = sum I(p + tap) (Ix, Iy), through the same path as J below
        int ci[M::CPL];
        lane_cols<WIN>(ipx - R, w, lc.tcol_i, lane, ci);
        if (u8) corr4<ST, true, WIN>(W + buf * D::TRAW, D::RWI, 0, ci, lane, XY, S);
        else corr4<ST, false, WIN>(W + buf * D::TRAW, D::RWI, 0, ci, lane, XY, S);
        combine4(S, ax, ay, cx, cy);
        if (!owns) cx = cy = 0.f;
    }
    group_sum4<G>(sxx, syy, cx, cy, lane);
    sxy = group_sum<G>(sxy);
    const float det = det2(sxx, syy, sxy);
    const float dd = sxx - syy;
    const float lmax = 0.5f * ((sxx + syy) + sqrtf(fmaf(dd, dd, 4.0f * sxy * sxy)));
    // lambda_min = det / lambda_max >= tau_n and > 0, decided without the
    // division (lambda_max > 0 whenever lambda_min > 0; non-finite sums fail)
    if (!(det >= tau_n * lmax) || !(det > 0.f)) return OMT_PT_LOST_EIG;
    const float inv_det = 1.0f / det;
    // Prefetch the next template (next level, or the next point's top level)
    // into the other buffer while this level iterates.
    if (nx.has) {
        __syncwarp(gm);
        issue_template<ST, WIN>(nx.P, nx.w, nx.h, nx.tm, nx.u8, nx.ipx, nx.ipy, 1 - buf, lane, W,
                                f, pf.tcol_i, pf.tcol_g);
        pf.valid = true;
        pf.buf = 1 - buf;
    }
    // the search region has landed; the prefetch may still run
    if (!fill_wait<G>(f, BUF_SEARCH)) return OMT_PT_LOST_TIMEOUT;
    if (c0_ok) search_edges<ST, WIN>(h, tms, W, lc, lane);
    __syncwarp(gm);
    // The window stays inside the tracking bounds while its integer centre
    // j = ip + floor(a + g + nu) satisfies -R <= j <= w - 1 + R (at the
    // upper bound only with a zero fraction): in terms of a + g + nu, the
    // closed interval [lo, hi] below (integers, exact in float).  A
    // non-finite centre fails the test too.
    const float lox = (float)(-R - ipx), hix = (float)(w - 1 + R - ipx);
    const float loy = (float)(-R - ipy), hiy = (float)(h - 1 + R - ipy);
    bool staged = c0_ok;
    float cfx = 0.f, cfy = 0.f;  // floor of a + g + nu where S was correlated
    bool cached = false;
    while (k < max_iter) {
        const float ccx = agx + nux, ccy = agy + nuy;
        if (!(ccx >= lox && ccx <= hix && ccy >= loy && ccy <= hiy)) return OMT_PT_LOST_OOB;
        const float fcx = floorf(ccx), fcy = floorf(ccy);
        const float bx = ccx - fcx, by = ccy - fcy;
        if (!cached || fcx != cfx || fcy != cfy) {
            const int jx = ipx + (int)fcx, jy = ipy + (int)fcy;
            if (!staged || abs(jx - sjx) > MARGIN || abs(jy - sjy) > MARGIN) {
                __syncwarp(gm);
                copy_search<ST, WIN>(J, w, h, tms, u8, jx, jy, lane, W, f, lc);
                if (!fill_wait<G>(f, BUF_SEARCH)) return OMT_PT_LOST_TIMEOUT;
                search_edges<ST, WIN>(h, tms, W, lc, lane);
                __syncwarp(gm);
                sjx = jx;
                sjy = jy;
                staged = true;
            }
            int cj[M::CPL];
            lane_cols<WIN>(jx - R, w, lc.scol, lane, cj);
            const int oy = jy - sjy + MARGIN;
            if (u8) corr4<ST, true, WIN>(W + D::UNION, D::RWJ, oy, cj, lane, XY, S);
            else corr4<ST, false, WIN>(W + D::UNION, D::RWJ, oy, cj, lane, XY, S);
            cfx = fcx;
            cfy = fcy;
            cached = true;
        }
        float sx, sy;
        combine4(S, bx, by, sx, sy);
        if (!owns) sx = sy = 0.f;
        group_sum2<G>(sx, sy, lane);
        const float bbx = cx - sx, bby = cy - sy;  // b = sum (I - J) grad I
        const float ex = (syy * bbx - sxy * bby) * inv_det;
        const float ey = (sxx * bby - sxy * bbx) * inv_det;
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
// A point the warp holds but cannot track because one of its waits ran out
// (Fills): reported at its input position, no iterations.
__device__ __forceinline__ void lost_timeout(float2 u, int i, float2 *out, uint8_t *status,
                                             uint8_t *iters, int levels, int lane) {
    if (lane == 0) {
        out[i] = u;
        status[i] = (uint8_t)OMT_PT_LOST_TIMEOUT;
    }
    if (iters && lane < levels) iters[(int64_t)i * levels + lane] = 0;
}

// What tracking one point gives: its position, status and iterations per
// level (8 bits each).  The caller writes them out, so that no output
// pointer stays live while the point is tracked.
struct PointResult {
    float2 v;
    int st;
    unsigned long long itp;
};

// The next point's top-level template for the prefetch of the finest level.
template <int WIN>
__device__ __forceinline__ NextTemplate next_top(bool has, float2 un, const LevelView *Pn,
                                                 const CUtensorMap *tmn, int levels) {
    NextTemplate nx;
    const float st0 = __int_as_float((127 - (levels - 1)) << 23);
    nx.has = has && fabsf(un.x) <= 16777216.f && fabsf(un.y) <= 16777216.f;
    nx.P = &Pn[levels - 1];
    nx.w = nx.has ? Pn[levels - 1].w : 1;
    nx.h = nx.has ? Pn[levels - 1].h : 1;
    nx.tm = level_maps(tmn, levels - 1);
    nx.u8 = levels - 1 == 0;
    nx.ipx = (int)floorf(un.x * st0);
    nx.ipy = (int)floorf(un.y * st0);
    return nx;
}

// The whole pyramidal iteration for one point u (the whole warp); P, J are
// the frame-t and frame-(t+1) level views, tm their maps (or null).
// next() gives the next point's top-level template (NextTemplate), called
// at the finest level only.  A point with a non-finite coordinate or one
// beyond 2^24 px is lost outside the frame without a window (its integer
// positions would not fit); a point whose wait ran out comes back
// OMT_PT_LOST_TIMEOUT at its input position with no iterations.
template <int ST, int WIN, class NextFn>
__device__ __forceinline__ PointResult lk_point(const LevelView *P, const LevelView *J, int levels,
                                                int max_iter, float eps2, float tau_n, float2 u,
                                                const CUtensorMap *tm, unsigned *W, Fills &f,
                                                Prefetch &pf, NextFn next, bool force_fail) {
    constexpr int G = lk_group<WIN>();
    const int lane = group_lane<G>();
    PointResult r;
    r.v = u;
    r.itp = 0ull;
    if (!(fabsf(u.x) <= 16777216.f) || !(fabsf(u.y) <= 16777216.f)) {
        fill_drain<G>(f);
        pf.valid = false;
        r.st = OMT_PT_LOST_OOB;
        return r;
    }
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f;
    int st = OMT_PT_OK;
    bool nonconv = false;
    // level sizes, read once (both frames share them)
    const int w0 = P[0].w, h0 = P[0].h;

    for (int L = levels - 1; L >= 0; --L) {
        const float sc = __int_as_float((127 - L) << 23);  // 2^-L, exact
        const int wl = ((w0 - 1) >> L) + 1, hl = ((h0 - 1) >> L) + 1;  // (w + 1) >> 1 per level
        NextTemplate nx;
        if (L > 0) {
            const float s1 = __int_as_float((127 - (L - 1)) << 23);
            nx.has = true;
            nx.P = &P[L - 1];
            nx.w = ((w0 - 1) >> (L - 1)) + 1;
            nx.h = ((h0 - 1) >> (L - 1)) + 1;
            nx.tm = level_maps(tm, L - 1);
            nx.u8 = L - 1 == 0;
            nx.ipx = (int)floorf(u.x * s1);
            nx.ipy = (int)floorf(u.y * s1);
        } else {
            nx = next();
        }
        float nux, nuy;
        int k;
        bool conv;
        st = track_level<ST, WIN>(&P[L], &J[L], wl, hl, u.x * sc, u.y * sc, gx, gy, max_iter,
                                  eps2, tau_n, lane, L == 0, level_maps(tm, L), W, f, pf, nx,
                                  nux, nuy, k, conv, L == levels - 1 && force_fail);
        r.itp |= (unsigned long long)k << (8 * L);
        if (st == OMT_PT_LOST_TIMEOUT) {
            // give the point up; the kernel lands what else is in flight
            // (bounded) before it exits
            pf.valid = false;
            r.st = OMT_PT_LOST_TIMEOUT;
            r.itp = 0ull;
            return r;
        }
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
    if (st != OMT_PT_OK) {
        // a lost point leaves its prefetch (for a level it will not reach)
        // unused, and maybe its search region in flight: land them and
        // forget them
        fill_drain<G>(f);
        pf.valid = false;
    } else {
        const float ox = u.x + dx, oy = u.y + dy;
        if (!(ox >= 0.f && ox <= (float)(w0 - 1) && oy >= 0.f && oy <= (float)(h0 - 1)))
            st = OMT_PT_LOST_OOB;
        else
            r.v = make_float2(ox, oy);
    }
    if (st == OMT_PT_OK && nonconv) st |= OMT_PT_NONCONV;
    r.st = st;
    return r;
}

// Writes a point's result: position and status by lane 0, the iterations
// of level L by lane L.
__device__ __forceinline__ void put_point(const PointResult &r, int i, float2 *out,
                                          uint8_t *status, uint8_t *iters, int levels, int lane) {
    if (lane == 0) {
        out[i] = r.v;
        status[i] = (uint8_t)r.st;
    }
    if (iters && lane < levels) iters[(int64_t)i * levels + lane] = (uint8_t)(r.itp >> (8 * lane));
}

// ------------------------------------------------------ forward-backward
// A point tracked u -> v keeps its status only if the backward run v -> u'
// is OK and the round trip closes: |u' - u| <= fb_max (FP32, level-0 px);
// else it becomes LOST_FB.  Lost forward points are left as they are.
__device__ __forceinline__ void fb_apply(float2 u, float2 u_back, uint8_t status_back,
                                         float fb_max, uint8_t &status) {
    if (!(status & OMT_PT_OK)) return;
    if (status_back & OMT_PT_LOST_TIMEOUT) {   // the backward run was not made
        status = (uint8_t)OMT_PT_LOST_TIMEOUT;
        return;
    }
    const float dx = u_back.x - u.x, dy = u_back.y - u.y;
    const bool closes = (status_back & OMT_PT_OK) && sqrtf(fmaf(dx, dx, dy * dy)) <= fb_max;
    if (!closes) status = (uint8_t)OMT_PT_LOST_FB;
}

__global__ void fb_check_kernel(const float2 *pts, const float2 *pts_back,
                                const uint8_t *status_back, int n_max, const int32_t *n_dev,
                                float fb_max, uint8_t *status) {
    int n = n_max;
    if (n_dev) n = min(n, *n_dev);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint8_t st = status[i];
        fb_apply(pts[i], pts_back[i], status_back[i], fb_max, st);
        status[i] = st;
    }
}

// This group's staging words in the block's dynamic shared memory, from its
// first 128-byte boundary (tensor copies land on 128-byte boundaries; every
// group's share is a multiple of 128 bytes).
template <int ST, int WIN>
__device__ __forceinline__ unsigned *warp_words() {
    extern __shared__ __align__(128) unsigned lk_smem[];
    const unsigned lead = (128u - (smem_u32(lk_smem) & 127u)) & 127u;
    return lk_smem + lead / 4 + (size_t)(threadIdx.x / lk_group<WIN>()) * Dims<ST, WIN>::WORDS;
}

template <int ST, int WIN>
constexpr size_t stage_bytes(int warps = LK_WARPS) {
    return (size_t)warps * (32 / lk_group<WIN>()) * Dims<ST, WIN>::WORDS * 4 + 128;
}

template <int ST, int WIN>
__global__ void __launch_bounds__(LK_MAX_NT) lk_kernel(const __grid_constant__ LKArgs a) {
    unsigned *W = warp_words<ST, WIN>();
    int n = a.n_max;
    if (a.n_dev) {
        const int m = *a.n_dev;
        n = m < n ? m : n;
    }
    constexpr int G = lk_group<WIN>();
    const int glane = group_lane<G>();
    const int ngroups = gridDim.x * (LK_NT / G);
    Fills f;
    fills_init<G>(f, W + Dims<ST, WIN>::BAR, glane);
    const CUtensorMap *tm = all_maps(a.tm_ok, a.levels) ? a.tm : nullptr;
    Prefetch pf;
    pf.valid = false;
    for (int i = blockIdx.x * (LK_NT / G) + (int)(threadIdx.x / G); i < n; i += ngroups) {
        if (f.pend & FILL_FAILED) {   // a wait ran out: the group's later points are given up
            lost_timeout(a.pts[i], i, a.out, a.status, a.iters, a.levels, glane);
            continue;
        }
        const int nxt = i + ngroups;
        auto next = [&]() {
            const bool has = nxt < n;
            return next_top<WIN>(has, has ? a.pts[nxt] : make_float2(0.f, 0.f), a.P, tm, a.levels);
        };
        const PointResult r = lk_point<ST, WIN>(a.P, a.J, a.levels, a.max_iter, a.eps2, a.tau_n,
                                                a.pts[i], tm, W, f, pf, next,
                                                (long long)i == lk_fail_point);
        put_point(r, i, a.out, a.status, a.iters, a.levels, glane);
    }
    fill_drain<G>(f);
}

// Queue positions [lo, hi) of a batch that a failed warp holds: reported
// OMT_PT_LOST_TIMEOUT (out of line: only a failed warp gets here).
template <bool backward>
__device__ __noinline__ void give_up_batch(const uint8_t *table, const int32_t *pre, int lo,
                                           int hi, int lane) {
    const BatchView t(table);
    const BatchHeader &h = t.hdr();
    for (int q = lo; q < hi; ++q) {
        const int sq = find_segment(pre, h.nstreams, q);
        const StreamEntry &eq = t.stream(sq);
        const int iq = q - pre[sq];
        if constexpr (backward) {
            lost_timeout(eq.pts_out[iq], iq, eq.pts_back, eq.status_back, nullptr, h.levels, lane);
            if (lane == 0)
                fb_apply(eq.pts[iq], eq.pts_back[iq], eq.status_back[iq], h.fb_max, eq.status[iq]);
        } else {
            lost_timeout(eq.pts[iq], iq, eq.pts_out, eq.status, eq.iters, h.levels, lane);
        }
    }
}

// All points of all streams of a batch: the per-stream counts come from the
// CSR offsets written by the corner step; each CTA forms their prefix in
// shared memory.  Warps take `chunk` consecutive points at a time from a
// work queue (a counter in the table's header, zeroed before the launch), so
// points of uneven cost balance over the warps; a warp takes its next chunk
// before the last point of the current one, whose finest level then
// prefetches the next point's top-level template.
template <int ST, int WIN, bool backward>
__global__ void __launch_bounds__(LK_MAX_NT) __maxnreg__(lk_batch_regs<WIN>())
    lk_batch_kernel(const uint8_t *table, int chunk) {
    __shared__ int32_t pre[OMT_BATCH_MAX_STREAMS + 1];
    unsigned *W = warp_words<ST, WIN>();
    const BatchView t(table);
    const BatchHeader &h = t.hdr();
    if constexpr (backward) {
        if (!h.fb_on) return;  // a table packed without the check
    }
    unsigned *queue = const_cast<unsigned *>(&h.work[0]);
    const int ns = h.nstreams;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        // the streams' point counts, a lane per stream, and their prefix
        int acc = 0;
        for (int b = 0; b < ns; b += 32) {
            const int s = b + lane;
            int c = 0;
            if (s < ns) {
                const StreamEntry &e = t.stream(s);
                c = e.offsets[e.nboxes];
            }
            int v = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(FULL_MASK, v, o);
                if (lane >= o) v += u;
            }
            if (s < ns) pre[s + 1] = acc + v;
            acc += __shfl_sync(FULL_MASK, v, 31);
        }
        if (lane == 0) pre[0] = 0;
    }
    __syncthreads();
    const int total = pre[ns];
    constexpr int G = lk_group<WIN>();
    const int glane = group_lane<G>();
    auto take = [&]() -> int {
        unsigned b = 0;
        if (glane == 0) b = atomicAdd(queue, (unsigned)chunk);
        b = __shfl_sync(group_mask<G>(), b, 0, G);
        return b < (unsigned)total ? (int)b : total;
    };
    Fills f;
    fills_init<G>(f, W + Dims<ST, WIN>::BAR, glane);
    Prefetch pf;
    pf.valid = false;
    int g = take(), end = g + chunk;
    int s = g < total ? find_segment(pre, ns, g) : 0;
    while (g < total) {
        int gn = g + 1;
        if (gn >= end || gn >= total) {
            gn = take();
            end = gn + chunk;
        }
        const int i = g - pre[s];
        const bool has_next = gn < total;
        const int sn = has_next ? find_segment(pre, ns, gn) : s;
        PointResult r;
        {
            const StreamEntry &e = t.stream(s);
            // forward: frame t -> t+1 from the corners; backward: frame t+1 -> t
            // from the forward results
            const float2 u = (backward ? e.pts_out : e.pts)[i];
            auto next = [&]() {
                const StreamEntry &en = t.stream(sn);
                const float2 un = has_next ? (backward ? en.pts_out : en.pts)[gn - pre[sn]]
                                           : make_float2(0.f, 0.f);
                return next_top<WIN>(has_next, un, backward ? en.P_next : en.P,
                                     stream_maps(t, sn, h.levels, backward), h.levels);
            };
            r = lk_point<ST, WIN>(backward ? e.P_next : e.P, backward ? e.P : e.P_next, h.levels,
                                  h.max_iter, h.eps2, h.tau_n, u,
                                  stream_maps(t, s, h.levels, backward), W, f, pf, next,
                                  (long long)g == lk_fail_point);
        }
        {
            const StreamEntry &e = t.stream(s);
            if constexpr (backward) {
                put_point(r, i, e.pts_back, e.status_back, nullptr, h.levels, glane);
                if (glane == 0)
                    fb_apply(e.pts[i], e.pts_back[i], e.status_back[i], h.fb_max, e.status[i]);
            } else {
                put_point(r, i, e.pts_out, e.status, e.iters, h.levels, glane);
            }
        }
        if (f.pend & FILL_FAILED) {
            // a wait ran out: the points this group holds (the rest of its
            // chunk, or the chunk it took next) are given up, and it takes
            // no more work
            give_up_batch<backward>(table, pre, gn, end < total ? end : total, glane);
            break;
        }
        g = gn;
        s = sn;
    }
    fill_drain<G>(f);
}

// A CTA of LK_NT threads tracks LK_NT / G points at a time; the grid
// covers the points once, at most 32 CTAs per SM.
template <int ST, int W>
cudaError_t launch_plain(const LKArgs &a, int sms, cudaStream_t s) {
    if (cudaFuncSetAttribute(lk_kernel<ST, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stage_bytes<ST, W>()) != cudaSuccess)
        return cudaGetLastError();
    const int per = LK_NT / lk_group<W>();
    const int need = (a.n_max + per - 1) / per, cap = sms * 32;
    lk_kernel<ST, W><<<need < cap ? need : cap, LK_NT, stage_bytes<ST, W>(), s>>>(a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_st(const LKArgs &a, int win, int sms, cudaStream_t s) {
    switch (win) {
#define OMT_LK_CASE(W)                                                                    \
    case W:                                                                               \
        return launch_plain<ST, W>(a, sms, s);
        OMT_LK_CASE(3) OMT_LK_CASE(5) OMT_LK_CASE(7) OMT_LK_CASE(9) OMT_LK_CASE(11)
        OMT_LK_CASE(13) OMT_LK_CASE(15) OMT_LK_CASE(17) OMT_LK_CASE(19) OMT_LK_CASE(21)
        OMT_LK_CASE(23) OMT_LK_CASE(25) OMT_LK_CASE(27) OMT_LK_CASE(29) OMT_LK_CASE(31)
#undef OMT_LK_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int ST, int WIN, bool backward>
cudaError_t launch_batch_dir(const uint8_t *table, int sms, int warps, int ctas_per_sm, int chunk,
                             cudaStream_t s) {
    // no more warps per CTA than their staging areas fit in shared memory
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int fit = optin / (int)stage_bytes<ST, WIN>(1);
    if (warps > fit) warps = fit > 0 ? fit : 1;
    const size_t smem = stage_bytes<ST, WIN>(warps);
    e = cudaFuncSetAttribute(lk_batch_kernel<ST, WIN, backward>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lk_batch_kernel<ST, WIN, backward>, 32 * warps,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    // the work queue starts at 0 for every launch
    e = cudaMemsetAsync(const_cast<uint8_t *>(table) + offsetof(BatchHeader, work), 0,
                        sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    lk_batch_kernel<ST, WIN, backward><<<sms * per_sm, 32 * warps, smem, s>>>(table, chunk);
    return cudaGetLastError();
}

template <int ST, int WIN>
cudaError_t launch_batch_win(const uint8_t *table, int sms, int warps, int ctas_per_sm, int chunk,
                             int backward, cudaStream_t s) {
    if (backward) return launch_batch_dir<ST, WIN, true>(table, sms, warps, ctas_per_sm, chunk, s);
    return launch_batch_dir<ST, WIN, false>(table, sms, warps, ctas_per_sm, chunk, s);
}

template <int ST>
cudaError_t launch_batch_st(const uint8_t *table, int win, int sms, int warps, int ctas_per_sm,
                            int chunk, int backward, cudaStream_t s) {
    switch (win) {
#define OMT_LK_CASE(W) \
    case W: return launch_batch_win<ST, W>(table, sms, warps, ctas_per_sm, chunk, backward, s);
        OMT_LK_CASE(3) OMT_LK_CASE(5) OMT_LK_CASE(7) OMT_LK_CASE(9) OMT_LK_CASE(11)
        OMT_LK_CASE(13) OMT_LK_CASE(15) OMT_LK_CASE(17) OMT_LK_CASE(19) OMT_LK_CASE(21)
        OMT_LK_CASE(23) OMT_LK_CASE(25) OMT_LK_CASE(27) OMT_LK_CASE(29) OMT_LK_CASE(31)
#undef OMT_LK_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// ------------------------------------------------------------ tensor maps
namespace {

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled tensor_map_encoder() {
    static const EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiled) nullptr;
        }
        return (EncodeTiled)p;
    }();
    return fn;
}

// Encoded maps are kept by their parameters: a caller that re-packs the
// same pyramid buffers every step pays for each map once.
struct MapKey {
    const void *base;
    int64_t pitch;
    int w, h, dtype, box_w, box_h;
    bool operator==(const MapKey &o) const {
        return base == o.base && pitch == o.pitch && w == o.w && h == o.h && dtype == o.dtype &&
               box_w == o.box_w && box_h == o.box_h;
    }
};
struct MapKeyHash {
    size_t operator()(const MapKey &k) const {
        uint64_t x = (uint64_t)(uintptr_t)k.base ^ ((uint64_t)k.pitch << 17);
        x ^= ((uint64_t)k.w << 32) ^ ((uint64_t)k.h << 8) ^ ((uint64_t)k.dtype << 56);
        x ^= ((uint64_t)k.box_w << 40) ^ ((uint64_t)k.box_h << 24);
        x *= 0x9E3779B97F4A7C15ull;
        return (size_t)(x ^ (x >> 29));
    }
};
constexpr size_t MAP_CACHE_MAX = 8192;

// A 2D map of a plane of h rows of w elements (pitch bytes apart) read in
// boxes of box_w x box_h elements, zero-filled outside the plane.
bool encode_2d(CUtensorMap *m, CUtensorMapDataType dt, const void *base, int w, int h,
               int64_t pitch, int box_w, int box_h) {
    static std::mutex mu;
    static std::unordered_map<MapKey, CUtensorMap, MapKeyHash> cache;
    const MapKey key{base, pitch, w, h, (int)dt, box_w, box_h};
    std::lock_guard<std::mutex> lock(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) {
        *m = it->second;
        return true;
    }
    const EncodeTiled enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t elem[2] = {1, 1};
    if (enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (cache.size() >= MAP_CACHE_MAX) cache.clear();
    cache.emplace(key, *m);
    return true;
}

template <int ST, int WIN>
uint32_t encode_win(const omt_pyramid &P, const omt_pyramid &J, CUtensorMap *out) {
    using D = Dims<ST, WIN>;
    const CUtensorMapDataType dg = D::GSZ == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                               : CU_TENSOR_MAP_DATA_TYPE_INT64;
    uint32_t ok = 0;
    for (int L = 0; L < P.levels && L < OMT_MAX_LEVELS; ++L) {
        const int esz = L == 0 ? 1 : D::ESZ;
        const CUtensorMapDataType di = esz == 1   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                       : esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_UINT32;
        const LevelView p = level_view(P, L), j = level_view(J, L);
        CUtensorMap *m = out + LK_MAPS * L;
        if (encode_2d(m + LK_MAP_TI, di, p.img, p.w, p.h, p.img_pitch, D::RWI * 4 / esz, D::T) &&
            encode_2d(m + LK_MAP_TG, dg, p.grad, p.w, p.h, p.grad_pitch, D::RWG * 4 / D::GSZ, D::T) &&
            encode_2d(m + LK_MAP_S, di, j.img, j.w, j.h, j.img_pitch, D::RWJ * 4 / esz, D::SH))
            ok |= 7u << (LK_MAPS * L);
    }
    return ok;
}

template <int ST>
uint32_t encode_st(const omt_pyramid &P, const omt_pyramid &J, int win, CUtensorMap *out) {
    switch (win) {
#define OMT_LK_CASE(W) \
    case W: return encode_win<ST, W>(P, J, out);
        OMT_LK_CASE(3) OMT_LK_CASE(5) OMT_LK_CASE(7) OMT_LK_CASE(9) OMT_LK_CASE(11)
        OMT_LK_CASE(13) OMT_LK_CASE(15) OMT_LK_CASE(17) OMT_LK_CASE(19) OMT_LK_CASE(21)
        OMT_LK_CASE(23) OMT_LK_CASE(25) OMT_LK_CASE(27) OMT_LK_CASE(29) OMT_LK_CASE(31)
#undef OMT_LK_CASE
        default: return 0;
    }
}

}  // namespace

bool encode_plane_map(const void *base, int esz, int w, int h, int64_t pitch, int box_w, int box_h,
                      CUtensorMap *out) {
    if (((uintptr_t)base & 15) || (pitch & 15) || w < 1 || h < 1) return false;
    const CUtensorMapDataType dt = esz == 1   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                              : CU_TENSOR_MAP_DATA_TYPE_UINT32;
    return encode_2d(out, dt, base, w, h, pitch, box_w, box_h);
}

uint32_t encode_lk_maps(const omt_pyramid &P, const omt_pyramid &J, int win, CUtensorMap *out) {
    if (P.storage == OMT_F32) return encode_st<OMT_F32>(P, J, win, out);
    return encode_st<OMT_F16>(P, J, win, out);
}

cudaError_t lk_fail_point_set(long long point) {
    return cudaMemcpyToSymbol(lk_fail_point, &point, sizeof(point));
}

cudaError_t lk_wait_timeouts_take(unsigned *count) {
    unsigned zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(count, lk_wait_timeouts, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(lk_wait_timeouts, &zero, sizeof(unsigned));
    return e;
}

cudaError_t launch_lk_batch(const uint8_t *table, int storage, int win, int warps,
                            int ctas_per_sm, int chunk, int backward, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (warps <= 0) warps = LK_WARPS;
    if (chunk <= 0) chunk = 1;
    if (storage == OMT_F32)
        return launch_batch_st<OMT_F32>(table, win, sms, warps, ctas_per_sm, chunk, backward, s);
    return launch_batch_st<OMT_F16>(table, win, sms, warps, ctas_per_sm, chunk, backward, s);
}

cudaError_t launch_fb_check(const float2 *pts, const float2 *pts_back, const uint8_t *status_back,
                            int n_max, const int32_t *n_dev, float fb_max, uint8_t *status,
                            cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    const int nt = 256;
    int blocks = (n_max + nt - 1) / nt;
    if (blocks > 148 * 16) blocks = 148 * 16;
    fb_check_kernel<<<blocks, nt, 0, s>>>(pts, pts_back, status_back, n_max, n_dev, fb_max,
                                          status);
    return cudaGetLastError();
}

cudaError_t launch_lk(const omt_pyramid &prev, const omt_pyramid &next, const float2 *pts,
                      int n_max, const int32_t *n_dev, const omt_params &prm, float2 *out,
                      uint8_t *status, uint8_t *iters, cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    LKArgs a;
    a.tm_ok = encode_lk_maps(prev, next, prm.win, a.tm);
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
    if (prev.storage == OMT_F32) return launch_st<OMT_F32>(a, prm.win, sms, s);
    return launch_st<OMT_F16>(a, prm.win, sms, s);
}

}  // namespace omt

