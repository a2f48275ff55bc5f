// corners.cu -- K2: Shi-Tomasi response and per-box corner selection.
//
// The response walk: 28x64 strips of level 0, one warp each (only strips
// that touch an eligible pixel of some box when boxes are given), all in
// registers: integer Scharr -> 3x3 structure tensor -> exact
// R = (a+c) - isqrt((a-c)^2 + 4b^2) -> non-strict 3x3 maximum flag, the
// value R | flag << 30 of every pixel.
//
// Corner selection, per call (four launches after a reset of the per-box
// counters):
//   1. list_kernel       the response walk into a shared-memory copy of the
//                        strip; then, for every box the strip overlaps, R_max
//                        of the box's pixels in the strip (atomic max) and
//                        the keys (R << 32 | ~(y*W + x)) of its local maxima
//                        with R > 0, appended to the box's candidate list
//                        (CAND_CAP keys, one atomic per box and strip).
//   2. overflow_kernel   the response walk into the frame-sized uint32 map,
//                        only for strips that touch a box whose list
//                        overflowed (none on ordinary frames).
//   3. select_kernel     one CTA per box: the candidates from its list (or,
//                        after an overflow, from one pass over its map),
//                        bitonic sort in shared memory, greedy minimum-
//                        distance acceptance by one warp.  Boxes with more
//                        candidates than fit in shared memory are consumed in
//                        descending chunks found by an exact MSD radix select
//                        over the keys.
//   4. compact_kernel    exclusive scan of the per-box counts into the CSR
//                        offsets and a copy of the kept points, box by box.
// omt_corner_response runs the walk into the map alone.
// Everything is integer arithmetic, so the result equals the definition bit
// for bit, and the atomics only change the order in which unique keys are
// gathered, never the sorted order.
#include <type_traits>

#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr uint32_t R_MASK = 0x3FFFFFFFu;
constexpr uint32_t MAX_FLAG = 1u << 30;

// ----------------------------------------------------------- exact isqrt
// floor(sqrt(D)) for D < 2^58 given f, any float within a relative 2^-20 of
// D, without branches: the hardware square-root approximation of f is within a
// relative 2^-19 of sqrt(D) (within 2^10 for sqrt(D) < 2^29), and one
// Newton step on the exact residual leaves it within one unit of
// floor(sqrt(D)) (the step's overshoot e^2 / (2 s) stays below 0.1, its
// float rounding below 1e-3), which one comparison each way settles.
__device__ __forceinline__ uint32_t isqrt_est(uint64_t D, float f) {
    float sf;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(sf) : "f"(f));
    int s = (int)sf;  // < 2^30
    const int64_t r = (int64_t)D - (int64_t)((uint64_t)(uint32_t)s * (uint32_t)s);
    s += s > 0 ? (int)floorf(__fdividef((float)r, 2.0f * (float)s)) : 0;
    s = s < 0 ? 0 : s;
    const uint64_t sq = (uint64_t)(uint32_t)s * (uint32_t)s;
    const uint64_t sq1 = sq + 2 * (uint64_t)(uint32_t)s + 1;  // (s + 1)^2
    return (uint32_t)(s - (sq > D ? 1 : 0) + (sq1 <= D ? 1 : 0));
}

// ------------------------------------------------------ response map kernel
// A warp walks a strip of RW = 28 columns down RH = 64 rows of level 0, all
// in registers.  Lane l holds column x = x0 - 2 + l; lanes 2..29 own the
// strip's columns, the others supply the halo.  Per row step a lane loads
// its column's texel of the new bottom row (the three rows around the step's
// gradient row slide down; reflected rows at the frame's top and bottom are
// read afresh), takes the neighbouring columns from lanes l-1 and l+1 by
// shuffles (lanes 0 and 31 load theirs), forms the raw Scharr gradient, and
// the 3x1 sums of the structure tensor products from its neighbours'
// gradients; the 1x3 sums come from the two previous rows kept in registers.  The response of
// the row above follows (exact integer square root), and the non-strict 3x3
// maximum flag of the row above that is decided from the 3-column maxima of
// three response rows.  A gradient position outside the frame takes the
// gradient of its reflect-101 image (a lane shuffle for columns; for rows the
// three texel rows are reflected around the reflected row).
constexpr int RW = 28, RH = 64, RNT = 256, RWARPS = RNT / 32;
// The list kernel keeps one strip's values (RW x RH words) per warp in
// shared memory: 4 warps per CTA.
constexpr int LNT = 128, LWARPS = LNT / 32;
// Keys a box's candidate list holds; a box with more candidates takes the
// map path (the select kernel's shared key capacity).
constexpr int CAND_CAP = 1024;

struct RespArgs {
    const uint8_t *img;
    int64_t pitch;
    int w, h;
    uint32_t *out;        // w*h, row-major, no padding
    const float4 *boxes;  // nullptr: whole frame
    int nboxes;
    uint64_t *cand;       // nboxes x CAND_CAP candidate keys
    uint32_t *cstate;     // per box: key count, R_max; then the overflow word
    uint32_t *any_overflow;  // batched step: set when any stream's list overflows, or null
};

// A candidate's sort key: R above the complemented pixel index, so that
// descending keys run by R descending, then raster index ascending.
__device__ __forceinline__ uint64_t make_key(uint32_t R, uint32_t idx) {
    return ((uint64_t)R << 32) | (uint64_t)(0xFFFFFFFFu - idx);
}

// Whether the strip tile at (x0, y0) holds an eligible pixel of some box
// (always, without boxes); with only_overflow, of some box whose candidate
// list overflowed.  Warp-uniform.
__device__ __forceinline__ bool strip_needed(const RespArgs &a, int x0, int y0, int lane,
                                             bool only_overflow = false) {
    if (!a.boxes) return true;
    const int x1 = min(x0 + RW - 1, a.w - 1), y1 = min(y0 + RH - 1, a.h - 1);
    for (int b0 = 0; b0 < a.nboxes; b0 += 32) {
        const int b = b0 + lane;
        bool hit = false;
        if (b < a.nboxes && (!only_overflow || a.cstate[2 * b] > (uint32_t)CAND_CAP)) {
            int xlo, xhi, ylo, yhi;
            if (box_pixel_range(a.boxes[b], a.w, a.h, xlo, xhi, ylo, yhi))
                hit = xlo <= x1 && xhi >= x0 && ylo <= y1 && yhi >= y0;
        }
        if (__any_sync(FULL_MASK, hit)) return true;
    }
    return false;
}

// The response walk of the strip whose first output column is x0 and first
// output row oy; every pixel of the strip inside the frame is handed to
// put(yf, x, R | flag) exactly once, by the lane that owns its column
// (lanes 2 .. 29).
template <class Put>
__device__ __forceinline__ void response_strip(const RespArgs &a, int x0, int oy, int lane,
                                               Put put) {
    const int x = x0 - 2 + lane;
    const bool inx = x >= 0 && x < a.w;
    const int cx = reflect101(x, a.w);
    const bool edge = lane == 0 || lane == 31;
    const int ex = reflect101(lane == 0 ? x - 1 : x + 1, a.w);  // edge lanes' outer column
    // Outside the frame a lane takes the gradient of its mirror column's
    // lane; only strips that reach a frame edge need the exchange.
    const bool mirror = x0 - 2 < 0 || x0 + 29 >= a.w;
    int src = lane;
    if (!inx) src = min(max(reflect101(x, a.w) - (x0 - 2), 0), 31);
    // texels of the three rows around the gradient row: own column (v),
    // left (l) and right (q) neighbours; m, 0, p = rows above, at, below
    int vm = 0, v0 = 0, vp = 0, lm = 0, l0 = 0, lp = 0, qm = 0, q0 = 0, qp = 0;
    int Ha2 = 0, Hb2 = 0, Hc2 = 0, Ha1 = 0, Hb1 = 0, Hc1 = 0;  // 3x1 sums, rows g-2, g-1
    uint32_t Rp = 0, M2 = 0, M1 = 0;  // R of row g-2; 3-column maxima of rows g-3, g-2
    // texels of row g+1 loaded one step early by the sliding steps (nv, ne)
    int nv = 0, ne = 0;
    // One step: gradient row g = oy - 2 + s.  SLIDE steps (rows g-1 .. g+1
    // inside the frame, after the first step) shift the rows read by the
    // previous step and take row g+1 from the prefetch; the others read the
    // three (reflected) rows afresh.  The sliding steps are one contiguous
    // range of s, so the loops below need no per-step branch between them.
    auto step = [&](int s, auto slide) {
        const int g = oy - 2 + s;
        if constexpr (decltype(slide)::value) {
            vm = v0;
            v0 = vp;
            lm = l0;
            l0 = lp;
            qm = q0;
            q0 = qp;
            vp = nv;
            const int ep = ne;
            // the next step's row g+2 (clamped: the last sliding step's
            // prefetch is not used)
            const uint8_t *r3 = a.img + (int64_t)min(g + 2, a.h - 1) * a.pitch;
            nv = __ldg(r3 + cx);
            ne = edge ? (int)__ldg(r3 + ex) : 0;
            lp = __shfl_up_sync(FULL_MASK, vp, 1);
            qp = __shfl_down_sync(FULL_MASK, vp, 1);
            lp = lane == 0 ? ep : lp;
            qp = lane == 31 ? ep : qp;
        } else {
            const int py = reflect101(g, a.h);
            const uint8_t *r0 = a.img + (int64_t)reflect101(py - 1, a.h) * a.pitch;
            const uint8_t *r1 = a.img + (int64_t)py * a.pitch;
            const uint8_t *r2 = a.img + (int64_t)reflect101(py + 1, a.h) * a.pitch;
            vm = __ldg(r0 + cx);
            v0 = __ldg(r1 + cx);
            vp = __ldg(r2 + cx);
            int em = 0, e0 = 0, ep = 0;
            if (edge) {
                em = __ldg(r0 + ex);
                e0 = __ldg(r1 + ex);
                ep = __ldg(r2 + ex);
            }
            lm = __shfl_up_sync(FULL_MASK, vm, 1);
            l0 = __shfl_up_sync(FULL_MASK, v0, 1);
            lp = __shfl_up_sync(FULL_MASK, vp, 1);
            qm = __shfl_down_sync(FULL_MASK, vm, 1);
            q0 = __shfl_down_sync(FULL_MASK, v0, 1);
            qp = __shfl_down_sync(FULL_MASK, vp, 1);
            lm = lane == 0 ? em : lm;
            l0 = lane == 0 ? e0 : l0;
            lp = lane == 0 ? ep : lp;
            qm = lane == 31 ? em : qm;
            q0 = lane == 31 ? e0 : q0;
            qp = lane == 31 ? ep : qp;
        }
        int gx = 3 * (qm - lm) + 10 * (q0 - l0) + 3 * (qp - lp);
        int gy = 3 * (lp - lm) + 10 * (vp - vm) + 3 * (qp - qm);
        if (mirror) {
            gx = __shfl_sync(FULL_MASK, gx, src);
            gy = __shfl_sync(FULL_MASK, gy, src);
        }
        // 3x1 sums of the tensor products over columns x-1 .. x+1
        const int gxl = __shfl_up_sync(FULL_MASK, gx, 1), gyl = __shfl_up_sync(FULL_MASK, gy, 1);
        const int gxr = __shfl_down_sync(FULL_MASK, gx, 1), gyr = __shfl_down_sync(FULL_MASK, gy, 1);
        const int Ha0 = gxl * gxl + gx * gx + gxr * gxr;
        const int Hb0 = gxl * gyl + gx * gy + gxr * gyr;
        const int Hc0 = gyl * gyl + gy * gy + gyr * gyr;

        // response of row g - 1 (its tensor is complete: rows g-2 .. g);
        // computed by every lane, kept where the pixel is in the frame
        const int ta = Ha2 + Ha1 + Ha0, tb = Hb2 + Hb1 + Hb0, tc = Hc2 + Hc1 + Hc0;
        const int amc = ta - tc;  // |a - c| < 2^28
        const uint64_t D = (uint64_t)((int64_t)amc * amc) + 4ull * (uint64_t)((int64_t)tb * tb);
        const float fa = (float)amc, fb = (float)tb;
        const float f = fmaf(fa, fa, 4.0f * fb * fb);
        const uint32_t Rv = (uint32_t)((int64_t)ta + tc - (int64_t)isqrt_est(D, f));
        const uint32_t Rn = inx && g - 1 >= 0 && g - 1 < a.h ? Rv : 0u;
        const uint32_t Mn =
            max(Rn, max(__shfl_up_sync(FULL_MASK, Rn, 1), __shfl_down_sync(FULL_MASK, Rn, 1)));

        // row g - 2: its value and maximum flag (a predicated store)
        const int yf = g - 2;
        const bool interior = x >= 1 && x <= a.w - 2 && yf >= 1 && yf <= a.h - 2;
        const uint32_t flag = interior && Rp >= max(M2, max(M1, Mn)) ? MAX_FLAG : 0u;
        if (s >= 4 && yf < a.h && lane >= 2 && lane <= 29 && inx) put(yf, x, Rp | flag);
        Ha2 = Ha1;
        Hb2 = Hb1;
        Hc2 = Hc1;
        Ha1 = Ha0;
        Hb1 = Hb0;
        Hc1 = Hc0;
        M2 = M1;
        M1 = Mn;
        Rp = Rn;
    };
    using Fresh = std::integral_constant<bool, false>;
    using Slide = std::integral_constant<bool, true>;
    constexpr int STEPS = RH + 4;
    // sliding steps: s >= 1 with 2 <= g <= h - 2, i.e. s in [s_a, s_b]
    const int s_a = max(1, 4 - oy), s_b = min(STEPS - 1, a.h - oy);
    int s = 0;
#pragma unroll 1
    for (; s < min(s_a, STEPS); ++s) step(s, Fresh{});
    if (s_a <= s_b) {
        const uint8_t *r = a.img + (int64_t)(oy - 2 + s_a + 1) * a.pitch;  // row g(s_a) + 1
        nv = __ldg(r + cx);
        ne = edge ? (int)__ldg(r + ex) : 0;
#pragma unroll 1
        for (s = s_a; s <= s_b; ++s) step(s, Slide{});
    }
#pragma unroll 1
    for (; s < STEPS; ++s) step(s, Fresh{});
}

// Tile t of a w x h frame: strip column and row block.
__device__ __forceinline__ void strip_origin(int t, int w, int &x0, int &y0) {
    const int tx = (w + RW - 1) / RW;
    const int ty = t / tx;
    x0 = (t - ty * tx) * RW;
    y0 = ty * RH;
}

// The map form: every value into the frame-sized map.
__device__ __forceinline__ void strip_to_map(const RespArgs &a, int x0, int y0, int lane) {
    response_strip(a, x0, y0, lane,
                   [&](int yf, int x, uint32_t v) { a.out[(int64_t)yf * a.w + x] = v; });
}

// The list form: the strip's values into this warp's shared copy, then, for
// each box the strip overlaps, its part of the box's R_max (atomic max) and
// the keys of its local maxima with R > 0, appended to the box's list (one
// atomic per box and strip: count, reserve, write).  Appends past CAND_CAP
// are dropped; the count still grows, marking the overflow, and the
// stream's overflow word is set.  Every pixel of the frame lies in exactly
// one strip, so a box's list ends with the keys of exactly its candidates
// whenever it did not overflow (in an order that depends on the schedule;
// the select kernel sorts them).
__device__ __forceinline__ void strip_to_lists(const RespArgs &a, int x0, int y0, int lane,
                                               uint32_t *buf) {
    response_strip(a, x0, y0, lane,
                   [&](int yf, int x, uint32_t v) { buf[(yf - y0) * RW + (x - x0)] = v; });
    __syncwarp();
    const int x1 = min(x0 + RW - 1, a.w - 1), y1 = min(y0 + RH - 1, a.h - 1);
    const int x = x0 + lane;  // lane c reads strip column c
    const uint32_t *cp = buf + (lane < RW ? lane : 0);
    for (int b0 = 0; b0 < a.nboxes; b0 += 32) {
        const int b = b0 + lane;
        int xlo = 0, xhi = -1, ylo = 0, yhi = -1;
        bool hit = false;
        if (b < a.nboxes && box_pixel_range(a.boxes[b], a.w, a.h, xlo, xhi, ylo, yhi))
            hit = xlo <= x1 && xhi >= x0 && ylo <= y1 && yhi >= y0;
        unsigned m = __ballot_sync(FULL_MASK, hit);
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const int bx0 = max(__shfl_sync(FULL_MASK, xlo, j), x0);
            const int bx1 = min(__shfl_sync(FULL_MASK, xhi, j), x1);
            const int by0 = max(__shfl_sync(FULL_MASK, ylo, j), y0);
            const int by1 = min(__shfl_sync(FULL_MASK, yhi, j), y1);
            const int box = b0 + j;
            const bool col = lane < RW && x >= bx0 && x <= bx1;
            uint32_t rm = 0;
            int c = 0;
            for (int y = by0; y <= by1; ++y) {
                const uint32_t v = col ? cp[(y - y0) * RW] : 0u;
                const uint32_t R = v & R_MASK;
                rm = max(rm, R);
                c += (v & MAX_FLAG) && R > 0;
            }
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL_MASK, incl, o);
                if (lane >= o) incl += t;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rm = max(rm, __shfl_xor_sync(FULL_MASK, rm, o));
            const int total = __shfl_sync(FULL_MASK, incl, 31);
            uint32_t base = 0;
            if (lane == 0) {
                uint32_t *st = a.cstate + 2 * box;
                if (rm) atomicMax(st + 1, rm);
                if (total) {
                    base = atomicAdd(st, (uint32_t)total);
                    if (base + (uint32_t)total > (uint32_t)CAND_CAP) {
                        a.cstate[2 * a.nboxes] = 1u;
                        if (a.any_overflow) *a.any_overflow = 1u;
                    }
                }
            }
            base = __shfl_sync(FULL_MASK, base, 0);
            if (total && base < (uint32_t)CAND_CAP) {
                uint32_t pos = base + (uint32_t)(incl - c);
                uint64_t *out = a.cand + (int64_t)box * CAND_CAP;
                for (int y = by0; y <= by1 && c > 0; ++y) {
                    const uint32_t v = col ? cp[(y - y0) * RW] : 0u;
                    const uint32_t R = v & R_MASK;
                    if ((v & MAX_FLAG) && R > 0) {
                        if (pos < (uint32_t)CAND_CAP) out[pos] = make_key(R, (uint32_t)(y * a.w + x));
                        ++pos;
                        --c;
                    }
                }
            }
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(RNT) response_kernel(RespArgs a, int total) {
    const int lane = threadIdx.x & 31;
    for (int t = blockIdx.x * RWARPS + (threadIdx.x >> 5); t < total; t += gridDim.x * RWARPS) {
        int x0, y0;
        strip_origin(t, a.w, x0, y0);
        if (strip_needed(a, x0, y0, lane)) strip_to_map(a, x0, y0, lane);
    }
}

// The strips of a frame for the candidate lists (boxes given).
__global__ void __launch_bounds__(LNT) list_kernel(RespArgs a, int total) {
    __shared__ uint32_t strip[LWARPS][RW * RH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = blockIdx.x * LWARPS + warp; t < total; t += gridDim.x * LWARPS) {
        int x0, y0;
        strip_origin(t, a.w, x0, y0);
        if (strip_needed(a, x0, y0, lane)) strip_to_lists(a, x0, y0, lane, strip[warp]);
    }
}

// The map, only where a box's list overflowed (the stream's overflow word).
__global__ void __launch_bounds__(RNT) overflow_kernel(RespArgs a, int total) {
    if (a.cstate[2 * a.nboxes] == 0u) return;
    const int lane = threadIdx.x & 31;
    for (int t = blockIdx.x * RWARPS + (threadIdx.x >> 5); t < total; t += gridDim.x * RWARPS) {
        int x0, y0;
        strip_origin(t, a.w, x0, y0);
        if (strip_needed(a, x0, y0, lane, true)) strip_to_map(a, x0, y0, lane);
    }
}

__device__ __forceinline__ RespArgs stream_resp_args(const StreamEntry &e, uint32_t *any_overflow) {
    RespArgs a;
    a.img = e.P[0].img;
    a.pitch = e.P[0].img_pitch;
    a.w = e.w;
    a.h = e.h;
    a.out = e.rmap;
    a.boxes = e.boxes;
    a.nboxes = e.nboxes;
    a.cand = e.cand;
    a.cstate = e.cstate;
    a.any_overflow = any_overflow;
    return a;
}

// Per-box counters and R_max, and the overflow word, of every stream back
// to zero (a CTA per stream).
__global__ void reset_lists_batch_kernel(const uint8_t *table) {
    const BatchView t(table);
    const int si = blockIdx.x;
    if (si >= t.nstreams()) return;
    const StreamEntry &e = t.stream(si);
    for (int i = threadIdx.x; i <= 2 * e.nboxes; i += blockDim.x) e.cstate[i] = 0u;
    if (si == 0 && threadIdx.x == 0) {
        uint32_t *work = const_cast<uint32_t *>(t.hdr().work);
        work[1] = 0u;
        work[2] = 0u;
    }
}

__global__ void __launch_bounds__(LNT) list_batch_kernel(const uint8_t *table) {
    __shared__ uint32_t strip[LWARPS][RW * RH];
    const BatchView t(table);
    const int32_t *pre = t.resp_prefix();
    const int total = pre[t.nstreams()];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *queue = const_cast<uint32_t *>(t.hdr().work) + 2;
    for (;;) {
        // the next strip, one atomic per warp and strip (strips differ in
        // cost, so a static stride leaves a tail of warps with one strip more)
        uint32_t take = 0;
        if (lane == 0) take = atomicAdd(queue, 1u);
        const int gi = (int)__shfl_sync(FULL_MASK, take, 0);
        if (gi >= total) break;
        const int si = find_segment(pre, t.nstreams(), gi);
        const StreamEntry &e = t.stream(si);
        if (e.nboxes == 0) continue;
        const RespArgs a = stream_resp_args(e, const_cast<uint32_t *>(t.hdr().work) + 1);
        int x0, y0;
        strip_origin(gi - pre[si], e.w, x0, y0);
        if (strip_needed(a, x0, y0, lane)) strip_to_lists(a, x0, y0, lane, strip[warp]);
    }
}

// Every stream's strips that touch an overflowed box; a step without an
// overflow leaves after one load per CTA.
__global__ void __launch_bounds__(RNT) overflow_batch_kernel(const uint8_t *table) {
    const BatchView t(table);
    if (t.hdr().work[1] == 0u) return;
    const int32_t *pre = t.resp_prefix();
    const int total = pre[t.nstreams()];
    const int lane = threadIdx.x & 31;
    for (int gi = blockIdx.x * RWARPS + (threadIdx.x >> 5); gi < total; gi += gridDim.x * RWARPS) {
        const int si = find_segment(pre, t.nstreams(), gi);
        const StreamEntry &e = t.stream(si);
        if (e.nboxes == 0 || e.cstate[2 * e.nboxes] == 0u) continue;
        const RespArgs a = stream_resp_args(e, nullptr);
        int x0, y0;
        strip_origin(gi - pre[si], e.w, x0, y0);
        if (strip_needed(a, x0, y0, lane, true)) strip_to_map(a, x0, y0, lane);
    }
}

// ------------------------------------------------------------ select kernel
constexpr int SNT = 128;
constexpr int SCAP = 1024;   // candidate keys held in shared memory
static_assert(CAND_CAP == SCAP, "a box's whole list fits the shared keys");
constexpr int GCAP = 4096;   // cells of the accepted-point grid in shared memory

// Keys sorted per chunk for a box keeping up to maxc corners: enough for the
// greedy pass to usually finish in one chunk (it rejects some candidates).
__host__ __device__ __forceinline__ int chunk_keys(int maxc) {
    int t = 64;
    while (t < 2 * maxc && t < SCAP) t <<= 1;
    return t;
}

// Dynamic shared memory of the select kernels for boxes of up to acc_cap
// corners: keys[SCAP] | sorted chunk | accepted points | grid cells.
__host__ __device__ __forceinline__ size_t select_smem_bytes(int acc_cap) {
    return (size_t)SCAP * 8 + (size_t)chunk_keys(acc_cap) * 8 + (size_t)acc_cap * 8 +
           (size_t)GCAP * 2;
}

struct SelectArgs {
    const uint32_t *rmap;
    int w, h;
    const float4 *boxes;
    int maxc;
    int qnum, qden;
    int64_t md2c;   // reject when dx^2 + dy^2 < md2c (= ceil(fl32(min_dist^2)))
    int dmax;       // largest |dx| with dx^2 < md2c
    int cell;       // side of the accepted-point grid cells, max(1, floor(sqrt(md2c / 2)))
    float2 *pad_pts;
    int32_t *pad_counts;
    const uint64_t *cand;   // per box: CAND_CAP candidate keys (list_kernel)
    const uint32_t *cstate; // per box: key count, R_max; null: map path only
};

// One compare-exchange of the bitonic network for the key at index i, held
// by this lane, against index i ^ j in the same warp (j < 32).
__device__ __forceinline__ uint64_t bitonic_step(uint64_t x, int i, int j, int k) {
    const uint64_t y = __shfl_xor_sync(FULL_MASK, x, j);
    const bool up = (i & k) == 0, lower = (i & j) == 0;
    const bool take_min = lower == up;
    return take_min ? (x < y ? x : y) : (x < y ? y : x);
}

// Ascending bitonic sort of keys[0..N), N a power of two, 32 <= N <= SCAP.
// Exchanges between indices less than 32 apart run inside a warp with
// shuffles (one key per lane); the wider ones through shared memory with a
// barrier per stage.
__device__ void bitonic_sort(uint64_t *keys, int N) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = warp * 32; b < N; b += SNT) {
        uint64_t x = keys[b + lane];
        for (int k = 2; k <= 32; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) x = bitonic_step(x, b + lane, j, k);
        keys[b + lane] = x;
    }
    __syncthreads();
    for (int k = 64; k <= N; k <<= 1) {
        for (int j = k >> 1; j >= 32; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += SNT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t x = keys[i], y = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        keys[i] = y;
                        keys[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
        for (int b = warp * 32; b < N; b += SNT) {
            uint64_t x = keys[b + lane];
            for (int j = 16; j > 0; j >>= 1) x = bitonic_step(x, b + lane, j, k);
            keys[b + lane] = x;
        }
        __syncthreads();
    }
}

// Grid of accepted points over a box's eligible pixels: cells of side
// `cell` with 2 (cell-1)^2 < md2c hold at most one accepted point each, so a
// candidate only checks the cells within dmax pixels of itself.
// The accepted points of a box, for the minimum-distance test: an
// occupancy bitmap of the box's pixels when the test's disc is small and the
// bitmap fits (bits), else a grid of cells holding an accepted point's index
// (cells), else none (the whole list is checked).
struct AccGrid {
    uint32_t *bits;  // row r of the box: bits[r * wpr ...], bit c = column xlo + c
    int16_t *cells;
    int gx, gy, xlo, ylo;
    int nx, rows, wpr;
};

// Whether an accepted point lies within the minimum distance of (xr, yr)
// (box-relative), from the occupancy bitmap: the rows |dy| <= dmax, in each
// the columns with dx^2 + dy^2 < md2c.
__device__ __forceinline__ bool bitmap_conflict(const AccGrid &g, int xr, int yr, int dmax,
                                                int64_t md2c) {
    for (int dy = -dmax; dy <= dmax; ++dy) {
        const int r = yr + dy;
        if (r < 0 || r >= g.rows) continue;
        int dx = dmax;
        while (dx > 0 && (int64_t)dx * dx + (int64_t)dy * dy >= md2c) --dx;
        const int c0 = max(xr - dx, 0), c1 = min(xr + dx, g.nx - 1);
        const uint32_t *row = g.bits + r * g.wpr;
        const int w0 = c0 >> 5, w1 = c1 >> 5;  // c1 - c0 <= 14: at most two words
        const uint64_t v = (uint64_t)row[w0] | (w1 != w0 ? (uint64_t)row[w1] << 32 : 0ull);
        const uint64_t mask = ((1ull << (c1 - c0 + 1)) - 1ull) << (c0 & 31);
        if (v & mask) return true;
    }
    return false;
}

// Greedy minimum-distance acceptance over the n largest keys of the sorted
// array (descending order from index N-1), by warp 0.  nacc is shared.
__device__ void greedy(const SelectArgs &a, int box, const uint64_t *keys, int N, int n,
                       int2 *acc, int *s_nacc, const AccGrid &g) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int nacc = *s_nacc;
    for (int base = 0; base < n && nacc < a.maxc; base += 32) {
        const int j = base + lane;
        const bool valid = j < n;
        const uint64_t key = valid ? keys[N - 1 - j] : 0ull;
        const uint32_t idx = 0xFFFFFFFFu - (uint32_t)key;
        const int y = (int)(idx / (uint32_t)a.w), x = (int)(idx - (uint32_t)y * (uint32_t)a.w);
        // a key always names a pixel of the box; anything else (a corrupted
        // input) is refused rather than indexing the grid out of range
        bool ok = valid && x >= g.xlo && y >= g.ylo && x < g.xlo + g.nx && y < g.ylo + g.rows;
        if (ok && a.md2c > 0) {
            if (g.bits) {
                ok = !bitmap_conflict(g, x - g.xlo, y - g.ylo, a.dmax, a.md2c);
            } else if (g.cells) {
                const int cx0 = max(x - a.dmax - g.xlo, 0) / a.cell;
                const int cx1 = min((x + a.dmax - g.xlo) / a.cell, g.gx - 1);
                const int cy0 = max(y - a.dmax - g.ylo, 0) / a.cell;
                const int cy1 = min((y + a.dmax - g.ylo) / a.cell, g.gy - 1);
                for (int cy = cy0; cy <= cy1 && ok; ++cy)
                    for (int cx = cx0; cx <= cx1; ++cx) {
                        const int t = g.cells[cy * g.gx + cx];
                        if (t >= 0) {
                            const int2 q = acc[t];
                            const int64_t dx = x - q.x, dy = y - q.y;
                            if (dx * dx + dy * dy < a.md2c) {
                                ok = false;
                                break;
                            }
                        }
                    }
            } else {
                for (int t = 0; t < nacc && ok; ++t) {
                    const int2 q = acc[t];
                    const int64_t dx = x - q.x, dy = y - q.y;
                    if (dx * dx + dy * dy < a.md2c) ok = false;
                }
            }
        }
        // The group in order: a candidate is kept iff it passed the test
        // against the points kept before the group (ok) and no earlier kept
        // candidate of the group lies within the minimum distance.  Each
        // lane first forms the mask of the group's earlier candidates within
        // that distance of its own (all lanes at once); the scan then keeps
        // the first undecided candidate and drops the later ones its lane
        // conflicts with, until none is left or max_corners is reached.
        unsigned undecided = __ballot_sync(FULL_MASK, ok);
        unsigned earlier = 0;  // bit q: candidate q < lane lies within the minimum distance
        if (a.md2c > 0 && (undecided & (undecided - 1u))) {
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                const int xq = __shfl_sync(FULL_MASK, x, q), yq = __shfl_sync(FULL_MASK, y, q);
                const int64_t dx = x - xq, dy = y - yq;
                if (q < lane && dx * dx + dy * dy < a.md2c) earlier |= 1u << q;
            }
        }
        unsigned kept = 0;
        int room = a.maxc - nacc;
        while (undecided && room > 0) {
            const int src = __ffs(undecided) - 1;
            kept |= 1u << src;
            --room;
            undecided &= ~(1u << src) & ~__ballot_sync(FULL_MASK, (earlier >> src) & 1u);
        }
        // the kept candidates, written by their own lanes in the group's order
        if ((kept >> lane) & 1u) {
            const int slot = nacc + __popc(kept & ((1u << lane) - 1u));
            acc[slot] = make_int2(x, y);
            if (g.bits)
                atomicOr(&g.bits[(y - g.ylo) * g.wpr + ((x - g.xlo) >> 5)], 1u << ((x - g.xlo) & 31));
            else if (g.cells)
                g.cells[((y - g.ylo) / a.cell) * g.gx + (x - g.xlo) / a.cell] = (int16_t)slot;
            a.pad_pts[(int64_t)box * a.maxc + slot] = make_float2((float)x, (float)y);
        }
        nacc += __popc(kept);
        __syncwarp();
    }
    if (lane == 0) *s_nacc = nacc;
}

// A lower bound `lo` such that exactly k of the keys in [lo_bound, hi)
// among keys[0..n) are >= lo (1 <= k <= their count; keys are unique): the
// k-th largest key, or the prefix of a digit bin that holds exactly the
// keys still needed (then no lower digit matters).  8-bit MSD radix select;
// whole CTA, result in the return value of every thread.
__device__ uint64_t kth_largest(const uint64_t *keys, int n, uint64_t lo_bound, uint64_t hi, int k,
                                unsigned *hist, int *s_sel, int *s_k) {
    const int tid = threadIdx.x;
    uint64_t prefix = 0, pmask = 0;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += SNT) hist[i] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += SNT) {
            const uint64_t key = keys[i];
            if (key >= lo_bound && key < hi && (key & pmask) == prefix)
                atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            // lane l holds bins 255-8l .. 248-8l; scan from the top
            unsigned c[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = hist[255 - 8 * tid - q];
                sum += c[q];
            }
            unsigned incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(FULL_MASK, incl, o);
                if (tid >= o) incl += v;
            }
            const unsigned excl = incl - sum;
            const unsigned hit = __ballot_sync(FULL_MASK, incl >= (unsigned)k);
            if (tid == __ffs(hit) - 1) {
                unsigned cum = excl;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (cum + c[q] >= (unsigned)k) {
                        // a bin holding exactly the keys still needed ends the search
                        *s_sel = (255 - 8 * tid - q) | (cum + c[q] == (unsigned)k ? 256 : 0);
                        *s_k = k - (int)cum;
                        break;
                    }
                    cum += c[q];
                }
            }
        }
        __syncthreads();
        const int sel = *s_sel;
        prefix |= (uint64_t)(sel & 255) << shift;
        pmask |= 0xFFull << shift;
        k = *s_k;
        __syncthreads();
        if (sel & 256) break;
    }
    return prefix;
}

// Gathers into keys[] (up to SCAP of them, counted in *count) the keys of
// the box's local maxima with R > 0 and, with QUALITY, qden * R > thr; a warp
// per row, eight loads in flight per lane.  Returns this lane's R_max.
template <bool QUALITY>
__device__ __forceinline__ uint32_t gather_keys(const SelectArgs &a, int xlo, int xhi, int ylo,
                                                int yhi, int64_t thr, uint64_t *keys, int *count) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t m = 0;
    for (int y = ylo + warp; y <= yhi; y += SNT / 32) {
        const uint32_t *row = a.rmap + (int64_t)y * a.w;
        for (int x = xlo + lane; x <= xhi; x += 256) {
            uint32_t v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = x + 32 * q <= xhi ? __ldg(row + x + 32 * q) : 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t R = v[q] & R_MASK;
                m = max(m, R);
                if ((v[q] & MAX_FLAG) && R > 0 && (!QUALITY || (int64_t)a.qden * R > thr)) {
                    const int pos = atomicAdd(count, 1);
                    if (pos < SCAP) keys[pos] = make_key(R, (uint32_t)(y * a.w + x + 32 * q));
                }
            }
        }
    }
    return m;
}

// Corners of one box, whole CTA.  Shared memory: keys[SCAP] | chunk[T] |
// acc[acc_cap] | cells[GCAP] in the dynamic area.
__device__ void select_box(const SelectArgs &a, int box, int acc_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *keys = (uint64_t *)smem;
    uint64_t *chunk = keys + SCAP;
    int2 *acc = (int2 *)(chunk + chunk_keys(acc_cap));
    int16_t *cells = (int16_t *)(acc + acc_cap);
    __shared__ unsigned hist[256];
    __shared__ int s_count, s_nacc, s_sel, s_k;
    __shared__ uint32_t s_rmax;
    const int tid = threadIdx.x;
    __syncthreads();

    int xlo, xhi, ylo, yhi;
    if (!box_pixel_range(a.boxes[box], a.w, a.h, xlo, xhi, ylo, yhi) || a.maxc == 0) {
        if (tid == 0) a.pad_counts[box] = 0;
        return;
    }
    const int nx = xhi - xlo + 1;
    const int E = nx * (yhi - ylo + 1);
    AccGrid g;
    g.xlo = xlo;
    g.ylo = ylo;
    g.gx = (nx + a.cell - 1) / a.cell;
    g.gy = (yhi - ylo + a.cell) / a.cell;
    g.nx = nx;
    g.rows = yhi - ylo + 1;
    g.wpr = (nx + 31) >> 5;
    // the bitmap shares the grid's shared memory (GCAP int16 = GCAP / 2 words)
    g.bits = (a.md2c > 0 && a.dmax <= 7 && (int64_t)g.wpr * g.rows <= GCAP / 2)
                 ? (uint32_t *)cells : nullptr;
    g.cells = (!g.bits && a.md2c > 0 && (int64_t)g.gx * g.gy <= GCAP) ? cells : nullptr;
    if (g.bits)
        for (int i = tid; i < g.wpr * g.rows; i += SNT) g.bits[i] = 0u;
    else if (g.cells)
        for (int i = tid; i < g.gx * g.gy; i += SNT) g.cells[i] = -1;

    // One pass over the eligible pixels (a warp per row): R_max, and the keys
    // of every local maximum with R > 0 while they fit.
    const int lane = tid & 31;
    if (tid == 0) {
        s_rmax = 0;
        s_count = 0;
        s_nacc = 0;
    }
    __syncthreads();
    // The box's candidates: from its list when it holds them all (with R_max
    // from the list kernel), else from one pass over its map.
    const uint32_t listed = a.cstate ? a.cstate[2 * box] : 0xFFFFFFFFu;
    if (listed <= (uint32_t)CAND_CAP) {
        const uint64_t *src = a.cand + (int64_t)box * CAND_CAP;
        for (int i = tid; i < (int)listed; i += SNT) keys[i] = src[i];
        if (tid == 0) {
            s_rmax = a.cstate[2 * box + 1];
            s_count = (int)listed;
        }
    } else {
        uint32_t m = gather_keys<false>(a, xlo, xhi, ylo, yhi, 0, keys, &s_count);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL_MASK, m, o));
        if (lane == 0) atomicMax(&s_rmax, m);
    }
    __syncthreads();
    const int64_t thr = (int64_t)a.qnum * (int64_t)s_rmax;
    int total = s_count;
    if (total > SCAP) {
        // Overflow: gather again, keeping only the keys that pass the
        // quality test (R > thr / qden); they usually fit.
        __syncthreads();
        if (tid == 0) s_count = 0;
        __syncthreads();
        gather_keys<true>(a, xlo, xhi, ylo, yhi, thr, keys, &s_count);
        __syncthreads();
        total = s_count;
    }

    if (total <= SCAP) {
        // Candidates pass the quality test iff R > thr / qden, i.e. they are
        // the keys >= vmin.  Take them in descending chunks of T keys: radix
        // select the chunk's smallest key, gather, sort, greedy.
        const int64_t rth = thr / a.qden;  // largest R that fails
        const uint64_t vmin = rth >= (int64_t)R_MASK ? ~0ull : (uint64_t)(rth + 1) << 32;
        const int T = chunk_keys(a.maxc);
        uint64_t hi = ~0ull;
        for (int round = 0; round <= total / T + 1; ++round) {
            if (tid == 0) s_k = 0;
            __syncthreads();
            int cnt = 0;
            for (int i = tid; i < total; i += SNT) cnt += keys[i] >= vmin && keys[i] < hi;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
            if (lane == 0 && cnt) atomicAdd(&s_k, cnt);
            __syncthreads();
            const int rem = s_k;
            if (rem == 0) break;
            const uint64_t lo = rem <= T ? vmin : kth_largest(keys, total, vmin, hi, T, hist, &s_sel, &s_k);
            if (tid == 0) s_count = 0;
            __syncthreads();
            for (int i = tid; i < total; i += SNT) {
                const uint64_t key = keys[i];
                if (key >= lo && key < hi) chunk[atomicAdd(&s_count, 1)] = key;
            }
            __syncthreads();
            const int n = s_count;  // = min(rem, T)
            int N = 32;
            while (N < n) N <<= 1;
            for (int i = n + tid; i < N; i += SNT) chunk[i] = 0ull;
            __syncthreads();
            bitonic_sort(chunk, N);
            greedy(a, box, chunk, N, n, acc, &s_nacc, g);
            __syncthreads();
            if (s_nacc >= a.maxc || rem <= T) break;
            hi = lo;
        }
    } else {
        // Descending chunks of SCAP keys: lo = the SCAP-th largest key below hi.
        // Each round consumes exactly SCAP keys below hi, so total / SCAP + 1
        // rounds exhaust the box; the bound only makes that explicit.
        uint64_t hi = ~0ull;
        const int max_rounds = total / SCAP + 2;
        for (int round = 0; round < max_rounds; ++round) {
            uint64_t prefix = 0, pmask = 0;
            int k = SCAP;
            bool take_all = false;
            for (int shift = 56; shift >= 0; shift -= 8) {
                for (int i = tid; i < 256; i += SNT) hist[i] = 0;
                __syncthreads();
                for (int i = tid; i < E; i += SNT) {
                    const int y = ylo + i / nx, x = xlo + i % nx;
                    const uint32_t v = __ldg(a.rmap + (int64_t)y * a.w + x);
                    const uint32_t R = v & R_MASK;
                    if ((v & MAX_FLAG) && R > 0 && (int64_t)a.qden * R > thr) {
                        const uint64_t key = make_key(R, (uint32_t)(y * a.w + x));
                        if (key < hi && (key & pmask) == prefix)
                            atomicAdd(&hist[(key >> shift) & 255u], 1u);
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    unsigned cum = 0, tot = 0;
                    for (int b = 0; b < 256; ++b) tot += hist[b];
                    if (shift == 56 && tot <= (unsigned)k) {
                        s_sel = -1;
                    } else {
                        int sel = 0;
                        for (int b = 255; b >= 0; --b) {
                            if (cum + hist[b] >= (unsigned)k) {
                                sel = b;
                                break;
                            }
                            cum += hist[b];
                        }
                        s_sel = sel;
                        s_k = k - (int)cum;
                    }
                }
                __syncthreads();
                if (s_sel < 0) {
                    take_all = true;
                    break;
                }
                prefix |= (uint64_t)s_sel << shift;
                pmask |= 0xFFull << shift;
                k = s_k;
                __syncthreads();
            }
            const uint64_t lo = take_all ? 0ull : prefix;
            if (tid == 0) s_count = 0;
            __syncthreads();
            for (int i = tid; i < E; i += SNT) {
                const int y = ylo + i / nx, x = xlo + i % nx;
                const uint32_t v = __ldg(a.rmap + (int64_t)y * a.w + x);
                const uint32_t R = v & R_MASK;
                if ((v & MAX_FLAG) && R > 0 && (int64_t)a.qden * R > thr) {
                    const uint64_t key = make_key(R, (uint32_t)(y * a.w + x));
                    if (key >= lo && key < hi) {
                        const int pos = atomicAdd(&s_count, 1);
                        if (pos < SCAP) keys[pos] = key;
                    }
                }
            }
            __syncthreads();
            const int n = min(s_count, SCAP);
            int N = 32;
            while (N < n) N <<= 1;
            for (int i = n + tid; i < N; i += SNT) keys[i] = 0ull;
            __syncthreads();
            bitonic_sort(keys, N);
            greedy(a, box, keys, N, n, acc, &s_nacc, g);
            __syncthreads();
            if (take_all || s_nacc >= a.maxc || lo == 0ull || lo >= hi) break;
            hi = lo;
            __syncthreads();
        }
    }
    if (tid == 0) a.pad_counts[box] = s_nacc;
}

__global__ void __launch_bounds__(SNT) select_kernel(SelectArgs a) {
    select_box(a, blockIdx.x, a.maxc);
}

__global__ void __launch_bounds__(SNT, 8) select_batch_kernel(const uint8_t *table, int acc_cap) {
    const BatchView t(table);
    const BatchHeader &h = t.hdr();
    const int32_t *pre = t.box_prefix();
    const int total = pre[t.nstreams()];
    for (int gb = blockIdx.x; gb < total; gb += gridDim.x) {
        const int si = find_segment(pre, t.nstreams(), gb);
        const StreamEntry &e = t.stream(si);
        SelectArgs a;
        a.rmap = e.rmap;
        a.w = e.w;
        a.h = e.h;
        a.boxes = e.boxes;
        a.maxc = e.maxc;
        a.qnum = h.qnum;
        a.qden = h.qden;
        a.md2c = h.md2c;
        a.dmax = h.dmax;
        a.cell = h.cell;
        a.pad_pts = e.pad_pts;
        a.pad_counts = e.pad_counts;
        a.cand = e.cand;
        a.cstate = e.cstate;
        select_box(a, gb - pre[si], acc_cap);
    }
}

// ----------------------------------------------------------- compact kernel
constexpr int CNT = 1024;

__device__ __forceinline__ void compact_stream(const int32_t *pad_counts, const float2 *pad_pts,
                                               int nboxes, int maxc, float2 *pts,
                                               int32_t *offsets) {
    __shared__ int warp_tot[CNT / 32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nboxes; base += CNT) {
        const int b = base + tid;
        const int c = b < nboxes ? pad_counts[b] : 0;
        int v = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL_MASK, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) warp_tot[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(FULL_MASK, t, o);
                if (lane >= o) t += u;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int carry = s_carry;
        const int excl = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + v - c;
        if (b < nboxes) offsets[b] = excl;
        __syncthreads();
        if (tid == CNT - 1) s_carry = carry + warp_tot[CNT / 32 - 1];
        __syncthreads();
    }
    if (tid == 0) offsets[nboxes] = s_carry;
    __syncthreads();
    for (int b = wid; b < nboxes; b += CNT / 32) {
        const int c = pad_counts[b], o = offsets[b];
        for (int i = lane; i < c; i += 32) pts[o + i] = pad_pts[(int64_t)b * maxc + i];
    }
}

__global__ void __launch_bounds__(CNT) compact_kernel(const int32_t *pad_counts,
                                                      const float2 *pad_pts, int nboxes,
                                                      int maxc, float2 *pts, int32_t *offsets) {
    compact_stream(pad_counts, pad_pts, nboxes, maxc, pts, offsets);
}

__global__ void __launch_bounds__(CNT) compact_batch_kernel(const uint8_t *table) {
    const BatchView t(table);
    const int si = blockIdx.x;
    if (si >= t.nstreams()) return;
    const StreamEntry &e = t.stream(si);
    compact_stream(e.pad_counts, e.pad_pts, e.nboxes, e.maxc, e.pts, e.offsets);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

size_t select_scratch_bytes(int w, int h, int nboxes, int max_corners, bool lists) {
    const size_t map = align256((size_t)w * h * 4) + align256((size_t)nboxes * max_corners * 8) +
                       align256((size_t)nboxes * 4 + 4);
    if (!lists) return map;
    return map + align256((size_t)nboxes * CAND_CAP * 8) + align256((size_t)nboxes * 8 + 4);
}

void select_scratch_split(void *scratch, int w, int h, int nboxes, int max_corners, bool lists,
                          SelectScratch &out) {
    uint8_t *sp = (uint8_t *)scratch;
    out.rmap = (uint32_t *)sp;
    sp += align256((size_t)w * h * 4);
    out.pad_pts = (float2 *)sp;
    sp += align256((size_t)nboxes * max_corners * 8);
    out.pad_counts = (int32_t *)sp;
    sp += align256((size_t)nboxes * 4 + 4);
    out.cand = lists ? (uint64_t *)sp : nullptr;
    sp += align256((size_t)nboxes * CAND_CAP * 8);
    out.cstate = lists ? (uint32_t *)sp : nullptr;
}

cudaError_t launch_corner_response(const omt_pyramid &pyr, uint32_t *out, const float4 *boxes,
                                   int nboxes, cudaStream_t s) {
    RespArgs a;
    a.img = (const uint8_t *)pyr.base + pyr.lv[0].img_off;
    a.pitch = pyr.lv[0].img_pitch;
    a.w = pyr.w;
    a.h = pyr.h;
    a.out = out;
    a.boxes = boxes;
    a.nboxes = nboxes;
    a.cand = nullptr;
    a.cstate = nullptr;
    a.any_overflow = nullptr;
    const int total = response_tiles(pyr.w, pyr.h);
    response_kernel<<<(total + RWARPS - 1) / RWARPS, RNT, 0, s>>>(a, total);
    return cudaGetLastError();
}

cudaError_t launch_select_corners(const omt_pyramid &pyr, const float4 *boxes, int nboxes,
                                  const omt_params &prm, void *scratch, float2 *pts,
                                  int32_t *offsets, bool lists, cudaStream_t s) {
    SelectScratch sc;
    select_scratch_split(scratch, pyr.w, pyr.h, nboxes, prm.max_corners, lists, sc);
    uint32_t *rmap = sc.rmap;
    float2 *pad_pts = sc.pad_pts;
    int32_t *pad_counts = sc.pad_counts;

    cudaError_t e;
    if (nboxes > 0 && !lists) {
        // the map of every strip that touches a box
        e = launch_corner_response(pyr, rmap, boxes, nboxes, s);
        if (e != cudaSuccess) return e;
    } else if (nboxes > 0) {
        // candidate lists, then the map where a list overflowed
        e = cudaMemsetAsync(sc.cstate, 0, ((size_t)nboxes * 2 + 1) * 4, s);
        if (e != cudaSuccess) return e;
        RespArgs r;
        r.img = (const uint8_t *)pyr.base + pyr.lv[0].img_off;
        r.pitch = pyr.lv[0].img_pitch;
        r.w = pyr.w;
        r.h = pyr.h;
        r.out = rmap;
        r.boxes = boxes;
        r.nboxes = nboxes;
        r.cand = sc.cand;
        r.cstate = sc.cstate;
        r.any_overflow = nullptr;
        const int tiles = response_tiles(pyr.w, pyr.h);
        list_kernel<<<(tiles + LWARPS - 1) / LWARPS, LNT, 0, s>>>(r, tiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        overflow_kernel<<<(tiles + RWARPS - 1) / RWARPS, RNT, 0, s>>>(r, tiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nboxes > 0) {
        SelectArgs a;
        a.rmap = rmap;
        a.w = pyr.w;
        a.h = pyr.h;
        a.boxes = boxes;
        a.maxc = prm.max_corners;
        a.qnum = prm.quality_num;
        a.qden = prm.quality_den;
        const float md2 = prm.min_dist * prm.min_dist;
        a.md2c = (int64_t)ceil((double)md2);
        a.dmax = 0;
        while ((int64_t)(a.dmax + 1) * (a.dmax + 1) < a.md2c) ++a.dmax;
        a.cell = 1;
        while (2 * (int64_t)(a.cell + 1) * (a.cell + 1) <= a.md2c) ++a.cell;
        a.pad_pts = pad_pts;
        a.pad_counts = pad_counts;
        a.cand = sc.cand;
        a.cstate = sc.cstate;
        const size_t smem = select_smem_bytes(prm.max_corners);
        e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        select_kernel<<<nboxes, SNT, smem, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    compact_kernel<<<1, CNT, 0, s>>>(pad_counts, pad_pts, nboxes, prm.max_corners, pts, offsets);
    return cudaGetLastError();
}

int response_tiles(int w, int h) { return ((w + RW - 1) / RW) * ((h + RH - 1) / RH); }

cudaError_t launch_corners_batch(const uint8_t *table, int max_streams, int max_resp_tiles,
                                 int max_boxes, int max_corners, int list_ctas_per_sm,
                                 int select_ctas_per_sm, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    reset_lists_batch_kernel<<<max_streams > 0 ? max_streams : 1, 256, 0, s>>>(table);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int grid = (max_resp_tiles + LWARPS - 1) / LWARPS;
    const int list_cap = sms * (list_ctas_per_sm > 0 ? list_ctas_per_sm : 16);
    grid = grid < list_cap ? grid : list_cap;
    list_batch_kernel<<<grid > 0 ? grid : 1, LNT, 0, s>>>(table);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    grid = (max_resp_tiles + RWARPS - 1) / RWARPS;
    grid = grid < sms * 8 ? grid : sms * 8;
    overflow_batch_kernel<<<grid > 0 ? grid : 1, RNT, 0, s>>>(table);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (max_boxes > 0) {
        const size_t smem = select_smem_bytes(max_corners);
        e = cudaFuncSetAttribute(select_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_batch_kernel, SNT, smem);
        if (per_sm < 1) per_sm = 1;
        if (select_ctas_per_sm > 0 && select_ctas_per_sm < per_sm) per_sm = select_ctas_per_sm;
        grid = max_boxes < sms * per_sm ? max_boxes : sms * per_sm;
        select_batch_kernel<<<grid, SNT, smem, s>>>(table, max_corners);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    compact_batch_kernel<<<max_streams > 0 ? max_streams : 1, CNT, 0, s>>>(table);
    return cudaGetLastError();
}

}  // namespace omt
