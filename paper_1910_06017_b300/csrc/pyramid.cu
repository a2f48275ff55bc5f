// pyramid.cu -- K1: Gaussian pyramid and Scharr gradients (Section V-A,
// preprocessing).
//
// One launch per level L (in the batched form, levels >= 1 launched as
// programmatic dependents of the level above); each CTA streams 128x32
// tiles of level L (of every stream, in the batched form) through a ring of
// staged tiles in shared
// memory (tile_ring): a producer warp copies a tile and its halo (2 rows,
// and on the left the texels up to a 16-byte boundary) by one 2D tensor
// copy per tile, four consumer warps compute it.  Each consumer thread owns
// 4 adjacent columns and 8 consecutive rows of the tile: it reads the 11
// staged rows it needs, forms the horizontal Scharr difference and
// smoothing and the horizontal binomial sums, combines them vertically, and
// stores 4 gradient pairs per row, 2 texels of level L+1 at each even row,
// and at level 0 the u8 copy.  Level 0 (u8) computes on pairs of pixels in
// the halves of 32-bit registers (SWAR).
//
// Exactness: the Scharr weights 3/32 and 10/32 and the integer binomial
// weights with a final 1/256 keep every value that is dyadic-exact in FP32
// (pyramid levels 0-2, gradients of levels 0-1) bit-identical to the
// definition.  From level 2 on, a level's values need more bits than FP32
// sums keep, so those launches form the sums exactly in 64-bit fixed point
// (a level-L value, stored or not, is a multiple of 2^-8L: each reduction
// divides by 2^8 and rounding only coarsens) and round once: the stored
// value is the correctly rounded result of the definition applied to the
// level above as stored, in both storages (half outputs go through a
// round-to-odd FP32 value, which makes the second rounding exact).
#include <cstring>

#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int TX = 128;        // tile width
constexpr int TY = 32;         // tile height (even: level L+1 rows align)
constexpr int RPT = 4;         // rows per thread
constexpr int SROWS = TY + 4;  // staged rows: the tile and 2 halo rows each side
constexpr int NT = 256;        // threads per CTA: 32 column groups x 8 row groups
static_assert(TY == RPT * (NT / 32), "tile rows");

enum Fmt { FMT_U8 = 0, FMT_H16 = 1, FMT_F32 = 2 };  // storage of level L's texels
enum Path { PATH_FLOAT = 0, PATH_SPLIT = 1, PATH_INT64 = 2 };  // how a level's sums stay exact

template <int FMT>
struct Stage {
    static constexpr int ESZ = FMT == FMT_U8 ? 1 : (FMT == FMT_H16 ? 2 : 4);
    // staged columns start at the 16-byte boundary at or below column ox-4
    static constexpr int LEAD = FMT == FMT_U8 ? 16 : (FMT == FMT_H16 ? 8 : 4);  // texels before ox
    static constexpr int RB = ((LEAD + TX + 4) * ESZ + 15) / 16 * 16;            // bytes per staged row
};

struct LevelArgs {
    const uint8_t *src;   // level L: u8 frame (L = 0) or the pyramid's level plane
    int64_t src_pitch;
    int w, h;             // level L size
    bool vec_ok;          // src base and pitch are 16-byte aligned
    uint8_t *copy;        // level-0 u8 copy (L = 0 only)
    int64_t copy_pitch;
    uint8_t *grad;        // level-L gradient plane
    int64_t grad_pitch;
    uint8_t *next;        // level L+1 image plane or nullptr
    int64_t next_pitch;
    int nw, nh;           // level L+1 size
    int frac;             // 0: FP32 sums (exact for levels 0, 1); else the fixed-point
                          // fraction bits of level L's values (8 L, at most 40)
};

// Fixed-point fraction bits for the sums over level L (see the header).
__host__ __device__ __forceinline__ int level_frac(int L) { return L < 2 ? 0 : (L > 5 ? 40 : 8 * L); }

template <int FMT>
__device__ __forceinline__ float texel_value(unsigned bits) {
    if (FMT == FMT_U8) return (float)bits;
    if (FMT == FMT_H16) return __half2float(__ushort_as_half((unsigned short)bits)) + 128.0f;
    return __uint_as_float(bits);
}

// Values of tile columns 4g-2 .. 4g+5 of staged row r.
template <int FMT>
__device__ __forceinline__ void staged_row(const uint8_t *st, int r, int g, float m[8]) {
    using S = Stage<FMT>;
    const uint8_t *row = st + r * S::RB;
    if (FMT == FMT_U8) {
        // texels 4g+14 .. 4g+21 of the staged row: words g+3 .. g+5
        const unsigned *w = (const unsigned *)row + g + 3;
        const unsigned w0 = w[0], w1 = w[1], w2 = w[2];
        m[0] = (float)((w0 >> 16) & 0xFFu);
        m[1] = (float)(w0 >> 24);
#pragma unroll
        for (int c = 0; c < 4; ++c) m[2 + c] = (float)((w1 >> (8 * c)) & 0xFFu);
        m[6] = (float)(w2 & 0xFFu);
        m[7] = (float)((w2 >> 8) & 0xFFu);
    } else if (FMT == FMT_H16) {
        // halves 4g+6 .. 4g+13: words 2g+3 .. 2g+6
        const unsigned *w = (const unsigned *)row + 2 * g + 3;
        const unsigned w0 = w[0];
        const uint2 w12 = *(const uint2 *)(w + 1);
        const unsigned w3 = w[3];
        const unsigned u[4] = {w0, w12.x, w12.y, w3};
#pragma unroll
        for (int c = 0; c < 8; ++c) m[c] = texel_value<FMT>((u[c >> 1] >> (16 * (c & 1))) & 0xFFFFu);
    } else {
        // floats 4g+2 .. 4g+9
        const float *f = (const float *)row + 4 * g + 2;
        const float2 p0 = *(const float2 *)f;
        const float4 p1 = *(const float4 *)(f + 2);
        const float2 p2 = *(const float2 *)(f + 6);
        m[0] = p0.x;
        m[1] = p0.y;
        m[2] = p1.x;
        m[3] = p1.y;
        m[4] = p1.z;
        m[5] = p1.w;
        m[6] = p2.x;
        m[7] = p2.y;
    }
}

template <int ST>
__device__ __forceinline__ void store_grads(const LevelArgs &a, int y, int x, const float gx[4],
                                            const float gy[4]) {
    uint8_t *row = a.grad + (int64_t)y * a.grad_pitch;
    const bool full = x + 3 < a.w;
    if (ST == OMT_F32) {
        if (full) {
            float4 *p = (float4 *)(row + 8 * (int64_t)x);
            p[0] = make_float4(gx[0], gy[0], gx[1], gy[1]);
            p[1] = make_float4(gx[2], gy[2], gx[3], gy[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (x + c < a.w) ((float2 *)row)[x + c] = make_float2(gx[c], gy[c]);
        }
    } else {
        unsigned g[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const __half2 t = __floats2half2_rn(gx[c], gy[c]);
            g[c] = *(const unsigned *)&t;
        }
        if (full) {
            *(uint4 *)(row + 4 * (int64_t)x) = make_uint4(g[0], g[1], g[2], g[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (x + c < a.w) ((unsigned *)row)[x + c] = g[c];
        }
    }
}

template <int ST>
__device__ __forceinline__ void store_next(const LevelArgs &a, int Y, int X0, float v0, float v1) {
    if (Y >= a.nh || X0 >= a.nw) return;
    uint8_t *row = a.next + (int64_t)Y * a.next_pitch;
    if (ST == OMT_F32) {
        if (X0 + 1 < a.nw) ((float2 *)row)[X0 >> 1] = make_float2(v0, v1);
        else ((float *)row)[X0] = v0;
    } else {
        if (X0 + 1 < a.nw) ((__half2 *)row)[X0 >> 1] = __floats2half2_rn(v0 - 128.0f, v1 - 128.0f);
        else ((__half *)row)[X0] = __float2half_rn(v0 - 128.0f);
    }
}

// store_next for values already in the stored domain (half storage: I - 128).
template <int ST>
__device__ __forceinline__ void store_next_stored(const LevelArgs &a, int Y, int X0, float v0,
                                                  float v1) {
    if (Y >= a.nh || X0 >= a.nw) return;
    uint8_t *row = a.next + (int64_t)Y * a.next_pitch;
    if (ST == OMT_F32) {
        if (X0 + 1 < a.nw) ((float2 *)row)[X0 >> 1] = make_float2(v0, v1);
        else ((float *)row)[X0] = v0;
    } else {
        if (X0 + 1 < a.nw) ((__half2 *)row)[X0 >> 1] = __floats2half2_rn(v0, v1);
        else ((__half *)row)[X0] = __float2half_rn(v0);
    }
}

// ------------------------------------------------------- level 0 in SWAR
// Level 0 is integer: every sum the level needs fits 16 bits (the raw
// Scharr gradients in [-4080, 4080], the 5-tap binomial of a row at most
// 4080 and of five rows at most 65280), so it runs on pairs of pixels held
// as the two 16-bit halves of a 32-bit register -- pixels (c, c+2): the
// even pair (4g, 4g+2) and the odd pair (4g+1, 4g+3) of a thread's four
// columns -- with 32-bit integer instructions.  Differences carry a bias
// (256, then 4096 after the vertical pass) so that no half goes negative
// and no carry crosses between halves.  The results convert to float
// exactly (2^23 + v from the bits, then one fused multiply-add), so the
// stored values are those of compute_tile bit for bit.
constexpr unsigned SW_BIAS1 = 0x01000100u;   // 256 in each half
constexpr unsigned SW_BIAS2 = 0x10001000u;   // 4096 in each half
constexpr unsigned SW_MAGIC = 0x4B000000u;   // the bits of 2^23

struct SwRow {
    unsigned de, dof;   // biased horizontal differences, even / odd pair
    unsigned se, so;    // horizontal Scharr smoothing 3, 10, 3
    unsigned be;        // horizontal binomial 1, 4, 6, 4, 1 (even pair)
};

// The horizontal sums for columns x .. x+3 of one row, from the words of
// its columns x-4 .. x-1, x .. x+3 and x+4 .. x+7.
__device__ __forceinline__ SwRow sw_row(unsigned w0, unsigned w1, unsigned w2) {
    const unsigned E0 = w0 & 0x00FF00FFu, E1 = w1 & 0x00FF00FFu, E2 = w2 & 0x00FF00FFu;
    const unsigned O0 = __byte_perm(w0, 0u, 0x4341), O1 = __byte_perm(w1, 0u, 0x4341);
    // (x[c + k], x[c + 2 + k]) for the even pair c = 4g at k = -2 .. 2 are
    // A, B, E1, O1, C; for the odd pair c = 4g + 1 (k = -1 .. 1) B... E1,
    // O1, C
    const unsigned A = __byte_perm(E0, E1, 0x5432), B = __byte_perm(O0, O1, 0x5432);
    const unsigned C = __byte_perm(E1, E2, 0x5432);
    SwRow o;
    o.de = O1 + SW_BIAS1 - B;
    o.dof = C + SW_BIAS1 - E1;
    const unsigned te = B + O1, to = E1 + C;
    o.se = 3u * te + 10u * E1;
    o.so = 3u * to + 10u * O1;
    o.be = A + C + 4u * te + 6u * E1;
    return o;
}

// The lane of v (0: low half, 1: high half) as the float 2^23 + v.
__device__ __forceinline__ float sw_float(unsigned v, int half) {
    return __uint_as_float(__byte_perm(v, SW_MAGIC, half ? 0x7632 : 0x7610));
}

// This thread's share of a staged 128x32 level-0 tile, in SWAR (staged
// row bytes 4g-4 .. 4g+7 of the tile are words g+3 .. g+5 of the row).
template <int ST, int RPT = omt::RPT>
__device__ __forceinline__ void compute_tile_u8(const LevelArgs &a, int ox, int oy, const uint8_t *st,
                                                int q = threadIdx.x >> 5) {
    const int g = threadIdx.x & 31;   // columns 4g .. 4g+3 of the tile
    // q: rows RPT q .. RPT q + RPT-1 of the tile
    const int x = ox + 4 * g;
    if (x >= a.w) return;
    const int y0 = oy + RPT * q;
    SwRow h[RPT + 3];
    const float2 g_scale = make_float2(1.0f / 32.0f, 1.0f / 32.0f);
    const float2 g_off = make_float2(-(8388608.0f + 4096.0f) / 32.0f, -(8388608.0f + 4096.0f) / 32.0f);
#pragma unroll
    for (int k = 0; k < RPT + 3; ++k) {
        const unsigned *w = (const unsigned *)(st + (RPT * q + k) * Stage<FMT_U8>::RB) + g + 3;
        const unsigned w0 = w[0], w1 = w[1], w2 = w[2];
        h[k] = sw_row(w0, w1, w2);
        // the u8 copy of rows y0 .. y0+RPT-1
        if (a.copy && k >= 2 && k < RPT + 2 && y0 + k - 2 < a.h) {
            uint8_t *dst = a.copy + (int64_t)(y0 + k - 2) * a.copy_pitch + x;
            if (x + 3 < a.w) {
                *(unsigned *)dst = w1;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (x + c < a.w) dst[c] = (uint8_t)(w1 >> (8 * c));
            }
        }
        // gradients of row y0 + k - 3 (rows k-2 .. k are in): 4096 + raw
        if (k >= 3 && y0 + k - 3 < a.h) {
            const unsigned gxe = 3u * (h[k - 2].de + h[k].de) + 10u * h[k - 1].de;
            const unsigned gxo = 3u * (h[k - 2].dof + h[k].dof) + 10u * h[k - 1].dof;
            const unsigned gye = h[k].se + SW_BIAS2 - h[k - 2].se;
            const unsigned gyo = h[k].so + SW_BIAS2 - h[k - 2].so;
            // pixels 4g, 4g+1, 4g+2, 4g+3: (even lo, odd lo, even hi, odd hi)
            float gx[4], gy[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const unsigned vx = (c & 1) ? gxo : gxe, vy = (c & 1) ? gyo : gye;
                const float2 p = __ffma2_rn(make_float2(sw_float(vx, c >> 1), sw_float(vy, c >> 1)),
                                            g_scale, g_off);
                gx[c] = p.x;
                gy[c] = p.y;
            }
            store_grads<ST>(a, y0 + k - 3, x, gx, gy);
        }
        // level 1 row (y0 + k - 4) / 2 at even rows (rows k-4 .. k are in):
        // columns 2g, 2g+1 from the even pair
        if (a.next && k >= 4 && ((k & 1) == 0)) {
            const unsigned L1 = (h[k - 4].be + h[k].be) + 4u * (h[k - 3].be + h[k - 1].be) + 6u * h[k - 2].be;
            const float2 v = __ffma2_rn(make_float2(sw_float(L1, 0), sw_float(L1, 1)),
                                        make_float2(1.0f / 256.0f, 1.0f / 256.0f),
                                        make_float2(-32768.0f, -32768.0f));   // exact: L1 / 256
            store_next<ST>(a, (y0 >> 1) + (k - 4) / 2, x >> 1, v.x, v.y);
        }
    }
}

// This thread's share of the staged 128x32 tile of level L at (ox, oy).
template <int ST, int FMT, int RPT = omt::RPT>
__device__ __forceinline__ void compute_tile(const LevelArgs &a, int ox, int oy, const uint8_t *st,
                                             int q = threadIdx.x >> 5) {
    const int g = threadIdx.x & 31;   // columns 4g .. 4g+3 of the tile
    // q: rows RPT q .. RPT q + RPT-1 of the tile
    const int x = ox + 4 * g;
    if (x >= a.w) return;
    const int y0 = oy + RPT * q;
    // tile row t is staged row t + 2; this thread reads tile rows y0-oy-2 ..
    // y0-oy+RPT (k = 0 .. RPT+2) and emits each output once its rows are in
    float d[RPT + 3][4], hh[RPT + 3][4], hs[RPT + 3][2];
#pragma unroll
    for (int k = 0; k < RPT + 3; ++k) {
        float m[8];
        staged_row<FMT>(st, RPT * q + k, g, m);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            d[k][c] = m[c + 3] - m[c + 1];
            hh[k][c] = fmaf(10.0f / 32.0f, m[c + 2], (3.0f / 32.0f) * (m[c + 1] + m[c + 3]));
        }
        hs[k][0] = (m[0] + m[4]) + 4.0f * (m[1] + m[3]) + 6.0f * m[2];
        hs[k][1] = (m[2] + m[6]) + 4.0f * (m[3] + m[5]) + 6.0f * m[4];
        if (FMT == FMT_U8 && a.copy && k >= 2 && k < RPT + 2 && y0 + k - 2 < a.h) {
            uint8_t *dst = a.copy + (int64_t)(y0 + k - 2) * a.copy_pitch + x;
            const uint8_t *srow = st + (RPT * q + k) * Stage<FMT>::RB;
            if (x + 3 < a.w) {
                *(unsigned *)dst = ((const unsigned *)srow)[g + 4];
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (x + c < a.w) dst[c] = srow[16 + 4 * g + c];
            }
        }
        // gradients of row y0 + k - 3 (rows k-2 .. k are in)
        if (k >= 3 && k < RPT + 3 && y0 + k - 3 < a.h) {
            float gx[4], gy[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                gx[c] = fmaf(10.0f / 32.0f, d[k - 1][c], (3.0f / 32.0f) * (d[k - 2][c] + d[k][c]));
                gy[c] = hh[k][c] - hh[k - 2][c];
            }
            store_grads<ST>(a, y0 + k - 3, x, gx, gy);
        }
        // level L+1 row (y0 + k - 4) / 2 at even rows (rows k-4 .. k are in)
        if (a.next && k >= 4 && ((k & 1) == 0)) {
            float o[2];
#pragma unroll
            for (int c = 0; c < 2; ++c)
                o[c] = ((hs[k - 4][c] + hs[k][c]) + 4.0f * (hs[k - 3][c] + hs[k - 1][c]) +
                        6.0f * hs[k - 2][c]) * (1.0f / 256.0f);
            store_next<ST>(a, (y0 >> 1) + (k - 4) / 2, x >> 1, o[0], o[1]);
        }
    }
}

// ------------------------------------------------------------ exact sums
// 2^e as a float, e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// s as a float rounded to odd (truncate, then set the last bit if inexact):
// rounding that to half precision gives the correctly rounded half of s.
__device__ __forceinline__ float ll2float_odd(long long s) {
    const float f = __ll2float_rz(s);
    return __float2ll_rz(f) == s ? f : __int_as_float(__float_as_int(f) | 1);
}

// Values of tile columns 4g-2 .. 4g+5 of staged row r as integers v 2^frac.
template <int FMT>
__device__ __forceinline__ void staged_row_fixed(const uint8_t *st, int r, int g, float scale,
                                                 long long off, long long q[8]) {
    using S = Stage<FMT>;
    const uint8_t *row = st + r * S::RB;
    if (FMT == FMT_H16) {
        const unsigned *w = (const unsigned *)row + 2 * g + 3;
        const unsigned u[4] = {w[0], w[1], w[2], w[3]};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float h = __half2float(__ushort_as_half((unsigned short)((u[c >> 1] >> (16 * (c & 1))) & 0xFFFFu)));
            q[c] = __float2ll_rn(h * scale) + off;   // half(I - 128) 2^frac + 128 2^frac
        }
    } else {
        const float *f = (const float *)row + 4 * g + 2;
#pragma unroll
        for (int c = 0; c < 8; ++c) q[c] = __float2ll_rn(f[c] * scale);
    }
}

// The stored value of the integer s times 2^-e (correctly rounded).
template <int ST>
__device__ __forceinline__ float fixed_out(long long s, int e) {
    if (ST == OMT_F32) return __ll2float_rn(s) * pow2f(-e);
    return ll2float_odd(s) * pow2f(-e);   // the half store rounds it once more, exactly
}

template <int ST>
__device__ __forceinline__ void store_grads_fixed(const LevelArgs &a, int y, int x,
                                                  const long long gx[4], const long long gy[4]) {
    float fx[4], fy[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        fx[c] = fixed_out<ST>(gx[c], a.frac + 5);
        fy[c] = fixed_out<ST>(gy[c], a.frac + 5);
    }
    store_grads<ST>(a, y, x, fx, fy);
}

// compute_tile with the sums in 64-bit fixed point (levels >= 2).
template <int ST, int FMT, int RPT = omt::RPT>
__device__ __forceinline__ void compute_tile_fixed(const LevelArgs &a, int ox, int oy,
                                                   const uint8_t *st, int q = threadIdx.x >> 5) {
    const int g = threadIdx.x & 31;
    const int x = ox + 4 * g;
    if (x >= a.w) return;
    const int y0 = oy + RPT * q;
    const float scale = pow2f(a.frac);
    const long long off = 128ll << a.frac;
    long long d[RPT + 3][4], hh[RPT + 3][4], hs[RPT + 3][2];
#pragma unroll
    for (int k = 0; k < RPT + 3; ++k) {
        long long m[8];
        staged_row_fixed<FMT>(st, RPT * q + k, g, scale, off, m);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            d[k][c] = m[c + 3] - m[c + 1];
            hh[k][c] = 10 * m[c + 2] + 3 * (m[c + 1] + m[c + 3]);
        }
        hs[k][0] = (m[0] + m[4]) + 4 * (m[1] + m[3]) + 6 * m[2];
        hs[k][1] = (m[2] + m[6]) + 4 * (m[3] + m[5]) + 6 * m[4];
        if (k >= 3 && k < RPT + 3 && y0 + k - 3 < a.h) {
            long long gx[4], gy[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                gx[c] = 10 * d[k - 1][c] + 3 * (d[k - 2][c] + d[k][c]);
                gy[c] = hh[k][c] - hh[k - 2][c];
            }
            store_grads_fixed<ST>(a, y0 + k - 3, x, gx, gy);
        }
        if (a.next && k >= 4 && ((k & 1) == 0)) {
            float o[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                long long v = (hs[k - 4][c] + hs[k][c]) + 4 * (hs[k - 3][c] + hs[k - 1][c]) +
                              6 * hs[k - 2][c];
                // half storage keeps I - 128: subtract before the one rounding
                if (ST == OMT_F16) v -= 128ll << (a.frac + 8);
                o[c] = fixed_out<ST>(v, a.frac + 8);
            }
            store_next_stored<ST>(a, (y0 >> 1) + (k - 4) / 2, x >> 1, o[0], o[1]);
        }
    }
}

// ------------------------------------------------------ split FP32 sums
// A level-2 or level-3 value v (a multiple of 2^-16 or 2^-24 below 256) is
// split into hi = v rounded to a multiple of 2^-8 and lo = v - hi (|lo| <=
// 2^-9): every FP32 sum compute_tile forms is then exact for hi and for lo
// separately (at most 24 significant bits each), and the output is their
// sum rounded once -- to nearest for FP32 storage, to odd for half storage,
// whose store then rounds once more, exactly.
__device__ __forceinline__ void split_hi_lo(float v, float &hi, float &lo) {
    const float C = 49152.0f;   // 1.5 * 2^15: v + C has a 2^-8 ulp
    hi = (v + C) - C;
    lo = v - hi;
}

// a + b rounded to nearest (ST F32) or to odd (ST F16), a and b exact.
template <int ST>
__device__ __forceinline__ float sum_out(float a, float b) {
    const float s = __fadd_rn(a, b);
    if (ST == OMT_F32) return s;
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));  // a + b = s + e
    if (e == 0.0f || (__float_as_int(s) & 1)) return s;
    // s is even and inexact: the odd neighbour on e's side
    const int away = (e > 0.0f) == (s > 0.0f) ? 1 : -1;   // magnitude up or down
    return s == 0.0f ? e : __int_as_float(__float_as_int(s) + away);
}

// Tile columns 4g-2 .. 4g+5 of staged row r, split (values I, not I - 128).
template <int FMT>
__device__ __forceinline__ void staged_row_split(const uint8_t *st, int r, int g, float hi[8],
                                                 float lo[8]) {
    using S = Stage<FMT>;
    const uint8_t *row = st + r * S::RB;
    if (FMT == FMT_H16) {
        const unsigned *w = (const unsigned *)row + 2 * g + 3;
        const unsigned u[4] = {w[0], w[1], w[2], w[3]};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float h = __half2float(__ushort_as_half((unsigned short)((u[c >> 1] >> (16 * (c & 1))) & 0xFFFFu)));
            float hh;
            split_hi_lo(h, hh, lo[c]);   // |h| <= 128: the same 2^-8 grid
            hi[c] = hh + 128.0f;
        }
    } else {
        const float *f = (const float *)row + 4 * g + 2;
#pragma unroll
        for (int c = 0; c < 8; ++c) split_hi_lo(f[c], hi[c], lo[c]);
    }
}

// compute_tile with every sum formed on the hi and lo parts (levels 2-3).
template <int ST, int FMT, int RPT = omt::RPT>
__device__ __forceinline__ void compute_tile_split(const LevelArgs &a, int ox, int oy,
                                                   const uint8_t *st, int q = threadIdx.x >> 5) {
    const int g = threadIdx.x & 31;
    const int x = ox + 4 * g;
    if (x >= a.w) return;
    const int y0 = oy + RPT * q;
    float d[2][RPT + 3][4], hh[2][RPT + 3][4], hs[2][RPT + 3][2];
#pragma unroll
    for (int k = 0; k < RPT + 3; ++k) {
        float m[2][8];
        staged_row_split<FMT>(st, RPT * q + k, g, m[0], m[1]);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                d[p][k][c] = m[p][c + 3] - m[p][c + 1];
                hh[p][k][c] = fmaf(10.0f / 32.0f, m[p][c + 2], (3.0f / 32.0f) * (m[p][c + 1] + m[p][c + 3]));
            }
            hs[p][k][0] = (m[p][0] + m[p][4]) + 4.0f * (m[p][1] + m[p][3]) + 6.0f * m[p][2];
            hs[p][k][1] = (m[p][2] + m[p][6]) + 4.0f * (m[p][3] + m[p][5]) + 6.0f * m[p][4];
        }
        if (k >= 3 && k < RPT + 3 && y0 + k - 3 < a.h) {
            float gx[4], gy[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float px[2], py[2];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    px[p] = fmaf(10.0f / 32.0f, d[p][k - 1][c], (3.0f / 32.0f) * (d[p][k - 2][c] + d[p][k][c]));
                    py[p] = hh[p][k][c] - hh[p][k - 2][c];
                }
                gx[c] = sum_out<ST>(px[0], px[1]);
                gy[c] = sum_out<ST>(py[0], py[1]);
            }
            store_grads<ST>(a, y0 + k - 3, x, gx, gy);
        }
        if (a.next && k >= 4 && ((k & 1) == 0)) {
            float o[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float n[2];
#pragma unroll
                for (int p = 0; p < 2; ++p)
                    n[p] = (hs[p][k - 4][c] + hs[p][k][c]) + 4.0f * (hs[p][k - 3][c] + hs[p][k - 1][c]) +
                           6.0f * hs[p][k - 2][c];
                // 256 (I - 128) for half storage: exact on the hi part
                if (ST == OMT_F16) n[0] -= 32768.0f;
                o[c] = sum_out<ST>(n[0], n[1]) * (1.0f / 256.0f);
            }
            store_next_stored<ST>(a, (y0 >> 1) + (k - 4) / 2, x >> 1, o[0], o[1]);
        }
    }
}

// Arguments of level L of the pyramid a batch entry builds (frame t+1).
__device__ __forceinline__ void level_args_from_entry(const StreamEntry &e, int L, int levels,
                                                      LevelArgs &a) {
    const LevelView &v = e.P_next[L];
    a.w = v.w;
    a.h = v.h;
    if (L == 0) {
        a.src = e.frame;
        a.src_pitch = e.frame_pitch;
        a.vec_ok = (((uintptr_t)e.frame | (uintptr_t)e.frame_pitch) & 15) == 0;
        a.copy = const_cast<uint8_t *>(v.img);
        a.copy_pitch = v.img_pitch;
    } else {
        a.src = v.img;
        a.src_pitch = v.img_pitch;
        a.vec_ok = true;
        a.copy = nullptr;
        a.copy_pitch = 0;
    }
    a.grad = const_cast<uint8_t *>(v.grad);
    a.grad_pitch = v.grad_pitch;
    a.frac = level_frac(L);
    if (L + 1 < levels) {
        const LevelView &n = e.P_next[L + 1];
        a.next = const_cast<uint8_t *>(n.img);
        a.next_pitch = n.img_pitch;
        a.nw = n.w;
        a.nh = n.h;
    } else {
        a.next = nullptr;
        a.next_pitch = 0;
        a.nw = a.nh = 0;
    }
}

// -------------------------------------------------------------- TMA ring
// Every level streams through a ring of RING_STAGES staged tiles per CTA:
// one producer warp copies each 128 x 32 tile with its halo (Stage<FMT>'s
// box: LEAD texels left, 2 rows above, RB bytes x SROWS rows) global ->
// shared by one 2D tensor copy, whose completion the stage's "full"
// mbarrier counts; four consumer warps compute the tile (8 rows each) and
// release the stage on its "empty" mbarrier.  No CTA-wide barrier in the
// steady state: the producer runs up to RING_STAGES tiles ahead.  A plane
// without a tensor map (a frame whose base or pitch is not 16-byte aligned)
// is copied by the producer warp's plain loads instead.  Outside the plane
// the copy holds zeros; tiles at the plane's edge replace the halo texels
// that outputs read by their reflect-101 images (rows, then columns) before
// computing.  Every wait gives up after one second (counted in
// pyr_wait_timeouts), and a CTA whose wait ran out stops, after landing its
// copies in flight.
constexpr int RING_STAGES = 4;
constexpr int RING_CONS = 4;                    // consumer warps
constexpr int RING_NT = 32 * (RING_CONS + 1);   // and the producer warp
constexpr int RING_RPT = TY / RING_CONS;        // rows per consumer thread
constexpr unsigned long long RING_WAIT_NS = 1000000000ull;
static_assert(L0_BOX_W == Stage<FMT_U8>::RB && L0_BOX_H == SROWS, "the level-0 box is a staged tile");

template <int FMT>
struct Ring {
    static constexpr int ESZ = Stage<FMT>::ESZ;
    static constexpr int LEAD = Stage<FMT>::LEAD;
    static constexpr int RB = Stage<FMT>::RB;            // bytes per staged row
    static constexpr int BOX_W = RB / ESZ;                // texels per staged row
    static constexpr unsigned TILE = (unsigned)RB * SROWS;
    static_assert(TILE % 128 == 0, "stages on 128-byte boundaries");
};

struct RingBars {
    uint64_t full[RING_STAGES], empty[RING_STAGES];
    int ok[2];   // consumers: tile k's stage landed, in slot k & 1 (set by thread 0)
};

template <int FMT>
__host__ __device__ constexpr size_t ring_bytes() {
    return (size_t)RING_STAGES * Ring<FMT>::TILE + sizeof(RingBars);
}

__device__ unsigned pyr_wait_timeouts;

__device__ __forceinline__ unsigned ring_smem(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool ring_try_wait(const uint64_t *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(ring_smem(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long ring_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// One thread's bounded wait for the phase of parity `parity` to complete.
__device__ __forceinline__ bool ring_wait(const uint64_t *bar, unsigned parity) {
    if (ring_try_wait(bar, parity)) return true;
    const unsigned long long t0 = ring_ns();
    while (!ring_try_wait(bar, parity))
        if (ring_ns() - t0 > RING_WAIT_NS) {
            atomicAdd(&pyr_wait_timeouts, 1u);
            return false;
        }
    return true;
}
__device__ __forceinline__ void ring_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(ring_smem(bar)) : "memory");
}
__device__ __forceinline__ void ring_consumers_sync() {
    asm volatile("bar.sync 1, %0;\n" ::"n"(32 * RING_CONS) : "memory");
}

// The producer warp fills stage `st` with the box of tile (ox, oy): by the
// tensor map, or (no map) by plain loads, zero outside the plane.
template <int FMT>
__device__ __forceinline__ void ring_fill(const LevelArgs &a, const CUtensorMap *map, int ox, int oy,
                                          uint8_t *st, uint64_t *full, int lane) {
    using RG = Ring<FMT>;
    if (map) {
        if (lane == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ring_smem(full)),
                         "r"(RG::TILE)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(ring_smem(st)),
                "l"((unsigned long long)map), "r"(ox - RG::LEAD), "r"(oy - 2), "r"(ring_smem(full))
                : "memory");
        }
        return;
    }
    for (int i = lane; i < SROWS * RG::BOX_W; i += 32) {
        const int r = i / RG::BOX_W, c = i - r * RG::BOX_W;
        const int y = oy - 2 + r, x = ox - RG::LEAD + c;
        const bool in = y >= 0 && y < a.h && x >= 0 && x < a.w;
        const uint8_t *src = a.src + (int64_t)(in ? y : 0) * a.src_pitch + (int64_t)(in ? x : 0) * RG::ESZ;
        uint8_t *dst = st + r * RG::RB + c * RG::ESZ;
        if (RG::ESZ == 1) *dst = in ? *src : 0;
        else if (RG::ESZ == 2) *(unsigned short *)dst = in ? *(const unsigned short *)src : 0;
        else *(unsigned *)dst = in ? *(const unsigned *)src : 0u;
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) ring_arrive(full);
}

// Halo texels of an edge tile that outputs read (rows -2, -1, h, h+1 and
// columns -2, -1, w, w+1) take their reflect-101 images from inside the
// box: rows first, then columns (so corners reflect both ways).  The four
// consumer warps share the work; sources outside the box are never read
// texels, and are skipped.
template <int FMT>
__device__ __forceinline__ void ring_fix_edges(const LevelArgs &a, int ox, int oy, uint8_t *st, int t) {
    using RG = Ring<FMT>;
    const int y0 = oy - 2, x0 = ox - RG::LEAD;
    for (int i = t; i < 4 * (RG::RB / 4); i += 32 * RING_CONS) {
        const int k = i / (RG::RB / 4), c = i - k * (RG::RB / 4);
        const int y = k < 2 ? k - 2 : a.h + (k - 2);   // -2, -1, h, h+1
        const int r = y - y0, rr = reflect101(y, a.h) - y0;
        if (r < 0 || r >= SROWS || rr < 0 || rr >= SROWS) continue;
        ((unsigned *)(st + r * RG::RB))[c] = ((const unsigned *)(st + rr * RG::RB))[c];
    }
    ring_consumers_sync();
    for (int i = t; i < 4 * SROWS; i += 32 * RING_CONS) {
        const int k = i / SROWS, r = i - k * SROWS;
        const int x = k < 2 ? k - 2 : a.w + (k - 2);   // -2, -1, w, w+1
        const int c = x - x0, cc = reflect101(x, a.w) - x0;
        if (c < 0 || c >= RG::BOX_W || cc < 0 || cc >= RG::BOX_W) continue;
        uint8_t *row = st + r * RG::RB;
        if (RG::ESZ == 1) row[c] = row[cc];
        else if (RG::ESZ == 2) ((unsigned short *)row)[c] = ((const unsigned short *)row)[cc];
        else ((unsigned *)row)[c] = ((const unsigned *)row)[cc];
    }
    ring_consumers_sync();
}

// The ring over the CTA's tiles g = blockIdx.x, += gridDim.x, < total;
// resolve(g, args, ox, oy, map) names a tile (map: its plane's tensor map
// or null) and is called by every thread for every tile.
template <int ST, int FMT, int PATH, typename Resolve>
__device__ __forceinline__ void tile_ring(uint8_t *smem, int total, Resolve resolve) {
    using RG = Ring<FMT>;
    RingBars &R = *(RingBars *)(smem + (size_t)RING_STAGES * RG::TILE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < RING_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ring_smem(&R.full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(ring_smem(&R.empty[s])),
                         "r"(RING_CONS)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (warp == RING_CONS) {
        // producer
        int k = 0;
        for (int g = blockIdx.x; g < total; g += gridDim.x, ++k) {
            const int s = k % RING_STAGES;
            if (k >= RING_STAGES) {
                bool ok = true;
                if (lane == 0) ok = ring_wait(&R.empty[s], ((k / RING_STAGES) - 1) & 1);
                if (!__shfl_sync(FULL_MASK, ok, 0)) break;
            }
            LevelArgs a;
            int ox, oy;
            const CUtensorMap *map;
            resolve(g, a, ox, oy, map);
            ring_fill<FMT>(a, map, ox, oy, smem + (size_t)s * RG::TILE, &R.full[s], lane);
        }
        // land the copies still in flight (bounded) before the CTA exits
        if (lane == 0)
            for (int j = k - RING_STAGES > 0 ? k - RING_STAGES : 0; j < k; ++j)
                ring_wait(&R.full[j % RING_STAGES], (j / RING_STAGES) & 1);
        return;
    }
    // consumers: thread 0 waits for each stage, the four warps follow
    int k = 0;
    for (int g = blockIdx.x; g < total; g += gridDim.x, ++k) {
        const int s = k % RING_STAGES;
        // two slots: thread 0 writes tile k+1's only after every consumer
        // has passed tile k's barrier, i.e. read tile k's
        if (threadIdx.x == 0) R.ok[k & 1] = ring_wait(&R.full[s], (k / RING_STAGES) & 1);
        ring_consumers_sync();
        if (!R.ok[k & 1]) break;
        LevelArgs a;
        int ox, oy;
        const CUtensorMap *map;
        resolve(g, a, ox, oy, map);
        uint8_t *st = smem + (size_t)s * RG::TILE;
        if (ox == 0 || oy == 0 || ox + TX + 2 > a.w || oy + TY + 2 > a.h) {
            ring_fix_edges<FMT>(a, ox, oy, st, threadIdx.x);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // before the next copy
        }
        if constexpr (FMT == FMT_U8) compute_tile_u8<ST, RING_RPT>(a, ox, oy, st, warp);
        else if constexpr (PATH == PATH_INT64) compute_tile_fixed<ST, FMT, RING_RPT>(a, ox, oy, st, warp);
        else if constexpr (PATH == PATH_SPLIT) compute_tile_split<ST, FMT, RING_RPT>(a, ox, oy, st, warp);
        else compute_tile<ST, FMT, RING_RPT>(a, ox, oy, st, warp);
        __syncwarp();
        if (lane == 0) ring_arrive(&R.empty[s]);
    }
}

// One level of one frame (plain call).
template <int ST, int FMT, int PATH>
__global__ void __launch_bounds__(RING_NT) pyramid_level_kernel(const LevelArgs a, int tiles_x, int total,
                                                                const __grid_constant__ CUtensorMap map,
                                                                int map_ok) {
    extern __shared__ __align__(128) uint8_t ring_smem_raw[];
    tile_ring<ST, FMT, PATH>(ring_smem_raw, total,
                             [&](int g, LevelArgs &t, int &ox, int &oy, const CUtensorMap *&m) {
                                 const int ty = g / tiles_x, tx = g - ty * tiles_x;
                                 t = a;
                                 ox = tx * TX;
                                 oy = ty * TY;
                                 m = map_ok ? &map : nullptr;
                             });
}

// Level L of every stream of a batch: every stream's level arguments, tile
// prefix and map flag are copied into shared memory once per CTA, so
// naming a tile reads no global memory.
template <int FMT>
__host__ __device__ constexpr size_t batch_smem_bytes(int max_streams) {
    return ring_bytes<FMT>() + (size_t)max_streams * sizeof(LevelArgs) +
           ((size_t)max_streams + 1) * sizeof(int) + (size_t)max_streams * sizeof(int);
}

template <int ST, int FMT, int PATH>
__global__ void __launch_bounds__(RING_NT) pyramid_batch_kernel(const uint8_t *table, int L) {
    extern __shared__ __align__(128) uint8_t ring_smem_raw[];
    const BatchView t(table);
    const int ns = t.nstreams(), cap = t.hdr().max_streams;
    LevelArgs *sa = (LevelArgs *)(ring_smem_raw + ring_bytes<FMT>());
    int *spre = (int *)(sa + cap);
    int *sok = spre + cap + 1;
    for (int i = threadIdx.x; i < ns; i += RING_NT) {
        level_args_from_entry(t.stream(i), L, t.levels(), sa[i]);
        sok[i] = (int)((t.stream(i).pyr_maps_ok >> L) & 1u);
    }
    for (int i = threadIdx.x; i <= ns; i += RING_NT) spre[i] = t.pyr_prefix(L)[i];
    __syncthreads();
    // levels >= 1 are launched dependent on the level above: the table
    // reads above overlap its tail; its planes are read only after this
    pdl_begin();
    tile_ring<ST, FMT, PATH>(ring_smem_raw, spre[ns],
                             [&](int g, LevelArgs &a, int &ox, int &oy, const CUtensorMap *&m) {
                                 const int si = find_segment(spre, ns, g);
                                 a = sa[si];
                                 const int tiles_x = (a.w + TX - 1) / TX;
                                 const int local = g - spre[si];
                                 const int ty = local / tiles_x, tx = local - ty * tiles_x;
                                 ox = tx * TX;
                                 oy = ty * TY;
                                 m = sok[si] ? t.pyr_map(si, L) : nullptr;
                             });
}

// CTAs for `tiles` tiles: at most the number resident on the device at
// once (the kernels stride over the rest).  Sets the kernel's dynamic shared
// memory limit whenever a launch needs more than the last one set on the
// device; cap and cap_smem are the caller's per-kernel caches of resident
// CTAs and of that limit, per device.
template <typename K>
cudaError_t grid_for(K kernel, int tiles, size_t smem, int *cap, size_t *cap_smem, int &grid,
                     int nt) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cap[dev] == 0 || smem > cap_smem[dev]) {
        int sms = 0, per_sm = 0;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, smem);
        if (e != cudaSuccess) return e;
        cap[dev] = sms * (per_sm < 1 ? 1 : per_sm);
        cap_smem[dev] = smem;
    }
    grid = tiles < 1 ? 1 : (tiles < cap[dev] ? tiles : cap[dev]);
    return cudaSuccess;
}

bool encode_level_map(const uint8_t *base, int esz, int w, int h, int64_t pitch, CUtensorMap *out) {
    switch (esz) {
        case 1: return encode_plane_map(base, 1, w, h, pitch, Ring<FMT_U8>::BOX_W, SROWS, out);
        case 2: return encode_plane_map(base, 2, w, h, pitch, Ring<FMT_H16>::BOX_W, SROWS, out);
        default: return encode_plane_map(base, 4, w, h, pitch, Ring<FMT_F32>::BOX_W, SROWS, out);
    }
}

// Level 0 reads the u8 frame; level 1 sums in FP32 (exact); levels 2-3
// split their values in two FP32 parts (exact); deeper levels sum in 64-bit
// fixed point.
__host__ __device__ __forceinline__ int level_path(int frac) {
    return frac == 0 ? PATH_FLOAT : (frac <= 24 ? PATH_SPLIT : PATH_INT64);
}

template <int ST, int FMT, int PATH>
cudaError_t launch_level_k(const LevelArgs &a, cudaStream_t s) {
    const int tiles_x = (a.w + TX - 1) / TX, total = tiles_x * ((a.h + TY - 1) / TY);
    alignas(64) CUtensorMap map;
    memset(&map, 0, sizeof(map));
    const int map_ok = encode_level_map(a.src, Ring<FMT>::ESZ, a.w, a.h, a.src_pitch, &map) ? 1 : 0;
    const size_t smem = ring_bytes<FMT>();
    static int cap[64] = {0};
    static size_t cap_smem[64] = {0};
    int grid = 0;
    cudaError_t e = grid_for(pyramid_level_kernel<ST, FMT, PATH>, total, smem, cap, cap_smem, grid, RING_NT);
    if (e != cudaSuccess) return e;
    pyramid_level_kernel<ST, FMT, PATH><<<grid, RING_NT, smem, s>>>(a, tiles_x, total, map, map_ok);
    return cudaGetLastError();
}

template <int ST, int FMT>
cudaError_t launch_level(const LevelArgs &a, cudaStream_t s) {
    switch (FMT == FMT_U8 ? PATH_FLOAT : level_path(a.frac)) {
        case PATH_SPLIT: return launch_level_k<ST, FMT, PATH_SPLIT>(a, s);
        case PATH_INT64: return launch_level_k<ST, FMT, PATH_INT64>(a, s);
        default: return launch_level_k<ST, FMT, PATH_FLOAT>(a, s);
    }
}

template <int ST, int FMT, int PATH>
cudaError_t launch_batch_level_k(const uint8_t *table, int L, int max_tiles, int max_streams,
                                 int ctas_per_sm, cudaStream_t s) {
    const size_t smem = batch_smem_bytes<FMT>(max_streams);
    static int cap[64] = {0};
    static size_t cap_smem[64] = {0};
    int grid = 0;
    cudaError_t e = grid_for(pyramid_batch_kernel<ST, FMT, PATH>, max_tiles, smem, cap, cap_smem, grid, RING_NT);
    if (e != cudaSuccess) return e;
    if (ctas_per_sm > 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (grid > sms * ctas_per_sm) grid = sms * ctas_per_sm;
    }
    if (L > 0) {
        // scheduled while level L-1 drains (pdl_begin waits for it)
        e = launch_pdl(pyramid_batch_kernel<ST, FMT, PATH>, dim3(grid), dim3(RING_NT), smem, s,
                       table, L);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    pyramid_batch_kernel<ST, FMT, PATH><<<grid, RING_NT, smem, s>>>(table, L);
    return cudaGetLastError();
}

template <int ST, int FMT>
cudaError_t launch_batch_level(const uint8_t *table, int L, int max_tiles, int max_streams,
                               int ctas_per_sm, cudaStream_t s) {
    switch (FMT == FMT_U8 ? PATH_FLOAT : level_path(level_frac(L))) {
        case PATH_SPLIT:
            return launch_batch_level_k<ST, FMT, PATH_SPLIT>(table, L, max_tiles, max_streams, ctas_per_sm, s);
        case PATH_INT64:
            return launch_batch_level_k<ST, FMT, PATH_INT64>(table, L, max_tiles, max_streams, ctas_per_sm, s);
        default:
            return launch_batch_level_k<ST, FMT, PATH_FLOAT>(table, L, max_tiles, max_streams, ctas_per_sm, s);
    }
}

}  // namespace

cudaError_t launch_pyramid(const uint8_t *frame, int w, int h, size_t pitch,
                           const omt_pyramid &pyr, cudaStream_t s) {
    uint8_t *base = (uint8_t *)pyr.base;
    for (int L = 0; L < pyr.levels; ++L) {
        LevelArgs a;
        const omt_level &lv = pyr.lv[L];
        a.w = lv.w;
        a.h = lv.h;
        if (L == 0) {
            a.src = frame;
            a.src_pitch = (int64_t)pitch;
            a.vec_ok = (((uintptr_t)frame | (uintptr_t)pitch) & 15) == 0;
            a.copy = base + lv.img_off;
            a.copy_pitch = lv.img_pitch;
        } else {
            a.src = base + lv.img_off;
            a.src_pitch = lv.img_pitch;
            a.vec_ok = true;
            a.copy = nullptr;
            a.copy_pitch = 0;
        }
        a.grad = base + lv.grad_off;
        a.grad_pitch = lv.grad_pitch;
        a.frac = level_frac(L);
        if (L + 1 < pyr.levels) {
            a.next = base + pyr.lv[L + 1].img_off;
            a.next_pitch = pyr.lv[L + 1].img_pitch;
            a.nw = pyr.lv[L + 1].w;
            a.nh = pyr.lv[L + 1].h;
        } else {
            a.next = nullptr;
            a.next_pitch = 0;
            a.nw = a.nh = 0;
        }
        cudaError_t e;
        if (pyr.storage == OMT_F32)
            e = L == 0 ? launch_level<OMT_F32, FMT_U8>(a, s) : launch_level<OMT_F32, FMT_F32>(a, s);
        else
            e = L == 0 ? launch_level<OMT_F16, FMT_U8>(a, s) : launch_level<OMT_F16, FMT_H16>(a, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pyramid_batch(const uint8_t *table, int levels, int storage, int max_tiles[],
                                 int max_streams, int ctas_per_sm, cudaStream_t s) {
    for (int L = 0; L < levels; ++L) {
        const int mt = max_tiles[L] > 0 ? max_tiles[L] : 1;
        const int c = ctas_per_sm;
        cudaError_t e;
        if (storage == OMT_F32)
            e = L == 0 ? launch_batch_level<OMT_F32, FMT_U8>(table, L, mt, max_streams, c, s)
                       : launch_batch_level<OMT_F32, FMT_F32>(table, L, mt, max_streams, c, s);
        else
            e = L == 0 ? launch_batch_level<OMT_F16, FMT_U8>(table, L, mt, max_streams, c, s)
                       : launch_batch_level<OMT_F16, FMT_H16>(table, L, mt, max_streams, c, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

uint32_t encode_pyramid_maps(const uint8_t *frame, int64_t frame_pitch, const omt_pyramid &pyr,
                             CUtensorMap *out) {
    uint32_t ok = 0;
    if (encode_level_map(frame, 1, pyr.w, pyr.h, frame_pitch, &out[0])) ok |= 1u;
    const int esz = pyr.storage == OMT_F32 ? 4 : 2;
    for (int L = 1; L < pyr.levels && L < OMT_MAX_LEVELS; ++L) {
        const omt_level &lv = pyr.lv[L];
        if (encode_level_map((const uint8_t *)pyr.base + lv.img_off, esz, lv.w, lv.h, lv.img_pitch,
                             &out[L]))
            ok |= 1u << L;
    }
    return ok;
}

cudaError_t pyr_wait_timeouts_take(unsigned *count) {
    unsigned zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(count, pyr_wait_timeouts, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(pyr_wait_timeouts, &zero, sizeof(unsigned));
    return e;
}

int pyramid_tiles(int w, int h) { return ((w + TX - 1) / TX) * ((h + TY - 1) / TY); }

}  // namespace omt
