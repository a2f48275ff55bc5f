// pyramid.cu -- K1: Gaussian pyramid and Scharr gradients (Section V-A,
// preprocessing).
//
// One launch per level L.  A 256-thread CTA owns a 128x32 tile of level L:
// it stages the tile plus a 2-pixel reflect-101 halo in shared memory
// (interior tiles with aligned 4-byte or 16-byte row loads, border tiles
// element by element through the reflect-101 map), writes the tile's
// gradients (Ix, Iy) with conflict-free shared reads and coalesced stores,
// and writes the 64x16 tile of level L+1 that decimates it.  Level 0 also copies the u8
// frame into the pyramid buffer.  Sums use the integer binomial weights and
// scale by a power of two at the end, so every value that is dyadic-exact in
// FP32 (levels 0-2) comes out bit-identical to the definition.
#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int TX = 128;  // level-L tile width
constexpr int TY = 32;   // level-L tile height
constexpr int NT = 256;  // threads per CTA
constexpr int SX = TX + 4, SY = TY + 4;
constexpr int HX = TX / 2;  // level L+1 tile width

struct LevelArgs {
    const uint8_t *src;   // level L: u8 frame (L = 0) or the pyramid's level plane
    int64_t src_pitch;
    int w, h;             // level L size
    int level;
    bool vec_ok;          // src rows are 4-byte aligned (pointer and pitch)
    uint8_t *copy;        // level-0 u8 copy (L = 0 only)
    int64_t copy_pitch;
    uint8_t *grad;        // level-L gradient plane
    int64_t grad_pitch;
    uint8_t *next;        // level L+1 image plane or nullptr
    int64_t next_pitch;
    int nw, nh;           // level L+1 size
};

template <int ST>
__device__ __forceinline__ float load_src(const LevelArgs &a, int x, int y) {
    const uint8_t *row = a.src + (int64_t)y * a.src_pitch;
    if (a.level == 0) return (float)row[x];
    if (ST == OMT_F32) return ((const float *)row)[x];
    return __half2float(((const __half *)row)[x]) + 128.0f;
}

// Stage level L over [ox-2, ox+TX+2) x [oy-2, oy+TY+2) into s.
template <int ST>
__device__ __forceinline__ void stage_tile(const LevelArgs &a, int ox, int oy, float (*s)[SX]) {
    const int tid = threadIdx.x;
    const bool interior = ox - 4 >= 0 && oy - 2 >= 0 && ox + TX + 4 <= a.w && oy + TY + 2 <= a.h;
    if (interior && a.vec_ok) {
        if (a.level == 0 || ST == OMT_F16) {
            // 4-byte words from column ox-4 (4-aligned): 4 u8 or 2 half texels each
            const int per = a.level == 0 ? 4 : 2;
            const int nwords = (TX + 8) / per;
            for (int i = tid; i < SY * nwords; i += NT) {
                const int r = i / nwords, k = i - r * nwords;
                const uint8_t *row = a.src + (int64_t)(oy - 2 + r) * a.src_pitch;
                const int x = ox - 4 + k * per;  // first texel of the word
                const unsigned wv = __ldg((const unsigned *)(row + (int64_t)x * (per == 4 ? 1 : 2)));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q >= per) break;
                    const int c = x + q - (ox - 2);
                    if (c < 0 || c >= SX) continue;
                    float v;
                    if (per == 4) v = (float)((wv >> (8 * q)) & 0xFFu);
                    else v = __half2float(__ushort_as_half((unsigned short)(wv >> (16 * q)))) + 128.0f;
                    s[r][c] = v;
                }
            }
        } else {
            // float4 from column ox-4 (16-byte aligned)
            const int nq = (TX + 8) / 4;
            for (int i = tid; i < SY * nq; i += NT) {
                const int r = i / nq, k = i - r * nq;
                const float4 v = __ldg((const float4 *)(a.src + (int64_t)(oy - 2 + r) * a.src_pitch) +
                                       (ox - 4) / 4 + k);
                const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = 4 * k + q - 2;
                    if (c >= 0 && c < SX) s[r][c] = e[q];
                }
            }
        }
    } else {
        for (int i = tid; i < SX * SY; i += NT) {
            const int r = i / SX, c = i - r * SX;
            s[r][c] = load_src<ST>(a, reflect101(ox - 2 + c, a.w), reflect101(oy - 2 + r, a.h));
        }
    }
}

// Arguments of level L of the pyramid a batch entry builds (frame t+1).
__device__ __forceinline__ void level_args_from_entry(const StreamEntry &e, int L, int levels,
                                                      LevelArgs &a) {
    const LevelView &v = e.P_next[L];
    a.level = L;
    a.w = v.w;
    a.h = v.h;
    if (L == 0) {
        a.src = e.frame;
        a.src_pitch = e.frame_pitch;
        a.vec_ok = (((uintptr_t)e.frame | (uintptr_t)e.frame_pitch) & 3) == 0;
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

// One 128x32 tile of level L at (ox, oy): gradients of the tile and the
// 64x16 tile of level L+1 that decimates it.  Callers loop over tiles with
// the whole CTA; the leading barrier keeps tiles from overlapping in the
// shared arrays.
template <int ST>
__device__ __forceinline__ void pyramid_tile(const LevelArgs &a, int ox, int oy) {
    __shared__ float s[SY][SX];
    __shared__ float hs[SY][HX];
    const int tid = threadIdx.x;
    __syncthreads();
    stage_tile<ST>(a, ox, oy, s);
    if (a.copy) {
        // u8 copy of the tile, 4 bytes per thread where the row allows
        for (int i = tid; i < TY * (TX / 4); i += NT) {
            const int r = i / (TX / 4), k = i - r * (TX / 4);
            const int x = ox + 4 * k, y = oy + r;
            if (y >= a.h || x >= a.w) continue;
            uint8_t *dst = a.copy + (int64_t)y * a.copy_pitch + x;
            const uint8_t *src = a.src + (int64_t)y * a.src_pitch + x;
            if (x + 3 < a.w && a.vec_ok) {
                *(unsigned *)dst = __ldg((const unsigned *)src);
            } else {
                for (int q = 0; q < 4 && x + q < a.w; ++q) dst[q] = src[q];
            }
        }
    }
    __syncthreads();

    // Scharr gradients, intensity per level pixel.  Thread (tx, ty) takes
    // columns tx + 32 q and rows 4 ty + rr: conflict-free shared reads, and a
    // warp stores 32 consecutive pixels of a row.
    {
        const int tx = tid & 31, ty = tid >> 5;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int r = 4 * ty + rr;
            const int y = oy + r;
            if (y >= a.h) break;
            const int R = r + 2;
            uint8_t *row = a.grad + (int64_t)y * a.grad_pitch;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = tx + 32 * q, x = ox + c;
                if (x >= a.w) break;
                const int C = c + 2;
                float gx = 3.0f * (s[R - 1][C + 1] - s[R - 1][C - 1]);
                gx += 10.0f * (s[R][C + 1] - s[R][C - 1]);
                gx += 3.0f * (s[R + 1][C + 1] - s[R + 1][C - 1]);
                float gy = 3.0f * (s[R + 1][C - 1] - s[R - 1][C - 1]);
                gy += 10.0f * (s[R + 1][C] - s[R - 1][C]);
                gy += 3.0f * (s[R + 1][C + 1] - s[R - 1][C + 1]);
                gx *= (1.0f / 32.0f);
                gy *= (1.0f / 32.0f);
                if (ST == OMT_F32) ((float2 *)row)[x] = make_float2(gx, gy);
                else ((__half2 *)row)[x] = __floats2half2_rn(gx, gy);
            }
        }
    }
    if (a.next) {
        // Binomial reduce to level L+1: horizontal pass at the even columns...
        for (int i = tid; i < SY * HX; i += NT) {
            const int r = i / HX, X = i - r * HX;
            const int c = 2 * X + 2;
            hs[r][X] = (s[r][c - 2] + s[r][c + 2]) + 4.0f * (s[r][c - 1] + s[r][c + 1]) + 6.0f * s[r][c];
        }
        __syncthreads();
        // ...then vertical at the even rows, scaled by 1/256: thread (X, Y0)
        // takes rows Y0 + 4 q of column X.
        const int X = tid & (HX - 1), Y0 = tid / HX;
        const int gX = ox / 2 + X;
        if (gX < a.nw) {
#pragma unroll
            for (int q = 0; q < (TY / 2) / (NT / HX); ++q) {
                const int Y = Y0 + (NT / HX) * q;
                const int gY = oy / 2 + Y;
                if (gY >= a.nh) break;
                const int r = 2 * Y + 2;
                const float v = ((hs[r - 2][X] + hs[r + 2][X]) + 4.0f * (hs[r - 1][X] + hs[r + 1][X]) +
                                 6.0f * hs[r][X]) * (1.0f / 256.0f);
                uint8_t *row = a.next + (int64_t)gY * a.next_pitch;
                if (ST == OMT_F32) ((float *)row)[gX] = v;
                else ((__half *)row)[gX] = __float2half_rn(v - 128.0f);
            }
        }
    }
}

template <int ST>
__global__ void __launch_bounds__(NT) pyramid_level_kernel(LevelArgs a) {
    pyramid_tile<ST>(a, blockIdx.x * TX, blockIdx.y * TY);
}

// Level L of every stream of a batch: a grid-stride loop over the batch's
// tiles (tile prefix per stream in the table).
template <int ST>
__global__ void __launch_bounds__(NT) pyramid_batch_kernel(const uint8_t *table, int L) {
    const BatchView t(table);
    const int *pre = t.pyr_prefix(L);
    const int total = pre[t.nstreams()];
    for (int g = blockIdx.x; g < total; g += gridDim.x) {
        const int si = find_segment(pre, t.nstreams(), g);
        const StreamEntry &e = t.stream(si);
        const int tiles_x = (e.P_next[L].w + TX - 1) / TX;
        const int local = g - pre[si];
        const int ty = local / tiles_x, tx = local - ty * tiles_x;
        LevelArgs a;
        level_args_from_entry(e, L, t.levels(), a);
        pyramid_tile<ST>(a, tx * TX, ty * TY);
    }
}

}  // namespace

cudaError_t launch_pyramid(const uint8_t *frame, int w, int h, size_t pitch,
                           const omt_pyramid &pyr, cudaStream_t s) {
    uint8_t *base = (uint8_t *)pyr.base;
    for (int L = 0; L < pyr.levels; ++L) {
        LevelArgs a;
        const omt_level &lv = pyr.lv[L];
        a.level = L;
        a.w = lv.w;
        a.h = lv.h;
        if (L == 0) {
            a.src = frame;
            a.src_pitch = (int64_t)pitch;
            a.vec_ok = (((uintptr_t)frame | (uintptr_t)pitch) & 3) == 0;
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
        dim3 grid((lv.w + TX - 1) / TX, (lv.h + TY - 1) / TY);
        if (pyr.storage == OMT_F32) pyramid_level_kernel<OMT_F32><<<grid, NT, 0, s>>>(a);
        else pyramid_level_kernel<OMT_F16><<<grid, NT, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pyramid_batch(const uint8_t *table, int levels, int storage, int max_tiles[],
                                 cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int L = 0; L < levels; ++L) {
        const int cap = sms * 8;
        const int grid = max_tiles[L] < cap ? (max_tiles[L] > 0 ? max_tiles[L] : 1) : cap;
        if (storage == OMT_F32) pyramid_batch_kernel<OMT_F32><<<grid, NT, 0, s>>>(table, L);
        else pyramid_batch_kernel<OMT_F16><<<grid, NT, 0, s>>>(table, L);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int pyramid_tiles(int w, int h) { return ((w + TX - 1) / TX) * ((h + TY - 1) / TY); }

}  // namespace omt
