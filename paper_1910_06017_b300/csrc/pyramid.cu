// pyramid.cu -- K1: Gaussian pyramid and Scharr gradients (Section V-A,
// preprocessing).
//
// One launch per level L.  A CTA owns a 64x16 tile of level L: it stages
// the tile plus a 2-pixel reflect-101 halo in shared memory (coalesced
// loads), writes the tile's gradients (Ix, Iy), and writes the 32x8 tile of
// level L+1 that decimates it.  Level 0 also copies the u8 frame into the
// pyramid buffer.  Sums use the integer binomial weights and scale by a power
// of two at the end, so every value that is dyadic-exact in FP32 (levels 0-2)
// comes out bit-identical to the definition.
#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int TX = 64;  // level-L tile width
constexpr int TY = 16;  // level-L tile height
constexpr int NT = 256; // threads per CTA
constexpr int SX = TX + 4, SY = TY + 4;

struct LevelArgs {
    const uint8_t *src;   // level L: u8 frame (L = 0) or the pyramid's level plane
    int64_t src_pitch;
    int w, h;             // level L size
    int level;
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
        a.copy = const_cast<uint8_t *>(v.img);
        a.copy_pitch = v.img_pitch;
    } else {
        a.src = v.img;
        a.src_pitch = v.img_pitch;
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

// One 64x16 tile of level L at (ox, oy): gradients of the tile and the
// 32x8 tile of level L+1 that decimates it.  Callers loop over tiles with
// the whole CTA; the leading barrier keeps tiles from overlapping in the
// shared arrays.
template <int ST>
__device__ __forceinline__ void pyramid_tile(const LevelArgs &a, int ox, int oy) {
    __shared__ float s[SY][SX];
    __shared__ float hs[SY][TX / 2];
    const int tid = threadIdx.x;
    __syncthreads();

    // Stage level L with a reflect-101 halo of 2.
    for (int i = tid; i < SX * SY; i += NT) {
        const int r = i / SX, c = i - r * SX;
        const int x = reflect101(ox - 2 + c, a.w), y = reflect101(oy - 2 + r, a.h);
        s[r][c] = load_src<ST>(a, x, y);
    }
    if (a.copy) {
        for (int i = tid; i < TX * TY; i += NT) {
            const int r = i / TX, c = i - r * TX;
            const int x = ox + c, y = oy + r;
            if (x < a.w && y < a.h) a.copy[(int64_t)y * a.copy_pitch + x] = a.src[(int64_t)y * a.src_pitch + x];
        }
    }
    __syncthreads();

    // Scharr gradients of the tile, intensity per level pixel.
    for (int i = tid; i < TX * TY; i += NT) {
        const int r = i / TX, c = i - r * TX;
        const int x = ox + c, y = oy + r;
        if (x >= a.w || y >= a.h) continue;
        const int R = r + 2, C = c + 2;
        float gx = 3.0f * (s[R - 1][C + 1] - s[R - 1][C - 1]);
        gx += 10.0f * (s[R][C + 1] - s[R][C - 1]);
        gx += 3.0f * (s[R + 1][C + 1] - s[R + 1][C - 1]);
        float gy = 3.0f * (s[R + 1][C - 1] - s[R - 1][C - 1]);
        gy += 10.0f * (s[R + 1][C] - s[R - 1][C]);
        gy += 3.0f * (s[R + 1][C + 1] - s[R - 1][C + 1]);
        gx *= (1.0f / 32.0f);
        gy *= (1.0f / 32.0f);
        uint8_t *row = a.grad + (int64_t)y * a.grad_pitch;
        if (ST == OMT_F32) ((float2 *)row)[x] = make_float2(gx, gy);
        else ((__half2 *)row)[x] = __floats2half2_rn(gx, gy);
    }
    if (a.next) {
        // Binomial reduce to level L+1: horizontal pass at the even columns...
        for (int i = tid; i < SY * (TX / 2); i += NT) {
            const int r = i / (TX / 2), X = i - r * (TX / 2);
            const int c = 2 * X + 2;
            hs[r][X] = (s[r][c - 2] + s[r][c + 2]) + 4.0f * (s[r][c - 1] + s[r][c + 1]) + 6.0f * s[r][c];
        }
        __syncthreads();
        // ...then vertical at the even rows, scaled by 1/256.
        for (int i = tid; i < (TX / 2) * (TY / 2); i += NT) {
            const int Y = i / (TX / 2), X = i - Y * (TX / 2);
            const int gXo = ox / 2 + X, gYo = oy / 2 + Y;
            if (gXo >= a.nw || gYo >= a.nh) continue;
            const int r = 2 * Y + 2;
            float v = (hs[r - 2][X] + hs[r + 2][X]) + 4.0f * (hs[r - 1][X] + hs[r + 1][X]) + 6.0f * hs[r][X];
            v *= (1.0f / 256.0f);
            uint8_t *row = a.next + (int64_t)gYo * a.next_pitch;
            if (ST == OMT_F32) ((float *)row)[gXo] = v;
            else ((__half *)row)[gXo] = __float2half_rn(v - 128.0f);
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
            a.copy = base + lv.img_off;
            a.copy_pitch = lv.img_pitch;
        } else {
            a.src = base + lv.img_off;
            a.src_pitch = lv.img_pitch;
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
