// static_scratch.cu -- omt_select_corners_static: corner selection for
// callers that cannot hand the library a scratch buffer.
//
// Some callers cannot allocate device memory at the moment they need
// corners: a plugin running inside a host application that owns the CUDA
// allocator, a real-time loop that must never call cudaMalloc (it can
// synchronise the device and stall every other stream), or code that only
// receives input and output pointers from its framework.  For them the
// scratch that omt_select_corners takes from the caller lives here instead,
// in one fixed device array that every GPU loading this library keeps until
// the process exits.
#include <mutex>

#include "omt_internal.cuh"

namespace {

// The library's own scratch for omt_select_corners_static (see omt.h).
static __device__ __align__(256) unsigned char g_select_scratch[OMT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {};

// Device address of g_select_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the real address is
// looked up once per device, with that device current, and cached.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OMT_ECUDA;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess || !p) return OMT_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return OMT_OK;
}

}  // namespace

extern "C" int omt_select_corners_static(const omt_pyramid *pyr, const float *boxes,
                                         int32_t nboxes, const omt_params *prm, float *pts,
                                         int32_t *offsets, void *stream) {
    if (omt_validate_params(prm) != OMT_OK || !pyr || nboxes < 0) return OMT_EINVAL;
    if (nboxes > 0 && (!boxes || ((uintptr_t)boxes & 15) || !pts || ((uintptr_t)pts & 7)))
        return OMT_EINVAL;
    if (!offsets) return OMT_EINVAL;
    if (pyr->w < 1 || pyr->h < 1) return OMT_EINVAL;
    // the map path: its scratch is the response map and the per-box corner
    // slots, without the candidate lists
    const size_t need = omt::select_scratch_bytes(pyr->w, pyr->h, nboxes, prm->max_corners, false);
    if (need == 0 || need > (size_t)OMT_STATIC_SCRATCH_BYTES) return OMT_ENOMEM;
    void *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != OMT_OK) return rc;
    return omt::select_corners_entry(pyr, boxes, nboxes, prm, scratch, need, pts, offsets, false,
                                     stream);
}
