// api.cu -- the C-ABI of libomt: host-side validation, pyramid layout and
// dispatch to the kernels.  Every check happens before the first launch.
#include <math.h>
#include <string.h>

#include "omt_internal.cuh"

using namespace omt;

namespace {

constexpr int32_t kVersion = 400;  // 0.4.0: K1/K2 launch shapes in omt_batch_caps

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool shape_ok(int32_t w, int32_t h, int32_t levels, int32_t storage) {
    return w >= 1 && h >= 1 && (int64_t)w * h <= (int64_t)1 << 31 && w <= (1 << 16) &&
           h <= (1 << 16) && levels >= 1 && levels <= OMT_MAX_LEVELS &&
           (storage == OMT_F32 || storage == OMT_F16);
}

// Plane layout of a pyramid; returns the total byte count.
size_t layout(int32_t w, int32_t h, int32_t levels, int32_t storage, omt_level *lv) {
    size_t off = 0;
    const size_t esz = storage == OMT_F32 ? 4 : 2;
    int32_t lw = w, lh = h;
    for (int L = 0; L < levels; ++L) {
        omt_level l;
        l.w = lw;
        l.h = lh;
        l.img_pitch = (int64_t)align_up((size_t)lw * (L == 0 ? 1 : esz), 128);
        l.img_off = (int64_t)off;
        off = align_up(off + (size_t)l.img_pitch * lh, 256);
        l.grad_pitch = (int64_t)align_up((size_t)lw * 2 * esz, 128);
        l.grad_off = (int64_t)off;
        off = align_up(off + (size_t)l.grad_pitch * lh, 256);
        if (lv) lv[L] = l;
        lw = (lw + 1) >> 1;
        lh = (lh + 1) >> 1;
    }
    return off;
}

bool pyr_ok(const omt_pyramid *p) {
    if (!p || !p->base || !shape_ok(p->w, p->h, p->levels, p->storage)) return false;
    if (((uintptr_t)p->base & 255) != 0) return false;
    omt_level lv[OMT_MAX_LEVELS];
    const size_t need = layout(p->w, p->h, p->levels, p->storage, lv);
    if (p->bytes < need) return false;
    return memcmp(lv, p->lv, sizeof(omt_level) * p->levels) == 0;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

int from_cuda(cudaError_t e) { return e == cudaSuccess ? OMT_OK : OMT_ECUDA; }

}  // namespace

namespace omt {
int select_corners_entry(const omt_pyramid *pyr, const float *boxes, int32_t nboxes,
                         const omt_params *prm, void *scratch, size_t scratch_bytes, float *pts,
                         int32_t *offsets, bool lists, void *stream) {
    if (omt_validate_params(prm) != OMT_OK || !pyr_ok(pyr) || nboxes < 0) return OMT_EINVAL;
    if (nboxes > 0 && (!boxes || !aligned(boxes, 16) || !pts || !aligned(pts, 8)))
        return OMT_EINVAL;
    if (!offsets || !scratch || !aligned(scratch, 256)) return OMT_EINVAL;
    if ((int64_t)nboxes * prm->max_corners > ((int64_t)1 << 31) - 1) return OMT_EINVAL;
    if (scratch_bytes < select_scratch_bytes(pyr->w, pyr->h, nboxes, prm->max_corners, lists))
        return OMT_ENOMEM;
    return from_cuda(launch_select_corners(*pyr, (const float4 *)boxes, nboxes, *prm, scratch,
                                           (float2 *)pts, offsets, lists, (cudaStream_t)stream));
}
}  // namespace omt

extern "C" {

void omt_default_params(omt_params *p) {
    if (!p) return;
    p->levels = 3;
    p->win = 21;
    p->max_iter = 30;
    p->eps = 0.01f;
    p->min_eig = 1e-3f;
    p->quality_num = 1;
    p->quality_den = 100;
    p->min_dist = 5.0f;
    p->max_corners = 50;
    p->storage = OMT_F32;
    p->aggregator = 0;
    p->fb_max = -1.0f;
}

int omt_validate_params(const omt_params *p) {
    if (!p) return OMT_EINVAL;
    if (p->levels < 1 || p->levels > OMT_MAX_LEVELS) return OMT_EINVAL;
    if (p->win < OMT_MIN_WIN || p->win > OMT_MAX_WIN || (p->win & 1) == 0) return OMT_EINVAL;
    if (p->max_iter < 1 || p->max_iter > 255) return OMT_EINVAL;
    if (!(p->eps >= 0.0f) || !isfinite(p->eps)) return OMT_EINVAL;
    if (!(p->min_eig >= 0.0f) || !isfinite(p->min_eig)) return OMT_EINVAL;
    if (p->quality_num < 0 || p->quality_den < 1 || p->quality_num > 65535 ||
        p->quality_den > 65535)
        return OMT_EINVAL;
    if (!(p->min_dist >= 0.0f) || !(p->min_dist <= 65536.0f)) return OMT_EINVAL;
    if (p->max_corners < 0 || p->max_corners > OMT_MAX_CORNERS) return OMT_EINVAL;
    if (p->storage != OMT_F32 && p->storage != OMT_F16) return OMT_EINVAL;
    if (p->aggregator < 0 || p->aggregator > 2) return OMT_EINVAL;
    if (p->fb_max != p->fb_max) return OMT_EINVAL;  // NaN
    return OMT_OK;
}

size_t omt_pyramid_bytes(int32_t w, int32_t h, int32_t levels, int32_t storage) {
    if (!shape_ok(w, h, levels, storage)) return 0;
    return layout(w, h, levels, storage, nullptr);
}

int omt_pyramid_init(omt_pyramid *pyr, int32_t w, int32_t h, int32_t levels, int32_t storage,
                     void *base, size_t bytes) {
    if (!pyr || !base || !shape_ok(w, h, levels, storage) || !aligned(base, 256))
        return OMT_EINVAL;
    memset(pyr, 0, sizeof(*pyr));
    const size_t need = layout(w, h, levels, storage, pyr->lv);
    if (bytes < need) return OMT_ENOMEM;
    pyr->w = w;
    pyr->h = h;
    pyr->levels = levels;
    pyr->storage = storage;
    pyr->base = base;
    pyr->bytes = bytes;
    return OMT_OK;
}

int omt_build_pyramid(const uint8_t *frame, int32_t w, int32_t h, size_t pitch,
                      const omt_params *prm, const omt_pyramid *pyr, void *stream) {
    if (!frame || omt_validate_params(prm) != OMT_OK || !pyr_ok(pyr)) return OMT_EINVAL;
    if (pyr->w != w || pyr->h != h || pyr->levels != prm->levels || pyr->storage != prm->storage)
        return OMT_EINVAL;
    if (pitch < (size_t)w) return OMT_EINVAL;
    return from_cuda(launch_pyramid(frame, w, h, pitch, *pyr, (cudaStream_t)stream));
}

int omt_corner_response(const omt_pyramid *pyr, uint32_t *out, void *stream) {
    if (!pyr_ok(pyr) || !out || !aligned(out, 4)) return OMT_EINVAL;
    return from_cuda(launch_corner_response(*pyr, out, nullptr, 0, (cudaStream_t)stream));
}

size_t omt_corner_scratch_bytes(int32_t w, int32_t h, int32_t nboxes, int32_t max_corners) {
    if (w < 1 || h < 1 || nboxes < 0 || max_corners < 0 || max_corners > OMT_MAX_CORNERS)
        return 0;
    return select_scratch_bytes(w, h, nboxes, max_corners);
}


int omt_select_corners(const omt_pyramid *pyr, const float *boxes, int32_t nboxes,
                       const omt_params *prm, void *scratch, size_t scratch_bytes, float *pts,
                       int32_t *offsets, void *stream) {
    return select_corners_entry(pyr, boxes, nboxes, prm, scratch, scratch_bytes, pts, offsets,
                                true, stream);
}

int omt_lk_track(const omt_pyramid *prev, const omt_pyramid *next, const float *pts,
                 int32_t n_max, const int32_t *n_dev, const omt_params *prm, float *pts_out,
                 uint8_t *status, uint8_t *iters, void *stream) {
    if (omt_validate_params(prm) != OMT_OK || !pyr_ok(prev) || !pyr_ok(next)) return OMT_EINVAL;
    if (prev->w != next->w || prev->h != next->h || prev->levels != next->levels ||
        prev->storage != next->storage || prev->levels != prm->levels ||
        prev->storage != prm->storage)
        return OMT_EINVAL;
    if (n_max < 0) return OMT_EINVAL;
    if (n_max > 0 && (!pts || !pts_out || !status || !aligned(pts, 8) || !aligned(pts_out, 8)))
        return OMT_EINVAL;
    return from_cuda(launch_lk(*prev, *next, (const float2 *)pts, n_max, n_dev, *prm,
                               (float2 *)pts_out, status, iters, (cudaStream_t)stream));
}

int omt_update_boxes(const float *boxes, const int32_t *offsets, const float *pts,
                     const float *pts_out, const uint8_t *status, int32_t nboxes,
                     const omt_params *prm, float *boxes_out, int32_t *nvalid, void *stream) {
    if (omt_validate_params(prm) != OMT_OK || nboxes < 0) return OMT_EINVAL;
    if (nboxes == 0) return OMT_OK;
    if (!boxes || !offsets || !boxes_out || !aligned(boxes, 16) || !aligned(boxes_out, 16))
        return OMT_EINVAL;
    if (boxes == boxes_out) return OMT_EINVAL;
    if (!pts || !pts_out || !status || !aligned(pts, 8) || !aligned(pts_out, 8))
        return OMT_EINVAL;
    return from_cuda(launch_update_boxes((const float4 *)boxes, offsets, (const float2 *)pts,
                                         (const float2 *)pts_out, status, nboxes,
                                         prm->aggregator, (float4 *)boxes_out, nvalid,
                                         (cudaStream_t)stream));
}

namespace {

bool caps_ok(const omt_batch_caps *c) {
    return c && c->max_streams >= 1 && c->max_streams <= OMT_BATCH_MAX_STREAMS &&
           c->max_boxes >= 0 && c->max_w >= 1 && c->max_h >= 1 && c->max_w <= (1 << 16) &&
           c->max_h <= (1 << 16) && c->max_corners >= 0 && c->max_corners <= OMT_MAX_CORNERS &&
           c->lk_warps >= 0 && c->lk_warps <= 8 && c->lk_ctas_per_sm >= 0 &&
           c->lk_ctas_per_sm <= 32 && c->lk_chunk >= 0 && c->lk_chunk <= 16 &&
           c->pyr_ctas_per_sm >= 0 && c->pyr_ctas_per_sm <= 32 && c->corner_ctas_per_sm >= 0 &&
           c->corner_ctas_per_sm <= 32 && c->select_ctas_per_sm >= 0 &&
           c->select_ctas_per_sm <= 32 && c->reserved == 0;
}

void fill_levels(const omt_pyramid &p, LevelView *out) {
    for (int L = 0; L < OMT_MAX_LEVELS; ++L) out[L] = level_view(p, L < p.levels ? L : 0);
}

}  // namespace

size_t omt_batch_table_bytes(const omt_batch_caps *caps) {
    if (!caps_ok(caps)) return 0;
    return batch_table_bytes(caps->max_streams);
}

int omt_batch_pack(const omt_batch_stream *streams, int32_t nstreams, const omt_params *prm,
                   const omt_batch_caps *caps, void *table, size_t table_bytes) {
    if (omt_validate_params(prm) != OMT_OK || !caps_ok(caps) || !table) return OMT_EINVAL;
    if (nstreams < 0 || nstreams > caps->max_streams || (nstreams > 0 && !streams))
        return OMT_EINVAL;
    if (prm->max_corners > caps->max_corners) return OMT_EINVAL;
    const size_t need = batch_table_bytes(caps->max_streams);
    if (table_bytes < need) return OMT_ENOMEM;
    uint8_t *base = (uint8_t *)table;
    memset(base, 0, need);
    BatchHeader &h = *(BatchHeader *)base;
    h.nstreams = nstreams;
    h.max_streams = caps->max_streams;
    h.levels = prm->levels;
    h.storage = prm->storage;
    h.win = prm->win;
    h.max_iter = prm->max_iter;
    h.qnum = prm->quality_num;
    h.qden = prm->quality_den;
    h.aggregator = prm->aggregator;
    h.eps2 = prm->eps * prm->eps;
    h.tau_n = prm->min_eig * (float)(prm->win * prm->win);
    h.fb_max = prm->fb_max;
    h.fb_on = prm->fb_max >= 0.0f;
    const float md2 = prm->min_dist * prm->min_dist;
    h.md2c = (int64_t)ceil((double)md2);
    h.dmax = 0;
    while ((int64_t)(h.dmax + 1) * (h.dmax + 1) < h.md2c) ++h.dmax;
    h.cell = 1;
    while (2 * (int64_t)(h.cell + 1) * (h.cell + 1) <= h.md2c) ++h.cell;
    h.bytes = (int64_t)need;
    BatchView v(base);
    int32_t *pyr_pre[OMT_MAX_LEVELS];
    for (int L = 0; L < OMT_MAX_LEVELS; ++L) pyr_pre[L] = const_cast<int32_t *>(v.pyr_prefix(L));
    int32_t *resp_pre = const_cast<int32_t *>(v.resp_prefix());
    int32_t *box_pre = const_cast<int32_t *>(v.box_prefix());
    StreamEntry *ent = (StreamEntry *)(base + batch_entries_offset(caps->max_streams));
    int64_t boxes_total = 0;
    for (int i = 0; i < nstreams; ++i) {
        const omt_batch_stream &b = streams[i];
        const omt_pyramid &P = b.prev, &N = b.next;
        if (!pyr_ok(&P) || !pyr_ok(&N)) return OMT_EINVAL;
        if (P.w != N.w || P.h != N.h || P.levels != prm->levels || N.levels != prm->levels ||
            P.storage != prm->storage || N.storage != prm->storage)
            return OMT_EINVAL;
        if (P.base == N.base) return OMT_EINVAL;
        if (P.w > caps->max_w || P.h > caps->max_h) return OMT_EINVAL;
        if (!b.frame || b.frame_pitch < (size_t)P.w) return OMT_EINVAL;
        if (b.nboxes < 0 || b.max_corners < 0 || b.max_corners > caps->max_corners) return OMT_EINVAL;
        if ((int64_t)b.nboxes * b.max_corners > ((int64_t)1 << 31) - 1) return OMT_EINVAL;
        if (b.nboxes > 0) {
            if (!b.boxes || !aligned(b.boxes, 16) || !b.boxes_out || !aligned(b.boxes_out, 16) ||
                b.boxes == b.boxes_out)
                return OMT_EINVAL;
            if (!b.pts || !b.pts_out || !b.status || !aligned(b.pts, 8) || !aligned(b.pts_out, 8))
                return OMT_EINVAL;
            if (h.fb_on && (!b.pts_back || !b.status_back || !aligned(b.pts_back, 8)))
                return OMT_EINVAL;
        }
        if (!b.offsets || !b.scratch || !aligned(b.scratch, 256)) return OMT_EINVAL;
        if (b.scratch_bytes < select_scratch_bytes(P.w, P.h, b.nboxes, b.max_corners))
            return OMT_ENOMEM;
        StreamEntry &e = ent[i];
        fill_levels(P, e.P);
        fill_levels(N, e.P_next);
        e.frame = b.frame;
        e.frame_pitch = (int64_t)b.frame_pitch;
        e.boxes = (const float4 *)b.boxes;
        e.boxes_out = (float4 *)b.boxes_out;
        e.nvalid = b.nvalid;
        e.pts = (float2 *)b.pts;
        e.pts_out = (float2 *)b.pts_out;
        e.status = b.status;
        e.iters = b.iters;
        e.pts_back = h.fb_on ? (float2 *)b.pts_back : nullptr;
        e.status_back = h.fb_on ? b.status_back : nullptr;
        e.offsets = b.offsets;
        {
            SelectScratch sc;
            select_scratch_split(b.scratch, P.w, P.h, b.nboxes, b.max_corners, true, sc);
            e.rmap = sc.rmap;
            e.pad_pts = sc.pad_pts;
            e.pad_counts = sc.pad_counts;
            e.cand = sc.cand;
            e.cstate = sc.cstate;
        }
        e.w = P.w;
        e.h = P.h;
        e.nboxes = b.nboxes;
        e.maxc = b.max_corners;
        {
            // the host table may be only 16-byte aligned: encode aside, then
            // copy; backward maps (templates on frame t+1) only for the
            // forward-backward check
            alignas(64) CUtensorMap tm[2][OMT_MAX_LEVELS * LK_MAPS];
            memset(tm, 0, sizeof(tm));
            e.tm_ok = encode_lk_maps(P, N, prm->win, tm[0]);
            e.tm_ok_back = h.fb_on ? encode_lk_maps(N, P, prm->win, tm[1]) : 0u;
            memcpy(base + batch_maps_offset(caps->max_streams) +
                       sizeof(CUtensorMap) * (size_t)i * 2 * OMT_MAX_LEVELS * LK_MAPS,
                   tm, sizeof(tm));
        }
        {
            alignas(64) CUtensorMap pm[OMT_MAX_LEVELS];
            memset(pm, 0, sizeof(pm));
            e.pyr_maps_ok = encode_pyramid_maps(b.frame, (int64_t)b.frame_pitch, N, pm);
            memcpy(base + batch_pyr_maps_offset(caps->max_streams) +
                       sizeof(CUtensorMap) * (size_t)i * OMT_MAX_LEVELS,
                   pm, sizeof(pm));
        }
        for (int L = 0; L < prm->levels; ++L)
            pyr_pre[L][i + 1] = pyr_pre[L][i] + pyramid_tiles(P.lv[L].w, P.lv[L].h);
        resp_pre[i + 1] = resp_pre[i] + response_tiles(P.w, P.h);
        boxes_total += b.nboxes;
        if (boxes_total > caps->max_boxes) return OMT_EINVAL;
        box_pre[i + 1] = (int32_t)boxes_total;
    }
    h.total_boxes = (int32_t)boxes_total;
    return OMT_OK;
}

int omt_batch_upload(const void *table, const omt_batch_caps *caps, void *dev_table,
                     size_t dev_table_bytes, void *stream) {
    if (!caps_ok(caps) || !table || !dev_table || !aligned(dev_table, 256)) return OMT_EINVAL;
    const size_t need = batch_table_bytes(caps->max_streams);
    if (dev_table_bytes < need) return OMT_ENOMEM;
    const BatchHeader &h = *(const BatchHeader *)table;
    if (h.max_streams != caps->max_streams || h.bytes != (int64_t)need || h.nstreams < 0 ||
        h.nstreams > caps->max_streams || h.total_boxes > caps->max_boxes)
        return OMT_EINVAL;
    return from_cuda(cudaMemcpyAsync(dev_table, table, need, cudaMemcpyHostToDevice,
                                     (cudaStream_t)stream));
}

int omt_batch_phase(const void *dev_table, const omt_batch_caps *caps, const omt_params *prm,
                    int32_t phase, void *stream) {
    if (omt_validate_params(prm) != OMT_OK || !caps_ok(caps) || !dev_table ||
        !aligned(dev_table, 256))
        return OMT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const uint8_t *dt = (const uint8_t *)dev_table;
    switch (phase) {
        case OMT_PHASE_PYRAMID: {
            int max_tiles[OMT_MAX_LEVELS];
            int lw = caps->max_w, lh = caps->max_h;
            for (int L = 0; L < prm->levels; ++L) {
                max_tiles[L] = caps->max_streams * pyramid_tiles(lw, lh);
                lw = (lw + 1) >> 1;
                lh = (lh + 1) >> 1;
            }
            return from_cuda(launch_pyramid_batch(dt, prm->levels, prm->storage, max_tiles,
                                                  caps->max_streams, caps->pyr_ctas_per_sm, s));
        }
        case OMT_PHASE_CORNERS:
            return from_cuda(launch_corners_batch(
                dt, caps->max_streams, caps->max_streams * response_tiles(caps->max_w, caps->max_h),
                caps->max_boxes, caps->max_corners, caps->corner_ctas_per_sm,
                caps->select_ctas_per_sm, s));
        case OMT_PHASE_FB:
            if (!(prm->fb_max >= 0.0f)) return OMT_OK;
            return from_cuda(launch_lk_batch(dt, prm->storage, prm->win, caps->lk_warps,
                                             caps->lk_ctas_per_sm, caps->lk_chunk, 1, s));
        case OMT_PHASE_LK:
            return from_cuda(launch_lk_batch(dt, prm->storage, prm->win, caps->lk_warps,
                                             caps->lk_ctas_per_sm, caps->lk_chunk, 0, s));
        case OMT_PHASE_BOXES:
            return from_cuda(launch_update_boxes_batch(dt, caps->max_boxes, prm->aggregator, s));
        default:
            return OMT_EINVAL;
    }
}

int omt_batch_step(const void *table, const omt_batch_caps *caps, const omt_params *prm,
                   void *dev_table, size_t dev_table_bytes, void *stream) {
    if (omt_validate_params(prm) != OMT_OK || !caps_ok(caps) || !table || !dev_table)
        return OMT_EINVAL;
    const BatchHeader &h = *(const BatchHeader *)table;
    if (h.levels != prm->levels || h.storage != prm->storage || h.win != prm->win ||
        h.max_iter != prm->max_iter)
        return OMT_EINVAL;
    if (h.fb_max != prm->fb_max || h.aggregator != prm->aggregator) return OMT_EINVAL;
    int rc = omt_batch_upload(table, caps, dev_table, dev_table_bytes, stream);
    static const int order[] = {OMT_PHASE_PYRAMID, OMT_PHASE_CORNERS, OMT_PHASE_LK, OMT_PHASE_FB,
                                OMT_PHASE_BOXES};
    for (int k = 0; rc == OMT_OK && k < 5; ++k)
        rc = omt_batch_phase(dev_table, caps, prm, order[k], stream);
    return rc;
}

int omt_iou_matrix(const float *a, int32_t na, const float *b, int32_t nb, double *iou,
                   void *stream) {
    if (na < 0 || nb < 0) return OMT_EINVAL;
    if (na == 0 || nb == 0) return OMT_OK;
    if (!a || !b || !iou || !aligned(a, 16) || !aligned(b, 16) || !aligned(iou, 8)) return OMT_EINVAL;
    return from_cuda(launch_iou_matrix(a, na, b, nb, iou, (cudaStream_t)stream));
}

int omt_fb_check(const float *pts, const float *pts_back, const uint8_t *status_back,
                 int32_t n_max, const int32_t *n_dev, float fb_max, uint8_t *status,
                 void *stream) {
    if (fb_max != fb_max || n_max < 0) return OMT_EINVAL;
    if (n_max == 0) return OMT_OK;
    if (!pts || !pts_back || !status_back || !status || !aligned(pts, 8) || !aligned(pts_back, 8))
        return OMT_EINVAL;
    return from_cuda(launch_fb_check((const float2 *)pts, (const float2 *)pts_back, status_back,
                                     n_max, n_dev, fb_max, status, (cudaStream_t)stream));
}

void omt_default_flow_params(omt_flow_params *p) {
    if (!p) return;
    p->st_theta = 0.125f;
    p->st_alpha = 0.95f;
    p->st_k = 2.0f;
    p->st_iters = 100;
    p->lambda = 10.0f;
    p->eps = 0.05f;
    p->warps = 3;
    p->iters = 30;
    p->block = 2;
}

namespace {
bool flow_params_ok(const omt_flow_params *p) {
    return p && p->st_theta > 0.0f && isfinite(p->st_theta) && isfinite(p->st_alpha) &&
           isfinite(p->st_k) && p->st_iters >= 0 && p->st_iters <= 100000 && p->lambda >= 0.0f &&
           isfinite(p->lambda) && p->eps >= 0.0f && isfinite(p->eps) && p->warps >= 1 &&
           p->warps <= 100 && p->iters >= 1 && p->iters <= 100000 &&
           (p->block == 1 || p->block == 2);
}
}  // namespace

size_t omt_structure_texture_scratch_bytes(int32_t w, int32_t h) {
    if (w < 1 || h < 1 || w > (1 << 16) || h > (1 << 16)) return 0;
    return st_scratch_bytes(w, h);
}

size_t omt_tvl1_scratch_bytes(int32_t w, int32_t h) {
    if (w < 1 || h < 1 || w > (1 << 16) || h > (1 << 16)) return 0;
    return tvl1_scratch_bytes(w, h);
}

int omt_structure_texture(const uint8_t *frame, int32_t w, int32_t h, size_t pitch,
                          const omt_flow_params *fp, uint8_t *texture, size_t tpitch,
                          void *scratch, size_t scratch_bytes, void *stream) {
    if (!flow_params_ok(fp) || !frame || !texture || !scratch || w < 1 || h < 1 ||
        w > (1 << 16) || h > (1 << 16) || pitch < (size_t)w || tpitch < (size_t)w)
        return OMT_EINVAL;
    if (scratch_bytes < st_scratch_bytes(w, h)) return OMT_ENOMEM;
    return from_cuda(launch_structure_texture(frame, w, h, pitch, *fp, texture, tpitch, scratch,
                                              (cudaStream_t)stream));
}

int omt_tvl1_flow(const omt_pyramid *prev, const omt_pyramid *next, const omt_flow_params *fp,
                  float *flow, void *scratch, size_t scratch_bytes, void *stream) {
    if (!flow_params_ok(fp) || !pyr_ok(prev) || !pyr_ok(next) || !flow || !scratch ||
        !aligned(flow, 8))
        return OMT_EINVAL;
    if (prev->w != next->w || prev->h != next->h || prev->levels != next->levels ||
        prev->storage != OMT_F32 || next->storage != OMT_F32 || prev->base == next->base)
        return OMT_EINVAL;
    if (scratch_bytes < tvl1_scratch_bytes(prev->w, prev->h)) return OMT_ENOMEM;
    return from_cuda(launch_tvl1(*prev, *next, *fp, (float2 *)flow, scratch, (cudaStream_t)stream));
}

int omt_box_mean_flow(const float *flow, int32_t w, int32_t h, const float *boxes, int32_t nboxes,
                      float *boxes_out, void *stream) {
    if (nboxes < 0 || w < 1 || h < 1) return OMT_EINVAL;
    if (nboxes == 0) return OMT_OK;
    if (!flow || !boxes || !boxes_out || !aligned(flow, 8) || !aligned(boxes, 16) ||
        !aligned(boxes_out, 16) || boxes == boxes_out)
        return OMT_EINVAL;
    return from_cuda(launch_box_mean_flow((const float2 *)flow, w, h, (const float4 *)boxes,
                                          nboxes, (float4 *)boxes_out, (cudaStream_t)stream));
}

int32_t omt_working_level(int32_t w, int32_t h) {
    (void)h;
    return w <= 1280 ? 0 : (w <= 2560 ? 1 : 2);
}

int omt_level_u8(const omt_pyramid *pyr, int32_t level, uint8_t *out, size_t pitch,
                 void *stream) {
    if (!pyr_ok(pyr) || pyr->storage != OMT_F32 || level < 0 || level >= pyr->levels || !out ||
        pitch < (size_t)pyr->lv[level].w)
        return OMT_EINVAL;
    return from_cuda(launch_level_u8(*pyr, level, out, pitch, (cudaStream_t)stream));
}

int omt_scale_boxes(const float *boxes, int32_t n, float scale, float *boxes_out, void *stream) {
    if (n < 0 || scale != scale) return OMT_EINVAL;
    if (n == 0) return OMT_OK;
    if (!boxes || !boxes_out || !aligned(boxes, 16) || !aligned(boxes_out, 16)) return OMT_EINVAL;
    return from_cuda(launch_scale_boxes((const float4 *)boxes, n, scale, (float4 *)boxes_out,
                                        (cudaStream_t)stream));
}

int omt_lk_wait_timeouts(uint32_t *count) {
    if (!count) return OMT_EINVAL;
    unsigned c = 0, cp = 0;
    int r = from_cuda(lk_wait_timeouts_take(&c));
    if (r == OMT_OK) r = from_cuda(pyr_wait_timeouts_take(&cp));
    c += cp;
    *count = c;
    if (r != OMT_OK) return r;
    return c ? OMT_ETIMEOUT : OMT_OK;
}

int omt_debug_fail_lk_wait(int64_t point) {
    return from_cuda(lk_fail_point_set(point < 0 ? -1 : (long long)point));
}

size_t omt_assign_workspace_bytes(int32_t na, int32_t nb) {
    if (na < 0 || nb < 0) return 0;
    return assign_workspace(na > nb ? na : nb);
}

int omt_assign(const double *iou, int32_t na, int32_t nb, const uint8_t *active, double iou_min,
               void *workspace, size_t workspace_bytes, int32_t *match_a, int32_t *match_b) {
    if (na < 0 || nb < 0 || iou_min != iou_min) return OMT_EINVAL;
    if ((na > 0 && !match_a) || (nb > 0 && !match_b) || (na > 0 && nb > 0 && !iou))
        return OMT_EINVAL;
    if (workspace_bytes < omt_assign_workspace_bytes(na, nb) || (!workspace && (na || nb)))
        return OMT_ENOMEM;
    assign_max_iou(iou, na, nb, active, iou_min, workspace, match_a, match_b);
    return OMT_OK;
}

int omt_update_tracks(const float *boxes_s, const uint8_t *active_s, int32_t ns,
                      const float *boxes_d, int32_t nd, const int32_t *match_s,
                      const int32_t *match_d, float *boxes_out, uint8_t *active_out,
                      int32_t *n_out) {
    if (ns < 0 || nd < 0 || !n_out) return OMT_EINVAL;
    if ((ns > 0 && (!boxes_s || !active_s || !match_s)) || (nd > 0 && (!boxes_d || !match_d)) ||
        (ns + nd > 0 && (!boxes_out || !active_out)))
        return OMT_EINVAL;
    int n = 0;
    for (int i = 0; i < ns; ++i, ++n) {
        const bool keep = active_s[i] && match_s[i] >= 0 && match_s[i] < nd;
        memcpy(boxes_out + 4 * n, keep ? boxes_d + 4 * match_s[i] : boxes_s + 4 * i, 4 * sizeof(float));
        active_out[n] = keep ? 1 : 0;
    }
    for (int j = 0; j < nd; ++j) {
        if (match_d[j] >= 0) continue;
        memcpy(boxes_out + 4 * n, boxes_d + 4 * j, 4 * sizeof(float));
        active_out[n++] = 1;
    }
    *n_out = n;
    return OMT_OK;
}

const char *omt_error_string(int32_t code) {
    switch (code) {
        case OMT_OK: return "success";
        case OMT_EINVAL: return "invalid argument";
        case OMT_ENOMEM: return "caller buffer too small";
        case OMT_ECUDA: return "CUDA launch or runtime error";
        case OMT_ETIMEOUT: return "bounded device wait timed out";
        case OMT_ECHECK: return "device-side check failed";
        default: return "unknown error";
    }
}

int32_t omt_version(void) { return kVersion; }

}  // extern "C"
