// match.cu -- matching and update phases (Section V-A): the IoU of every
// predicted scene object against every detection (device, FP64 with no
// fused operations, so the matrix is reproducible bit for bit), the
// globally optimal assignment of the IoU score (host, the Hungarian method
// of Kuhn 1955 as shortest augmenting paths over column potentials), and
// the update of the scene-object list.
#include <math.h>
#include <string.h>

#include "omt_internal.cuh"

namespace omt {
namespace {

constexpr int MT = 16;  // a CTA computes a 16 x 16 block of pairs

// IoU of two half-open boxes: areas of the clipped extents, the
// intersection's extents clipped at 0, union = (area_a + area_b) - inter.
__device__ __forceinline__ double iou_pair(float4 a, float4 b) {
    const double aw = fmax(__dsub_rn(a.z, a.x), 0.0), ah = fmax(__dsub_rn(a.w, a.y), 0.0);
    const double bw = fmax(__dsub_rn(b.z, b.x), 0.0), bh = fmax(__dsub_rn(b.w, b.y), 0.0);
    const double iw = fmax(__dsub_rn(fmin((double)a.z, (double)b.z), fmax((double)a.x, (double)b.x)), 0.0);
    const double ih = fmax(__dsub_rn(fmin((double)a.w, (double)b.w), fmax((double)a.y, (double)b.y)), 0.0);
    const double inter = __dmul_rn(iw, ih);
    const double uni = __dsub_rn(__dadd_rn(__dmul_rn(aw, ah), __dmul_rn(bw, bh)), inter);
    return uni > 0.0 ? __ddiv_rn(inter, uni) : 0.0;
}

__global__ void __launch_bounds__(MT * MT) iou_kernel(const float4 *a, int na, const float4 *b, int nb,
                                                      double *out) {
    __shared__ float4 sa[MT], sb[MT];
    const int i0 = blockIdx.y * MT, j0 = blockIdx.x * MT;
    const int t = threadIdx.y * MT + threadIdx.x;
    if (t < MT && i0 + t < na) sa[t] = a[i0 + t];
    if (t >= MT && t < 2 * MT && j0 + t - MT < nb) sb[t - MT] = b[j0 + t - MT];
    __syncthreads();
    const int i = i0 + threadIdx.y, j = j0 + threadIdx.x;
    if (i < na && j < nb) out[(int64_t)i * nb + j] = iou_pair(sa[threadIdx.y], sb[threadIdx.x]);
}

}  // namespace

cudaError_t launch_iou_matrix(const float *a, int na, const float *b, int nb, double *out,
                              cudaStream_t s) {
    if (na == 0 || nb == 0) return cudaSuccess;
    dim3 grid((nb + MT - 1) / MT, (na + MT - 1) / MT), block(MT, MT);
    iou_kernel<<<grid, block, 0, s>>>((const float4 *)a, na, (const float4 *)b, nb, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ assignment
// Minimum-cost perfect matching of an n x n matrix given by cost(i, j), by
// successive shortest augmenting paths: each row in turn is joined to the
// matching by a Dijkstra search over the columns with reduced costs
// cost(i, j) - v[j] (v: column potentials, updated after each search so
// that reduced costs stay non-negative on the matched edges), then the path
// is flipped.  O(n^3) time, O(n) memory in `ws`.
struct AssignWork {
    double *v, *dist;
    int *row_of_col, *col_of_row, *pred;
    unsigned char *scanned;
};

size_t assign_workspace(int n) {
    return (size_t)(n + 1) * (2 * sizeof(double) + 3 * sizeof(int) + 1) + 64;
}

template <typename Cost>
static void shortest_path_assign(int n, Cost cost, AssignWork w) {
    for (int j = 0; j < n; ++j) {
        w.v[j] = 0.0;
        w.row_of_col[j] = -1;
    }
    for (int i = 0; i < n; ++i) w.col_of_row[i] = -1;
    for (int f = 0; f < n; ++f) {
        for (int j = 0; j < n; ++j) {
            w.dist[j] = cost(f, j) - w.v[j];
            w.pred[j] = f;
            w.scanned[j] = 0;
        }
        int sink = -1;
        double mu = 0.0;
        int nscan = 0;
        while (sink < 0) {
            // the closest unscanned column (lowest index among equals)
            int jm = -1;
            for (int j = 0; j < n; ++j)
                if (!w.scanned[j] && (jm < 0 || w.dist[j] < w.dist[jm])) jm = j;
            mu = w.dist[jm];
            w.scanned[jm] = 1;
            ++nscan;
            const int i = w.row_of_col[jm];
            if (i < 0) {
                sink = jm;
                break;
            }
            // relax through the row matched to jm
            const double base = mu - (cost(i, jm) - w.v[jm]);
            for (int k = 0; k < n; ++k) {
                if (w.scanned[k]) continue;
                const double alt = base + cost(i, k) - w.v[k];
                if (alt < w.dist[k]) {
                    w.dist[k] = alt;
                    w.pred[k] = i;
                }
            }
        }
        // potentials of the scanned columns keep reduced costs non-negative
        for (int j = 0; j < n; ++j)
            if (w.scanned[j] && j != sink) w.v[j] += w.dist[j] - mu;
        // flip the path from the sink back to row f
        int j = sink;
        for (;;) {
            const int i = w.pred[j];
            w.row_of_col[j] = i;
            const int prev = w.col_of_row[i];
            w.col_of_row[i] = j;
            if (i == f) break;
            j = prev;
        }
    }
}

void assign_max_iou(const double *iou, int na, int nb, const uint8_t *active, double iou_min,
                    void *ws, int32_t *match_a, int32_t *match_b) {
    for (int i = 0; i < na; ++i) match_a[i] = -1;
    for (int j = 0; j < nb; ++j) match_b[j] = -1;
    const int n = na > nb ? na : nb;
    if (n == 0) return;
    uint8_t *p = (uint8_t *)(((uintptr_t)ws + 15) & ~(uintptr_t)15);
    AssignWork w;
    w.v = (double *)p;
    w.dist = w.v + (n + 1);
    w.row_of_col = (int *)(w.dist + (n + 1));
    w.col_of_row = w.row_of_col + (n + 1);
    w.pred = w.col_of_row + (n + 1);
    w.scanned = (unsigned char *)(w.pred + (n + 1));
    // score 0 on the padding and on inactive rows; minimise the negated IoU
    auto cost = [&](int i, int j) -> double {
        if (i >= na || j >= nb || (active && !active[i])) return 0.0;
        return -iou[(size_t)i * nb + j];
    };
    shortest_path_assign(n, cost, w);
    for (int i = 0; i < na; ++i) {
        const int j = w.col_of_row[i];
        if (j < nb && (!active || active[i]) && iou[(size_t)i * nb + j] > iou_min) {
            match_a[i] = j;
            match_b[j] = i;
        }
    }
}

}  // namespace omt
