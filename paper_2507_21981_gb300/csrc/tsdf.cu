// Depth -> TSDF fusion (Sec. III-B: a Gaussian node is turned back into a mesh by rendering
// multi-view depth maps and fusing them into a truncated signed distance field; the decimation
// that follows is not part of this library).
//
// A pre-pass writes every pixel's normalised depth d = D / A (NaN where A < min_alpha) into a
// packed array.  Then one thread per four consecutive voxels along x (one per voxel where the
// rows are not a multiple of four), x fastest (coalesced field reads and writes); each voxel
// takes the views in order: project the voxel centre, read d at the pixel holding
// the projection, sdf = d - z, skip when sdf < -trunc, f = min(1, sdf / trunc),
// F <- (W F + f) / (W + 1), W <- min(W + 1, max_weight).
// The field is read and written once per call whatever the number of views, so a call with
// many views is bound by the per-view arithmetic and the depth gathers (served by L2).
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kTsdfThreads = 256;

// Pre-pass: the normalised depth D / A of every pixel of every view into a packed array (NaN
// where A < min_alpha), so that the fusion makes one gather per (voxel, view) and no division.
// Thread = packed pixel q; views[v].q0 = first packed pixel of view v.
__global__ void __launch_bounds__(kTsdfThreads) k_tsdf_depth(const TsdfView* __restrict__ views, int V, int64_t n_pix,
                                                             float min_alpha, const float* __restrict__ depth,
                                                             const float* __restrict__ alpha, float* __restrict__ dn) {
    const int64_t q = (int64_t)blockIdx.x * kTsdfThreads + threadIdx.x;
    if (q >= n_pix) return;
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].q0 <= q) lo = mid; else hi = mid - 1;
    }
    const int64_t p = views[lo].pix_off + (q - views[lo].q0);
    const float a = alpha[p];
    dn[q] = a >= min_alpha ? __fdividef(depth[p], a) : __int_as_float(0x7fc00000);
}

// The block first copies the view table (up to kSmemViews views) into shared memory, so that
// the per-view camera fields are shared-memory broadcasts rather than cached global loads.
constexpr int kSmemViews = 64;

__global__ void __launch_bounds__(kTsdfThreads) k_tsdf(float* __restrict__ F, float* __restrict__ Wt, int nx, int ny,
                                                       int64_t n_vox, TsdfParams TP, const TsdfView* __restrict__ gviews,
                                                       int V, const float* __restrict__ dn) {
    __shared__ TsdfView s_views[kSmemViews];
    const bool in_smem = V <= kSmemViews;
    if (in_smem) {
        const int words = V * (int)(sizeof(TsdfView) / 4);
        const uint32_t* src = reinterpret_cast<const uint32_t*>(gviews);
        uint32_t* dst = reinterpret_cast<uint32_t*>(s_views);
        for (int w = threadIdx.x; w < words; w += kTsdfThreads) dst[w] = src[w];
        __syncthreads();
    }
    const TsdfView* __restrict__ views = in_smem ? s_views : gviews;
    const int64_t idx = (int64_t)blockIdx.x * kTsdfThreads + threadIdx.x;
    if (idx >= n_vox) return;
    const int i = (int)(idx % nx);
    const int64_t r = idx / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    const float px = fmaf((float)i + 0.5f, TP.voxel, TP.ox), py = fmaf((float)j + 0.5f, TP.voxel, TP.oy),
                pz = fmaf((float)k + 0.5f, TP.voxel, TP.oz);
    float f = F[idx], w = Wt[idx];
    for (int v = 0; v < V; ++v) {
        const TsdfView& cv = views[v];
        const float z = fmaf(cv.R[6], px, fmaf(cv.R[7], py, fmaf(cv.R[8], pz, cv.t[2])));
        if (!(z > 0.f)) continue;
        const float x = fmaf(cv.R[0], px, fmaf(cv.R[1], py, fmaf(cv.R[2], pz, cv.t[0])));
        const float y = fmaf(cv.R[3], px, fmaf(cv.R[4], py, fmaf(cv.R[5], pz, cv.t[1])));
        const float iz = __fdividef(1.f, z);
        const float u = fmaf(cv.fx * x, iz, cv.cx), vv = fmaf(cv.fy * y, iz, cv.cy);
        if (!(u >= 0.f) || !(vv >= 0.f) || !(u < (float)cv.W) || !(vv < (float)cv.H)) continue;
        const float d = __ldg(dn + cv.q0 + (int64_t)(int)vv * cv.W + (int)u);
        const float sdf = d - z;
        if (!(sdf >= -TP.trunc)) continue;              // also a pixel without coverage (NaN)
        const float fv = fminf(1.f, sdf * TP.inv_trunc);
        f = __fdividef(fmaf(w, f, fv), w + 1.f);
        w = fminf(w + 1.f, TP.max_weight);
    }
    F[idx] = f;
    Wt[idx] = w;
}

// Four consecutive voxels along x per thread (nx a multiple of 4, 16-byte aligned fields): the
// view's fields are read once for the four, the camera-space centre steps along x by the view's
// first rotation column times the voxel size, and the four projections are made before the
// four depth gathers, which are then in flight together.  Each voxel takes the views in order
// with the per-voxel update of k_tsdf.
__global__ void __launch_bounds__(kTsdfThreads) k_tsdf4(float* __restrict__ F, float* __restrict__ Wt, int nx, int ny,
                                                        int64_t n_vox, TsdfParams TP, const TsdfView* __restrict__ gviews,
                                                        int V, const float* __restrict__ dn) {
    __shared__ TsdfView s_views[kSmemViews];
    const bool in_smem = V <= kSmemViews;
    if (in_smem) {
        const int words = V * (int)(sizeof(TsdfView) / 4);
        const uint32_t* src = reinterpret_cast<const uint32_t*>(gviews);
        uint32_t* dst = reinterpret_cast<uint32_t*>(s_views);
        for (int w = threadIdx.x; w < words; w += kTsdfThreads) dst[w] = src[w];
        __syncthreads();
    }
    const TsdfView* __restrict__ views = in_smem ? s_views : gviews;
    const int64_t idx = ((int64_t)blockIdx.x * kTsdfThreads + threadIdx.x) * 4;
    if (idx >= n_vox) return;
    const int i = (int)(idx % nx);
    const int64_t r = idx / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    const float px = fmaf((float)i + 0.5f, TP.voxel, TP.ox), py = fmaf((float)j + 0.5f, TP.voxel, TP.oy),
                pz = fmaf((float)k + 0.5f, TP.voxel, TP.oz);
    const float4 f4 = *reinterpret_cast<const float4*>(F + idx), w4 = *reinterpret_cast<const float4*>(Wt + idx);
    float f[4] = {f4.x, f4.y, f4.z, f4.w}, w[4] = {w4.x, w4.y, w4.z, w4.w};
    for (int v = 0; v < V; ++v) {
        const TsdfView& cv = views[v];
        const float z0 = fmaf(cv.R[6], px, fmaf(cv.R[7], py, fmaf(cv.R[8], pz, cv.t[2])));
        const float x0 = fmaf(cv.R[0], px, fmaf(cv.R[1], py, fmaf(cv.R[2], pz, cv.t[0])));
        const float y0 = fmaf(cv.R[3], px, fmaf(cv.R[4], py, fmaf(cv.R[5], pz, cv.t[1])));
        const float sx = cv.R[0] * TP.voxel, sy = cv.R[3] * TP.voxel, sz = cv.R[6] * TP.voxel;
        float zm[4], d[4];
        int64_t pix[4];
        bool ok[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float z = fmaf((float)m, sz, z0);
            const float x = fmaf((float)m, sx, x0), y = fmaf((float)m, sy, y0);
            const float iz = __fdividef(1.f, z);
            const float u = fmaf(cv.fx * x, iz, cv.cx), vv = fmaf(cv.fy * y, iz, cv.cy);
            ok[m] = z > 0.f && u >= 0.f && vv >= 0.f && u < (float)cv.W && vv < (float)cv.H;
            pix[m] = ok[m] ? cv.q0 + (int64_t)(int)vv * cv.W + (int)u : 0;
            zm[m] = z;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) d[m] = ok[m] ? __ldg(dn + pix[m]) : 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float sdf = d[m] - zm[m];
            if (!ok[m] || !(sdf >= -TP.trunc)) continue;    // also a pixel without coverage (NaN)
            const float fv = fminf(1.f, sdf * TP.inv_trunc);
            f[m] = __fdividef(fmaf(w[m], f[m], fv), w[m] + 1.f);
            w[m] = fminf(w[m] + 1.f, TP.max_weight);
        }
    }
    *reinterpret_cast<float4*>(F + idx) = make_float4(f[0], f[1], f[2], f[3]);
    *reinterpret_cast<float4*>(Wt + idx) = make_float4(w[0], w[1], w[2], w[3]);
}

}  // namespace

void launch_tsdf(const Launch& L, float* F, float* W, int nx, int ny, int64_t n_vox, const TsdfParams& TP,
                 const TsdfView* views, int V, const float* depth, const float* alpha, float* dn, int64_t n_pix) {
    if (n_vox <= 0 || n_pix <= 0) return;
    k_tsdf_depth<<<(unsigned)((n_pix + kTsdfThreads - 1) / kTsdfThreads), kTsdfThreads, 0, L.stream>>>(
        views, V, n_pix, TP.min_alpha, depth, alpha, dn);
    const bool quads = nx % 4 == 0 && reinterpret_cast<uintptr_t>(F) % 16 == 0 && reinterpret_cast<uintptr_t>(W) % 16 == 0;
    if (quads)
        k_tsdf4<<<(unsigned)((n_vox / 4 + kTsdfThreads - 1) / kTsdfThreads), kTsdfThreads, 0, L.stream>>>(
            F, W, nx, ny, n_vox, TP, views, V, dn);
    else
        k_tsdf<<<(unsigned)((n_vox + kTsdfThreads - 1) / kTsdfThreads), kTsdfThreads, 0, L.stream>>>(F, W, nx, ny, n_vox,
                                                                                                     TP, views, V, dn);
    *L.launches += 2;
}

}  // namespace dgs
