// Tile ranges (K4) and front-to-back compositing of RGB + depth (K5).
//
// Sec. III-A: after sorting, every screen tile owns a contiguous run of depth-ordered
// Gaussians and each pixel alpha-blends them front to back.  Sec. III-C: the depth image is
// produced the same way, by alpha-compositing the camera-space z of the Gaussians.
//
// One block per tile, one thread per pixel.  The block walks its run in batches of
// blockDim records staged in shared memory; a pixel stops at the first Gaussian that would
// drive its transmittance below t_min (that Gaussian is not composited) and the block leaves
// the loop once all of its pixels have stopped (__syncthreads_count).
#include "dgs_internal.cuh"

namespace dgs {
namespace {

__global__ void k_ranges(const uint64_t* __restrict__ keys, uint32_t n, uint2* __restrict__ ranges, int n_tiles) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t t = keys[i] >> kZBits;
    if (t >= (uint64_t)n_tiles) return;   // dead pairs sort past every real tile
    if (i == 0 || (keys[i - 1] >> kZBits) != t) ranges[t].x = i;
    if (i + 1 == n || (keys[i + 1] >> kZBits) != t) ranges[t].y = i + 1;
}

__global__ void __launch_bounds__(256) k_composite(const ViewDesc* __restrict__ views, int v0, int nv,
                                                   const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                                   const Record* __restrict__ rec, Params P, float* __restrict__ out_rgb,
                                                   float* __restrict__ out_depth, float* __restrict__ out_alpha) {
    __shared__ float4 s0[256], s1[256], s2[256];
    const int gt = blockIdx.x;                 // tile within the group
    const int ga = gt + P.tile0;               // tile within the call
    // view of this tile: last view of the group whose tile_base <= ga
    int lo = v0, hi = v0 + nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= ga) lo = mid; else hi = mid - 1;
    }
    const ViewDesc& vd = views[lo];
    const int tile = ga - vd.tile_base;
    const int tx = tile % vd.tiles_x, ty = tile / vd.tiles_x;
    const int lx = threadIdx.x % P.tile_w, ly = threadIdx.x / P.tile_w;
    const int px = tx * P.tile_w + lx, py = ty * P.tile_h + ly;
    const bool inside = px < vd.W && py < vd.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 range = ranges[gt];
    const int nthreads = blockDim.x;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    bool done = !inside;
    for (uint32_t b = range.x; b < range.y; b += nthreads) {
        if (__syncthreads_count(done) == nthreads) break;
        const uint32_t i = b + threadIdx.x;
        if (i < range.y) {
            const Record& r = rec[vals[i]];
            s0[threadIdx.x] = r.r0;
            s1[threadIdx.x] = r.r1;
            s2[threadIdx.x] = r.r2;
        }
        __syncthreads();
        const int cnt = (int)umin((uint32_t)nthreads, range.y - b);
        for (int j = 0; j < cnt && !done; ++j) {
            const float4 a = s0[j], c = s1[j];
            const float dx = fx - a.x, dy = fy - a.y;
            const float t = fmaf(c.y, dy, dx);
            const float q = fmaf(c.x * t, t, c.z * dy * dy);
            if (q > P.q_max) continue;
            const float alpha = fminf(P.alpha_max, a.z * __expf(-0.5f * q));
            if (alpha < P.alpha_min) continue;
            const float Tn = T * (1.f - alpha);
            if (Tn < P.t_min) { done = true; break; }
            const float w = alpha * T;
            const float4 col = s2[j];
            C0 = fmaf(w, col.x, C0); C1 = fmaf(w, col.y, C1); C2 = fmaf(w, col.z, C2);
            D = fmaf(w, a.w, D);
            T = Tn;
        }
        __syncthreads();
    }
    if (inside) {
        const int64_t p = vd.pix_off + (int64_t)py * vd.W + px;
        out_rgb[p * 3 + 0] = fmaf(P.bg0, T, C0);
        out_rgb[p * 3 + 1] = fmaf(P.bg1, T, C1);
        out_rgb[p * 3 + 2] = fmaf(P.bg2, T, C2);
        out_depth[p] = D;
        if (out_alpha) out_alpha[p] = 1.f - T;
    }
}

}  // namespace

void launch_ranges(const Launch& L, const uint64_t* keys, uint32_t n, uint2* ranges, int n_tiles) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, L.stream);
    if (n == 0) return;
    k_ranges<<<(n + 255) / 256, 256, 0, L.stream>>>(keys, n, ranges, n_tiles);
    ++*L.launches;
}

void launch_composite(const Launch& L, const ViewDesc* views, int v0, int n_group_views, int n_tiles,
                      const uint2* ranges, const uint32_t* vals, const Record* records, const Params& P,
                      float* out_rgb, float* out_depth, float* out_alpha) {
    if (n_tiles == 0) return;
    k_composite<<<n_tiles, P.tile_w * P.tile_h, 0, L.stream>>>(views, v0, n_group_views, ranges, vals, records, P,
                                                               out_rgb, out_depth, out_alpha);
    ++*L.launches;
}

}  // namespace dgs
