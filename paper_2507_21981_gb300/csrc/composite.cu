// Tile ranges (K4) and front-to-back compositing of RGB + depth (K5).
//
// Sec. III-A: after sorting, every screen tile owns a contiguous run of depth-ordered
// Gaussians and each pixel alpha-blends them front to back.  Sec. III-C: the depth image is
// produced the same way, by alpha-compositing the camera-space z of the Gaussians.
//
// One block per tile, one thread per pixel, one warp per 8x4 sub-tile.  The block walks its run
// in batches of blockDim records staged in shared memory; a pixel stops at the first Gaussian
// that would drive its transmittance below t_min (that Gaussian is not composited) and the
// block leaves the loop once all of its pixels have stopped (__syncthreads_count).
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

// Does the ellipse {d^T Q d <= qlim}, Q = [[a, b], [b, c]], reach the rectangle of pixel
// centres [X0, X1] x [Y0, Y1] (relative to the mean)?  Minimum of q over the rectangle: 0 if
// the mean is inside, else the smallest of the four edge minima.
__device__ __forceinline__ bool ellipse_meets(float a, float b, float c, float ia, float ic, float qlim, float X0,
                                              float X1, float Y0, float Y1) {
    if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return true;
    float m = INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float X = e ? X1 : X0;
        const float Y = fminf(Y1, fmaxf(Y0, -b * X * ic));
        m = fminf(m, fmaf(a * X, X, fmaf(2.f * b * X, Y, c * Y * Y)));
        const float Yh = e ? Y1 : Y0;
        const float Xh = fminf(X1, fmaxf(X0, -b * Yh * ia));
        m = fminf(m, fmaf(a * Xh, Xh, fmaf(2.f * b * Xh, Yh, c * Yh * Yh)));
    }
    return m <= qlim;
}

// Block = one tile, warp = one 8x4 sub-tile of it, lane = one pixel.  Per batch of staged
// records the loader thread of each record computes the set of sub-tiles its ellipse can reach
// (box overlap, then the exact ellipse-rectangle test with the binning margin), and every warp
// evaluates only the records whose bit it holds, in list order.
__global__ void __launch_bounds__(256) k_composite(const ViewDesc* __restrict__ views, int v0, int nv,
                                                   const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                                   const Record* __restrict__ rec, Params P, float* __restrict__ out_rgb,
                                                   float* __restrict__ out_depth, float* __restrict__ out_alpha) {
    __shared__ float4 s0[256], s1[256], s2[256];
    __shared__ uint32_t s_mask[256];
    __shared__ uint8_t s_list[8][256];
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
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int sub_cols = P.tile_w >> 3;        // 8-pixel-wide sub-tiles per tile row
    const int tile_x0 = tx * P.tile_w, tile_y0 = ty * P.tile_h;
    const int wx0 = tile_x0 + (w % sub_cols) * 8, wy0 = tile_y0 + (w / sub_cols) * 4;
    const int px = wx0 + (lane & 7), py = wy0 + (lane >> 3);
    const bool inside = px < vd.W && py < vd.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 range = ranges[gt];
    const int nthreads = blockDim.x;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    bool done = !inside;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t b = range.x; b < range.y; b += nthreads) {
        if (__syncthreads_count(done) == nthreads) break;
        const uint32_t i = b + threadIdx.x;
        if (i < range.y) {
            const Record& r = rec[vals[i]];
            const float4 a = r.r0, q = r.r1;
            s0[threadIdx.x] = a;
            s1[threadIdx.x] = q;
            s2[threadIdx.x] = r.r2;
            // conic of the factored form q = qa (dx + qb dy)^2 + qc dy^2 and its pixel box
            const float ca = q.x, cb = q.x * q.y, cc = fmaf(q.x * q.y, q.y, q.z);
            const float hx = sqrtf(P.qbin * (q.y * q.y / q.z + 1.f / q.x)), hy = sqrtf(P.qbin / q.z);
            const float ia = 1.f / ca, ic = 1.f / cc;
            uint32_t m = 0;
            for (int k = 0; k < nwarps; ++k) {
                const int X0 = tile_x0 + (k % sub_cols) * 8, Y0 = tile_y0 + (k / sub_cols) * 4;
                const int X1 = min(X0 + 7, vd.W - 1), Y1 = min(Y0 + 3, vd.H - 1);
                if (X0 > X1 || Y0 > Y1) continue;
                const float dx0 = (float)X0 + 0.5f - a.x, dx1 = (float)X1 + 0.5f - a.x;
                const float dy0 = (float)Y0 + 0.5f - a.y, dy1 = (float)Y1 + 0.5f - a.y;
                if (dx0 > hx || dx1 < -hx || dy0 > hy || dy1 < -hy) continue;
                if (ellipse_meets(ca, cb, cc, ia, ic, P.qbin, dx0, dx1, dy0, dy1)) m |= 1u << k;
            }
            s_mask[threadIdx.x] = m;
        }
        __syncthreads();
        // this warp's records of the batch, in list order
        const int cnt = (int)umin((uint32_t)nthreads, range.y - b);
        int n_mine = 0;
        for (int base = 0; base < cnt; base += 32) {
            const int j = base + lane;
            const bool rel = j < cnt && ((s_mask[j] >> w) & 1u);
            const uint32_t bal = __ballot_sync(0xffffffffu, rel);
            if (rel) s_list[w][n_mine + __popc(bal & lt)] = (uint8_t)j;
            n_mine += __popc(bal);
        }
        __syncwarp();
        for (int k = 0; k < n_mine && !done; ++k) {
            const int j = s_list[w][k];
            const float4 a = s0[j], c = s1[j];
            const float dx = fx - a.x, dy = fy - a.y;
            const float t = fmaf(c.y, dy, dx);
            const float q = fmaf(c.x * t, t, c.z * dy * dy);
            if (q > P.q_max) continue;
            const float alpha = fminf(P.alpha_max, a.z * __expf(-0.5f * q));
            if (alpha < P.alpha_min) continue;
            const float Tn = T * (1.f - alpha);
            if (Tn < P.t_min) { done = true; break; }
            const float wgt = alpha * T;
            const float4 col = s2[j];
            C0 = fmaf(wgt, col.x, C0); C1 = fmaf(wgt, col.y, C1); C2 = fmaf(wgt, col.z, C2);
            D = fmaf(wgt, a.w, D);
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
