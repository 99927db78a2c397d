// Tile ranges (K4) and front-to-back compositing of RGB + depth (K5).
//
// Sec. III-A: after sorting, every screen tile owns a contiguous run of depth-ordered
// Gaussians and each pixel alpha-blends them front to back.  Sec. III-C: the depth image is
// produced the same way, by alpha-compositing the camera-space z of the Gaussians.
//
// One block per tile, one warp per 8x4 sub-tile, one thread per pixel.  A pixel stops at the
// first Gaussian that would drive its transmittance below t_min (that Gaussian is not
// composited); a warp stops once all of its pixels have.
#include "dgs_internal.cuh"

namespace dgs {
namespace {

// Thread = 4 consecutive sorted keys (one 16-byte load); a run starts where the key's tile
// differs from the one before and ends where it differs from the one after.
__global__ void k_ranges(const uint32_t* __restrict__ keys, uint32_t n, const uint32_t* __restrict__ d_n,
                         uint2* __restrict__ ranges, int n_tiles) {
    const uint32_t i4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4u;
    if (d_n) n = min(n, *d_n);
    if (i4 >= n) return;
    uint32_t k[6];                                  // k[0] = key before, k[5] = key after
    if (i4 + 4 <= n) {
        const uint4 q = *reinterpret_cast<const uint4*>(keys + i4);
        k[1] = q.x; k[2] = q.y; k[3] = q.z; k[4] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) k[1 + j] = i4 + j < n ? keys[i4 + j] : 0u;
    }
    k[0] = i4 > 0 ? keys[i4 - 1] : 0u;
    k[5] = i4 + 4 < n ? keys[i4 + 4] : 0u;
#pragma unroll
    for (int j = 0; j < 6; ++j) k[j] &= kTileMask;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t i = i4 + j;
        if (i >= n) break;
        const uint32_t t = k[1 + j];
        if (t >= (uint32_t)n_tiles) continue;       // dead pairs sort past every real tile
        if (i == 0 || k[j] != t) ranges[t].x = i;
        if (i + 1 == n || k[2 + j] != t) ranges[t].y = i + 1;
    }
}

// Block = one tile, warp = one 8x4 sub-tile, lane = one pixel.  Warps are independent (no
// block barrier): each walks the tile's list 32 entries at a time, keeps the entries whose
// sub-tile mask (written by binning: the ellipse reaches a pixel centre of the sub-tile, exact
// test with the binning margin) holds its bit -- one coalesced key load and a ballot per 32
// entries -- gathers their records into its own shared memory in list order and composites
// them; it stops once its 32 pixels have terminated.  AUG: the view's image randomisation is
// applied to the RGB before it is stored.
template <bool COUNT, bool AUG>
__global__ void __launch_bounds__(256, 6) k_composite(const ViewDesc* __restrict__ views, int v0, int nv,
                                                   const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
                                                   const uint32_t* __restrict__ vals,
                                                   const Record* __restrict__ rec, Params P, float* __restrict__ out_rgb,
                                                   float* __restrict__ out_depth, float* __restrict__ out_alpha,
                                                   unsigned long long* __restrict__ work) {
    __shared__ float4 s_rec[8][3][32];
    if (sort_failed(P.err)) return;            // the lists are not valid: nothing to composite
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
    const int sub_cols = P.tile_w >> 3;        // 8-pixel-wide sub-tiles per tile row
    const int wx0 = tx * P.tile_w + (w % sub_cols) * 8, wy0 = ty * P.tile_h + (w / sub_cols) * 4;
    const int wx1 = min(wx0 + 7, vd.W - 1), wy1 = min(wy0 + 3, vd.H - 1);
    if (wx0 > wx1 || wy0 > wy1) return;        // sub-tile outside the image
    const int px = wx0 + (lane & 7), py = wy0 + (lane >> 3);
    const bool inside = px < vd.W && py < vd.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 range = ranges[gt];
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    bool done = !inside;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t wbit = 1u << (kTileBits + w);
    float4* const sr0 = s_rec[w][0];
    float4* const sr1 = s_rec[w][1];
    float4* const sr2 = s_rec[w][2];
    uint32_t n_eval = 0, n_reach = 0, n_comp = 0;
    // the key and value of the next chunk are loaded while the current chunk composites, so a
    // chunk waits on one level of loads (its records) instead of three
    uint32_t key_n = 0, val_n = 0;
    if (range.x + lane < range.y) { key_n = __ldg(keys + range.x + lane); val_n = __ldg(vals + range.x + lane); }
    for (uint32_t base = range.x; base < range.y; base += 32) {
        if (__all_sync(0xffffffffu, done)) break;
        const uint32_t i = base + lane;
        const uint32_t val = val_n;
        // (debug builds check every entry of the range, whichever sub-tiles it reaches)
        const bool ok = i >= range.y || in_bounds(val, P.n_rec, P.err, kSiteCompositeRecord);
        const bool rel = i < range.y && (key_n & wbit) && ok;
        if (i + 32 < range.y) { key_n = __ldg(keys + i + 32); val_n = __ldg(vals + i + 32); }
        const uint32_t m = __ballot_sync(0xffffffffu, rel);
        if (m == 0) continue;
        if (rel) {
            const Record* r = rec + val;
            const float4 a = r->r0, q = r->r1, col = r->r2;
            const int pos = __popc(m & lt);
            sr0[pos] = a; sr2[pos] = col;
            sr1[pos] = make_float4(kHalfLog2e * q.x, q.y, kHalfLog2e * q.z, 0.f);
        }
        __syncwarp();
        const int n = __popc(m);
        if (COUNT) n_eval += done ? 0u : (uint32_t)n;
        for (int k = 0; k < n && !done; ++k) {
            const float4 g0 = sr0[k], g1 = sr1[k];
            float t;
            const float pe = pixel_exponent(g1.x, g1.y, g1.z, fx - g0.x, fy - g0.y, t);
            if (pe < P.p_min) continue;
            if (COUNT) ++n_reach;
            const float alpha = fminf(P.alpha_max, g0.z * fast_exp2(pe));
            if (alpha < P.alpha_min) continue;
            const float Tn = fmaf(-alpha, T, T);   // T (1 - alpha), one rounding
            if (Tn < P.t_min) { done = true; break; }
            if (COUNT) ++n_comp;
            const float wgt = alpha * T;
            const float4 g2 = sr2[k];
            C0 = fmaf(wgt, g2.x, C0); C1 = fmaf(wgt, g2.y, C1); C2 = fmaf(wgt, g2.z, C2);
            D = fmaf(wgt, g0.w, D);
            T = Tn;
        }
        __syncwarp();
    }
    if (COUNT) {
        const uint32_t a = __reduce_add_sync(0xffffffffu, n_eval), b = __reduce_add_sync(0xffffffffu, n_reach),
                       cc = __reduce_add_sync(0xffffffffu, n_comp);
        if (lane == 0) { atomicAdd(work + 0, a); atomicAdd(work + 1, b); atomicAdd(work + 2, cc); }
    }
    if (inside) {
        const int64_t p = vd.pix_off + (int64_t)py * vd.W + px;
        float r = fmaf(P.bg0, T, C0), g = fmaf(P.bg1, T, C1), b = fmaf(P.bg2, T, C2);
        if (AUG) {
            const dgs_augment& a = P.aug[lo];
            augment_pixel(a, a.overlay_beta != 0.f ? overlay_pixel(P.overlay, P.ov_w, P.ov_h, a, px, py) : nullptr,
                          r, g, b);
        }
        out_rgb[p * 3 + 0] = r;
        out_rgb[p * 3 + 1] = g;
        out_rgb[p * 3 + 2] = b;
        out_depth[p] = D;
        if (out_alpha) out_alpha[p] = 1.f - T;
    }
}

}  // namespace

void launch_ranges(const Launch& L, const uint32_t* keys, uint32_t n, uint2* ranges, int n_tiles,
                   const uint32_t* d_n) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, L.stream);
    if (n == 0) return;
    const uint32_t threads = (n + 3) / 4;
    k_ranges<<<(threads + 255) / 256, 256, 0, L.stream>>>(keys, n, d_n, ranges, n_tiles);
    ++*L.launches;
}

void launch_composite(const Launch& L, const ViewDesc* views, int v0, int n_group_views, int n_tiles,
                      const uint2* ranges, const uint32_t* keys, const uint32_t* vals, const Record* records,
                      const Params& P, float* out_rgb, float* out_depth, float* out_alpha, unsigned long long* work) {
    if (n_tiles == 0) return;
    auto* kern = work ? (P.aug ? k_composite<true, true> : k_composite<true, false>)
                      : (P.aug ? k_composite<false, true> : k_composite<false, false>);
    kern<<<n_tiles, P.tile_w * P.tile_h, 0, L.stream>>>(views, v0, n_group_views, ranges, keys, vals, records, P, out_rgb,
                                                        out_depth, out_alpha, work);
    ++*L.launches;
}

}  // namespace dgs
