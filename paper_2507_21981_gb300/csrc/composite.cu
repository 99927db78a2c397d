// Tile ranges (K4) and front-to-back compositing of RGB + depth (K5).
//
// Sec. III-A: after sorting, every screen tile owns a contiguous run of depth-ordered
// Gaussians and each pixel alpha-blends them front to back.  Sec. III-C: the depth image is
// produced the same way, by alpha-compositing the camera-space z of the Gaussians.
//
// Two warps per block (two 8x4 sub-tiles of one tile), one thread per pixel.  A pixel stops at the
// first Gaussian that would drive its transmittance below t_min (that Gaussian is not
// composited); a warp stops once all of its pixels have.
#include <algorithm>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

// Thread = 4 consecutive sorted keys at a time (one 16-byte load), grid-stride over the live
// keys (the grid is sized for the capacity, at most a few waves); a run starts where the key's
// tile differs from the one before and ends where it differs from the one after.  A key names
// (view in group, tile in view); its tile in the group is the view's first tile + tile in view.
__global__ void k_ranges(const uint32_t* __restrict__ keys, uint32_t n, const uint32_t* __restrict__ d_n,
                         uint2* __restrict__ ranges, int n_tiles, const ViewDesc* __restrict__ views, int v0, int nv,
                         int tile0, int tbits) {
    if (d_n) n = min(n, *d_n);
    const uint32_t stride = gridDim.x * blockDim.x * 4u;
    for (uint32_t i4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4u; i4 < n; i4 += stride) {
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
        const bool first = i == 0 || k[j] != t, last = i + 1 == n || k[2 + j] != t;
        if (!first && !last) continue;              // the view is decoded at run ends only
        const uint32_t vg = t >> tbits;
        if (vg >= (uint32_t)nv) continue;           // dead pairs sort past every real tile
        const uint32_t gt = (uint32_t)(views[v0 + vg].tile_base - tile0) + (t & ((1u << tbits) - 1u));
        if (gt >= (uint32_t)n_tiles) continue;      // (only keys of a sort that gave up waiting)
        if (first) ranges[gt].x = i;
        if (last) ranges[gt].y = i + 1;
    }
    }
}

// Heaviest tiles first (the longest-processing-time rule of list scheduling): a view group with
// few waves of tiles is otherwise finished by the blocks of its longest lists while most SMs
// idle, so the compositors take their tiles in descending order of list length, bucketed at 8
// steps per octave of length.  One block; within a bucket the order is arbitrary.
__device__ __forceinline__ uint32_t length_bucket(uint2 r) {
    const uint32_t c = r.y - r.x + 1u;              // >= 1
    const uint32_t oct = 31u - (uint32_t)__clz(c);  // floor(log2 c), 0..31
    const uint32_t frac = oct >= 3 ? (c >> (oct - 3)) & 7u : (c << (3 - oct)) & 7u;
    return 255u - min(255u, oct * 8u + frac);       // heaviest first
}

__global__ void __launch_bounds__(1024) k_tile_order(const uint2* __restrict__ ranges, int n_tiles, uint32_t* order) {
    __shared__ uint32_t cnt[256];
    if (threadIdx.x < 256) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) atomicAdd(&cnt[length_bucket(ranges[t])], 1u);
    __syncthreads();
    if (threadIdx.x < 32) {                         // exclusive scan of the 256 counts, 8 per lane
        const int lane = threadIdx.x;
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) { v[j] = cnt[lane * 8 + j]; sum += v[j]; }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int j = 0; j < 8; ++j) { cnt[lane * 8 + j] = run; run += v[j]; }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) order[atomicAdd(&cnt[length_bucket(ranges[t])], 1u)] = t;
}

// One block: every tile's first checkpoint slot (an exclusive scan of its segments after the
// first, in tile order), then the (tile, segment) jobs of the adjoint in descending order of
// their length, bucketed as above; *n_jobs = their number.
__global__ void __launch_bounds__(1024) k_segment_jobs(const uint2* __restrict__ ranges, int n_tiles, Checkpoints ck) {
    __shared__ uint32_t cnt[256];
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto n_seg = [&](int t) { const uint2 r = ranges[t]; return (r.y - r.x + kSegEntries - 1) / kSegEntries; };
    if (tid < 256) cnt[tid] = 0;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int t0 = 0; t0 < n_tiles; t0 += blockDim.x) {
        const int t = t0 + tid;
        const uint32_t v = t < n_tiles ? max(n_seg(t), 1u) - 1u : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        uint32_t pre = s_carry, all = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            if (q < warp) pre += s_w[q];
            all += s_w[q];
        }
        if (t < n_tiles) ck.off[t] = pre + x - v;
        __syncthreads();
        if (tid == 0) s_carry += all;
        __syncthreads();
    }
    for (int t = tid; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t ns = n_seg(t);
        for (uint32_t sg = 0; sg < ns; ++sg) {
            const uint32_t a = r.x + sg * kSegEntries;
            atomicAdd(&cnt[length_bucket(make_uint2(a, min(r.y, a + kSegEntries) - 1u))], 1u);
        }
    }
    __syncthreads();
    if (tid < 32) {
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) { v[j] = cnt[tid * 8 + j]; sum += v[j]; }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int j = 0; j < 8; ++j) { cnt[tid * 8 + j] = run; run += v[j]; }
        if (tid == 31) *ck.n_jobs = run;
    }
    __syncthreads();
    for (int t = tid; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t ns = n_seg(t);
        for (uint32_t sg = 0; sg < ns; ++sg) {
            const uint32_t a = r.x + sg * kSegEntries;
            const uint32_t b = length_bucket(make_uint2(a, min(r.y, a + kSegEntries) - 1u));
            ck.jobs[atomicAdd(&cnt[b], 1u)] = make_uint2((uint32_t)t, sg);
        }
    }
}

// Block = kCompWarps sub-tiles of one tile, warp = one 8x4 sub-tile, lane = one pixel.  Warps are independent (no
// block barrier): each walks the tile's list 32 entries at a time, keeps the entries whose
// sub-tile mask (written by binning: the ellipse reaches a pixel centre of the sub-tile, exact
// test with the binning margin) holds its bit -- one coalesced key load and a ballot per 32
// entries -- gathers their records into its own shared memory in list order and composites
// them; it stops once its 32 pixels have terminated.  AUG: the view's image randomisation is
// applied to the RGB before it is stored.  CK: the per-pixel state is checkpointed at every
// segment start for the adjoint (see Checkpoints).
template <bool COUNT, bool AUG, bool CK>
__global__ void __launch_bounds__(kCompWarps * 32, (COUNT || AUG || CK) ? 20 : 24) k_composite(const ViewDesc* __restrict__ views, int v0, int nv,
                                                   const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
                                                   const uint32_t* __restrict__ vals,
                                                   const Record* __restrict__ rec, Params P, float* __restrict__ out_rgb,
                                                   float* __restrict__ out_depth, float* __restrict__ out_alpha,
                                                   unsigned long long* __restrict__ work,
                                                   const uint32_t* __restrict__ tile_order, Checkpoints ck) {
    __shared__ float4 s_rec[kCompWarps][3][32];
    if (sort_failed(P.err)) return;            // the lists are not valid: nothing to composite
    // kCompWarps sub-tiles of one tile per block: a block frees its slot as soon as its own
    // warps end, not when the tile's slowest sub-tile does
    const int bpt = (P.tile_w * P.tile_h) / (32 * kCompWarps);   // blocks per tile
    const int tb = (int)blockIdx.x / bpt;
    const int gt = tile_order ? (int)tile_order[tb] : tb;        // tile within the group
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
    const int lane = threadIdx.x & 31, bw = threadIdx.x >> 5;
    const int w = ((int)blockIdx.x - tb * bpt) * kCompWarps + bw;   // sub-tile within the tile
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
    float4* const sr0 = s_rec[bw][0];
    float4* const sr1 = s_rec[bw][1];
    float4* const sr2 = s_rec[bw][2];
    uint32_t n_eval = 0, n_reach = 0, n_comp = 0;
    // the key and value of the next chunk are loaded while the current chunk composites, so a
    // chunk waits on one level of loads (its records) instead of three
    uint32_t key_n = 0, val_n = 0;
    if (range.x + lane < range.y) { key_n = __ldg(keys + range.x + lane); val_n = __ldg(vals + range.x + lane); }
    const int n_sub = P.tile_w * P.tile_h / 32;
    uint32_t entered = 0, chunk = 0;            // segments entered, chunk index in the list
    for (uint32_t base = range.x; base < range.y; base += 32, ++chunk) {
        if (__all_sync(0xffffffffu, done)) break;
        if (CK && chunk % kSegChunks == 0) {      // a segment starts: the adjoint's checkpoint
            entered = chunk / kSegChunks + 1;
            if (chunk > 0)
                ck.st[((size_t)(ck.off[gt] + entered - 2) * n_sub + w) * 32 + lane] =
                    CkState{T, C0, C1, C2, D, done ? 1.f : 0.f};
        }
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
            sr1[pos] = make_float4(kHalfLog2e * q.x, q.y, kHalfLog2e * q.z, reach_threshold(P, a.z));
        }
        __syncwarp();
        const int n = __popc(m);
        if (COUNT) n_eval += done ? 0u : (uint32_t)n;
        for (int k = 0; k < n && !done; ++k) {
            const float4 g0 = sr0[k], g1 = sr1[k];
            float t;
            const float pe = pixel_exponent(g1.x, g1.y, g1.z, fx - g0.x, fy - g0.y, t);
            if (COUNT && pe >= P.p_min) ++n_reach;
            // without branches: a record outside the ellipse or below alpha_min gets alpha = 0,
            // and a step that would take T below t_min ends the pixel with weight 0; either
            // leaves T, C and D bit for bit unchanged (T - 0 T = T, C + 0 c = C)
            const bool hit = pe >= g1.w;
            const float alpha = hit ? fminf(P.alpha_max, g0.z * fast_exp2(pe)) : 0.f;
            const float Tn = fmaf(-alpha, T, T);   // T (1 - alpha), one rounding
            const bool stop = Tn < P.t_min;
            if (COUNT && hit && !stop) ++n_comp;
            const float wgt = stop ? 0.f : alpha * T;
            const float4 g2 = sr2[k];
            C0 = fmaf(wgt, g2.x, C0); C1 = fmaf(wgt, g2.y, C1); C2 = fmaf(wgt, g2.z, C2);
            D = fmaf(wgt, g0.w, D);
            T = stop ? T : Tn;
            done = stop;
        }
        __syncwarp();
    }
    if (CK && lane == 0) ck.last[(size_t)gt * n_sub + w] = entered;
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
                   const uint32_t* d_n, const ViewDesc* views, int nv, const Params& P) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, L.stream);
    if (n == 0) return;
    const uint32_t threads = (n + 3) / 4;
    const uint32_t blocks = std::min<uint32_t>((threads + 255) / 256, sm_count() * 8u);
    k_ranges<<<blocks, 256, 0, L.stream>>>(keys, n, d_n, ranges, n_tiles, views, (int)P.view0, nv,
                                                          P.tile0, P.tbits);
    ++*L.launches;
}

void launch_tile_order(const Launch& L, const uint2* ranges, int n_tiles, uint32_t* order) {
    if (n_tiles == 0) return;
    k_tile_order<<<1, 1024, 0, L.stream>>>(ranges, n_tiles, order);
    ++*L.launches;
}

void launch_segment_jobs(const Launch& L, const uint2* ranges, int n_tiles, const Checkpoints& ck) {
    if (n_tiles == 0) {
        cudaMemsetAsync(ck.n_jobs, 0, sizeof(uint32_t), L.stream);
        return;
    }
    k_segment_jobs<<<1, 1024, 0, L.stream>>>(ranges, n_tiles, ck);
    ++*L.launches;
}

void launch_composite(const Launch& L, const ViewDesc* views, int v0, int n_group_views, int n_tiles,
                      const uint2* ranges, const uint32_t* keys, const uint32_t* vals, const Record* records,
                      const Params& P, float* out_rgb, float* out_depth, float* out_alpha, unsigned long long* work,
                      const uint32_t* tile_order, const Checkpoints& ck) {
    if (n_tiles == 0) return;
    // checkpoints are for the adjoint, which never runs on randomised outputs
    const bool with_ck = ck.st != nullptr && !P.aug;
    auto* kern = with_ck ? (work ? k_composite<true, false, true> : k_composite<false, false, true>)
                 : work  ? (P.aug ? k_composite<true, true, false> : k_composite<true, false, false>)
                         : (P.aug ? k_composite<false, true, false> : k_composite<false, false, false>);
    const int bpt = (P.tile_w * P.tile_h) / (32 * kCompWarps);
    kern<<<n_tiles * bpt, kCompWarps * 32, 0, L.stream>>>(views, v0, n_group_views, ranges, keys, vals, records, P,
                                                          out_rgb, out_depth, out_alpha, work, tile_order, ck);
    ++*L.launches;
}

}  // namespace dgs
