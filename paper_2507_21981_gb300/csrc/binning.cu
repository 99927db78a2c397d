// Depth-ordered (tile, instance) pairs: tile-count scan (K3b) and pair emission (K3c).
//
// Sec. III-A: after projection every screen tile must receive the Gaussians that reach it in
// front-to-back order.  The projected instances are first sorted by depth key; here each
// instance's tile pairs are laid out in that order (an exclusive scan of the instances' pair
// counts taken in sorted order) and written by walking the instance's tile rectangle with the
// same exact test that counted them.  A stable sort by tile then leaves every tile's run in
// depth order, equal depths in emission (id) order.
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kScanThreads = 256, kScanItems = 16, kScanTile = kScanThreads * kScanItems;
constexpr int kPairWarps = 4;

__device__ __forceinline__ uint32_t live(uint32_t n, const uint32_t* d_n) { return d_n ? min(n, *d_n) : n; }

__device__ __forceinline__ uint32_t block_sum(uint32_t x) {
    __shared__ uint32_t s[kScanThreads / 32];
    x = __reduce_add_sync(0xffffffffu, x);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += s[w];
    return t;
}

// parts[b] = sum of ntile[order[i]] over partition b
__global__ void __launch_bounds__(kScanThreads) k_tscan_partial(const uint32_t* __restrict__ order,
                                                               const uint32_t* __restrict__ ntile, uint32_t n,
                                                               const uint32_t* __restrict__ d_n, uint32_t* parts,
                                                               const uint32_t* err) {
    if (sort_failed(err)) return;
    n = live(n, d_n);
    const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
    if (base >= n) return;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) s += ntile[order[i]];
    }
    s = block_sum(s);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// one block: exclusive scan of the live partitions' sums in place; poff[n] = the grand total
// and *total = min(grand total, cap)
__global__ void __launch_bounds__(kScanThreads) k_tscan_parts(uint32_t* parts, uint32_t n, const uint32_t* __restrict__ d_n,
                                                              uint32_t* poff, uint32_t cap, uint32_t* total) {
    __shared__ uint32_t s_w[kScanThreads / 32];
    n = live(n, d_n);
    const uint32_t np = (n + kScanTile - 1) / kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (uint32_t b0 = 0; b0 < np; b0 += kScanThreads) {
        const uint32_t i = b0 + threadIdx.x;
        const uint32_t x = i < np ? parts[i] : 0u;
        uint32_t y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        if (lane == 31) s_w[warp] = y;
        __syncthreads();
        uint32_t wpre = 0, all = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) {
            if (w < warp) wpre += s_w[w];
            all += s_w[w];
        }
        if (i < np) parts[i] = carry + wpre + y - x;
        carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        poff[n] = carry;
        *total = min(carry, cap);
    }
}

// poff[i] for i < n: thread t of block b scans 16 consecutive entries
__global__ void __launch_bounds__(kScanThreads) k_tscan_final(const uint32_t* __restrict__ order,
                                                             const uint32_t* __restrict__ ntile, uint32_t n,
                                                             const uint32_t* __restrict__ d_n,
                                                             const uint32_t* __restrict__ parts, uint32_t* poff,
                                                             const uint32_t* err) {
    __shared__ uint32_t s_w[kScanThreads / 32];
    if (sort_failed(err)) return;
    n = live(n, d_n);
    const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
    if (base >= n) return;
    const uint32_t i0 = base + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = i0 + j < n ? ntile[order[i0 + j]] : 0u;
        sum += v[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t y = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
    }
    if (lane == 31) s_w[warp] = y;
    __syncthreads();
    uint32_t run = parts[blockIdx.x] + y - sum;
    for (int w = 0; w < warp; ++w) run += s_w[w];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (i0 + j < n) poff[i0 + j] = run;
        run += v[j];
    }
}

// Per-warp state of the pair walk: item l is depth-ordered instance i0 + l.
struct PairWarp {
    float4 a[32];          // (u, v, qa, qb)
    float4 b[32];          // (qc, x-box, y-box, tile origin)
    float4 e[32];          // ellipse_extent of the instance
    int4 c[32];            // (rectangle width in tiles, first tile of the view in the group, view tiles_x, record)
    uint32_t excl[32], off[32], end[32], run[32];
};

__global__ void __launch_bounds__(kPairWarps * 32) k_pairs(const ViewDesc* __restrict__ views, int K,
                                                          const uint32_t* __restrict__ order,
                                                          const uint32_t* __restrict__ poff,
                                                          const Record* __restrict__ rec,
                                                          const InstInfo* __restrict__ info, uint32_t n,
                                                          const uint32_t* __restrict__ d_n, Params P,
                                                          uint32_t* __restrict__ tkeys, uint32_t* __restrict__ tvals,
                                                          uint32_t cap) {
    __shared__ PairWarp pw[kPairWarps];
    if (sort_failed(P.err)) return;
    n = live(n, d_n);
    const uint32_t w = (blockIdx.x * (uint32_t)blockDim.x + threadIdx.x) >> 5;
    if (w * 32u >= n) return;
    const int lane = (int)lane_id();
    PairWarp& S = pw[threadIdx.x >> 5];
    const uint32_t item = w * 32u + (uint32_t)lane;
    const bool act = item < n;
    uint32_t area = 0;
    if (act) {
        const uint32_t r = order[item];
        const Record& R = rec[r];
        const float4 r0 = R.r0, r1 = R.r1;
        const float byf = R.r2.w;
        const uint32_t bx = __float_as_uint(r1.w), by = __float_as_uint(byf);
        const int tx0 = (int)(bx & 0xFFFFu) >> P.tile_sx, tx1 = (int)(bx >> 16) >> P.tile_sx;
        const int ty0 = (int)(by & 0xFFFFu) >> P.tile_sy, ty1 = (int)(by >> 16) >> P.tile_sy;
        const ViewDesc& vd = views[info[r].view / (uint32_t)K];
        S.a[lane] = make_float4(r0.x, r0.y, r1.x, r1.y);
        S.b[lane] = make_float4(r1.z, r1.w, byf, pack_u16x2((uint32_t)tx0, (uint32_t)ty0));
        S.e[lane] = ellipse_extent(r1.x, r1.y, r1.z, P.qbin);
        S.c[lane] = make_int4(tx1 - tx0 + 1, vd.tile_base - P.tile0, vd.tiles_x, (int)r);
        S.off[lane] = poff[item];
        S.end[lane] = poff[item + 1];
        S.run[lane] = 0;
        area = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    }
    uint32_t incl = area;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t my = incl - area;
    S.excl[lane] = my;
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t base = 0; base < total; base += 32) {
        const int o = walk_owner_of(lane, act, act ? my : total, base);
        const uint32_t f = base + (uint32_t)lane;
        bool hit = false;
        int tx = 0, ty = 0;
        int4 cc = make_int4(0, 0, 0, 0);
        if (f < total) {
            cc = S.c[o];
            hit = walk_tile(S.a[o], S.b[o], cc.x, f - S.excl[o], P, tx, ty);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, hit ? o : -1);
        if (hit) {
            const uint32_t pos = S.off[o] + S.run[o] + __popc(peers & lt);
            if (pos < S.end[o] && pos < cap) {
                const float4 a = S.a[o], b = S.b[o];
                const uint32_t bx = __float_as_uint(b.y), by = __float_as_uint(b.z);
                const uint32_t sub = subtile_mask(a.x, a.y, a.z, a.w, b.x, S.e[o], (int)(bx & 0xFFFFu), (int)(bx >> 16),
                                                  (int)(by & 0xFFFFu), (int)(by >> 16), tx, ty, P);
                tkeys[pos] = (uint32_t)(cc.y + ty * cc.z + tx) | (sub << kTileBits);
                tvals[pos] = (uint32_t)cc.w;
            } else {
                atomicOr(P.err, pos < cap ? kErrMismatch : kErrCapacity);
            }
        }
        __syncwarp();
        if (hit && (peers & lt) == 0) S.run[o] += __popc(peers);
        __syncwarp();
    }
    // the emission count and this walk take the same decisions; pad a shortfall with dead keys
    if (act) {
        const uint32_t have = S.off[lane] + S.run[lane];
        if (have != S.end[lane]) {
            atomicOr(P.err, kErrMismatch);
            for (uint32_t q = have; q < S.end[lane] && q < cap; ++q) { tkeys[q] = ~0u; tvals[q] = 0; }
        }
    }
}

}  // namespace

size_t tile_scan_parts(uint32_t n) { return ((size_t)n + kScanTile - 1) / kScanTile + 1; }

void launch_tile_scan(const Launch& L, const uint32_t* order, const uint32_t* ntile, uint32_t n, const uint32_t* d_n,
                      uint32_t* poff, uint32_t* parts, uint32_t cap, uint32_t* total, const uint32_t* err) {
    const uint32_t blocks = (n + kScanTile - 1) / kScanTile;
    if (blocks) k_tscan_partial<<<blocks, kScanThreads, 0, L.stream>>>(order, ntile, n, d_n, parts, err);
    k_tscan_parts<<<1, kScanThreads, 0, L.stream>>>(parts, n, d_n, poff, cap, total);
    if (blocks) k_tscan_final<<<blocks, kScanThreads, 0, L.stream>>>(order, ntile, n, d_n, parts, poff, err);
    *L.launches += blocks ? 3 : 1;
}

void launch_pairs(const Launch& L, const ViewDesc* views, int K, const uint32_t* order, const uint32_t* poff,
                  const Record* records, const InstInfo* info, uint32_t n, const uint32_t* d_n, const Params& P,
                  uint32_t* tkeys, uint32_t* tvals, uint32_t cap) {
    if (n == 0) return;
    const uint32_t warps = (n + 31) / 32;
    const uint32_t blocks = (warps + kPairWarps - 1) / kPairWarps;
    k_pairs<<<blocks, kPairWarps * 32, 0, L.stream>>>(views, K, order, poff, records, info, n, d_n, P, tkeys, tvals, cap);
    ++*L.launches;
}

}  // namespace dgs
