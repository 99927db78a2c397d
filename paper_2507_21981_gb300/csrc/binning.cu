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
                                                               uint32_t* err) {
    if (sort_failed(err)) return;
    n = live(n, d_n);
    const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
    if (base >= n) return;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) {
            const uint32_t r = order[i];
            if (in_bounds(r, n, err, kSiteScanInstance)) s += ntile[r];
        }
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

// poff[i] for i < n: thread t of block b scans the 16 consecutive entries from 16 t of its tile
__global__ void __launch_bounds__(kScanThreads) k_tscan_final(const uint32_t* __restrict__ order,
                                                             const uint32_t* __restrict__ ntile, uint32_t n,
                                                             const uint32_t* __restrict__ d_n,
                                                             const uint32_t* __restrict__ parts, uint32_t* poff,
                                                             uint32_t* err) {
    __shared__ uint32_t s_w[kScanThreads / 32];
    // the counts of the block's kScanTile instances, gathered warp-striped (coalesced order
    // reads) into shared memory, one pad word per 16 against bank conflicts; each thread then
    // scans its kScanItems consecutive counts, and the offsets go back the same way
    __shared__ uint32_t s_v[kScanTile + kScanTile / 16];
    auto slot = [](int k) { return k + (k >> 4); };
    if (sort_failed(err)) return;
    n = live(n, d_n);
    const uint32_t base = blockIdx.x * (uint32_t)kScanTile;
    if (base >= n) return;
#pragma unroll 4
    for (int j = 0; j < kScanItems; ++j) {
        const int k = j * kScanThreads + threadIdx.x;
        uint32_t x = 0u;
        if (base + k < n) {
            const uint32_t r = order[base + k];
            if (in_bounds(r, n, err, kSiteScanInstance)) x = ntile[r];
        }
        s_v[slot(k)] = x;
    }
    __syncthreads();
    uint32_t v[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = s_v[slot(threadIdx.x * kScanItems + j)];
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
        s_v[slot(threadIdx.x * kScanItems + j)] = run;
        run += v[j];
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < kScanItems; ++j) {
        const int k = j * kScanThreads + threadIdx.x;
        if (base + k < n) poff[base + k] = s_v[slot(k)];
    }
}

// Sub-tile mask of tile column tx from the sub-row intervals [L, R] of its tile row (SR rows x SC
// columns of 8x4-pixel sub-tiles; bit s = sub-tile (s mod SC, s div SC)).
template <int SR, int SC>
__device__ __forceinline__ uint32_t row_mask(const float (&L)[SR], const float (&R)[SR], int tx, int tile_w) {
    uint32_t m = 0;
#pragma unroll
    for (int sy = 0; sy < SR; ++sy)
#pragma unroll
        for (int sx = 0; sx < SC; ++sx) {
            const float c0 = (float)(tx * tile_w + sx * 8) + 0.5f;
            if (L[sy] <= c0 + 7.f && R[sy] >= c0) m |= 1u << (sy * SC + sx);
        }
    return m;
}

// Per-warp state of the pair writer: item l is depth-ordered instance i0 + l.  Its pairs are
// written tile row by tile row: a row job (item, tile row) covers the run of tiles that row's
// band of the ellipse reaches (tile_row_run), in row-major order, at the item's next positions.
// Row jobs are taken 32 at a time, one per lane, and a lane writes its job's whole run (runs are
// short: about three tiles on the benchmark batch).
struct PairWarp {
    float4 a[32];          // (u, v, qb, qc)
    float4 e[32];          // ellipse_extent
    int4 box[32];          // pixel box (x0, x1, y0, y1)
    int4 c[32];            // (first tile row, view's first tile in the group, view tiles_x, record)
    uint32_t rexcl[32];    // exclusive prefix of the items' tile-row counts
    uint32_t off[32], end[32], run[32];
};

// SR x SC: sub-tile rows and columns of the tile shape (8x4-pixel sub-tiles).
template <int SR, int SC>
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
    const uint32_t full = 0xffffffffu;
    PairWarp& S = pw[threadIdx.x >> 5];
    const uint32_t item = w * 32u + (uint32_t)lane;
    const uint32_t r = item < n ? order[item] : 0u;
    const bool act = item < n && in_bounds(r, n, P.err, kSitePairsInstance);
    uint32_t nrows = 0;
    if (act) {
        const Record& R = rec[r];
        const float4 r0 = R.r0, r1 = R.r1;
        const uint32_t bx = __float_as_uint(r1.w), by = __float_as_uint(R.r2.w);
        const int x0 = (int)(bx & 0xFFFFu), x1 = (int)(bx >> 16), y0 = (int)(by & 0xFFFFu), y1 = (int)(by >> 16);
        const int ty0 = y0 >> P.tile_sy, ty1 = y1 >> P.tile_sy;
        const uint32_t view = info[r].view / (uint32_t)K;
        const ViewDesc& vd = views[view];
        S.a[lane] = make_float4(r0.x, r0.y, r1.y, r1.z);
        S.e[lane] = ellipse_extent(r1.x, r1.y, r1.z, P.qbin);
        S.box[lane] = make_int4(x0, x1, y0, y1);
        // tile keys: the view in the group above the tile's index in its view
        S.c[lane] = make_int4(ty0, (int)((view - P.view0) << P.tbits), vd.tiles_x, (int)r);
        S.off[lane] = poff[item];
        S.end[lane] = poff[item + 1];
        S.run[lane] = 0;
        nrows = (uint32_t)(ty1 - ty0 + 1);     // >= 1: walk_owner_of needs a unit per item
    }
    uint32_t incl = nrows;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total_rows = __shfl_sync(full, incl, 31);
    const uint32_t my_rexcl = incl - nrows;
    S.rexcl[lane] = my_rexcl;
    __syncwarp();
    for (uint32_t rb = 0; rb < total_rows; rb += 32) {
        // one row job per lane: its run of tiles and the sub-row intervals of its tile row
        const uint32_t j = rb + (uint32_t)lane;
        const bool jact = j < total_rows;
        const int o = walk_owner_of(lane, act, act ? my_rexcl : total_rows, rb);
        int nrun = 0, t0 = 0, row = 0;
        float L[SR], R[SR];
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), e = a;
        int4 bx = make_int4(0, 0, 0, 0);
        if (jact) {
            a = S.a[o]; e = S.e[o]; bx = S.box[o];
            row = S.c[o].x + (int)(j - S.rexcl[o]);
            // an instance without pairs (no row reaches a pixel centre, or a dead record of the
            // count pass's conservative cull, whose conic is all zero) writes none
            if (S.end[o] > S.off[o]) nrun = tile_row_run(a.x, a.y, a.z, a.w, e, bx.x, bx.y, bx.z, bx.w, row, P, t0);
        }
        // the job's first position: the item's pairs of earlier batches, plus the runs of its
        // earlier jobs in this batch (an item's jobs are consecutive lanes)
        uint32_t jincl = (uint32_t)nrun;
#pragma unroll
        for (int q = 1; q < 32; q <<= 1) {
            const uint32_t t = __shfl_up_sync(full, jincl, q);
            if (lane >= q) jincl += t;
        }
        const uint32_t jexcl = jincl - (uint32_t)nrun;
        const int seg0 = jact ? (int)(max(rb, S.rexcl[o]) - rb) : lane;
        const uint32_t seg_excl0 = __shfl_sync(full, jexcl, seg0);
        const int next_o = __shfl_down_sync(full, o, 1);
        const bool last_of_item = jact && (lane == 31 || j + 1 >= total_rows || next_o != o);
        if (nrun > 0) {
            const uint32_t first = S.off[o] + S.run[o] + (jexcl - seg_excl0);
            const uint32_t end = min(S.end[o], cap);
            const int4 cc = S.c[o];
            const uint32_t tile_row = (uint32_t)(cc.y + row * cc.z);
            // sub-row intervals of this tile row (unrolled: registers)
#pragma unroll
            for (int sy = 0; sy < SR; ++sy) {
                L[sy] = 1.f; R[sy] = 0.f;
                const int ry = row * (4 * SR) + sy * 4;
                const int py0 = max(ry, bx.z), py1 = min(ry + 3, bx.w);
                float l = (float)bx.x + 0.5f, rr = (float)bx.y + 0.5f;
                bool ok = py0 <= py1;
                if (ok && P.exact_tile_test) {
                    float bl, br;
                    ok = band_interval(a.x, a.y, a.z, a.w, e, (float)py0 + 0.5f, (float)py1 + 0.5f, P.qbin, bl, br);
                    l = fmaxf(l, bl);
                    rr = fminf(rr, br);
                }
                if (ok) { L[sy] = l; R[sy] = rr; }
            }
            for (int ti = 0; ti < nrun; ++ti) {
                const int tx = t0 + ti;
                const uint32_t sub = row_mask<SR, SC>(L, R, tx, 8 * SC);
                const uint32_t pos = first + (uint32_t)ti;
                if (pos < end) {
                    tkeys[pos] = (tile_row + (uint32_t)tx) | (sub << kTileBits);
                    tvals[pos] = (uint32_t)cc.w;
                } else {
                    atomicOr(P.err, pos < cap ? kErrMismatch : kErrCapacity);
                }
            }
        }
        __syncwarp();
        if (last_of_item) S.run[o] += jincl - seg_excl0;
        __syncwarp();
    }
    // the emission count and these runs take the same decisions; pad a shortfall with dead keys
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
                      uint32_t* poff, uint32_t* parts, uint32_t cap, uint32_t* total, uint32_t* err) {
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
    // one instantiation per tile shape (sub-tile rows x columns; at most 8 sub-tiles)
    auto kern = k_pairs<1, 1>;
    switch ((P.tile_h >> 2) * 16 + (P.tile_w >> 3)) {
        case 1 * 16 + 2: kern = k_pairs<1, 2>; break;
        case 1 * 16 + 4: kern = k_pairs<1, 4>; break;
        case 1 * 16 + 8: kern = k_pairs<1, 8>; break;
        case 2 * 16 + 1: kern = k_pairs<2, 1>; break;
        case 2 * 16 + 2: kern = k_pairs<2, 2>; break;
        case 2 * 16 + 4: kern = k_pairs<2, 4>; break;
        case 4 * 16 + 1: kern = k_pairs<4, 1>; break;
        case 4 * 16 + 2: kern = k_pairs<4, 2>; break;
        case 8 * 16 + 1: kern = k_pairs<8, 1>; break;
        default: break;
    }
    kern<<<blocks, kPairWarps * 32, 0, L.stream>>>(views, K, order, poff, records, info, n, d_n, P, tkeys, tvals, cap);
    ++*L.launches;
}

}  // namespace dgs
