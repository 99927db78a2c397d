// Stable LSD radix sort of (32-bit key, 32-bit value) pairs in the onesweep style (kernel K3).
//
// Sec. III-A: the 3DGS rasterizer orders the (tile, depth) pairs of every view with a fast
// GPU sort before blending.  Here the order is built in two stable sorts of 32-bit keys: the
// projected instances by depth key (28 bits) and then by their view in the view group (a more
// significant key carried by the values), then the (tile, instance) pairs -- emitted in that
// order -- by their tile within the view.  Stability carries the depth order, and the id order
// of equal depths, into every (view, tile) run.
//
// Structure: one upfront pass builds the histograms of every digit at once; then each digit is
// one kernel in which a block takes the next 3072-key partition from an atomic counter, ranks
// its keys by digit inside the block (per-bit warp ballots + per-warp counters), publishes its
// digit counts, scatters its keys into shared memory in digit order, and only then finds its
// global offset per digit by decoupled look-back over the partitions before it (status word =
// 2-bit flag | 30-bit count), which have had that long to publish their prefixes.  Measured on
// the benchmark's key sets (17.9M depth keys, 59.7M tile keys), the ballot ranking with 12 keys
// per thread at 4 blocks per SM sorts 13-17 % faster than warp-match ranking with 16 keys at 3
// blocks (either change alone gains nothing), and the late look-back 4 % faster than one right
// after the ranking.  Digits are D = ceil(bits / passes) bits wide with passes = ceil(bits / 8),
// the last pass taking the remaining bits so that exactly the requested key bits are sorted
// (bits above them keep their input order: the tile keys hold the view there, ordered by the
// depth sort before); measured on this path, wider digits (fewer passes) lose what they save to
// the scatter, whose runs per partition shrink to a few keys.  Look-back spins are bounded by
// a wall-clock limit (SortCtl::spin_ns, 1 s by default); on expiry the kernel sets
// kErrTimeout and finishes: its output is then not a permutation of the input, the kernels
// that use sorted values as indices return at once when they see kErrTimeout, and the host
// reports the timeout.
#include <algorithm>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 12;
constexpr int kTile = kThreads * kItems;          // 3072 keys per partition
constexpr int kWarps = kThreads / 32;
constexpr int kMaxD = 8;                          // widest digit: 256 bins
constexpr int kMaxR = 1 << kMaxD;
constexpr int kWindow = 4;                        // predecessors read per digit and look-back round
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kCountMask = (1u << 30) - 1u;
constexpr int kSmem = kTile * 8 + kWarps * kMaxR * 4;
constexpr int kKeysIn = 0, kKeysGather = 1, kKeysPacked = 2;   // where a pass's key comes from

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t live_count(uint32_t n, const uint32_t* d_n) { return d_n ? min(*d_n, n) : n; }

// Histograms of every pass's digit (digit width D) in one read of the keys; hist[p * kMaxR + b].
// Each warp counts into its own shared-memory copy (the copies are summed at the end).  RUNS:
// each thread counts 16 consecutive keys (four 16-byte loads) and issues one shared atomic per
// run of equal digits -- for keys whose high digits repeat over neighbours (tile keys emitted
// instance by instance, depth keys emitted node chunk by node chunk), whose lanes would
// otherwise all add to one counter; else a grid-stride loop with one atomic per key and pass.
template <bool RUNS>
__global__ void __launch_bounds__(kThreads) k_hist(const uint32_t* __restrict__ keys, uint32_t n,
                                                   const uint32_t* __restrict__ d_n, int passes, int D,
                                                   int last_bits, uint32_t* hist) {
    __shared__ uint32_t sh_all[kWarps][4 * kMaxR];   // one private histogram per warp
    uint32_t* sh = sh_all[threadIdx.x >> 5];
    n = live_count(n, d_n);
    // every pass's digit is D bits but the last one's, last_bits (the key bits above are not sorted)
    const uint32_t R = 1u << D;
    auto dmask = [&](int p) { return p == passes - 1 ? (1u << last_bits) - 1u : R - 1u; };
    for (int i = threadIdx.x; i < kWarps * 4 * kMaxR; i += kThreads) (&sh_all[0][0])[i] = 0;
    __syncthreads();
    if constexpr (RUNS) {
        const uint32_t stride = gridDim.x * kThreads * 16u;
        for (uint32_t base = (blockIdx.x * kThreads + threadIdx.x) * 16u; base < n; base += stride) {
            uint32_t k[16];
            if (base + 16 <= n) {
                const uint4* q = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint4 v = __ldg(q + j);
                    k[4 * j] = v.x; k[4 * j + 1] = v.y; k[4 * j + 2] = v.z; k[4 * j + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) k[j] = base + j < n ? keys[base + j] : 0u;
            }
            const int cnt = (int)min(16u, n - base);
            for (int p = 0; p < passes; ++p) {
                const uint32_t mask = dmask(p);
                uint32_t cur = (k[0] >> (D * p)) & mask, run = 1;
#pragma unroll
                for (int j = 1; j < 16; ++j) {
                    if (j >= cnt) break;
                    const uint32_t d = (k[j] >> (D * p)) & mask;
                    if (d == cur) { ++run; continue; }
                    atomicAdd(&sh[p * R + cur], run);
                    cur = d;
                    run = 1;
                }
                atomicAdd(&sh[p * R + cur], run);
            }
        }
    } else {
        for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
            const uint32_t k = keys[i];
            for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * R + ((k >> (D * p)) & dmask(p))], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * (int)R; i += kThreads) {
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += sh_all[w][i];
        if (t) atomicAdd(&hist[(i / R) * kMaxR + (i % R)], t);
    }
}

// one block, 256 threads: exclusive scan of each pass's R bins, in place (4 bins per thread)
__global__ void __launch_bounds__(256) k_hist_scan(uint32_t* hist, int passes, int R) {
    __shared__ uint32_t s_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = 0; p < passes; ++p) {
        uint32_t* h = hist + p * kMaxR;
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = threadIdx.x * 4 + j;
            v[j] = b < R ? h[b] : 0u;
            sum += v[j];
        }
        uint32_t y = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        if (lane == 31) s_w[warp] = y;
        __syncthreads();
        uint32_t run = y - sum;
        for (int w = 0; w < warp; ++w) run += s_w[w];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = threadIdx.x * 4 + j;
            if (b < R) h[b] = run;
            run += v[j];
        }
        __syncthreads();
    }
}

// One digit pass.  Thread t owns digits t, t + 256, ... (< 2^D) in the per-digit phases
// (prefix over warps, look-back, block scan); digits are (key >> shift) & (2^D - 1).
// MODE kKeysIn reads the keys; the other two derive a more significant key from the value (the
// keys sorted by the earlier passes are dropped): kKeysGather reads key = ind[value], kKeysPacked
// takes the value's high bits, key = value >> vshift.  Those two write no keys.  Every mode
// stores value & vmask (the last pass over packed values strips the key bits).  A null kout
// also skips the key writes (keys that no later pass reads).
template <int D, int MODE>
__global__ void __launch_bounds__(kThreads, 4) k_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n,
                                                      const uint32_t* __restrict__ d_n, int shift,
                                                      const uint32_t* __restrict__ digit_off, uint32_t* status,
                                                      uint32_t* counter, uint32_t* err, uint64_t spin_ns,
                                                      uint32_t mute_part, const uint32_t* __restrict__ ind, int vshift,
                                                      uint32_t vmask) {
    constexpr int R = 1 << D;
    constexpr uint32_t M = R - 1;
    constexpr int DPT = (R + kThreads - 1) / kThreads;   // digits per thread
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(smem);                          // kTile
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + kTile * 4);               // kTile
    uint32_t* s_whist = reinterpret_cast<uint32_t*>(smem + kTile * 8);              // kWarps x R
    __shared__ uint32_t s_dexcl[R];
    __shared__ uint32_t s_gbase[R];
    __shared__ uint32_t s_wsum[kWarps];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(counter, 1u);
    for (int i = tid; i < kWarps * R; i += kThreads) s_whist[i] = 0;
    __syncthreads();
    const uint32_t part = s_part;
    n = live_count(n, d_n);
    // a capacity-sized grid: partitions past the live count have no keys (and no later
    // partition looks back at them)
    if (part * (uint64_t)kTile >= n && part > 0) return;
    const uint32_t base = part * (uint32_t)kTile;

    uint32_t k[kItems], v[kItems], rank[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = base + warp * (kItems * 32) + j * 32 + lane;
        if (idx < n) {
            v[j] = vin[idx];
            // (a value outside 0..n-1, left by an earlier pass that gave up waiting, reads nothing)
            k[j] = MODE == kKeysGather ? (v[j] < n ? __ldg(ind + v[j]) : ~0u)
                   : MODE == kKeysPacked ? v[j] >> vshift
                                         : kin[idx];
        } else {
            k[j] = ~0u; v[j] = 0;
        }
    }
    // rank within the warp, in original order (round j covers 32 consecutive keys); the lanes
    // holding the same digit are found by one ballot per digit bit
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t* wh = s_whist + warp * R;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t dg = (k[j] >> shift) & M;
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const bool bit = (dg >> b) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        const uint32_t pre = wh[dg];
        rank[j] = pre + __popc(peers & lt);
        __syncwarp();
        if ((peers & lt) == 0) wh[dg] = pre + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per owned digit: exclusive prefix over warps and the partition total
    uint32_t total[DPT], excl[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid + q * kThreads;
        total[q] = 0;
        excl[q] = 0;
        if (d < R) {
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = s_whist[w * R + d];
                s_whist[w * R + d] = total[q];
                total[q] += c;
            }
        }
    }
    // publish this partition's digit counts at once (the inclusive prefix for partition 0);
    // partition mute_part (a test of the bounded wait, never a real partition index by
    // default) publishes nothing, so the partitions after it wait for it until spin_ns runs out
    const bool publish = part != mute_part;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid + q * kThreads;
        if (d < R && publish) st_relaxed(&status[(size_t)part * R + d], (part == 0 ? kFlagInc : kFlagAgg) | total[q]);
    }
    // block exclusive scan of the digit totals in digit order -> local digit offsets; slab q
    // holds digits [q * 256, q * 256 + 256)
    uint32_t carry = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        uint32_t x = total[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t wpre = 0, slab = 0;
        for (int w = 0; w < kWarps; ++w) {
            if (w < warp) wpre += s_wsum[w];
            slab += s_wsum[w];
        }
        const int d = tid + q * kThreads;
        if (d < R) s_dexcl[d] = carry + wpre + x - total[q];
        carry += slab;
        __syncthreads();
    }
    // local scatter: digit-major order inside the partition
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t dj = (k[j] >> shift) & M;
        const uint32_t pos = s_dexcl[dj] + s_whist[warp * R + dj] + rank[j];
        s_keys[pos] = k[j];
        s_vals[pos] = v[j];
    }
    // decoupled look-back over earlier partitions, all owned digits at once, after the local
    // scatter: the partitions before this one have had that long to publish their prefixes
    if (part > 0) {
        int64_t p[DPT];
        bool done[DPT];
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid + q * kThreads;
            done[q] = d >= R;
            p[q] = (int64_t)part - 1;
        }
        uint64_t t0 = 0;
        uint32_t spins = 0;
        while (true) {
            uint32_t sv[DPT][kWindow];
#pragma unroll
            for (int q = 0; q < DPT; ++q)
#pragma unroll
                for (int w = 0; w < kWindow; ++w)
                    sv[q][w] = (!done[q] && p[q] - w >= 0)
                                   ? ld_relaxed(&status[(size_t)(p[q] - w) * R + tid + q * kThreads]) : kFlagInc;
            bool all = true, stall = false;
#pragma unroll
            for (int q = 0; q < DPT; ++q) {
                if (done[q]) continue;
                bool stop = false;
#pragma unroll
                for (int w = 0; w < kWindow; ++w) {
                    if (stop || done[q]) continue;
                    const uint32_t f = sv[q][w] & ~kCountMask;
                    if (f == 0) { stop = true; continue; }
                    excl[q] += sv[q][w] & kCountMask;
                    if (f == kFlagInc) done[q] = true; else --p[q];
                }
                if (!done[q]) { all = false; stall |= stop; }
            }
            if (all) break;
            if (stall && (++spins & 1023u) == 0) {
                const uint64_t now = global_timer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > spin_ns) { atomicOr(err, kErrTimeout); break; }
            }
        }
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid + q * kThreads;
            if (d < R && publish) st_relaxed(&status[(size_t)part * R + d], kFlagInc | (excl[q] + total[q]));
        }
    }
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid + q * kThreads;
        if (d < R) s_gbase[d] = digit_off[d] + excl[q];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = tid; i < kTile; i += kThreads) {
        const uint32_t key = s_keys[i];
        const uint32_t dj = (key >> shift) & M;
        const uint32_t g = s_gbase[dj] + (uint32_t)i - s_dexcl[dj];
        // every live key lands below n (the padding keys, ~0, sort past the end and are dropped)
        if (kDebugChecks && key != ~0u && !in_bounds(g, n, err, kSiteSortScatter)) continue;
        if (g < n) {
            if (MODE == kKeysIn && kout) kout[g] = key;
            vout[g] = s_vals[i] & vmask;
        }
    }
}

using OnesweepFn = void (*)(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t, const uint32_t*, int,
                            const uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint64_t, uint32_t, const uint32_t*, int,
                            uint32_t);

template <int MODE>
OnesweepFn onesweep_for(int D) {
    switch (D) {
        case 1: return k_onesweep<1, MODE>;
        case 2: return k_onesweep<2, MODE>;
        case 3: return k_onesweep<3, MODE>;
        case 4: return k_onesweep<4, MODE>;
        case 5: return k_onesweep<5, MODE>;
        case 6: return k_onesweep<6, MODE>;
        case 7: return k_onesweep<7, MODE>;
        default: return k_onesweep<8, MODE>;
    }
}

// Histograms of the view passes' digits, from the count scan rather than from the values: view
// j of the group holds inst_off[view_tab[v0 + j + 1]] - inst_off[view_tab[v0 + j]] instance
// numbers.  One block; the bins are stored, not added.
__global__ void __launch_bounds__(kThreads) k_view_hist(const uint32_t* __restrict__ inst_off,
                                                        const int64_t* __restrict__ view_tab, int v0, int nv,
                                                        int passes, int D, int last_bits, uint32_t* hist) {
    __shared__ uint32_t sh[4 * kMaxR];
    const uint32_t R = 1u << D;
    for (int i = threadIdx.x; i < passes * (int)R; i += kThreads) sh[i] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < nv; j += kThreads) {
        const uint32_t c = inst_off[view_tab[v0 + j + 1]] - inst_off[view_tab[v0 + j]];
        if (!c) continue;
        for (int p = 0; p < passes; ++p) {
            const uint32_t mask = p == passes - 1 ? (1u << last_bits) - 1u : R - 1u;
            atomicAdd(&sh[p * R + (((uint32_t)j >> (D * p)) & mask)], c);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * (int)R; i += kThreads) hist[(i / R) * kMaxR + (i % R)] = sh[i];
}

}  // namespace

// Streaming multiprocessors of the current device (read once per process and device).
uint32_t sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        cached[dev] = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 152;
    }
    return (uint32_t)cached[dev];
}

int sort_passes(int key_bits) { return std::max(1, (key_bits + kMaxD - 1) / kMaxD); }

size_t sort_status_words(uint32_t n) { return ((size_t)n + kTile - 1) / kTile * kMaxR; }

void sort_prepare() {
    static bool attr_set = false;
    if (!attr_set) {
        for (int D = 1; D <= kMaxD; ++D) {
            cudaFuncSetAttribute(onesweep_for<kKeysIn>(D), cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
            cudaFuncSetAttribute(onesweep_for<kKeysGather>(D), cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
            cudaFuncSetAttribute(onesweep_for<kKeysPacked>(D), cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        }
        attr_set = true;
    }
}

// hist: [8 * 256] words, counters: [8] words, status: sort_status_words(n) words.
void launch_sort(const Launch& L, uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, uint32_t n,
                 int key_bits, uint32_t* hist, uint32_t* status, uint32_t* counters, uint32_t* err,
                 uint32_t** keys_out, uint32_t** vals_out, const uint32_t* d_n, SortCtl ctl, const ViewKey* vk) {
    *keys_out = keys;
    *vals_out = vals;
    // with a device-side count every pass runs (the output lands in the same buffer whatever
    // the count); a host-known count of 0 or 1 is already sorted
    if (n <= 1 && !d_n) return;
    if (n == 0) return;
    const int bits = std::max(1, key_bits);
    const int passes = sort_passes(bits);
    const int D = (bits + passes - 1) / passes;
    const int last_bits = bits - D * (passes - 1);      // exactly key_bits bits are sorted
    sort_prepare();
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kMaxR * passes, L.stream);
    cudaMemsetAsync(counters, 0, sizeof(uint32_t) * 8, L.stream);
    const int hist_blocks = (int)std::min<uint32_t>(4 * sm_count(), (n + kThreads * 8 - 1) / (kThreads * 8));
    if (ctl.runs) k_hist<true><<<hist_blocks, kThreads, 0, L.stream>>>(keys, n, d_n, passes, D, last_bits, hist);
    else k_hist<false><<<hist_blocks, kThreads, 0, L.stream>>>(keys, n, d_n, passes, D, last_bits, hist);
    k_hist_scan<<<1, 256, 0, L.stream>>>(hist, passes, 1 << D);
    *L.launches += 2;
    const uint32_t parts = (n + kTile - 1) / kTile;
    const bool by_view = vk && vk->bits > 0;
    uint32_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int Dp = p == passes - 1 ? last_bits : D;
        const OnesweepFn fn = onesweep_for<false>(Dp);
        // the view passes read no keys: the last key pass before them writes none
        uint32_t* kw = by_view && p == passes - 1 ? nullptr : ko;
        cudaMemsetAsync(status, 0, sizeof(uint32_t) * (size_t)(1 << Dp) * parts, L.stream);
        fn<<<parts, kThreads, kSmem, L.stream>>>(ki, vi, kw, vo, n, d_n, D * p, hist + p * kMaxR, status, counters + p,
                                                 err, ctl.spin_ns, p == 0 ? ctl.mute_part : 0xFFFFFFFFu, nullptr, 0,
                                                 0xFFFFFFFFu);
        ++*L.launches;
        uint32_t* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
    }
    // the most significant key, the view, derived from the values (their high bits, or vig[value]);
    // its histogram comes from the per-view counts of the count scan
    if (by_view) {
        const int ip = sort_passes(vk->bits);
        const int Di = (vk->bits + ip - 1) / ip;
        const int ilast = vk->bits - Di * (ip - 1);
        uint32_t* ih = hist + passes * kMaxR;
        k_view_hist<<<1, kThreads, 0, L.stream>>>(vk->inst_off, vk->view_tab, vk->v0, vk->nv, ip, Di, ilast, ih);
        k_hist_scan<<<1, 256, 0, L.stream>>>(ih, ip, 1 << Di);
        *L.launches += 2;
        const bool packed = vk->vshift > 0;
        for (int p = 0; p < ip; ++p) {
            const int Dp = p == ip - 1 ? ilast : Di;
            const OnesweepFn fi = packed ? onesweep_for<kKeysPacked>(Dp) : onesweep_for<kKeysGather>(Dp);
            const uint32_t vmask = packed && p == ip - 1 ? (1u << vk->vshift) - 1u : 0xFFFFFFFFu;
            cudaMemsetAsync(status, 0, sizeof(uint32_t) * (size_t)(1 << Dp) * parts, L.stream);
            fi<<<parts, kThreads, kSmem, L.stream>>>(ki, vi, ko, vo, n, d_n, Di * p, ih + p * kMaxR, status,
                                                     counters + passes + p, err, ctl.spin_ns, 0xFFFFFFFFu, vk->vig,
                                                     vk->vshift, vmask);
            ++*L.launches;
            uint32_t* tk = ki; ki = ko; ko = tk;
            uint32_t* tv = vi; vi = vo; vo = tv;
        }
    }
    *keys_out = by_view ? nullptr : ki;
    *vals_out = vi;
}

}  // namespace dgs
